// Arnoldi steps of the outer FGMRES in FP32-pair arithmetic.
//
// The fine-level Krylov basis is FP64, and one Arnoldi step with classical
// Gram-Schmidt and one reorthogonalisation (CGS2) costs about 32 (k + 1)
// FP64 multiply-adds per complex element against k + 1 basis vectors.  On
// GB300 the FP64 rate (two FMA per clock per SM) makes that the limit, not
// the memory traffic.  These kernels keep the FP64 vectors in memory, split
// every loaded value into a pair h + l of FP32 numbers with integer
// operations (tm_pair.cuh), and do the products and sums in pair arithmetic
// (about 47 significant bits); results written back are FP64.  Each vector
// update is fused with the reduction that follows it in CGS2, so one step
// reads the basis three times instead of four:
//   d1 = V^H w                       (launch_pdot_b)
//   w -= V d1;  d2 = V^H w           (launch_pcaxpy_dot_b)
//   w -= V d2;  n = |w|^2            (launch_pcaxpy_norm_b)
// Partial sums per CTA are converted to FP64 and reduced in a fixed order,
// so every result is deterministic.
#include "tm_kernels.h"
#include "tm_pair.cuh"

namespace tmamg {

namespace {

constexpr int kPairThreads = 256;
constexpr int kChunk = 8;  // basis vectors handled per CTA in registers

int pair_grid(long ncx) { return dot_grid_for(ncx); }

__device__ __forceinline__ cdf ld_pair(const double* __restrict__ p, long i) {
  const double2 v = reinterpret_cast<const double2*>(p)[i];
  return cx2pair(v.x, v.y);
}
__device__ __forceinline__ void st_pair(double* __restrict__ p, long i, cdf a) {
  reinterpret_cast<double2*>(p)[i] = make_double2(pair2d(a.r), pair2d(a.i));
}

// stage 1 of d_j = sum_i conj(X_j[i]) y[i] for j in the CTA's chunk of KC
// (KC = 4 for short bases: fewer registers, more warps in flight)
template <int KC>
__global__ void __launch_bounds__(kPairThreads) k_pdot_partial_b(const double* __restrict__ X, long xstr, long ldx,
                                                                 int k, const double* __restrict__ y, long ystr,
                                                                 long ncx, double* __restrict__ part,
                                                                 const int* __restrict__ active) {
  __shared__ double red[32 * 2 * KC];
  const int r = blockIdx.z;
  if (active && !active[r]) return;
  const int j0 = blockIdx.y * KC;
  cdf d[KC];
#pragma unroll
  for (int m = 0; m < KC; ++m) d[m] = cdf{{0.f, 0.f}, {0.f, 0.f}};
  const double* yr = y + r * ystr;
  const double* Xr = X + r * xstr + j0 * ldx;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    const cdf yv = ld_pair(yr, i);
#pragma unroll
    for (int jj = 0; jj < KC; ++jj)
      if (j0 + jj < k) cfmac_pp(d[jj], ld_pair(Xr + jj * ldx, i), yv);
  }
  double v[2 * KC];
#pragma unroll
  for (int jj = 0; jj < KC; ++jj) {
    v[2 * jj] = pair2d(d[jj].r);
    v[2 * jj + 1] = pair2d(d[jj].i);
  }
  block_allreduce<double, 2 * KC>(v, red);
  if (threadIdx.x < 2 * KC) {
    const int jj = threadIdx.x >> 1;
    if (j0 + jj < k)
      part[(((long)r * k + j0 + jj) * gridDim.x + blockIdx.x) * 2 + (threadIdx.x & 1)] = v[threadIdx.x];
  }
}

// y -= sum_j c_j X_j over all k vectors; MODE 1 (k <= KC) also forms the
// partial sums of d_j = X_j^H y with the updated y, MODE 2 those of |y|^2
template <int MODE, int KC = kChunk>
__global__ void __launch_bounds__(kPairThreads) k_pcaxpy_b(const double* __restrict__ X, long xstr, long ldx, int k,
                                                           const double* __restrict__ c, long cstr,
                                                           double* __restrict__ y, long ystr, long ncx,
                                                           double* __restrict__ part, const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char praw[];
  cdf* cs = reinterpret_cast<cdf*>(praw);  // -c_j as pairs, [k]
  double* red = reinterpret_cast<double*>(cs + k);
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const double* cr = c + r * cstr;
  for (int j = threadIdx.x; j < k; j += blockDim.x) cs[j] = cx2pair(-cr[2 * j], -cr[2 * j + 1]);
  __syncthreads();
  double* yr = y + r * ystr;
  const double* Xr = X + r * xstr;
  cdf d[MODE == 1 ? KC : 1];
#pragma unroll
  for (int m = 0; m < (MODE == 1 ? KC : 1); ++m) d[m] = cdf{{0.f, 0.f}, {0.f, 0.f}};
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    cdf acc = ld_pair(yr, i);
    if constexpr (MODE == 1) {
      cdf xs[KC];
#pragma unroll
      for (int j = 0; j < KC; ++j) xs[j] = cdf{{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
      for (int j = 0; j < KC; ++j) {
        if (j < k) {
          xs[j] = ld_pair(Xr + j * ldx, i);
          cfma_pp(acc, cs[j], xs[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < KC; ++j)
        if (j < k) cfmac_pp(d[j], xs[j], acc);
    } else {
      for (int j = 0; j < k; ++j) cfma_pp(acc, cs[j], ld_pair(Xr + j * ldx, i));
      if constexpr (MODE == 2) {
        fma_pp(d[0].r, acc.r, acc.r);
        fma_pp(d[0].r, acc.i, acc.i);
      }
    }
    st_pair(yr, i, acc);
  }
  if constexpr (MODE == 1) {
    double v[2 * KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      v[2 * j] = pair2d(d[j].r);
      v[2 * j + 1] = pair2d(d[j].i);
    }
    block_allreduce<double, 2 * KC>(v, red);
    if (threadIdx.x < 2 * KC) {
      const int j = threadIdx.x >> 1;
      if (j < k) part[(((long)r * k + j) * gridDim.x + blockIdx.x) * 2 + (threadIdx.x & 1)] = v[threadIdx.x];
    }
  } else if constexpr (MODE == 2) {
    double v[1] = {pair2d(d[0].r)};
    block_allreduce<double, 1>(v, red);
    if (threadIdx.x == 0) part[(long)r * gridDim.x + blockIdx.x] = v[0];
  }
}

// out[r * ostr + 2 j + {0,1}] = sum over the G partials of (r, j), fixed order
__global__ void k_preduce_b(const double* __restrict__ part, int G, int k, double* __restrict__ out, long ostr,
                            const int* __restrict__ active) {
  __shared__ double red[32 * 2];
  const int j = blockIdx.x, r = blockIdx.y;
  if (active && !active[r]) return;
  double d[2] = {0, 0};
  const double* p = part + ((long)r * k + j) * G * 2;
  for (int b = threadIdx.x; b < G; b += blockDim.x) {
    d[0] += p[2 * b];
    d[1] += p[2 * b + 1];
  }
  block_allreduce<double, 2>(d, red);
  if (threadIdx.x == 0) {
    out[r * ostr + 2 * j] = d[0];
    out[r * ostr + 2 * j + 1] = d[1];
  }
}

__global__ void k_preduce_norm_b(const double* __restrict__ part, int G, double* __restrict__ out,
                                 const int* __restrict__ active) {
  __shared__ double red[32];
  const int r = blockIdx.x;
  if (active && !active[r]) return;
  double d[1] = {0};
  for (int b = threadIdx.x; b < G; b += blockDim.x) d[0] += part[(long)r * G + b];
  block_allreduce<double, 1>(d, red);
  if (threadIdx.x == 0) out[r] = d[0];
}

// x += sum_j c_j Z_j, Z FP32 (exact in a pair), x FP64; active[r] = terms of rhs r (0: skip)
__global__ void __launch_bounds__(kPairThreads) k_plincomb_b(const float* __restrict__ Z, long zstr, long ldz, int k,
                                                             const double* __restrict__ c, long cstr,
                                                             double* __restrict__ x, long xstr, long ncx,
                                                             const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char praw[];
  cdf* cs = reinterpret_cast<cdf*>(praw);
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const int kr = active ? min(k, active[r]) : k;
  const double* cr = c + r * cstr;
  for (int j = threadIdx.x; j < kr; j += blockDim.x) cs[j] = cx2pair(cr[2 * j], cr[2 * j + 1]);
  __syncthreads();
  double* xr = x + r * xstr;
  const float* Zr = Z + r * zstr;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    cdf acc = ld_pair(xr, i);
    for (int j = 0; j < kr; ++j) {
      const float2 z = reinterpret_cast<const float2*>(Zr + j * ldz)[i];
      cfma_pf(acc, cs[j], cx<float>{z.x, z.y});
    }
    st_pair(xr, i, acc);
  }
}

size_t pair_smem(int k) { return (size_t)k * sizeof(cdf) + 32 * 2 * kChunk * sizeof(double); }
constexpr int kShort = 4;  // bases of at most 4 vectors take the 4-wide kernels

}  // namespace

void launch_pdot_b(const double* X, long xstr, long ldx, int k, const double* y, long ystr, long ncx, double* out,
                   long ostr, double* scratch, int nrhs, const int* active, cudaStream_t st) {
  const int G = pair_grid(ncx);
  if (k <= kShort)
    k_pdot_partial_b<kShort><<<dim3(G, 1, nrhs), kPairThreads, 0, st>>>(X, xstr, ldx, k, y, ystr, ncx, scratch,
                                                                        active);
  else
    k_pdot_partial_b<kChunk><<<dim3(G, (k + kChunk - 1) / kChunk, nrhs), kPairThreads, 0, st>>>(
        X, xstr, ldx, k, y, ystr, ncx, scratch, active);
  k_preduce_b<<<dim3(k, nrhs), 256, 0, st>>>(scratch, G, k, out, ostr, active);
}

int launch_pcaxpy_dot_b(const double* X, long xstr, long ldx, int k, const double* c, long cstr, double* y, long ystr,
                        long ncx, double* out, long ostr, double* scratch, int nrhs, const int* active,
                        cudaStream_t st) {
  const int G = pair_grid(ncx);
  if (k <= kShort) {
    k_pcaxpy_b<1, kShort><<<dim3(G, nrhs), kPairThreads, pair_smem(k), st>>>(X, xstr, ldx, k, c, cstr, y, ystr, ncx,
                                                                             scratch, active);
    k_preduce_b<<<dim3(k, nrhs), 256, 0, st>>>(scratch, G, k, out, ostr, active);
    return 2;
  }
  if (k <= kChunk) {
    k_pcaxpy_b<1><<<dim3(G, nrhs), kPairThreads, pair_smem(k), st>>>(X, xstr, ldx, k, c, cstr, y, ystr, ncx, scratch,
                                                                     active);
    k_preduce_b<<<dim3(k, nrhs), 256, 0, st>>>(scratch, G, k, out, ostr, active);
    return 2;
  }
  k_pcaxpy_b<0><<<dim3(G, nrhs), kPairThreads, pair_smem(k), st>>>(X, xstr, ldx, k, c, cstr, y, ystr, ncx, nullptr,
                                                                   active);
  launch_pdot_b(X, xstr, ldx, k, y, ystr, ncx, out, ostr, scratch, nrhs, active, st);
  return 3;
}

void launch_pcaxpy_norm_b(const double* X, long xstr, long ldx, int k, const double* c, long cstr, double* y,
                          long ystr, long ncx, double* nrm, double* scratch, int nrhs, const int* active,
                          cudaStream_t st) {
  const int G = pair_grid(ncx);
  k_pcaxpy_b<2><<<dim3(G, nrhs), kPairThreads, pair_smem(k), st>>>(X, xstr, ldx, k, c, cstr, y, ystr, ncx, scratch,
                                                                   active);
  k_preduce_norm_b<<<nrhs, 256, 0, st>>>(scratch, G, nrm, active);
}

void launch_plincomb_b(const float* Z, long zstr, long ldz, int k, const double* c, long cstr, double* x, long xstr,
                       long ncx, int nrhs, const int* active, cudaStream_t st) {
  k_plincomb_b<<<dim3(pair_grid(ncx), nrhs), kPairThreads, (size_t)k * sizeof(cdf), st>>>(Z, zstr, ldz, k, c, cstr,
                                                                                          x, xstr, ncx, active);
}

}  // namespace tmamg
