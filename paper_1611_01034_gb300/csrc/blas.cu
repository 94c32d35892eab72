// Level-1 vector kernels for the Krylov solvers (FGMRES on the fine level,
// GMRES on the coarsest level): casts, axpby, linear combinations, and
// inner products reduced deterministically in two stages (per-CTA partial
// sums into a scratch array, then one CTA per result in fixed order).
// Vectors are flat arrays of complex numbers stored as (re, im) pairs.  Inner
// products accumulate in the storage precision within a CTA (FP32 sums for
// FP32 fields: FP64 arithmetic is a small fraction of FP32 throughput on this
// GPU) and combine the per-CTA partial sums in FP64.
#include "tm_kernels.h"

namespace tmamg {

template <typename Ti, typename To>
__global__ void k_convert(const Ti* __restrict__ in, To* __restrict__ out, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = (To)in[i];
}

static inline int grid_for(long n, int threads = 256) {
  long b = (n + threads - 1) / threads;
  if (b > 152L * 16) b = 152L * 16;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename Ti, typename To>
void launch_convert(const Ti* in, To* out, long n_reals, cudaStream_t st) {
  k_convert<Ti, To><<<grid_for(n_reals), 256, 0, st>>>(in, out, n_reals);
}

template <typename T>
__global__ void k_zero(T* x, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) x[i] = T(0);
}
template <typename T>
void launch_zero(T* x, long n_reals, cudaStream_t st) {
  k_zero<T><<<grid_for(n_reals), 256, 0, st>>>(x, n_reals);
}

template <typename T>
__global__ void k_caxpby(cx<T> a, const T* __restrict__ x, cx<T> b, T* __restrict__ y, long ncx) {
  const cx<T>* xx = reinterpret_cast<const cx<T>*>(x);
  cx<T>* yy = reinterpret_cast<cx<T>*>(y);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x)
    yy[i] = a * xx[i] + b * yy[i];
}
template <typename T>
void launch_caxpby(double ar, double ai, const T* x, double br, double bi, T* y, long ncx, cudaStream_t st) {
  k_caxpby<T><<<grid_for(ncx), 256, 0, st>>>(cx<T>{(T)ar, (T)ai}, x, cx<T>{(T)br, (T)bi}, y, ncx);
}

// ---- multi-dot: out[j] = sum conj(X_j) y ------------------------------------
// stage 1: CTA (b, chunk) accumulates 8 dots over its slice, writes partials
template <typename T>
__global__ void k_multidot_partial(const T* __restrict__ X, long ldx, int k, const T* __restrict__ y, long ncx,
                                   double* __restrict__ part) {
  __shared__ T red[32 * 16];
  const int j0 = blockIdx.y * 8;
  T d[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) d[m] = 0;
  const cx<T>* yy = reinterpret_cast<const cx<T>*>(y);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    const cx<T> yv = yy[i];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      if (j0 + jj < k) {
        const cx<T> xv = reinterpret_cast<const cx<T>*>(X + (long)(j0 + jj) * ldx)[i];
        // conj(x) y as four fused multiply-adds (FP64 arithmetic is the limit on GB300)
        d[2 * jj] = fma(xv.r, yv.r, d[2 * jj]);
        d[2 * jj] = fma(xv.i, yv.i, d[2 * jj]);
        d[2 * jj + 1] = fma(xv.r, yv.i, d[2 * jj + 1]);
        d[2 * jj + 1] = fma(-xv.i, yv.r, d[2 * jj + 1]);
      }
    }
  }
  __shared__ T fin[16];
  block_reduce16<T>(d, red, fin);
  if (threadIdx.x < 16) {
    const int jj = threadIdx.x >> 1;
    if (j0 + jj < k) part[((long)(j0 + jj) * gridDim.x + blockIdx.x) * 2 + (threadIdx.x & 1)] = (double)fin[threadIdx.x];
  }
}

// stage 2: one CTA per result sums the partials in fixed order
__global__ void k_reduce_partials(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  __shared__ double red[32 * 2];
  const int j = blockIdx.x;
  double d[2] = {0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    d[0] += part[((long)j * nblocks + b) * 2];
    d[1] += part[((long)j * nblocks + b) * 2 + 1];
  }
  block_allreduce<double, 2>(d, red);
  if (threadIdx.x == 0) {
    out[2 * j] = d[0];
    out[2 * j + 1] = d[1];
  }
}

template <typename T>
void launch_multidot(const T* X, long ldx, int k, const T* y, long ncx, double* dev_out, double* scratch,
                     int nscratch_blocks, cudaStream_t st) {
  int G = grid_for(ncx);
  if (G > nscratch_blocks) G = nscratch_blocks;
  dim3 grid(G, (k + 7) / 8);
  k_multidot_partial<T><<<grid, 256, 0, st>>>(X, ldx, k, y, ncx, scratch);
  k_reduce_partials<<<k, 256, 0, st>>>(scratch, G, dev_out);
}

// ---- norms of nrhs vectors ----------------------------------------------------
template <typename T>
__global__ void k_norm2_partial(const T* __restrict__ x, long ncx, double* __restrict__ part) {
  __shared__ T red[32 * 2];
  const int r = blockIdx.y;
  const cx<T>* xx = reinterpret_cast<const cx<T>*>(x) + (long)r * ncx;
  T d[2] = {0, 0};
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    const cx<T> v = xx[i];
    d[0] = fma(v.r, v.r, d[0]);
    d[0] = fma(v.i, v.i, d[0]);
  }
  block_allreduce<T, 2>(d, red);
  if (threadIdx.x < 2) part[((long)r * gridDim.x + blockIdx.x) * 2 + threadIdx.x] = (double)d[threadIdx.x];
}

__global__ void k_reduce_norm(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  __shared__ double red[32];
  const int r = blockIdx.x;
  double d[1] = {0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) d[0] += part[((long)r * nblocks + b) * 2];
  block_allreduce<double, 1>(d, red);
  if (threadIdx.x == 0) out[r] = d[0];
}

template <typename T>
void launch_norm2(const T* x, long ncx, int nrhs, double* dev_out, double* scratch, int nscratch_blocks,
                  cudaStream_t st) {
  int G = grid_for(ncx);
  if (G * nrhs > nscratch_blocks) G = nscratch_blocks / nrhs;
  if (G < 1) G = 1;
  dim3 grid(G, nrhs);
  k_norm2_partial<T><<<grid, 256, 0, st>>>(x, ncx, scratch);
  k_reduce_norm<<<nrhs, 256, 0, st>>>(scratch, G, dev_out);
}

// ---- y -= sign * sum_j c_j X_j  (c device double2) ------------------------------
template <typename T>
__global__ void k_multi_caxpy(const T* __restrict__ X, long ldx, int k, const double* __restrict__ c, T sign,
                              T* __restrict__ y, long ncx) {
  __shared__ cx<T> cs_[128];  // -sign c_j, formed once per CTA
  for (int j = threadIdx.x; j < k; j += blockDim.x) cs_[j] = cx<T>{-sign * (T)c[2 * j], -sign * (T)c[2 * j + 1]};
  __syncthreads();
  cx<T>* yy = reinterpret_cast<cx<T>*>(y);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    cx<T> acc = yy[i];
    for (int j = 0; j < k; ++j) {
      const cx<T> xv = reinterpret_cast<const cx<T>*>(X + (long)j * ldx)[i];
      cfma(acc, cs_[j], xv);
    }
    yy[i] = acc;
  }
}
template <typename T>
void launch_multi_caxpy(const T* X, long ldx, int k, const double* c, double sign, T* y, long ncx,
                        cudaStream_t st) {
  k_multi_caxpy<T><<<grid_for(ncx), 256, 0, st>>>(X, ldx, k, c, (T)sign, y, ncx);
}

// ---- y += sum_j c_j X_j, mixed precision ------------------------------------------
template <typename Tx, typename Ty>
__global__ void k_lincomb(const Tx* __restrict__ X, long ldx, int k, const double* __restrict__ c,
                          Ty* __restrict__ y, long ncx) {
  cx<Ty>* yy = reinterpret_cast<cx<Ty>*>(y);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    cx<Ty> acc = yy[i];
    for (int j = 0; j < k; ++j) {
      const cx<Tx> xv = reinterpret_cast<const cx<Tx>*>(X + (long)j * ldx)[i];
      const cx<Ty> cj{(Ty)c[2 * j], (Ty)c[2 * j + 1]};
      cfma(acc, cj, cx<Ty>{(Ty)xv.r, (Ty)xv.i});
    }
    yy[i] = acc;
  }
}
template <typename Tx, typename Ty>
void launch_lincomb(const Tx* X, long ldx, int k, const double* c, Ty* y, long ncx, cudaStream_t st) {
  k_lincomb<Tx, Ty><<<grid_for(ncx), 256, 0, st>>>(X, ldx, k, c, y, ncx);
}

// ---- x_r *= s_r --------------------------------------------------------------------
template <typename T>
__global__ void k_scale(T* __restrict__ x, long ncx, const double* __restrict__ s, int inv_sqrt) {
  const int r = blockIdx.y;
  double sc = s[r];
  if (inv_sqrt) sc = sc > 0 ? 1.0 / sqrt(sc) : 0.0;
  const T f = (T)sc;
  T* xx = x + (long)r * 2 * ncx;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * ncx; i += (long)gridDim.x * blockDim.x)
    xx[i] *= f;
}
template <typename T>
void launch_scale(T* x, long ncx, int nrhs, const double* s, bool inv_sqrt, cudaStream_t st) {
  dim3 grid(grid_for(2 * ncx), nrhs);
  k_scale<T><<<grid, 256, 0, st>>>(x, ncx, s, inv_sqrt ? 1 : 0);
}

// ===========================================================================
// batched variants over right-hand sides (blockIdx.y or .z = rhs); each rhs
// uses the same grid decomposition as the single-rhs kernels above, so the
// per-rhs arithmetic is the same; masked (finished) right-hand sides skip.
// ===========================================================================
static inline int dot_grid(long ncx) {
  int G = grid_for(ncx);
  return G > kReduceBlocks ? kReduceBlocks : G;
}

long multidot_scratch_doubles(long ncx, int k, int nrhs) { return 2L * dot_grid(ncx) * k * nrhs; }
int dot_grid_for(long ncx) { return dot_grid(ncx); }

template <typename T>
__global__ void k_multidot_partial_b(const T* __restrict__ X, long xstr, long ldx, int k, const T* __restrict__ y,
                                     long ystr, long ncx, double* __restrict__ part, const int* __restrict__ active) {
  __shared__ T red[32 * 16];
  const int r = blockIdx.z;
  if (active && !active[r]) return;
  const int j0 = blockIdx.y * 8;
  T d[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) d[m] = 0;
  const cx<T>* yy = reinterpret_cast<const cx<T>*>(y + r * ystr);
  const T* Xr = X + r * xstr;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    const cx<T> yv = yy[i];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      if (j0 + jj < k) {
        const cx<T> xv = reinterpret_cast<const cx<T>*>(Xr + (long)(j0 + jj) * ldx)[i];
        // conj(x) y as four fused multiply-adds (FP64 arithmetic is the limit on GB300)
        d[2 * jj] = fma(xv.r, yv.r, d[2 * jj]);
        d[2 * jj] = fma(xv.i, yv.i, d[2 * jj]);
        d[2 * jj + 1] = fma(xv.r, yv.i, d[2 * jj + 1]);
        d[2 * jj + 1] = fma(-xv.i, yv.r, d[2 * jj + 1]);
      }
    }
  }
  __shared__ T fin[16];
  block_reduce16<T>(d, red, fin);
  if (threadIdx.x < 16) {
    const int jj = threadIdx.x >> 1;
    if (j0 + jj < k)
      part[(((long)r * k + j0 + jj) * gridDim.x + blockIdx.x) * 2 + (threadIdx.x & 1)] = (double)fin[threadIdx.x];
  }
}

__global__ void k_reduce_partials_b(const double* __restrict__ part, int nblocks, int k, double* __restrict__ out,
                                    long ostr, const int* __restrict__ active) {
  __shared__ double red[32 * 2];
  const int j = blockIdx.x, r = blockIdx.y;
  if (active && !active[r]) return;
  double d[2] = {0, 0};
  const double* p = part + ((long)r * k + j) * nblocks * 2;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    d[0] += p[2 * b];
    d[1] += p[2 * b + 1];
  }
  block_allreduce<double, 2>(d, red);
  if (threadIdx.x == 0) {
    out[r * ostr + 2 * j] = d[0];
    out[r * ostr + 2 * j + 1] = d[1];
  }
}

template <typename T>
void launch_multidot_b(const T* X, long xstr, long ldx, int k, const T* y, long ystr, long ncx, double* out, long ostr,
                       double* scratch, int nrhs, const int* active, cudaStream_t st) {
  const int G = dot_grid(ncx);
  dim3 grid(G, (k + 7) / 8, nrhs);
  k_multidot_partial_b<T><<<grid, 256, 0, st>>>(X, xstr, ldx, k, y, ystr, ncx, scratch, active);
  dim3 g2(k, nrhs);
  k_reduce_partials_b<<<g2, 256, 0, st>>>(scratch, G, k, out, ostr, active);
}

template <typename T>
__global__ void k_norm2_partial_b(const T* __restrict__ y, long ystr, long ncx, double* __restrict__ part,
                                  const int* __restrict__ active) {
  __shared__ T red[32 * 2];
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const cx<T>* yy = reinterpret_cast<const cx<T>*>(y + r * ystr);
  T d[2] = {0, 0};
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    const cx<T> v = yy[i];
    d[0] = fma(v.r, v.r, d[0]);
    d[0] = fma(v.i, v.i, d[0]);
  }
  block_allreduce<T, 2>(d, red);
  if (threadIdx.x < 2) part[((long)r * gridDim.x + blockIdx.x) * 2 + threadIdx.x] = (double)d[threadIdx.x];
}

__global__ void k_reduce_norm_b(const double* __restrict__ part, int nblocks, double* __restrict__ out,
                                const int* __restrict__ active) {
  __shared__ double red[32];
  const int r = blockIdx.x;
  if (active && !active[r]) return;
  double d[1] = {0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) d[0] += part[((long)r * nblocks + b) * 2];
  block_allreduce<double, 1>(d, red);
  if (threadIdx.x == 0) out[r] = d[0];
}

template <typename T>
void launch_norm2_b(const T* y, long ystr, long ncx, double* out, double* scratch, int nrhs, const int* active,
                    cudaStream_t st) {
  const int G = dot_grid(ncx);
  dim3 grid(G, nrhs);
  k_norm2_partial_b<T><<<grid, 256, 0, st>>>(y, ystr, ncx, scratch, active);
  k_reduce_norm_b<<<nrhs, 256, 0, st>>>(scratch, G, out, active);
}

template <typename T>
__global__ void k_multi_caxpy_b(const T* __restrict__ X, long xstr, long ldx, int k, const double* __restrict__ c,
                                long cstr, T* __restrict__ y, long ystr, long ncx, const int* __restrict__ active) {
  __shared__ cx<T> cs_[128];  // -c_j, formed once per CTA
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const double* cr = c + r * cstr;
  for (int j = threadIdx.x; j < k; j += blockDim.x) cs_[j] = cx<T>{-(T)cr[2 * j], -(T)cr[2 * j + 1]};
  __syncthreads();
  cx<T>* yy = reinterpret_cast<cx<T>*>(y + r * ystr);
  const T* Xr = X + r * xstr;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    cx<T> acc = yy[i];
    for (int j = 0; j < k; ++j) cfma(acc, cs_[j], reinterpret_cast<const cx<T>*>(Xr + (long)j * ldx)[i]);
    yy[i] = acc;
  }
}
template <typename T>
void launch_multi_caxpy_b(const T* X, long xstr, long ldx, int k, const double* c, long cstr, T* y, long ystr, long ncx,
                          int nrhs, const int* active, cudaStream_t st) {
  dim3 grid(grid_for(ncx), nrhs);
  k_multi_caxpy_b<T><<<grid, 256, 0, st>>>(X, xstr, ldx, k, c, cstr, y, ystr, ncx, active);
}

template <typename Tx, typename Ty>
__global__ void k_lincomb_b(const Tx* __restrict__ X, long xstr, long ldx, int k, const double* __restrict__ c,
                            long cstr, Ty* __restrict__ y, long ystr, long ncx, const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  if (active) k = min(k, active[r]);  // active[r] = number of terms for rhs r
  cx<Ty>* yy = reinterpret_cast<cx<Ty>*>(y + r * ystr);
  const Tx* Xr = X + r * xstr;
  const double* cr = c + r * cstr;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    cx<Ty> acc = yy[i];
    for (int j = 0; j < k; ++j) {
      const cx<Ty> cj{(Ty)cr[2 * j], (Ty)cr[2 * j + 1]};
      const cx<Tx> xv = reinterpret_cast<const cx<Tx>*>(Xr + (long)j * ldx)[i];
      cfma(acc, cj, cx<Ty>{(Ty)xv.r, (Ty)xv.i});
    }
    yy[i] = acc;
  }
}
template <typename Tx, typename Ty>
void launch_lincomb_b(const Tx* X, long xstr, long ldx, int k, const double* c, long cstr, Ty* y, long ystr,
                      long ncx, int nrhs, const int* active, cudaStream_t st) {
  dim3 grid(grid_for(ncx), nrhs);
  k_lincomb_b<Tx, Ty><<<grid, 256, 0, st>>>(X, xstr, ldx, k, c, cstr, y, ystr, ncx, active);
}

template <typename T>
__global__ void k_scale_copy_b(const T* __restrict__ src, long sstr, T* __restrict__ dst, long dstr,
                               const double* __restrict__ s, long ncx, const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  T f = T(1);
  if (s) {
    const double sc = s[r];
    f = (T)(sc > 0 ? 1.0 / sqrt(sc) : 0.0);
  }
  const T* a = src + r * sstr;
  T* b = dst + r * dstr;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * ncx; i += (long)gridDim.x * blockDim.x)
    b[i] = s ? a[i] * f : a[i];
}
template <typename T>
void launch_scale_copy_b(const T* src, long sstr, T* dst, long dstr, const double* s, long ncx, int nrhs,
                         const int* active, cudaStream_t st) {
  dim3 grid(grid_for(2 * ncx), nrhs);
  k_scale_copy_b<T><<<grid, 256, 0, st>>>(src, sstr, dst, dstr, s, ncx, active);
}

// --- the same steps taking the per-block partial sums of the preceding
// reduction directly (one launch less each): every CTA sums the partials in
// the same fixed order, CTA 0 also stores the result for the host.  Few
// partial blocks (kFusedParts) and few consumer CTAs per rhs (kFusedCtas) keep
// the redundant partial reads small. ---------------------------------------------
constexpr int kFusedParts = 16, kFusedCtas = 64;
static inline int fused_parts(long ncx) {
  const int G = dot_grid(ncx);
  return G < kFusedParts ? G : kFusedParts;
}
static inline int fused_ctas(long n) {
  const int G = grid_for(n);
  return G < kFusedCtas ? G : kFusedCtas;
}

template <typename T>
void launch_multidot_b_partials(const T* X, long xstr, long ldx, int k, const T* y, long ystr, long ncx,
                                double* scratch, int nrhs, const int* active, cudaStream_t st) {
  dim3 grid(fused_parts(ncx), (k + 7) / 8, nrhs);
  k_multidot_partial_b<T><<<grid, 256, 0, st>>>(X, xstr, ldx, k, y, ystr, ncx, scratch, active);
}

template <typename T>
__global__ void k_multi_caxpy_bp(const T* __restrict__ X, long xstr, long ldx, int k, const double* __restrict__ part,
                                 int G, double* __restrict__ cout_, long cstr, T* __restrict__ y, long ystr, long ncx,
                                 const int* __restrict__ active) {
  extern __shared__ double cs_[];  // [k][2]
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double* p = part + ((long)r * k + j) * G * 2;
    double a = 0, b = 0;
    for (int q = 0; q < G; ++q) {
      a += p[2 * q];
      b += p[2 * q + 1];
    }
    cs_[2 * j] = a;
    cs_[2 * j + 1] = b;
    if (blockIdx.x == 0) {
      cout_[r * cstr + 2 * j] = a;
      cout_[r * cstr + 2 * j + 1] = b;
    }
  }
  __syncthreads();
  cx<T>* yy = reinterpret_cast<cx<T>*>(y + r * ystr);
  const T* Xr = X + r * xstr;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    cx<T> acc = yy[i];
    for (int j = 0; j < k; ++j) {
      const cx<T> cj{(T)cs_[2 * j], (T)cs_[2 * j + 1]};
      cfma(acc, -cj, reinterpret_cast<const cx<T>*>(Xr + (long)j * ldx)[i]);
    }
    yy[i] = acc;
  }
}
template <typename T>
void launch_multi_caxpy_bp(const T* X, long xstr, long ldx, int k, const double* part, long ncx_dot, double* c,
                           long cstr, T* y, long ystr, long ncx, int nrhs, const int* active, cudaStream_t st) {
  dim3 grid(fused_ctas(ncx), nrhs);
  k_multi_caxpy_bp<T><<<grid, 256, (size_t)2 * k * sizeof(double), st>>>(X, xstr, ldx, k, part, fused_parts(ncx_dot),
                                                                        c, cstr, y, ystr, ncx, active);
}

template <typename T>
void launch_norm2_b_partials(const T* y, long ystr, long ncx, double* scratch, int nrhs, const int* active,
                             cudaStream_t st) {
  dim3 grid(fused_parts(ncx), nrhs);
  k_norm2_partial_b<T><<<grid, 256, 0, st>>>(y, ystr, ncx, scratch, active);
}

template <typename T>
__global__ void k_scale_copy_bp(const T* __restrict__ src, long sstr, T* __restrict__ dst, long dstr,
                                const double* __restrict__ part, int G, double* __restrict__ nrm, long ncx,
                                const int* __restrict__ active) {
  __shared__ double sc_;
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  if (threadIdx.x == 0) {
    double a = 0;
    for (int q = 0; q < G; ++q) a += part[((long)r * G + q) * 2];
    sc_ = a;
    if (blockIdx.x == 0) nrm[r] = a;
  }
  __syncthreads();
  const double sc = sc_;
  const T f = (T)(sc > 0 ? 1.0 / sqrt(sc) : 0.0);
  const T* a = src + r * sstr;
  T* b = dst + r * dstr;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * ncx; i += (long)gridDim.x * blockDim.x)
    b[i] = a[i] * f;
}
template <typename T>
void launch_scale_copy_bp(const T* src, long sstr, T* dst, long dstr, const double* part, double* nrm, long ncx,
                          int nrhs, const int* active, cudaStream_t st) {
  dim3 grid(fused_ctas(2 * ncx), nrhs);
  k_scale_copy_bp<T><<<grid, 256, 0, st>>>(src, sstr, dst, dstr, part, fused_parts(ncx), nrm, ncx, active);
}

template <typename T>
__global__ void k_sub_b(const T* __restrict__ x, long xstr, T* __restrict__ y, long ystr, long ncx,
                        const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const T* a = x + r * xstr;
  T* b = y + r * ystr;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * ncx; i += (long)gridDim.x * blockDim.x)
    b[i] = a[i] - b[i];
}
template <typename T>
void launch_sub_b(const T* x, long xstr, T* y, long ystr, long ncx, int nrhs, const int* active, cudaStream_t st) {
  dim3 grid(grid_for(2 * ncx), nrhs);
  k_sub_b<T><<<grid, 256, 0, st>>>(x, xstr, y, ystr, ncx, active);
}

#define TM_INST_BP(T)                                                                                        \
  template void launch_multidot_b_partials<T>(const T*, long, long, int, const T*, long, long, double*, int,    \
                                              const int*, cudaStream_t);                                       \
  template void launch_multi_caxpy_bp<T>(const T*, long, long, int, const double*, long, double*, long, T*,     \
                                         long, long, int, const int*, cudaStream_t);                           \
  template void launch_norm2_b_partials<T>(const T*, long, long, double*, int, const int*, cudaStream_t);       \
  template void launch_scale_copy_bp<T>(const T*, long, T*, long, const double*, double*, long, int,            \
                                        const int*, cudaStream_t);
TM_INST_BP(double)
TM_INST_BP(float)
#undef TM_INST_BP

#define TM_INST_B(T)                                                                                              \
  template void launch_multidot_b<T>(const T*, long, long, int, const T*, long, long, double*, long, double*, int, \
                                     const int*, cudaStream_t);                                                   \
  template void launch_multi_caxpy_b<T>(const T*, long, long, int, const double*, long, T*, long, long, int,      \
                                        const int*, cudaStream_t);                                                \
  template void launch_norm2_b<T>(const T*, long, long, double*, double*, int, const int*, cudaStream_t);         \
  template void launch_scale_copy_b<T>(const T*, long, T*, long, const double*, long, int, const int*,            \
                                       cudaStream_t);                                                             \
  template void launch_sub_b<T>(const T*, long, T*, long, long, int, const int*, cudaStream_t);
TM_INST_B(double)
TM_INST_B(float)
#undef TM_INST_B
template void launch_lincomb_b<double, double>(const double*, long, long, int, const double*, long, double*, long,
                                               long, int, const int*, cudaStream_t);
template void launch_lincomb_b<float, float>(const float*, long, long, int, const double*, long, float*, long, long,
                                             int, const int*, cudaStream_t);
template void launch_lincomb_b<float, double>(const float*, long, long, int, const double*, long, double*, long,
                                              long, int, const int*, cudaStream_t);

#define TM_INST(T)                                                                                    \
  template void launch_zero<T>(T*, long, cudaStream_t);                                               \
  template void launch_caxpby<T>(double, double, const T*, double, double, T*, long, cudaStream_t);   \
  template void launch_multidot<T>(const T*, long, int, const T*, long, double*, double*, int,        \
                                   cudaStream_t);                                                     \
  template void launch_multi_caxpy<T>(const T*, long, int, const double*, double, T*, long, cudaStream_t); \
  template void launch_norm2<T>(const T*, long, int, double*, double*, int, cudaStream_t);            \
  template void launch_scale<T>(T*, long, int, const double*, bool, cudaStream_t);
TM_INST(double)
TM_INST(float)
#undef TM_INST
template void launch_convert<double, float>(const double*, float*, long, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, long, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, long, cudaStream_t);
template void launch_convert<float, float>(const float*, float*, long, cudaStream_t);
template void launch_lincomb<double, double>(const double*, long, int, const double*, double*, long, cudaStream_t);
template void launch_lincomb<float, double>(const float*, long, int, const double*, double*, long, cudaStream_t);
template void launch_lincomb<float, float>(const float*, long, int, const double*, float*, long, cudaStream_t);

}  // namespace tmamg
