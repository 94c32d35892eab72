// Level-1 vector kernels for the Krylov solvers (FGMRES on the fine level,
// GMRES on the coarsest level): casts, axpby, linear combinations, and
// inner products reduced deterministically in two stages (per-CTA partial
// sums into a scratch array, then one CTA per result in fixed order).
// Vectors are flat arrays of complex numbers stored as (re, im) pairs; the
// inner products accumulate in FP64 whatever the storage precision.
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
  __shared__ double red[32 * 16];
  const int j0 = blockIdx.y * 8;
  double d[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) d[m] = 0;
  const cx<T>* yy = reinterpret_cast<const cx<T>*>(y);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    const cx<T> yv = yy[i];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      if (j0 + jj < k) {
        const cx<T> xv = reinterpret_cast<const cx<T>*>(X + (long)(j0 + jj) * ldx)[i];
        d[2 * jj] += (double)xv.r * yv.r + (double)xv.i * yv.i;
        d[2 * jj + 1] += (double)xv.r * yv.i - (double)xv.i * yv.r;
      }
    }
  }
  block_allreduce<double, 16>(d, red);
  if (threadIdx.x < 16) {
    const int jj = threadIdx.x >> 1;
    if (j0 + jj < k) part[((long)(j0 + jj) * gridDim.x + blockIdx.x) * 2 + (threadIdx.x & 1)] = d[threadIdx.x];
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
  __shared__ double red[32 * 2];
  const int r = blockIdx.y;
  const cx<T>* xx = reinterpret_cast<const cx<T>*>(x) + (long)r * ncx;
  double d[2] = {0, 0};
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    const cx<T> v = xx[i];
    d[0] += (double)v.r * v.r + (double)v.i * v.i;
  }
  block_allreduce<double, 2>(d, red);
  if (threadIdx.x < 2) part[((long)r * gridDim.x + blockIdx.x) * 2 + threadIdx.x] = d[threadIdx.x];
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
  cx<T>* yy = reinterpret_cast<cx<T>*>(y);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < ncx; i += (long)gridDim.x * blockDim.x) {
    cx<T> acc = yy[i];
    for (int j = 0; j < k; ++j) {
      const cx<T> cj{(T)(sign * (T)c[2 * j]), (T)(sign * (T)c[2 * j + 1])};
      const cx<T> xv = reinterpret_cast<const cx<T>*>(X + (long)j * ldx)[i];
      acc = acc - cj * xv;
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
