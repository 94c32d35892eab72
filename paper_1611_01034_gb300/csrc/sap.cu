// SAP smoother M of eq. (1): red/black multiplicative Schwarz with
// block-local minimal-residual solves (Sec. 1 of the paper: the smoother is
// the Schwarz Alternating Procedure and damps the UV modes).
//
// One launch processes every block of one colour.  One CTA owns one block,
// one thread one site.  The CTA
//   1. forms r = b - D x on its block with the full operator (neighbours in
//      the other colour are read from global memory; blocks of one colour are
//      never adjacent, so no CTA reads sites another CTA writes);
//   2. keeps r in shared memory and runs n_MR steps of
//        q = D_B r;  alpha = <q, r> / <q, q>;  e += alpha r;  r -= alpha q
//      with the Dirichlet block operator D_B (hops leaving the block are
//      dropped), the two inner products reduced by warp shuffles;
//   3. adds e to x.
// Block colour = parity of the sum of block coordinates; every dimension has
// an even number (>= 2) of blocks, so no block touches itself or a block of
// its own colour.
#include "tm_kernels.h"
#include "tm_stencil.cuh"

namespace tmamg {

template <typename T>
struct SapArgs {
  const T* gauge;
  const T* clover;
  const T* b;
  T* x;
  SapGeom sg;
  T mu;
  T bc;
  int n_mr;
  int colour;
  int nrhs;
};

template <typename T, int MU>
__device__ __forceinline__ void block_hops(const cx<T>* __restrict__ rs, int BS, int l, const int lc[4],
                                           const int lst[4], const T* __restrict__ gauge, const Lat& g, int s,
                                           const int c[4], const int blk[4], cx<T> (&acc)[12]) {
  if (lc[MU] < blk[MU] - 1) {
    cx<T> p[12];
    const int ln = l + lst[MU];
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = rs[k * BS + ln];
    hop_fwd_p<T, MU>(p, gauge, g.V, s, T(1), acc);
  }
  if (lc[MU] > 0) {
    cx<T> p[12];
    const int ln = l - lst[MU];
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = rs[k * BS + ln];
    hop_bwd_p<T, MU>(p, gauge, g.V, nb_bwd(g, s, c, MU), T(1), acc);
  }
}

// FP32: two CTAs per SM (128 registers); FP64 would spill heavily at that bound
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_sap(SapArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SapGeom& sg = a.sg;
  const Lat& g = sg.g;
  const int BS = sg.bsites;
  cx<T>* rs = reinterpret_cast<cx<T>*>(smem_raw);  // [12][BS]
  T* red = reinterpret_cast<T*>(rs + 12 * BS);     // [32 * 3]
  // consecutive CTAs take the same block for consecutive right-hand sides, so
  // the block's links and clover are read from DRAM once and then from L2
  const int rhs = blockIdx.x % a.nrhs;
  const long off = (long)rhs * NR_SPINOR * g.V;
  T* x = a.x + off;

  // the (blockIdx.x / nrhs)-th block of this colour
  int k = blockIdx.x / a.nrhs;
  const int nbxh = sg.nb[3] / 2;
  int bc4[4];
  const int bxh = k % nbxh;
  k /= nbxh;
  bc4[2] = k % sg.nb[2];
  k /= sg.nb[2];
  bc4[1] = k % sg.nb[1];
  bc4[0] = k / sg.nb[1];
  bc4[3] = 2 * bxh + ((bc4[0] + bc4[1] + bc4[2] + a.colour) & 1);

  const int l = threadIdx.x;
  const bool act = l < BS;
  int lc[4], c[4], lst[4];
  lst[3] = 1;
  lst[2] = sg.blk[3];
  lst[1] = sg.blk[3] * sg.blk[2];
  lst[0] = lst[1] * sg.blk[1];
  int s = 0;
  {
    int q = act ? l : 0;
    lc[3] = q % sg.blk[3];
    q /= sg.blk[3];
    lc[2] = q % sg.blk[2];
    q /= sg.blk[2];
    lc[1] = q % sg.blk[1];
    lc[0] = q / sg.blk[1];
#pragma unroll
    for (int d = 0; d < 4; ++d) c[d] = bc4[d] * sg.blk[d] + lc[d];
    s = ((c[0] * g.L[1] + c[1]) * g.L[2] + c[2]) * g.L[3] + c[3];
  }

  cx<T> r[12], e[12];
  const T half = T(0.5);
  if (act) {
    cx<T> acc[12], p[12];
    all_hops_global<T>(x, a.gauge, g, s, c, a.bc, acc);
    ld_cx<T, 12>(x, g.V, s, p);
    site_diag<T>(a.clover, g.V, s, a.mu, p, r);
#pragma unroll
    for (int i = 0; i < 12; ++i) r[i] = half * acc[i] - r[i];  // -D x
    if (a.b) {
      cx<T> bb[12];
      ld_cx<T, 12>(a.b + off, g.V, s, bb);
#pragma unroll
      for (int i = 0; i < 12; ++i) r[i] = r[i] + bb[i];
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) rs[i * BS + l] = r[i];
  }
#pragma unroll
  for (int i = 0; i < 12; ++i) e[i] = cx<T>{0, 0};

  for (int it = 0; it < a.n_mr; ++it) {
    __syncthreads();
    cx<T> q[12];
    T dots[3] = {0, 0, 0};
    if (act) {
      cx<T> acc[12];
#pragma unroll
      for (int i = 0; i < 12; ++i) acc[i] = cx<T>{0, 0};
      block_hops<T, 0>(rs, BS, l, lc, lst, a.gauge, g, s, c, sg.blk, acc);
      block_hops<T, 1>(rs, BS, l, lc, lst, a.gauge, g, s, c, sg.blk, acc);
      block_hops<T, 2>(rs, BS, l, lc, lst, a.gauge, g, s, c, sg.blk, acc);
      block_hops<T, 3>(rs, BS, l, lc, lst, a.gauge, g, s, c, sg.blk, acc);
      site_diag<T>(a.clover, g.V, s, a.mu, r, q);
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        q[i] = q[i] - half * acc[i];
        dots[0] = fma(q[i].r, r[i].r, fma(q[i].i, r[i].i, dots[0]));   // Re <q, r>
        dots[1] = fma(q[i].r, r[i].i, fma(-q[i].i, r[i].r, dots[1]));  // Im <q, r>
        dots[2] = fma(q[i].r, q[i].r, fma(q[i].i, q[i].i, dots[2]));   // <q, q>
      }
    }
    block_allreduce<T, 3>(dots, red);
    const cx<T> alpha = dots[2] > T(0) ? cx<T>{dots[0] / dots[2], dots[1] / dots[2]} : cx<T>{0, 0};
    if (act) {
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        cfma(e[i], alpha, r[i]);
        cfma(r[i], -alpha, q[i]);
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int i = 0; i < 12; ++i) rs[i * BS + l] = r[i];
    }
  }
  __syncthreads();
  if (act) {
    cx<T> p[12];
    ld_cx<T, 12>(x, g.V, s, p);
#pragma unroll
    for (int i = 0; i < 12; ++i) p[i] = p[i] + e[i];
    st_cx<T, 12>(x, g.V, s, p);
  }
}

template <typename T>
void launch_sap_colour(const T* gauge, const T* clover, const T* b, T* x, const SapGeom& sg, double mu,
                       double bc_t, int n_mr, int colour, int nrhs, cudaStream_t st) {
  const int threads = (sg.bsites + 31) / 32 * 32;
  const size_t smem = 12 * sg.bsites * sizeof(cx<T>) + 32 * 3 * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_sap<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  const int nblk_colour = sg.nb[0] * sg.nb[1] * sg.nb[2] * sg.nb[3] / 2;
  SapArgs<T> a{gauge, clover, b, x, sg, (T)mu, (T)bc_t, n_mr, colour, nrhs};
  dim3 grid(nblk_colour * nrhs);
  k_sap<T><<<grid, threads, smem, st>>>(a);
}

template void launch_sap_colour<double>(const double*, const double*, const double*, double*, const SapGeom&,
                                        double, double, int, int, int, cudaStream_t);
template void launch_sap_colour<float>(const float*, const float*, const float*, float*, const SapGeom&, double,
                                       double, int, int, int, cudaStream_t);

}  // namespace tmamg
