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
#include <type_traits>

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
  T rho;  // odd sites carry mu + rho
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
  const T mus = ((c[0] + c[1] + c[2] + c[3]) & 1) ? a.mu + a.rho : a.mu;
  if (act) {
    cx<T> acc[12], p[12];
    all_hops_global<T>(x, a.gauge, g, s, c, a.bc, acc);
    ld_cx<T, 12>(x, g.V, s, p);
    site_diag<T>(a.clover, g.V, s, mus, p, r);
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
      site_diag<T>(a.clover, g.V, s, mus, r, q);
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
                       double bc_t, int n_mr, int colour, int nrhs, cudaStream_t st, double rho) {
  const int threads = (sg.bsites + 31) / 32 * 32;
  const size_t smem = 12 * sg.bsites * sizeof(cx<T>) + 32 * 3 * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_sap<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  const int nblk_colour = sg.nb[0] * sg.nb[1] * sg.nb[2] * sg.nb[3] / 2;
  SapArgs<T> a{gauge, clover, b, x, sg, (T)mu, (T)bc_t, n_mr, colour, nrhs, (T)rho};
  dim3 grid(nblk_colour * nrhs);
  k_sap<T><<<grid, threads, smem, st>>>(a);
}

template void launch_sap_colour<double>(const double*, const double*, const double*, double*, const SapGeom&,
                                        double, double, int, int, int, cudaStream_t, double);
template void launch_sap_colour<float>(const float*, const float*, const float*, float*, const SapGeom&, double,
                                       double, int, int, int, cudaStream_t, double);

// ===========================================================================
// Odd-even block solve (Sec. 3: odd-even preconditioning is used in the
// smoother).  Within a block B (all dims even, origin on an even site, so the
// site parity (t+z+y+x) mod 2 splits it into two halves of BS/2 sites),
//   D_B = [[D_ee, D_eo], [D_oe, D_oo]],
// D_ee, D_oo the site-diagonal A(x) + i mu gamma5, D_eo, D_oe the Dirichlet
// intra-block hops.  The MR steps run on the Schur complement
//   S = D_ee - D_eo D_oo^-1 D_oe  over the even sites,
// with right-hand side r_e - D_eo D_oo^-1 r_o; afterwards
//   e_o = D_oo^-1 (r_o - D_oe e_e).
// One CTA owns one block and one right-hand side; thread j owns the j-th even
// and the j-th odd site (same t, z, y; x = 2 j_x + parity offset), so no lane
// idles in either half-step.  D_oo^-1 comes precomputed per odd site
// (launch_clover_inverse).
// ===========================================================================
namespace {

// index of a site within its parity class, from block-local coordinates
__device__ __forceinline__ int half_index(const int lc[4], const int blk[4]) {
  return ((lc[0] * blk[1] + lc[1]) * blk[2] + lc[2]) * (blk[3] / 2) + (lc[3] >> 1);
}

// acc += hops (Dirichlet, without the -1/2) from the neighbours of a site inside
// the block, whose values of the other parity are in shared memory src [12][HB]
template <typename T, int S>
__device__ __forceinline__ void oe_block_hops(const cx<T>* __restrict__ src, int HB, const int lc[4],
                                              const int blk[4], const void* __restrict__ gauge, const Lat& g, int s,
                                              const int c[4], cx<T> (&acc)[12]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cx<T>{0, 0};
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    if (lc[mu] < blk[mu] - 1) {
      int ln[4] = {lc[0], lc[1], lc[2], lc[3]};
      ln[mu] += 1;
      const int j = half_index(ln, blk);
      cx<T> p[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) p[k] = src[k * HB + j];
      switch (mu) {
        case 0: hop_fwd_p<T, 0, S>(p, gauge, g.V, s, T(1), acc); break;
        case 1: hop_fwd_p<T, 1, S>(p, gauge, g.V, s, T(1), acc); break;
        case 2: hop_fwd_p<T, 2, S>(p, gauge, g.V, s, T(1), acc); break;
        default: hop_fwd_p<T, 3, S>(p, gauge, g.V, s, T(1), acc); break;
      }
    }
    if (lc[mu] > 0) {
      int ln[4] = {lc[0], lc[1], lc[2], lc[3]};
      ln[mu] -= 1;
      const int j = half_index(ln, blk);
      cx<T> p[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) p[k] = src[k * HB + j];
      const int sb = nb_bwd(g, s, c, mu);
      switch (mu) {
        case 0: hop_bwd_p<T, 0, S>(p, gauge, g.V, sb, T(1), acc); break;
        case 1: hop_bwd_p<T, 1, S>(p, gauge, g.V, sb, T(1), acc); break;
        case 2: hop_bwd_p<T, 2, S>(p, gauge, g.V, sb, T(1), acc); break;
        default: hop_bwd_p<T, 3, S>(p, gauge, g.V, sb, T(1), acc); break;
      }
    }
  }
}

// y = D_oo^-1 p at odd site s: two general 6x6 complex blocks, 36 float4 /
// double2-pair chunks per odd site, compact odd index s >> 1
template <typename T, int S>
__device__ __forceinline__ void apply_dinv(const void* __restrict__ dinv, long Vh, int s, const cx<T> (&p)[12],
                                           cx<T> (&y)[12]) {
  const long so = s >> 1;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      cx<T> m[6];
      const long off = (long)(h * 6 + i) * 12 * Vh;  // row i of block h: 6 complex
      if constexpr (S == ST_NATIVE)
        ld_cx<T, 6>(static_cast<const T*>(dinv) + off, Vh, so, m);
      else
        ld_cx16<T, S, 6>(static_cast<const unsigned short*>(dinv) + off, Vh, so, m);
      cx<T> acc = m[0] * p[6 * h];
#pragma unroll
      for (int j = 1; j < 6; ++j) cfma(acc, m[j], p[6 * h + j]);
      y[6 * h + i] = acc;
    }
  }
}

// r = b - D x at site s (full operator, neighbours from global memory; b may be null)
template <typename T, int S = ST_NATIVE>
__device__ __forceinline__ void sap_residual_site(const T* __restrict__ x, const T* __restrict__ b,
                                                  const void* __restrict__ gauge, const void* __restrict__ clover,
                                                  const Lat& g, int s, const int c[4], T bc, T mu, cx<T> (&r)[12]) {
  cx<T> acc[12], p[12];
  all_hops_global<T, S>(x, gauge, g, s, c, bc, acc);
  ld_cx<T, 12>(x, g.V, s, p);
  site_diag<T, S>(clover, g.V, s, mu, p, r);
#pragma unroll
  for (int i = 0; i < 12; ++i) r[i] = T(0.5) * acc[i] - r[i];
  if (b) {
    ld_cx<T, 12>(b, g.V, s, p);
#pragma unroll
    for (int i = 0; i < 12; ++i) r[i] = r[i] + p[i];
  }
}

}  // namespace

template <typename T>
struct SapOeArgs {
  const void* gauge;  // links, clover and D_oo^-1 as T, or in 16 bits (kernel parameter S)
  const void* clover;
  const void* dinv;
  const T* b;
  T* x;
  SapGeom sg;
  T mu;
  T bc;
  int n_mr;
  int colour;
  int nrhs;
  T rho;  // odd sites carry mu + rho (D_oo^-1 is built with it)
};

// The kernel walks 2 n_MR + 3 half-steps, odd and even alternating, so that the
// hop gather, D_oo^-1 and the site-diagonal term each appear once in the code
// (the instruction cache holds the loop):
//   step 0 (odd):            u_o = D_oo^-1 r_o
//   step 1 (even):           rho = r_e - D_eo u_o
//   step 2k (odd, k >= 1):   t_o = D_oo^-1 D_oe rho
//   step 2k+1 (even):        q = D_ee rho - D_eo t_o; MR update of e_e, rho
//   step 2 n_MR + 2 (odd):   e_o = D_oo^-1 (r_o - D_oe e_e); x += e
// (D_eo, D_oe = -1/2 times the intra-block hops.)
template <typename T, int S>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 3 : 2) k_sap_oe(SapOeArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SapGeom& sg = a.sg;
  const Lat& g = sg.g;
  const int HB = sg.bsites / 2;
  cx<T>* ev = reinterpret_cast<cx<T>*>(smem_raw);  // [12][HB] even-site values (rho, then e_e)
  cx<T>* od = ev + 12 * HB;                         // [12][HB] odd-site values (u_o, t_o)
  cx<T>* ro = od + 12 * HB;                         // [12][HB] r_o
  T* red = reinterpret_cast<T*>(ro + 12 * HB);      // [32 * 3]
  const int rhs = blockIdx.x % a.nrhs;
  const long off = (long)rhs * NR_SPINOR * g.V;
  T* x = a.x + off;
  const long Vh = g.V / 2;

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

  const int j = threadIdx.x;
  const bool act = j < HB;
  // block-local coordinates of the j-th even site; the j-th odd site differs in x only
  int lce[4];
  int pr;
  {
    int q = act ? j : 0;
    const int bxh2 = sg.blk[3] / 2;
    const int xh = q % bxh2;
    q /= bxh2;
    lce[2] = q % sg.blk[2];
    q /= sg.blk[2];
    lce[1] = q % sg.blk[1];
    lce[0] = q / sg.blk[1];
    pr = (lce[0] + lce[1] + lce[2]) & 1;
    lce[3] = 2 * xh + pr;
  }
  auto site_of = [&](int parity, int (&lc)[4], int (&c)[4]) {
    lc[0] = lce[0];
    lc[1] = lce[1];
    lc[2] = lce[2];
    lc[3] = lce[3] - pr + (pr ^ parity);
#pragma unroll
    for (int d = 0; d < 4; ++d) c[d] = bc4[d] * sg.blk[d] + lc[d];
    return ((c[0] * g.L[1] + c[1]) * g.L[2] + c[2]) * g.L[3] + c[3];
  };
  const T half = T(0.5);

  // r = b - D x on the odd (pass 0, -> shared r_o) and the even site (pass 1, -> rho)
  cx<T> rho[12];
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    if (act) {
      int lc[4], c[4];
      const int s = site_of(pass ^ 1, lc, c);
      sap_residual_site<T, S>(x, a.b ? a.b + off : nullptr, a.gauge, a.clover, g, s, c, a.bc,
                              pass == 0 ? a.mu + a.rho : a.mu, rho);
      if (pass == 0) {
#pragma unroll
        for (int i = 0; i < 12; ++i) ro[i * HB + j] = rho[i];
      }
    }
  }
  cx<T> e[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) e[i] = cx<T>{0, 0};
  const int nsteps = 2 * a.n_mr + 3;
#pragma unroll 1
  for (int st = 0; st < nsteps; ++st) {
    const int parity = (st & 1) ^ 1;  // even steps work on odd sites
    __syncthreads();
    cx<T> acc[12];
    int lc[4], c[4];
    const int s = site_of(parity, lc, c);
    if (act && st > 0) oe_block_hops<T, S>(parity ? ev : od, HB, lc, sg.blk, a.gauge, g, s, c, acc);
    if (parity) {
      // odd site: y = D_oo^-1 in
      if (act) {
        cx<T> in[12], y[12];
        const bool last = st == nsteps - 1;
#pragma unroll
        for (int i = 0; i < 12; ++i) {
          if (st == 0)
            in[i] = ro[i * HB + j];
          else if (last)
            in[i] = ro[i * HB + j] + half * acc[i];
          else
            in[i] = -half * acc[i];
        }
        apply_dinv<T, S>(a.dinv, Vh, s, in, y);
        if (!last) {
#pragma unroll
          for (int i = 0; i < 12; ++i) od[i * HB + j] = y[i];
        } else {
          // x_o += e_o, x_e += e_e
          cx<T> p[12];
          ld_cx<T, 12>(x, g.V, s, p);
#pragma unroll
          for (int i = 0; i < 12; ++i) p[i] = p[i] + y[i];
          st_cx<T, 12>(x, g.V, s, p);
          int lc2[4], c2[4];
          const int s2 = site_of(0, lc2, c2);
          ld_cx<T, 12>(x, g.V, s2, p);
#pragma unroll
          for (int i = 0; i < 12; ++i) p[i] = p[i] + e[i];
          st_cx<T, 12>(x, g.V, s2, p);
        }
      }
    } else {
      const int kk = (st - 1) / 2;  // MR steps done before this one
      if (st == 1) {
        if (act) {
#pragma unroll
          for (int i = 0; i < 12; ++i) rho[i] = rho[i] + half * acc[i];
        }
      } else {
        cx<T> q[12];
        T dots[3] = {0, 0, 0};
        if (act) {
          site_diag<T, S>(a.clover, g.V, s, a.mu, rho, q);
#pragma unroll
          for (int i = 0; i < 12; ++i) {
            q[i] = q[i] + half * acc[i];
            dots[0] = fma(q[i].r, rho[i].r, fma(q[i].i, rho[i].i, dots[0]));   // Re <q, rho>
            dots[1] = fma(q[i].r, rho[i].i, fma(-q[i].i, rho[i].r, dots[1]));  // Im <q, rho>
            dots[2] = fma(q[i].r, q[i].r, fma(q[i].i, q[i].i, dots[2]));       // <q, q>
          }
        }
        block_allreduce<T, 3>(dots, red);
        const cx<T> alpha = dots[2] > T(0) ? cx<T>{dots[0] / dots[2], dots[1] / dots[2]} : cx<T>{0, 0};
        if (act) {
#pragma unroll
          for (int i = 0; i < 12; ++i) {
            cfma(e[i], alpha, rho[i]);
            cfma(rho[i], -alpha, q[i]);
          }
        }
      }
      // the next odd step gathers rho, or e_e after the last MR step (step 2 n_MR + 1)
      if (act) {
        const bool store_e = kk == a.n_mr;
#pragma unroll
        for (int i = 0; i < 12; ++i) ev[i * HB + j] = store_e ? e[i] : rho[i];
      }
    }
  }
}

template <typename T, int S>
void sap_oe_s(const SapOeArgs<T>& a, int nblocks, int threads, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_sap_oe<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  k_sap_oe<T, S><<<dim3(nblocks), threads, smem, st>>>(a);
}

template <typename T>
void launch_sap_oe_colour(const void* gauge, const void* clover, const void* dinv, const T* b, T* x,
                          const SapGeom& sg, double mu, double bc_t, int n_mr, int colour, int nrhs, cudaStream_t st,
                          double rho, int s16) {
  const int HB = sg.bsites / 2;
  const int threads = (HB + 31) / 32 * 32;
  const size_t smem = 3 * 12 * (size_t)HB * sizeof(cx<T>) + 32 * 3 * sizeof(T);
  const int nblk_colour = sg.nb[0] * sg.nb[1] * sg.nb[2] * sg.nb[3] / 2;
  SapOeArgs<T> a{gauge, clover, dinv, b, x, sg, (T)mu, (T)bc_t, n_mr, colour, nrhs, (T)rho};
  if constexpr (std::is_same<T, float>::value) {
    if (s16 == ST_F16) return sap_oe_s<T, ST_F16>(a, nblk_colour * nrhs, threads, smem, st);
    if (s16 == ST_BF16) return sap_oe_s<T, ST_BF16>(a, nblk_colour * nrhs, threads, smem, st);
  }
  sap_oe_s<T, ST_NATIVE>(a, nblk_colour * nrhs, threads, smem, st);
}

template void launch_sap_oe_colour<double>(const void*, const void*, const void*, const double*, double*,
                                           const SapGeom&, double, double, int, int, int, cudaStream_t, double, int);
template void launch_sap_oe_colour<float>(const void*, const void*, const void*, const float*, float*,
                                          const SapGeom&, double, double, int, int, int, cudaStream_t, double, int);

// ===========================================================================
// D_oo^-1 for the odd-even block solve: per odd site the inverses of the two
// chiral 6x6 blocks A_h(x) + i s_h mu (s_0 = -1, s_1 = +1: gamma5 of the
// chirality), Gauss-Jordan with partial pivoting in FP64, stored row-major
// per block as 12 rows of 6 complex, chunked SoA over the V/2 odd sites
// (compact index s >> 1).
// ===========================================================================
namespace {
template <typename T>
__global__ void k_clover_inverse(const double* __restrict__ c64, T* __restrict__ dinv, Lat g, double mu, int* err,
                                 int parity) {
  const long so = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long Vh = g.V / 2;
  if (so >= Vh) return;
  // odd site with compact index so: x-row so / (X/2), x = 2 (so % (X/2)) + parity offset
  const long row = so / (g.L[3] / 2);
  const int xh = (int)(so % (g.L[3] / 2));
  int c[4];
  c[2] = (int)(row % g.L[2]);
  c[1] = (int)((row / g.L[2]) % g.L[1]);
  c[0] = (int)(row / ((long)g.L[2] * g.L[1]));
  c[3] = 2 * xh + (((c[0] + c[1] + c[2]) & 1) ^ parity);
  const int s = ((c[0] * g.L[1] + c[1]) * g.L[2] + c[2]) * g.L[3] + c[3];
  double m72[72];
  ld_re<double, 72>(c64, g.V, s, m72);
  for (int h = 0; h < 2; ++h) {
    cx<double> M[6][12];
    const double* m = m72 + 36 * h;
    for (int i = 0; i < 6; ++i)
      for (int jj = 0; jj < 12; ++jj) M[i][jj] = cx<double>{jj - 6 == i ? 1.0 : 0.0, 0.0};
    for (int i = 0; i < 6; ++i) M[i][i] = cx<double>{m[i], (h == 0 ? -mu : mu)};
    int kk = 6;
    for (int i = 0; i < 6; ++i)
      for (int jj = i + 1; jj < 6; ++jj) {
        M[i][jj] = cx<double>{m[kk], m[kk + 1]};
        M[jj][i] = cx<double>{m[kk], -m[kk + 1]};
        kk += 2;
      }
    for (int col = 0; col < 6; ++col) {
      int piv = col;
      double best = norm2(M[col][col]);
      for (int i = col + 1; i < 6; ++i)
        if (norm2(M[i][col]) > best) {
          best = norm2(M[i][col]);
          piv = i;
        }
      if (!(best > 0)) {
        atomicOr(err, ERRF_SINGULAR);
        return;
      }
      if (piv != col)
        for (int jj = 0; jj < 12; ++jj) {
          const cx<double> t = M[col][jj];
          M[col][jj] = M[piv][jj];
          M[piv][jj] = t;
        }
      const cx<double> pv = M[col][col];
      const double pn = norm2(pv);
      const cx<double> inv{pv.r / pn, -pv.i / pn};
      for (int jj = 0; jj < 12; ++jj) M[col][jj] = inv * M[col][jj];
      for (int i = 0; i < 6; ++i) {
        if (i == col) continue;
        const cx<double> f = M[i][col];
        for (int jj = 0; jj < 12; ++jj) M[i][jj] = M[i][jj] - f * M[col][jj];
      }
    }
    for (int i = 0; i < 6; ++i) {
      cx<T> row6[6];
      for (int jj = 0; jj < 6; ++jj) row6[jj] = cx<T>{(T)M[i][6 + jj].r, (T)M[i][6 + jj].i};
      st_cx<T, 6>(dinv + (long)(h * 6 + i) * 12 * Vh, Vh, so, row6);
    }
  }
}
}  // namespace

template <typename T>
void launch_clover_inverse(const double* c64, T* dinv, const Lat& g, double mu, int* err, cudaStream_t st,
                           int parity) {
  const long Vh = g.V / 2;
  k_clover_inverse<T><<<(unsigned)((Vh + 63) / 64), 64, 0, st>>>(c64, dinv, g, mu, err, parity);
}
template void launch_clover_inverse<double>(const double*, double*, const Lat&, double, int*, cudaStream_t, int);
template void launch_clover_inverse<float>(const double*, float*, const Lat&, double, int*, cudaStream_t, int);

}  // namespace tmamg
