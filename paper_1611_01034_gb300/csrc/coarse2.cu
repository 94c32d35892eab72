// The first coarse level of the three-level hierarchy (Sec. 2 of the paper:
// the standard DD-alphaAMG setup has three levels, 4^4 then 2^4 aggregates):
// SAP on the 9-point coarse stencil, the level-1 aggregation P2 (thin QR per
// aggregate and chirality), restriction/prolongation between levels 1 and 2,
// and the Galerkin product D_c2 = P2^dagger D_c1 P2.
//
// Level-1 vectors are [Vc1][n1] complex (n1 = 2 Nv1, chirality -1 first), P2
// is N_v2 such fields (field j holds column j of P2_{a,chi} in the chirality-chi
// half of every site of aggregate a), D_c1 and D_c2 are stored like the first
// coarse operator: [site][9 blocks][col][row].
#include <cuda_fp16.h>

#include "tm_kernels.h"

namespace tmamg {

// D_c1 block entry: stored in T (S = ST_NATIVE), or as 16-bit (re, im) pairs
// (ST_F16, ST_BF16; arithmetic stays in T)
template <typename T, int S>
__device__ __forceinline__ cx<T> ld_blk(const void* __restrict__ Dc, long idx) {
  if constexpr (S != ST_NATIVE) {
    const float2 f = unpack16x2<S>(__ldg(reinterpret_cast<const unsigned*>(Dc) + idx));
    return cx<T>{(T)f.x, (T)f.y};
  } else {
    return reinterpret_cast<const cx<T>*>(Dc)[idx];
  }
}

__device__ __forceinline__ int c_nb(const Lat& g, int s, int t) {
  if (t == 0) return s;
  int c[4];
  site_coords(g, s, c);
  const int mu = (t - 1) >> 1;
  return ((t - 1) & 1) ? nb_bwd(g, s, c, mu) : nb_fwd(g, s, c, mu);
}

// ===========================================================================
// coarse SAP: one colour; CTA = one block of level-1 sites, thread = (site, row)
// ===========================================================================
template <typename T, int H>
__global__ void k_csap(const void* __restrict__ Dc, const T* __restrict__ b, T* __restrict__ x, CSapGeom sg, T mu,
                       int n_mr, int colour, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = sg.n, BS = sg.bsites;
  cx<T>* rs = reinterpret_cast<cx<T>*>(smem_raw);  // [BS][n]
  T* red = reinterpret_cast<T*>(rs + (size_t)BS * n);
  const Lat& g = sg.g;
  const long off = (long)(blockIdx.x % nrhs) * g.V * n;  // right-hand sides fastest (block reuse in L2)
  const cx<T>* bb = b ? reinterpret_cast<const cx<T>*>(b) + off : nullptr;
  cx<T>* xx = reinterpret_cast<cx<T>*>(x) + off;
  int k = blockIdx.x / nrhs;
  const int nbxh = sg.nb[3] / 2;
  int bc4[4];
  const int bxh = k % nbxh;
  k /= nbxh;
  bc4[2] = k % sg.nb[2];
  k /= sg.nb[2];
  bc4[1] = k % sg.nb[1];
  bc4[0] = k / sg.nb[1];
  bc4[3] = 2 * bxh + ((bc4[0] + bc4[1] + bc4[2] + colour) & 1);
  const int l = threadIdx.x / n, row = threadIdx.x % n;
  const bool act = l < BS;
  int lc[4], c[4], lst[4];
  lst[3] = 1;
  lst[2] = sg.blk[3];
  lst[1] = sg.blk[3] * sg.blk[2];
  lst[0] = lst[1] * sg.blk[1];
  {
    int q = act ? l : 0;
    lc[3] = q % sg.blk[3];
    q /= sg.blk[3];
    lc[2] = q % sg.blk[2];
    q /= sg.blk[2];
    lc[1] = q % sg.blk[1];
    lc[0] = q / sg.blk[1];
  }
  for (int d = 0; d < 4; ++d) c[d] = bc4[d] * sg.blk[d] + lc[d];
  const int s = ((c[0] * g.L[1] + c[1]) * g.L[2] + c[2]) * g.L[3] + c[3];
  const long B = (long)s * 9 * n * n;  // block entries of site s
  const T sg5 = row < n / 2 ? -mu : mu;  // i mu Gamma5_c
  cx<T> r{0, 0}, e{0, 0};
  if (act) {
    cx<T> acc{0, 0};
    for (int t = 0; t < 9; ++t) {
      const cx<T>* src = xx + (long)c_nb(g, s, t) * n;
      const long Bt = B + (long)t * n * n;
#pragma unroll 8
      for (int col = 0; col < n; ++col) cfma(acc, ld_blk<T, H>(Dc, Bt + (long)col * n + row), src[col]);
    }
    const cx<T> xs = xx[(long)s * n + row];
    acc.r -= sg5 * xs.i;
    acc.i += sg5 * xs.r;
    r = (bb ? bb[(long)s * n + row] : cx<T>{0, 0}) - acc;
    rs[(size_t)l * n + row] = r;
  }
  for (int it = 0; it < n_mr; ++it) {
    __syncthreads();
    cx<T> q{0, 0};
    T dots[3] = {0, 0, 0};
    if (act) {
      for (int t = 0; t < 9; ++t) {
        int ln = l;
        if (t > 0) {
          const int mu_d = (t - 1) >> 1;
          const bool bwd = (t - 1) & 1;
          if (bwd ? lc[mu_d] == 0 : lc[mu_d] == sg.blk[mu_d] - 1) continue;  // leaves the block
          ln = bwd ? l - lst[mu_d] : l + lst[mu_d];
        }
        const long Bt = B + (long)t * n * n;
        const cx<T>* src = rs + (size_t)ln * n;
#pragma unroll 8
        for (int col = 0; col < n; ++col) cfma(q, ld_blk<T, H>(Dc, Bt + (long)col * n + row), src[col]);
      }
      q.r -= sg5 * r.i;
      q.i += sg5 * r.r;
      dots[0] = q.r * r.r + q.i * r.i;
      dots[1] = q.r * r.i - q.i * r.r;
      dots[2] = q.r * q.r + q.i * q.i;
    }
    block_allreduce<T, 3>(dots, red);
    const cx<T> alpha = dots[2] > T(0) ? cx<T>{dots[0] / dots[2], dots[1] / dots[2]} : cx<T>{0, 0};
    if (act) {
      cfma(e, alpha, r);
      cfma(r, -alpha, q);
    }
    __syncthreads();
    if (act) rs[(size_t)l * n + row] = r;
  }
  __syncthreads();
  if (act) xx[(long)s * n + row] = xx[(long)s * n + row] + e;
}

// The same colour for up to RB right-hand sides per CTA: every block entry a
// thread loads serves all of them (the separate-rhs form reads the block's
// D_c1 entries once per right-hand side and MR step).  Each right-hand side
// keeps its own residual, correction and MR coefficients.
template <typename T, int H, int RB>
__global__ void __launch_bounds__(768) k_csap_b(const void* __restrict__ Dc, const T* __restrict__ b, T* __restrict__ x, CSapGeom sg, T mu,
                         int n_mr, int colour, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = sg.n, BS = sg.bsites;
  cx<T>* rs = reinterpret_cast<cx<T>*>(smem_raw);  // [RB][BS][n]
  T* red = reinterpret_cast<T*>(rs + (size_t)RB * BS * n);
  const Lat& g = sg.g;
  const int ngrp = (nrhs + RB - 1) / RB;
  const int r0 = (blockIdx.x % ngrp) * RB;  // groups of right-hand sides fastest (block reuse in L2)
  const int R = min(RB, nrhs - r0);
  const long vs = (long)g.V * n;  // complex numbers per level-1 vector
  int k = blockIdx.x / ngrp;
  const int nbxh = sg.nb[3] / 2;
  int bc4[4];
  const int bxh = k % nbxh;
  k /= nbxh;
  bc4[2] = k % sg.nb[2];
  k /= sg.nb[2];
  bc4[1] = k % sg.nb[1];
  bc4[0] = k / sg.nb[1];
  bc4[3] = 2 * bxh + ((bc4[0] + bc4[1] + bc4[2] + colour) & 1);
  const int l = threadIdx.x / n, row = threadIdx.x % n;
  const bool act = l < BS;
  int lc[4], c[4], lst[4];
  lst[3] = 1;
  lst[2] = sg.blk[3];
  lst[1] = sg.blk[3] * sg.blk[2];
  lst[0] = lst[1] * sg.blk[1];
  {
    int q = act ? l : 0;
    lc[3] = q % sg.blk[3];
    q /= sg.blk[3];
    lc[2] = q % sg.blk[2];
    q /= sg.blk[2];
    lc[1] = q % sg.blk[1];
    lc[0] = q / sg.blk[1];
  }
  for (int d = 0; d < 4; ++d) c[d] = bc4[d] * sg.blk[d] + lc[d];
  const int s = ((c[0] * g.L[1] + c[1]) * g.L[2] + c[2]) * g.L[3] + c[3];
  const long B = (long)s * 9 * n * n;
  const T sg5 = row < n / 2 ? -mu : mu;
  const cx<T>* xx = reinterpret_cast<const cx<T>*>(x) + r0 * vs;
  const cx<T>* bb = b ? reinterpret_cast<const cx<T>*>(b) + r0 * vs : nullptr;
  cx<T> r[RB], e[RB];
#pragma unroll
  for (int j = 0; j < RB; ++j) r[j] = e[j] = cx<T>{0, 0};
  if (act) {
    cx<T> acc[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) acc[j] = cx<T>{0, 0};
    for (int t = 0; t < 9; ++t) {
      const long src = (long)c_nb(g, s, t) * n;
      const long Bt = B + (long)t * n * n;
#pragma unroll 4
      for (int col = 0; col < n; ++col) {
        const cx<T> m = ld_blk<T, H>(Dc, Bt + (long)col * n + row);
#pragma unroll
        for (int j = 0; j < RB; ++j)
          if (j < R) cfma(acc[j], m, xx[j * vs + src + col]);
      }
    }
#pragma unroll
    for (int j = 0; j < RB; ++j) {
      if (j < R) {
        const cx<T> xs = xx[j * vs + (long)s * n + row];
        acc[j].r -= sg5 * xs.i;
        acc[j].i += sg5 * xs.r;
        r[j] = (bb ? bb[j * vs + (long)s * n + row] : cx<T>{0, 0}) - acc[j];
        rs[((size_t)j * BS + l) * n + row] = r[j];
      }
    }
  }
  for (int it = 0; it < n_mr; ++it) {
    __syncthreads();
    cx<T> q[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) q[j] = cx<T>{0, 0};
    T dots[3 * RB];
#pragma unroll
    for (int j = 0; j < 3 * RB; ++j) dots[j] = 0;
    if (act) {
      for (int t = 0; t < 9; ++t) {
        int ln = l;
        if (t > 0) {
          const int mu_d = (t - 1) >> 1;
          const bool bwd = (t - 1) & 1;
          if (bwd ? lc[mu_d] == 0 : lc[mu_d] == sg.blk[mu_d] - 1) continue;  // leaves the block
          ln = bwd ? l - lst[mu_d] : l + lst[mu_d];
        }
        const long Bt = B + (long)t * n * n;
#pragma unroll 4
        for (int col = 0; col < n; ++col) {
          const cx<T> m = ld_blk<T, H>(Dc, Bt + (long)col * n + row);
#pragma unroll
          for (int j = 0; j < RB; ++j)
            if (j < R) cfma(q[j], m, rs[((size_t)j * BS + ln) * n + col]);
        }
      }
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        q[j].r -= sg5 * r[j].i;
        q[j].i += sg5 * r[j].r;
        dots[3 * j] = q[j].r * r[j].r + q[j].i * r[j].i;
        dots[3 * j + 1] = q[j].r * r[j].i - q[j].i * r[j].r;
        dots[3 * j + 2] = q[j].r * q[j].r + q[j].i * q[j].i;
      }
    }
    block_allreduce<T, 3 * RB>(dots, red);
    if (act) {
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        const cx<T> alpha = dots[3 * j + 2] > T(0) ? cx<T>{dots[3 * j] / dots[3 * j + 2], dots[3 * j + 1] / dots[3 * j + 2]}
                                                   : cx<T>{0, 0};
        cfma(e[j], alpha, r[j]);
        cfma(r[j], -alpha, q[j]);
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int j = 0; j < RB; ++j)
        if (j < R) rs[((size_t)j * BS + l) * n + row] = r[j];
    }
  }
  __syncthreads();
  if (act) {
    cx<T>* xw = reinterpret_cast<cx<T>*>(x) + r0 * vs;
#pragma unroll
    for (int j = 0; j < RB; ++j)
      if (j < R) xw[j * vs + (long)s * n + row] = xw[j * vs + (long)s * n + row] + e[j];
  }
}

constexpr int kCsapRhs = 6;  // right-hand sides per CTA of the batched level-1 SAP

template <typename T, int H>
void csap_b(const void* Dc, const T* b, T* x, const CSapGeom& sg, double mu, int n_mr, int colour, int nrhs,
            cudaStream_t st) {
  const int threads = (sg.bsites * sg.n + 31) / 32 * 32;
  const size_t smem = (size_t)kCsapRhs * sg.bsites * sg.n * sizeof(cx<T>) + 32 * 3 * kCsapRhs * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_csap_b<T, H, kCsapRhs>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  const int ngrp = (nrhs + kCsapRhs - 1) / kCsapRhs;
  dim3 grid((unsigned)(sg.nb[0] * sg.nb[1] * sg.nb[2] * sg.nb[3] / 2) * (unsigned)ngrp);
  k_csap_b<T, H, kCsapRhs><<<grid, threads, smem, st>>>(Dc, b, x, sg, (T)mu, n_mr, colour, nrhs);
}

template <typename T>
void launch_csap_colour(const T* Dc, const T* b, T* x, const CSapGeom& sg, double mu, int n_mr, int colour,
                        int nrhs, cudaStream_t st, const void* Dc_half, int half_kind) {
  // several right-hand sides share every block-entry load (its 80 registers per
  // thread allow up to 768 threads: 2^4 blocks of N_v1 <= 24)
  if (nrhs > 1 && sizeof(T) == 4 && sg.bsites * sg.n <= 768) {
    if (Dc_half && half_kind == ST_BF16)
      csap_b<T, ST_BF16>(Dc_half, b, x, sg, mu, n_mr, colour, nrhs, st);
    else if (Dc_half)
      csap_b<T, ST_F16>(Dc_half, b, x, sg, mu, n_mr, colour, nrhs, st);
    else
      csap_b<T, ST_NATIVE>(Dc, b, x, sg, mu, n_mr, colour, nrhs, st);
    return;
  }
  const int threads = (sg.bsites * sg.n + 31) / 32 * 32;
  const size_t smem = (size_t)sg.bsites * sg.n * sizeof(cx<T>) + 32 * 3 * sizeof(T);
  dim3 grid((unsigned)(sg.nb[0] * sg.nb[1] * sg.nb[2] * sg.nb[3] / 2) * (unsigned)nrhs);
  if (Dc_half && half_kind == ST_BF16)
    k_csap<T, ST_BF16><<<grid, threads, smem, st>>>(Dc_half, b, x, sg, (T)mu, n_mr, colour, nrhs);
  else if (Dc_half)
    k_csap<T, ST_F16><<<grid, threads, smem, st>>>(Dc_half, b, x, sg, (T)mu, n_mr, colour, nrhs);
  else
    k_csap<T, ST_NATIVE><<<grid, threads, smem, st>>>(Dc, b, x, sg, (T)mu, n_mr, colour, nrhs);
}

// ===========================================================================
// level-1 aggregation
// ===========================================================================
// level-1 site of thread-site l of level-2 aggregate a, with local coordinates
__device__ __forceinline__ int cagg_site(const CAggGeom& ag, int a, int l, int lc[4]) {
  int ac[4];
  site_coords(ag.g2, a, ac);
  int q = l;
  lc[3] = q % ag.agg[3];
  q /= ag.agg[3];
  lc[2] = q % ag.agg[2];
  q /= ag.agg[2];
  lc[1] = q % ag.agg[1];
  lc[0] = q / ag.agg[1];
  int c[4];
  for (int d = 0; d < 4; ++d) c[d] = ac[d] * ag.agg[d] + lc[d];
  return ((c[0] * ag.g1.L[1] + c[1]) * ag.g1.L[2] + c[2]) * ag.g1.L[3] + c[3];
}

__device__ __forceinline__ int cagg_of(const CAggGeom& ag, int s1) {
  int c[4];
  site_coords(ag.g1, s1, c);
  return (((c[0] / ag.agg[0]) * ag.g2.L[1] + c[1] / ag.agg[1]) * ag.g2.L[2] + c[2] / ag.agg[2]) * ag.g2.L[3] +
         c[3] / ag.agg[3];
}

// CGS2 per (aggregate, chirality): thread = (site l, component i of the half)
template <typename T>
__global__ void k_corth(T* P2, CAggGeom ag, int* err) {
  __shared__ T red[32 * 16];
  const int a = blockIdx.x, chi = blockIdx.y;
  const int nv1 = ag.nv1, n1 = 2 * nv1, nv2 = ag.nv2;
  const int l = threadIdx.x / nv1, i = threadIdx.x % nv1;
  const bool act = l < ag.asites;
  int lc[4];
  const int s = act ? cagg_site(ag, a, l, lc) : 0;
  const long fstride = (long)ag.g1.V * n1;
  const long idx = (long)s * n1 + chi * nv1 + i;
  cx<T>* P = reinterpret_cast<cx<T>*>(P2);
  const T rank_tol = sizeof(T) == 8 ? T(1e-24) : T(1e-10);
  for (int j = 0; j < nv2; ++j) {
    cx<T> v = act ? P[j * fstride + idx] : cx<T>{0, 0};
    T t0[1] = {norm2(v)};
    block_allreduce<T, 1>(t0, red);
    const T n0 = t0[0];
    for (int pass = 0; pass < 2; ++pass) {
      for (int i0 = 0; i0 < j; i0 += 8) {
        T d[16];
        for (int m = 0; m < 16; ++m) d[m] = 0;
        if (act)
          for (int ii = 0; ii < 8 && i0 + ii < j; ++ii) {
            const cx<T> q = P[(i0 + ii) * fstride + idx];
            const cx<T> pr = cmulc(q, v);
            d[2 * ii] = pr.r;
            d[2 * ii + 1] = pr.i;
          }
        block_allreduce<T, 16>(d, red);
        if (act)
          for (int ii = 0; ii < 8 && i0 + ii < j; ++ii) {
            const cx<T> q = P[(i0 + ii) * fstride + idx];
            v = v - cx<T>{d[2 * ii], d[2 * ii + 1]} * q;
          }
      }
    }
    T t1[1] = {norm2(v)};
    block_allreduce<T, 1>(t1, red);
    T nn = t1[0];
    if (!(nn > rank_tol * n0) || !(nn > T(0))) {
      if (threadIdx.x == 0) atomicOr(err, ERRF_RANK);
      nn = T(1);
    }
    const T inv = T(1) / sqrt(nn);
    if (act) P[j * fstride + idx] = inv * v;
    __syncthreads();
  }
}

template <typename T>
void launch_corth(T* P2, const CAggGeom& ag, int* err, cudaStream_t st) {
  const int threads = (ag.asites * ag.nv1 + 31) / 32 * 32;
  dim3 grid(ag.g2.V, 2);
  k_corth<T><<<grid, threads, 0, st>>>(P2, ag, err);
}

// r2(a, chi*Nv2 + j) = sum_{x in a, i} conj(P2_j(x)[chi, i]) r1(x)[chi, i]
template <typename T>
__global__ void k_crestrict(const T* __restrict__ P2, const T* __restrict__ r1, T* __restrict__ r2, CAggGeom ag) {
  __shared__ T red[32 * 16];
  __shared__ T fin[16];
  const int a = blockIdx.x, rhs = blockIdx.y;
  const int n1 = 2 * ag.nv1, nv2 = ag.nv2;
  const int l = threadIdx.x / n1, cc = threadIdx.x % n1;
  const bool act = l < ag.asites;
  const int chi = cc >= ag.nv1;
  int lc[4];
  const int s = act ? cagg_site(ag, a, l, lc) : 0;
  const long fstride = (long)ag.g1.V * n1;
  const cx<T>* P = reinterpret_cast<const cx<T>*>(P2);
  const cx<T> rv = act ? reinterpret_cast<const cx<T>*>(r1)[(long)rhs * fstride + (long)s * n1 + cc] : cx<T>{0, 0};
  cx<T>* out = reinterpret_cast<cx<T>*>(r2) + ((long)rhs * ag.g2.V + a) * 2 * nv2;
  for (int j0 = 0; j0 < nv2; j0 += 4) {
    T d[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) d[m] = 0;
    if (act) {
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
        if (j0 + jj < nv2) {
          const cx<T> pr = cmulc(P[(j0 + jj) * fstride + (long)s * n1 + cc], rv);
          d[4 * jj + 2 * chi] = pr.r;
          d[4 * jj + 2 * chi + 1] = pr.i;
        }
    }
    block_reduce16<T>(d, red, fin);
    if (threadIdx.x < 8) {
      const int jj = threadIdx.x >> 1, h = threadIdx.x & 1;
      if (j0 + jj < nv2) out[h * nv2 + j0 + jj] = cx<T>{fin[4 * jj + 2 * h], fin[4 * jj + 2 * h + 1]};
    }
  }
}

template <typename T>
void launch_crestrict(const T* P2, const T* r1, T* r2, const CAggGeom& ag, int nrhs, cudaStream_t st) {
  const int threads = (ag.asites * 2 * ag.nv1 + 31) / 32 * 32;
  dim3 grid(ag.g2.V, nrhs);
  k_crestrict<T><<<grid, threads, 0, st>>>(P2, r1, r2, ag);
}

// x1(x)[chi, i] (+)= sum_j P2_j(x)[chi, i] e2(a(x), chi*Nv2 + j)
template <typename T>
__global__ void k_cprolong(const T* __restrict__ P2, const T* __restrict__ e2, T* __restrict__ x1, CAggGeom ag,
                           int accumulate) {
  const int n1 = 2 * ag.nv1, nv2 = ag.nv2;
  const long tot = (long)ag.g1.V * n1;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (e >= tot) return;
  const int s = (int)(e / n1), cc = (int)(e % n1);
  const int chi = cc >= ag.nv1;
  const int a = cagg_of(ag, s);
  const cx<T>* P = reinterpret_cast<const cx<T>*>(P2);
  const cx<T>* ev = reinterpret_cast<const cx<T>*>(e2) + ((long)rhs * ag.g2.V + a) * 2 * nv2 + chi * nv2;
  cx<T>* out = reinterpret_cast<cx<T>*>(x1) + (long)rhs * tot + e;
  cx<T> acc = accumulate ? *out : cx<T>{0, 0};
  for (int j = 0; j < nv2; ++j) cfma(acc, P[(long)j * tot + e], ev[j]);
  *out = acc;
}

template <typename T>
void launch_cprolong(const T* P2, const T* e2, T* x1, const CAggGeom& ag, int nrhs, bool accumulate,
                     cudaStream_t st) {
  const long tot = (long)ag.g1.V * 2 * ag.nv1;
  dim3 grid((unsigned)((tot + 255) / 256), nrhs);
  k_cprolong<T><<<grid, 256, 0, st>>>(P2, e2, x1, ag, accumulate ? 1 : 0);
}

// ===========================================================================
// D_c2 = P2^dagger D_c1(0) P2: one CTA per (block type t, level-2 site a)
// ===========================================================================
constexpr int kCBuildThreads = 256;
constexpr int kCBuildOut = 13;  // (2 Nv2)^2 <= 13 * 256

// f-th level-1 site (local index in the aggregate) visited by block type t
__device__ __forceinline__ int cblock_site(const CAggGeom& ag, int t, int f) {
  if (t == 0) return f;
  const int mu = (t - 1) >> 1;
  const int fixed = ((t - 1) & 1) ? 0 : ag.agg[mu] - 1;
  int lc[4], q = f;
  for (int d = 3; d >= 0; --d) {
    if (d == mu) {
      lc[d] = fixed;
    } else {
      lc[d] = q % ag.agg[d];
      q /= ag.agg[d];
    }
  }
  return ((lc[0] * ag.agg[1] + lc[1]) * ag.agg[2] + lc[2]) * ag.agg[3] + lc[3];
}

template <typename T>
__global__ void __launch_bounds__(kCBuildThreads) k_cbuild(const T* __restrict__ Dc1, const T* __restrict__ P2,
                                                           T* __restrict__ Dc2, CAggGeom ag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nv1 = ag.nv1, n1 = 2 * nv1, nv2 = ag.nv2, n2 = 2 * nv2;
  cx<T>* Ps = reinterpret_cast<cx<T>*>(smem_raw);  // [n1][nv2]  P2_j(x)[c]
  cx<T>* Us = Ps + (size_t)n1 * nv2;                 // [n1][n2]   u_k(x)[c]
  const int t = blockIdx.x, a = blockIdx.y;
  const int nsites = t == 0 ? ag.asites : ag.asites / ag.agg[(t - 1) >> 1];
  const long tot = (long)ag.g1.V * n1;
  const cx<T>* P = reinterpret_cast<const cx<T>*>(P2);
  cx<T> acc[kCBuildOut];
#pragma unroll
  for (int m = 0; m < kCBuildOut; ++m) acc[m] = cx<T>{0, 0};
  for (int f = 0; f < nsites; ++f) {
    int lc[4];
    const int l = cblock_site(ag, t, f);
    const int s = cagg_site(ag, a, l, lc);
    for (int e = threadIdx.x; e < n1 * nv2; e += blockDim.x) {
      const int cc = e / nv2, j = e % nv2;
      Ps[e] = P[(long)j * tot + (long)s * n1 + cc];
    }
    // columns k = chi' * Nv2 + j' of the block: B(x, nb) applied to the chirality-chi'
    // half of P2_j'(nb), summed over the couplings of block type t
    const cx<T>* B = reinterpret_cast<const cx<T>*>(Dc1) + (long)s * 9 * n1 * n1;
    for (int e = threadIdx.x; e < n1 * n2; e += blockDim.x) {
      const int cc = e / n2, k = e % n2;
      const int chi2 = k / nv2, j2 = k % nv2;
      cx<T> u{0, 0};
      for (int h = 0; h < 9; ++h) {
        bool use;
        if (t == 0) {
          if (h == 0) {
            use = true;
          } else {
            const int mu = (h - 1) >> 1;
            use = ((h - 1) & 1) ? lc[mu] > 0 : lc[mu] < ag.agg[mu] - 1;  // stays in the aggregate
          }
        } else {
          use = h == t;
        }
        if (!use) continue;
        const int nb = c_nb(ag.g1, s, h);
        const cx<T>* Bh = B + (long)h * n1 * n1;
        const cx<T>* src = P + (long)j2 * tot + (long)nb * n1 + chi2 * nv1;
        for (int col = 0; col < nv1; ++col) cfma(u, Bh[(long)(chi2 * nv1 + col) * n1 + cc], src[col]);
      }
      Us[e] = u;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kCBuildOut; ++m) {
      const int o = threadIdx.x + m * kCBuildThreads;
      if (o < n2 * n2) {
        const int row = o / n2, k = o % n2;
        const int chi = row / nv2, j = row % nv2;
        cx<T> sum = acc[m];
        for (int i = 0; i < nv1; ++i) {
          const int cc = chi * nv1 + i;
          cfmac(sum, Ps[(size_t)cc * nv2 + j], Us[(size_t)cc * n2 + k]);
        }
        acc[m] = sum;
      }
    }
    __syncthreads();
  }
  T* out = Dc2 + ((long)a * 9 + t) * n2 * n2 * 2;
#pragma unroll
  for (int m = 0; m < kCBuildOut; ++m) {
    const int o = threadIdx.x + m * kCBuildThreads;
    if (o < n2 * n2) {
      const int row = o / n2, k = o % n2;
      out[2 * ((long)k * n2 + row)] = acc[m].r;
      out[2 * ((long)k * n2 + row) + 1] = acc[m].i;
    }
  }
}

template <typename T>
void launch_cbuild(const T* Dc1, const T* P2, T* Dc2, const CAggGeom& ag, cudaStream_t st) {
  const size_t smem = (size_t)2 * ag.nv1 * 3 * ag.nv2 * sizeof(cx<T>);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_cbuild<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  dim3 grid(9, ag.g2.V);
  k_cbuild<T><<<grid, kCBuildThreads, smem, st>>>(Dc1, P2, Dc2, ag);
}

#define TM_INST(T)                                                                                           \
  template void launch_csap_colour<T>(const T*, const T*, T*, const CSapGeom&, double, int, int, int,       \
                                      cudaStream_t, const void*, int);                                       \
  template void launch_corth<T>(T*, const CAggGeom&, int*, cudaStream_t);                                   \
  template void launch_crestrict<T>(const T*, const T*, T*, const CAggGeom&, int, cudaStream_t);            \
  template void launch_cprolong<T>(const T*, const T*, T*, const CAggGeom&, int, bool, cudaStream_t);       \
  template void launch_cbuild<T>(const T*, const T*, T*, const CAggGeom&, cudaStream_t);
TM_INST(double)
TM_INST(float)
#undef TM_INST

}  // namespace tmamg
