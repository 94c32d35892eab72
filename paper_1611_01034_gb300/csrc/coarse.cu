// Aggregation-based interpolation P, restriction P^dagger, the coarse
// operator D_c = P^dagger D_W P (+ i mu_c Gamma5_c) and its odd-even Schur
// complement (Sec. 1 of the paper: P aggregates N_v test vectors and is
// Gamma5-compatible, D_c keeps Gamma5-hermiticity, the twisted-mass term stays
// diagonal, mu_c = delta mu on the coarsest grid; Sec. 3: odd-even
// preconditioning on the coarsest level).
//
// P is stored as N_v fine fields in the chunked spinor layout: field i holds
// column i of P_{a,0} on spins {0,1} and column i of P_{a,1} on spins {2,3}
// of every aggregate a.  The two chirality halves of a site are whole 16-byte
// chunks (12 reals each).  A coarse vector is [Vc][2 N_v] complex with index
// chi * N_v + i.  D_c is stored per coarse site as 9 blocks (self, then
// forward/backward per direction T, Z, Y, X), each column-major [col][row] so
// that one thread per row reads consecutive addresses.
#include "tm_kernels.h"
#include "tm_stencil.cuh"

namespace tmamg {

// fine site of thread l of aggregate a, with its local and global coordinates
__device__ __forceinline__ int agg_site(const AggGeom& ag, int a, int l, int lc[4], int c[4]) {
  int ac[4];
  site_coords(ag.gc, a, ac);
  int q = l;
  lc[3] = q % ag.agg[3];
  q /= ag.agg[3];
  lc[2] = q % ag.agg[2];
  q /= ag.agg[2];
  lc[1] = q % ag.agg[1];
  lc[0] = q / ag.agg[1];
#pragma unroll
  for (int d = 0; d < 4; ++d) c[d] = ac[d] * ag.agg[d] + lc[d];
  return ((c[0] * ag.g.L[1] + c[1]) * ag.g.L[2] + c[2]) * ag.g.L[3] + c[3];
}

__device__ __forceinline__ int coarse_of(const AggGeom& ag, const int c[4]) {
  return (((c[0] / ag.agg[0]) * ag.gc.L[1] + c[1] / ag.agg[1]) * ag.gc.L[2] + c[2] / ag.agg[2]) * ag.gc.L[3] +
         c[3] / ag.agg[3];
}

// ===========================================================================
// orthonormalisation: per (aggregate, chirality) classical Gram-Schmidt
// applied twice, giving the Q of the thin QR with a real positive R diagonal
// ===========================================================================
template <typename T>
__global__ void k_orthonormalise(T* P, AggGeom ag, int* err) {
  __shared__ T red[32 * 16];
  const int a = blockIdx.x, chi = blockIdx.y, nv = ag.nv;
  const int l = threadIdx.x;
  const bool act = l < ag.asites;
  int lc[4], c[4];
  const int s = act ? agg_site(ag, a, l, lc, c) : 0;
  const long V = ag.g.V;
  const long fstride = (long)NR_SPINOR * V;
  const long choff = 12L * chi * V;  // chunk offset of this chirality's 6 complex numbers
  // squared-norm ratio below which a column counts as linearly dependent
  const T rank_tol = sizeof(T) == 8 ? T(1e-24) : T(1e-10);
  for (int j = 0; j < nv; ++j) {
    cx<T> v[6];
    if (act) ld_cx<T, 6>(P + j * fstride + choff, V, s, v);
    else
      for (int k = 0; k < 6; ++k) v[k] = cx<T>{0, 0};
    T t0[1] = {0};
    for (int k = 0; k < 6; ++k) t0[0] += norm2(v[k]);
    block_allreduce<T, 1>(t0, red);
    const T n0 = t0[0];
    for (int pass = 0; pass < 2; ++pass) {
      for (int i0 = 0; i0 < j; i0 += 8) {
        T d[16];
        for (int m = 0; m < 16; ++m) d[m] = 0;
        if (act) {
          for (int ii = 0; ii < 8 && i0 + ii < j; ++ii) {
            cx<T> q[6];
            ld_cx<T, 6>(P + (i0 + ii) * fstride + choff, V, s, q);
            cx<T> acc{0, 0};
            for (int k = 0; k < 6; ++k) cfmac(acc, q[k], v[k]);
            d[2 * ii] = acc.r;
            d[2 * ii + 1] = acc.i;
          }
        }
        block_allreduce<T, 16>(d, red);
        if (act) {
          for (int ii = 0; ii < 8 && i0 + ii < j; ++ii) {
            cx<T> q[6];
            ld_cx<T, 6>(P + (i0 + ii) * fstride + choff, V, s, q);
            const cx<T> cc{d[2 * ii], d[2 * ii + 1]};
            for (int k = 0; k < 6; ++k) v[k] = v[k] - cc * q[k];
          }
        }
      }
    }
    T t1[1] = {0};
    for (int k = 0; k < 6; ++k) t1[0] += norm2(v[k]);
    block_allreduce<T, 1>(t1, red);
    T nn = t1[0];
    if (!(nn > rank_tol * n0) || !(nn > T(0))) {
      if (l == 0) atomicOr(err, ERRF_RANK);
      nn = T(1);
    }
    const T inv = T(1) / sqrt(nn);
    if (act) {
      for (int k = 0; k < 6; ++k) v[k] = inv * v[k];
      st_cx<T, 6>(P + j * fstride + choff, V, s, v);
    }
    __syncthreads();
  }
}

template <typename T>
void launch_orthonormalise(T* P, const AggGeom& ag, int* err, cudaStream_t st) {
  const int threads = (ag.asites + 31) / 32 * 32;
  dim3 grid(ag.gc.V, 2);
  k_orthonormalise<T><<<grid, threads, 0, st>>>(P, ag, err);
}

// ===========================================================================
// restriction  coarse(a, chi*Nv + i) = sum_{x in a, comp in chi} conj(P_i) fine
// ===========================================================================
// column i of P at site s, stored as T (S = ST_NATIVE) or in 16 bits
template <typename T, int S>
__device__ __forceinline__ void ld_pcol(const void* __restrict__ P, int i, long V, long s, cx<T> (&p)[12]) {
  if constexpr (S == ST_NATIVE)
    ld_cx<T, 12>(static_cast<const T*>(P) + (long)i * NR_SPINOR * V, V, s, p);
  else
    ld_cx16<T, S, 12>(static_cast<const unsigned short*>(P) + (long)i * NR_SPINOR * V, V, s, p);
}

template <typename T, int S>
__global__ void k_restrict(const void* __restrict__ P, const T* __restrict__ fine, T* __restrict__ coarse,
                           AggGeom ag, int nrhs) {
  __shared__ T red[32 * 16];
  __shared__ T fin[16];
  // right-hand sides fastest over the CTAs: an aggregate's P columns are reused from L2
  const int a = blockIdx.x / nrhs, rhs = blockIdx.x % nrhs, nv = ag.nv;
  const int l = threadIdx.x;
  const bool act = l < ag.asites;
  int lc[4], c[4];
  const int s = act ? agg_site(ag, a, l, lc, c) : 0;
  const long V = ag.g.V;
  cx<T> r[12];
  if (act) ld_cx<T, 12>(fine + (long)rhs * NR_SPINOR * V, V, s, r);
  cx<T>* out = reinterpret_cast<cx<T>*>(coarse) + ((long)rhs * ag.gc.V + a) * 2 * nv;
  for (int i0 = 0; i0 < nv; i0 += 4) {
    T d[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) d[m] = 0;
    if (act) {
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) {
        if (i0 + ii < nv) {
          cx<T> p[12];
          ld_pcol<T, S>(P, i0 + ii, V, s, p);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            cx<T> acc{0, 0};
#pragma unroll
            for (int k = 0; k < 6; ++k) cfmac(acc, p[6 * h + k], r[6 * h + k]);
            d[4 * ii + 2 * h] = acc.r;
            d[4 * ii + 2 * h + 1] = acc.i;
          }
        }
      }
    }
    block_reduce16<T>(d, red, fin);
    if (l < 8) {
      const int ii = l >> 1, h = l & 1;
      if (i0 + ii < nv) out[h * nv + i0 + ii] = cx<T>{fin[4 * ii + 2 * h], fin[4 * ii + 2 * h + 1]};
    }
  }
}

template <typename T>
void launch_restrict(const T* P, const T* fine, T* coarse, const AggGeom& ag, int nrhs, cudaStream_t st,
                     const void* P16, int p16) {
  const int threads = (ag.asites + 31) / 32 * 32;
  dim3 grid((unsigned)ag.gc.V * (unsigned)nrhs);
  if (P16 && p16 == ST_F16)
    k_restrict<T, ST_F16><<<grid, threads, 0, st>>>(P16, fine, coarse, ag, nrhs);
  else if (P16 && p16 == ST_BF16)
    k_restrict<T, ST_BF16><<<grid, threads, 0, st>>>(P16, fine, coarse, ag, nrhs);
  else
    k_restrict<T, ST_NATIVE><<<grid, threads, 0, st>>>(P, fine, coarse, ag, nrhs);
}

// ===========================================================================
// prolongation  fine(x, comp in chi) (+)= sum_i P_i(x, comp) coarse(a(x), chi*Nv + i)
// ===========================================================================
// RG right-hand sides per thread: every P value loaded serves all of them
// (with one right-hand side per thread the CTAs of the other right-hand sides
// read P again through L2)
template <typename T, bool ACC, int S, int RG>
__global__ void __launch_bounds__(128) k_prolong(const void* __restrict__ P, const T* __restrict__ coarse,
                                                 T* __restrict__ fine, AggGeom ag, int nrhs) {
  const int ngrp = (nrhs + RG - 1) / RG;
  const int s = (blockIdx.x / ngrp) * blockDim.x + threadIdx.x;  // right-hand-side groups fastest (P reuse)
  const int r0 = (blockIdx.x % ngrp) * RG, R = min(RG, nrhs - r0), nv = ag.nv;
  const long V = ag.g.V;
  if (s >= V) return;
  int c[4];
  site_coords(ag.g, s, c);
  const int a = coarse_of(ag, c);
  const long cstr = (long)ag.gc.V * 2 * nv;  // complex numbers per coarse vector
  const cx<T>* e = reinterpret_cast<const cx<T>*>(coarse) + (long)r0 * cstr + (long)a * 2 * nv;
  T* f = fine + (long)r0 * NR_SPINOR * V;
  cx<T> out[RG][12];
#pragma unroll
  for (int j = 0; j < RG; ++j) {
    if (ACC && j < R) {
      ld_cx<T, 12>(f + (long)j * NR_SPINOR * V, V, s, out[j]);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) out[j][k] = cx<T>{0, 0};
    }
  }
  for (int i = 0; i < nv; ++i) {
    cx<T> p[12];
    ld_pcol<T, S>(P, i, V, s, p);
#pragma unroll
    for (int j = 0; j < RG; ++j) {
      if (j < R) {
        const cx<T> e0 = e[j * cstr + i], e1 = e[j * cstr + nv + i];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          cfma(out[j][k], p[k], e0);
          cfma(out[j][6 + k], p[6 + k], e1);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < RG; ++j)
    if (j < R) st_cx<T, 12>(f + (long)j * NR_SPINOR * V, V, s, out[j]);
}

template <typename T, int S>
void prolong_s(const void* P, const T* coarse, T* fine, const AggGeom& ag, int nrhs, bool accumulate,
               cudaStream_t st) {
  constexpr int RG = sizeof(T) == 4 ? 3 : 1;
  const unsigned ngrp = (unsigned)((nrhs + RG - 1) / RG);
  dim3 grid((unsigned)((ag.g.V + 127) / 128) * ngrp);
  if (accumulate)
    k_prolong<T, true, S, RG><<<grid, 128, 0, st>>>(P, coarse, fine, ag, nrhs);
  else
    k_prolong<T, false, S, RG><<<grid, 128, 0, st>>>(P, coarse, fine, ag, nrhs);
}

template <typename T>
void launch_prolong(const T* P, const T* coarse, T* fine, const AggGeom& ag, int nrhs, bool accumulate,
                    cudaStream_t st, const void* P16, int p16) {
  if (P16 && p16 == ST_F16)
    prolong_s<T, ST_F16>(P16, coarse, fine, ag, nrhs, accumulate, st);
  else if (P16 && p16 == ST_BF16)
    prolong_s<T, ST_BF16>(P16, coarse, fine, ag, nrhs, accumulate, st);
  else
    prolong_s<T, ST_NATIVE>(P, coarse, fine, ag, nrhs, accumulate, st);
}

// 16-bit copy of n_cx FP32 complex numbers (element order kept)
template <int S>
__global__ void k_to16(const float2* __restrict__ in, unsigned* __restrict__ out, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    unsigned u;
    if constexpr (S == ST_F16) {
      const __half2 v = __float22half2_rn(in[i]);
      memcpy(&u, &v, 4);
    } else {
      const __nv_bfloat162 v = __float22bfloat162_rn(in[i]);
      memcpy(&u, &v, 4);
    }
    out[i] = u;
  }
}

void launch_to16(const float* in, void* out, long n_cx, int kind, cudaStream_t st) {
  long b = (n_cx + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (kind == ST_F16)
    k_to16<ST_F16><<<(int)b, 256, 0, st>>>(reinterpret_cast<const float2*>(in), static_cast<unsigned*>(out), n_cx);
  else
    k_to16<ST_BF16><<<(int)b, 256, 0, st>>>(reinterpret_cast<const float2*>(in), static_cast<unsigned*>(out), n_cx);
}

// ===========================================================================
// coarse operator build (local Galerkin projection, mu-free)
//   block 0:        P_a^dagger [A + hops inside a] P_a
//   block 1 + 2 mu: P_a^dagger [hops from a's upper mu-face into a + mu] P_{a+mu}
//   block 2 + 2 mu: P_a^dagger [hops from a's lower mu-face into a - mu] P_{a-mu}
// One CTA per (block t, aggregate a); the operator columns of a tile of sites
// are staged in shared memory, then projected onto P_a^dagger.
// ===========================================================================

// The two chirality columns (chi = 0, 1) of test vector j share the loads of
// P_j and of the link: with P_j masked to chirality 0 the projected half
// spinor is h = p_up, with P_j masked to chirality 1 it is h = -A p_dn, and each
// multiplies the link once.
// acc0/acc1 += sign (1 - gamma_MU) U (P_j masked to chi), U = U_MU(x) at sl
template <typename T, int MU>
__device__ __forceinline__ void hop_fwd_pair(const cx<T> (&p)[12], const T* __restrict__ gauge, int V, int sl,
                                             T sign, cx<T> (&acc0)[12], cx<T> (&acc1)[12]) {
  Link<T> U;
  ld_link(gauge, V, MU, sl, U);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int lo = 3 * (2 + gperm(MU, r)), ph = conjph(gphase(MU, r));
    cx<T> h[3], w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) h[k] = sign * p[3 * r + k];
    su3_mul(U, h, w);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc0[3 * r + k] = acc0[3 * r + k] + w[k];
      acc0[lo + k] = acc0[lo + k] - mulp(w[k], ph);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) h[k] = -sign * mulp(p[lo + k], gphase(MU, r));
    su3_mul(U, h, w);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc1[3 * r + k] = acc1[3 * r + k] + w[k];
      acc1[lo + k] = acc1[lo + k] - mulp(w[k], ph);
    }
  }
}

// acc0/acc1 += sign (1 + gamma_MU) U^dagger (P_j masked to chi), U = U_MU(x - MU) at sl
template <typename T, int MU>
__device__ __forceinline__ void hop_bwd_pair(const cx<T> (&p)[12], const T* __restrict__ gauge, int V, int sl,
                                             T sign, cx<T> (&acc0)[12], cx<T> (&acc1)[12]) {
  Link<T> U;
  ld_link(gauge, V, MU, sl, U);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int lo = 3 * (2 + gperm(MU, r)), ph = conjph(gphase(MU, r));
    cx<T> h[3], w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) h[k] = sign * p[3 * r + k];
    su3_dag_mul(U, h, w);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc0[3 * r + k] = acc0[3 * r + k] + w[k];
      acc0[lo + k] = acc0[lo + k] + mulp(w[k], ph);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) h[k] = sign * mulp(p[lo + k], gphase(MU, r));
    su3_dag_mul(U, h, w);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc1[3 * r + k] = acc1[3 * r + k] + w[k];
      acc1[lo + k] = acc1[lo + k] + mulp(w[k], ph);
    }
  }
}

template <typename T, int MU>
__device__ __forceinline__ void build_hops_pair(const T* __restrict__ P, const T* __restrict__ gauge,
                                                const AggGeom& ag, int s, const int c[4], const int lc[4], int j,
                                                int t, T bc, cx<T> (&acc0)[12], cx<T> (&acc1)[12]) {
  const Lat& g = ag.g;
  const T* Pj = P + (long)j * NR_SPINOR * g.V;
  const bool up = lc[MU] == ag.agg[MU] - 1, lo = lc[MU] == 0;
  // forward hop: inside a for t == 0 unless on the upper face; block 1+2MU on it
  if ((t == 0 && !up) || (t == 1 + 2 * MU && up)) {
    const int sf = nb_fwd(g, s, c, MU);
    cx<T> p[12];
    ld_cx<T, 12>(Pj, g.V, sf, p);
    const T sign = (MU == 0 && c[0] == g.L[0] - 1) ? bc : T(1);
    hop_fwd_pair<T, MU>(p, gauge, g.V, s, sign, acc0, acc1);
  }
  if ((t == 0 && !lo) || (t == 2 + 2 * MU && lo)) {
    const int sb = nb_bwd(g, s, c, MU);
    cx<T> p[12];
    ld_cx<T, 12>(Pj, g.V, sb, p);
    const T sign = (MU == 0 && c[0] == 0) ? bc : T(1);
    hop_bwd_pair<T, MU>(p, gauge, g.V, sb, sign, acc0, acc1);
  }
}

// operator columns k = j (chi = 0) and k = Nv + j (chi = 1) of block t at fine
// site s of aggregate a: u_chi = [D restricted to block t] (P_j masked to chi)
template <typename T>
__device__ __forceinline__ void column_op_pair(const T* __restrict__ gauge, const T* __restrict__ clover,
                                               const T* __restrict__ P, const AggGeom& ag, int s, const int c[4],
                                               const int lc[4], int j, int t, T bc, T rho, cx<T> (&u0)[12],
                                               cx<T> (&u1)[12]) {
  cx<T> acc0[12], acc1[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) acc0[q] = acc1[q] = cx<T>{0, 0};
  build_hops_pair<T, 0>(P, gauge, ag, s, c, lc, j, t, bc, acc0, acc1);
  build_hops_pair<T, 1>(P, gauge, ag, s, c, lc, j, t, bc, acc0, acc1);
  build_hops_pair<T, 2>(P, gauge, ag, s, c, lc, j, t, bc, acc0, acc1);
  build_hops_pair<T, 3>(P, gauge, ag, s, c, lc, j, t, bc, acc0, acc1);
  if (t == 0) {
    // the clover term is block diagonal in chirality: A P_j splits into the
    // chirality-0 rows of column j and the chirality-1 rows of column Nv + j;
    // an odd-site twisted-mass shift rho (i rho gamma5, also chirality
    // diagonal) is projected with it, the common twisted mass is added at apply
    cx<T> p[12], y[12];
    ld_cx<T, 12>(P + (long)j * NR_SPINOR * ag.g.V, ag.g.V, s, p);
    site_diag<T>(clover, ag.g.V, s, ((c[0] + c[1] + c[2] + c[3]) & 1) ? rho : T(0), p, y);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      u0[q] = y[q];
      u0[6 + q] = cx<T>{0, 0};
      u1[q] = cx<T>{0, 0};
      u1[6 + q] = y[6 + q];
    }
  } else {
#pragma unroll
    for (int q = 0; q < 12; ++q) u0[q] = u1[q] = cx<T>{0, 0};
  }
#pragma unroll
  for (int q = 0; q < 12; ++q) {
    u0[q] = u0[q] - T(0.5) * acc0[q];
    u1[q] = u1[q] - T(0.5) * acc1[q];
  }
}

// local site index within the aggregate of the f-th site that block t visits
// (all sites for t = 0, the sites of the crossed face otherwise)
__device__ __forceinline__ int block_site(const AggGeom& ag, int t, int f) {
  if (t == 0) return f;
  const int mu = (t - 1) >> 1;
  const int fixed = ((t - 1) & 1) ? 0 : ag.agg[mu] - 1;
  int lc[4], q = f;
#pragma unroll
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

constexpr int kBuildThreads = 256;
// register tiles of the projection: a thread owns kTR rows (one chirality) x KTC
// columns of a block, so every P value it loads from shared memory serves KTC
// outputs and every operator value kTR outputs; one tile per thread, KTC the
// smallest of 2, 3, 4 with 2 ceil(Nv / kTR) ceil(2 Nv / KTC) <= 256 tiles
// (KTC = 2 up to Nv = 21, 3 up to 27, 4 for 28)
constexpr int kTR = 4;

__host__ __device__ constexpr int build_tiles(int nv, int ktc) {
  return 2 * ((nv + kTR - 1) / kTR) * ((2 * nv + ktc - 1) / ktc);
}

// row strides (in complex numbers) of the staged P values and operator columns:
// each holds 12 * width entries of one site, padded to 1 mod 16 so that the
// threads of a warp, which take consecutive sites, store to distinct banks
__host__ __device__ __forceinline__ int build_row_stride(int width) {
  return 12 * width + ((1 - 12 * width) % 16 + 16) % 16;
}

// D_c(a, t) = P_a^dagger U_t, U_t = the 2 Nv operator columns of block t.
// One CTA per (t, a); the visited sites are processed in tiles of TS sites
// whose P values and U columns are staged in shared memory as
//   Ps[l * LP + comp * Nv + i],  Us[l * LU + comp * 2Nv + k],
// the staging threads taking consecutive sites so that neighbouring threads
// read neighbouring fine sites; then every thread accumulates its fixed
// outputs (row, col) in registers.
template <typename T, int KTC>
__global__ void __launch_bounds__(kBuildThreads, sizeof(T) == 4 ? 2 : 1) k_coarse_build(const T* __restrict__ gauge,
                                                                const T* __restrict__ clover,
                                                                const T* __restrict__ P, T* __restrict__ Dc,
                                                                AggGeom ag, T bc, int TS, T rho) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nv = ag.nv, n = 2 * nv;
  const int LP = build_row_stride(nv), LU = build_row_stride(n);
  cx<T>* Ps = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* Us = Ps + (size_t)TS * LP;
  const int t = blockIdx.x, a = blockIdx.y;
  const int nsites = t == 0 ? ag.asites : ag.asites / ag.agg[(t - 1) >> 1];
  const long V = ag.g.V;
  const int nib = (nv + kTR - 1) / kTR, nkb = (n + KTC - 1) / KTC;
  const bool owner = threadIdx.x < 2 * nib * nkb;
  cx<T> acc[kTR][KTC];
#pragma unroll
  for (int ri = 0; ri < kTR; ++ri)
#pragma unroll
    for (int kj = 0; kj < KTC; ++kj) acc[ri][kj] = cx<T>{0, 0};

  for (int f0 = 0; f0 < nsites; f0 += TS) {
    const int ts = min(TS, nsites - f0);
    // stage P_i at the tile's sites
    for (int e = threadIdx.x; e < ts * nv; e += blockDim.x) {
      const int l = e % ts, i = e / ts;
      int lc[4], c[4];
      const int s = agg_site(ag, a, block_site(ag, t, f0 + l), lc, c);
      cx<T> p[12];
      ld_cx<T, 12>(P + (long)i * NR_SPINOR * V, V, s, p);
#pragma unroll
      for (int q = 0; q < 12; ++q) Ps[(size_t)l * LP + q * nv + i] = p[q];
    }
    // operator columns at the tile's sites, both chiralities of one test vector per thread
    for (int e = threadIdx.x; e < ts * nv; e += blockDim.x) {
      const int l = e % ts, j = e / ts;
      int lc[4], c[4];
      const int s = agg_site(ag, a, block_site(ag, t, f0 + l), lc, c);
      cx<T> u0[12], u1[12];
      column_op_pair<T>(gauge, clover, P, ag, s, c, lc, j, t, bc, rho, u0, u1);
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        Us[(size_t)l * LU + q * n + j] = u0[q];
        Us[(size_t)l * LU + q * n + nv + j] = u1[q];
      }
    }
    __syncthreads();
    if (owner) {
      const int chi = threadIdx.x / (nib * nkb), rem = threadIdx.x % (nib * nkb);
      const int i0 = (rem / nkb) * kTR, k0 = (rem % nkb) * KTC;
      for (int l = 0; l < ts; ++l) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const cx<T>* pr = Ps + (size_t)l * LP + (6 * chi + q) * nv;
          const cx<T>* ur = Us + (size_t)l * LU + (6 * chi + q) * n;
          cx<T> pv[kTR], uv[KTC];
#pragma unroll
          for (int ri = 0; ri < kTR; ++ri) pv[ri] = i0 + ri < nv ? pr[i0 + ri] : cx<T>{0, 0};
#pragma unroll
          for (int kj = 0; kj < KTC; ++kj) uv[kj] = k0 + kj < n ? ur[k0 + kj] : cx<T>{0, 0};
#pragma unroll
          for (int ri = 0; ri < kTR; ++ri)
#pragma unroll
            for (int kj = 0; kj < KTC; ++kj) cfmac(acc[ri][kj], pv[ri], uv[kj]);
        }
      }
    }
    __syncthreads();
  }
  if (owner) {
    const int chi = threadIdx.x / (nib * nkb), rem = threadIdx.x % (nib * nkb);
    const int i0 = (rem / nkb) * kTR, k0 = (rem % nkb) * KTC;
    T* out = Dc + ((long)a * 9 + t) * n * n * 2;
#pragma unroll
    for (int ri = 0; ri < kTR; ++ri)
#pragma unroll
      for (int kj = 0; kj < KTC; ++kj) {
        const int row = chi * nv + i0 + ri, k = k0 + kj;
        if (i0 + ri < nv && k < n) {
          out[2 * ((long)k * n + row)] = acc[ri][kj].r;
          out[2 * ((long)k * n + row) + 1] = acc[ri][kj].i;
        }
      }
  }
}

// largest staged tile (sites) that keeps two CTAs per SM
static int build_ts_max(int nv, size_t real_bytes) {
  const size_t per_site = (size_t)(build_row_stride(nv) + build_row_stride(2 * nv)) * 2 * real_bytes;
  const size_t budget = 100 * 1024;
  int ts_max = (int)(budget / per_site);
  if (ts_max > 16) ts_max = 16;
  return ts_max < 1 ? 1 : ts_max;
}

BuildShape coarse_build_default(int nv, size_t real_bytes) {
  BuildShape b;
  // tile size whose TS * N_v staging items fill the CTA's rounds best (the
  // projection work does not depend on it); ties go to the larger tile
  double best = 0;
  for (int ts = 1; ts <= build_ts_max(nv, real_bytes); ++ts) {
    const int items = ts * nv, rounds = (items + kBuildThreads - 1) / kBuildThreads;
    const double fill = (double)items / (rounds * kBuildThreads);
    if (fill >= best) {
      best = fill;
      b.ts = ts;
    }
  }
  b.ktc = build_tiles(nv, 2) <= kBuildThreads ? 2 : build_tiles(nv, 3) <= kBuildThreads ? 3 : 4;
  return b;
}

std::vector<BuildShape> coarse_build_candidates(int nv, size_t real_bytes) {
  std::vector<BuildShape> out;
  for (int ktc = 2; ktc <= 4; ++ktc) {
    if (build_tiles(nv, ktc) > kBuildThreads) continue;
    for (int ts = 1; ts <= build_ts_max(nv, real_bytes); ++ts) out.push_back(BuildShape{ts, ktc});
  }
  return out;
}

// Every shape sums each D_c entry over the same sites and components in the
// same order, so all shapes give bit-identical blocks.
template <typename T>
void launch_coarse_build(const T* gauge, const T* clover, const T* P, T* Dc, const AggGeom& ag, double bc_t,
                         cudaStream_t st, BuildShape shape, double rho) {
  const int nv = ag.nv;
  const size_t per_site = (size_t)(build_row_stride(nv) + build_row_stride(2 * nv)) * sizeof(cx<T>);  // Ps + Us
  const BuildShape def = coarse_build_default(nv, sizeof(T));
  int TS = shape.ts > 0 ? shape.ts : def.ts;
  int ktc = shape.ktc > 0 ? shape.ktc : def.ktc;
  if (TS > build_ts_max(nv, sizeof(T)) || ktc < 2 || ktc > 4 || build_tiles(nv, ktc) > kBuildThreads) {
    TS = def.ts;  // a shape outside the candidate set falls back to the default
    ktc = def.ktc;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_coarse_build<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_coarse_build<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_coarse_build<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  dim3 grid(9, ag.gc.V);
  const size_t smem = TS * per_site;
  if (ktc == 2)
    k_coarse_build<T, 2><<<grid, kBuildThreads, smem, st>>>(gauge, clover, P, Dc, ag, (T)bc_t, TS, (T)rho);
  else if (ktc == 3)
    k_coarse_build<T, 3><<<grid, kBuildThreads, smem, st>>>(gauge, clover, P, Dc, ag, (T)bc_t, TS, (T)rho);
  else
    k_coarse_build<T, 4><<<grid, kBuildThreads, smem, st>>>(gauge, clover, P, Dc, ag, (T)bc_t, TS, (T)rho);
}

// number of 32-bit words in which a and b differ, added to *count
__global__ void k_count_mismatch(const unsigned* __restrict__ a, const unsigned* __restrict__ b, long n,
                                 unsigned long long* count) {
  unsigned long long c = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    c += a[i] != b[i];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

void launch_count_mismatch(const void* a, const void* b, long words, unsigned long long* count, cudaStream_t st) {
  long blocks = (words + 255) / 256;
  if (blocks > 152L * 8) blocks = 152L * 8;
  if (blocks < 1) blocks = 1;
  k_count_mismatch<<<(unsigned)blocks, 256, 0, st>>>(static_cast<const unsigned*>(a), static_cast<const unsigned*>(b),
                                                     words, count);
}

static_assert(build_tiles(21, 2) <= kBuildThreads && build_tiles(27, 3) <= kBuildThreads &&
                  build_tiles(28, 4) <= kBuildThreads,
              "one register tile per thread up to Nv = 28");

// ===========================================================================
// coarse stencil helpers
// ===========================================================================
// neighbour of coarse site a for block t (t = 0 self)
__device__ __forceinline__ int coarse_nb(const Lat& gc, int a, int t) {
  if (t == 0) return a;
  int c[4];
  site_coords(gc, a, c);
  const int mu = (t - 1) >> 1;
  return ((t - 1) & 1) ? nb_bwd(gc, a, c, mu) : nb_fwd(gc, a, c, mu);
}

// y = D_c(mu_c) v on the full coarse lattice; CTA per coarse site,
// threads (t, row): partial sums over columns, reduced over t in shared memory
template <typename T>
__global__ void k_coarse_apply(const T* __restrict__ Dc, const T* __restrict__ v, T* __restrict__ y, Lat gc, int nv,
                               T mu_c, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* part = reinterpret_cast<cx<T>*>(smem_raw);  // [9][n]
  const int n = 2 * nv;
  const int a = blockIdx.x / nrhs, rhs = blockIdx.x % nrhs;  // right-hand sides fastest (block reuse in L2)
  const int row = threadIdx.x % n, t = threadIdx.x / n;
  const cx<T>* vv = reinterpret_cast<const cx<T>*>(v) + (long)rhs * gc.V * n;
  if (t < 9) {
    const int nb = coarse_nb(gc, a, t);
    const cx<T>* src = vv + (long)nb * n;
    const cx<T>* B = reinterpret_cast<const cx<T>*>(Dc) + ((long)a * 9 + t) * n * n;
    cx<T> acc{0, 0};
#pragma unroll 8
    for (int col = 0; col < n; ++col) cfma(acc, B[(long)col * n + row], src[col]);
    part[t * n + row] = acc;
  }
  __syncthreads();
  if (threadIdx.x < n) {
    cx<T> acc = part[row];
    for (int q = 1; q < 9; ++q) acc = acc + part[q * n + row];
    const cx<T> x = vv[(long)a * n + row];
    const T sg = row < nv ? -mu_c : mu_c;  // i mu_c Gamma5_c
    acc.r -= sg * x.i;
    acc.i += sg * x.r;
    reinterpret_cast<cx<T>*>(y)[(long)rhs * gc.V * n + (long)a * n + row] = acc;
  }
}

// the same for up to RB right-hand sides per CTA: each block entry a thread
// loads serves all of them (one CTA per right-hand side reads every block
// once per right-hand side through L2)
template <typename T, int RB, int S>
__global__ void k_coarse_apply_b(const void* __restrict__ Dc, const T* __restrict__ v, T* __restrict__ y, Lat gc,
                                 int nv, T mu_c, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* part = reinterpret_cast<cx<T>*>(smem_raw);  // [RB][9][n]
  const int n = 2 * nv;
  const int ngrp = (nrhs + RB - 1) / RB;
  const int a = blockIdx.x / ngrp, r0 = (blockIdx.x % ngrp) * RB, R = min(RB, nrhs - r0);
  const int row = threadIdx.x % n, t = threadIdx.x / n;
  const long vs = (long)gc.V * n;
  const cx<T>* vv = reinterpret_cast<const cx<T>*>(v) + r0 * vs;
  if (t < 9) {
    const int nb = coarse_nb(gc, a, t);
    const long B = ((long)a * 9 + t) * n * n;
    cx<T> acc[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) acc[j] = cx<T>{0, 0};
#pragma unroll 4
    for (int col = 0; col < n; ++col) {
      cx<T> m;
      if constexpr (S == ST_NATIVE) {
        m = reinterpret_cast<const cx<T>*>(Dc)[B + (long)col * n + row];
      } else {
        const float2 f = unpack16x2<S>(__ldg(reinterpret_cast<const unsigned*>(Dc) + B + (long)col * n + row));
        m = cx<T>{(T)f.x, (T)f.y};
      }
#pragma unroll
      for (int j = 0; j < RB; ++j)
        if (j < R) cfma(acc[j], m, vv[j * vs + (long)nb * n + col]);
    }
#pragma unroll
    for (int j = 0; j < RB; ++j) part[(j * 9 + t) * n + row] = acc[j];
  }
  __syncthreads();
  if (threadIdx.x < n) {
    const T sg = row < nv ? -mu_c : mu_c;  // i mu_c Gamma5_c
    for (int j = 0; j < R; ++j) {
      cx<T> acc = part[(j * 9) * n + row];
      for (int q = 1; q < 9; ++q) acc = acc + part[(j * 9 + q) * n + row];
      const cx<T> x = vv[j * vs + (long)a * n + row];
      acc.r -= sg * x.i;
      acc.i += sg * x.r;
      reinterpret_cast<cx<T>*>(y)[(r0 + j) * vs + (long)a * n + row] = acc;
    }
  }
}

template <typename T>
void launch_coarse_apply(const T* Dc, const T* v, T* y, const Lat& gc, int nv, double mu_c, int nrhs,
                         cudaStream_t st, const void* Dc16, int kind16) {
  const int n = 2 * nv;
  const int threads = (9 * n + 31) / 32 * 32;
  if ((nrhs > 1 || Dc16) && sizeof(T) == 4) {
    constexpr int RB = 6;
    const unsigned ngrp = (unsigned)((nrhs + RB - 1) / RB);
    const size_t sm = (size_t)RB * 9 * n * sizeof(cx<T>);
    if (Dc16 && kind16 == ST_BF16)
      k_coarse_apply_b<T, RB, ST_BF16><<<(unsigned)gc.V * ngrp, threads, sm, st>>>(Dc16, v, y, gc, nv, (T)mu_c, nrhs);
    else if (Dc16)
      k_coarse_apply_b<T, RB, ST_F16><<<(unsigned)gc.V * ngrp, threads, sm, st>>>(Dc16, v, y, gc, nv, (T)mu_c, nrhs);
    else
      k_coarse_apply_b<T, RB, ST_NATIVE><<<(unsigned)gc.V * ngrp, threads, sm, st>>>(Dc, v, y, gc, nv, (T)mu_c, nrhs);
    return;
  }
  dim3 grid((unsigned)gc.V * (unsigned)nrhs);
  k_coarse_apply<T><<<grid, threads, 9 * n * sizeof(cx<T>), st>>>(Dc, v, y, gc, nv, (T)mu_c, nrhs);
}

// ===========================================================================
// odd-even on the coarse lattice
// ===========================================================================
// Gauss-Jordan inverse with partial pivoting of (self block + i mu_c G5c) at each odd site
template <typename T>
__global__ void k_oe_invert(const T* __restrict__ Dc, T* __restrict__ Dinv, OEGeom oe, T mu_c, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = 2 * oe.nv, w = 2 * n;
  cx<T>* M = reinterpret_cast<cx<T>*>(smem_raw);  // [n][2n] row-major augmented
  __shared__ int piv;
  __shared__ T fac_r[128], fac_i[128];
  const int k = blockIdx.x;
  const int a = oe.odd_site[k];
  const cx<T>* B = reinterpret_cast<const cx<T>*>(Dc) + (long)a * 9 * n * n;
  for (int e = threadIdx.x; e < n * w; e += blockDim.x) {
    const int r = e / w, cc = e % w;
    cx<T> val{0, 0};
    if (cc < n) {
      val = B[(long)cc * n + r];
      if (cc == r) val.i += (r < oe.nv ? -mu_c : mu_c);
    } else if (cc - n == r) {
      val = cx<T>{1, 0};
    }
    M[r * w + cc] = val;
  }
  __syncthreads();
  for (int col = 0; col < n; ++col) {
    if (threadIdx.x == 0) {
      int p = col;
      T best = norm2(M[col * w + col]);
      for (int r = col + 1; r < n; ++r) {
        const T v = norm2(M[r * w + col]);
        if (v > best) {
          best = v;
          p = r;
        }
      }
      if (!(best > T(0))) atomicOr(err, ERRF_SINGULAR);
      piv = p;
    }
    __syncthreads();
    const int p = piv;
    if (p != col) {
      for (int cc = threadIdx.x; cc < w; cc += blockDim.x) {
        const cx<T> tmp = M[col * w + cc];
        M[col * w + cc] = M[p * w + cc];
        M[p * w + cc] = tmp;
      }
    }
    __syncthreads();
    cx<T> pv = M[col * w + col];
    const T den = norm2(pv);
    const cx<T> inv = den > T(0) ? cx<T>{pv.r / den, -pv.i / den} : cx<T>{0, 0};
    __syncthreads();
    for (int cc = threadIdx.x; cc < w; cc += blockDim.x) M[col * w + cc] = M[col * w + cc] * inv;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      fac_r[r] = M[r * w + col].r;
      fac_i[r] = M[r * w + col].i;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * w; e += blockDim.x) {
      const int r = e / w, cc = e % w;
      if (r != col) {
        const cx<T> f{fac_r[r], fac_i[r]};
        M[r * w + cc] = M[r * w + cc] - f * M[col * w + cc];
      }
    }
    __syncthreads();
  }
  cx<T>* out = reinterpret_cast<cx<T>*>(Dinv) + (long)k * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int cc = e / n, r = e % n;  // column-major output
    out[(long)cc * n + r] = M[r * w + n + cc];
  }
}

template <typename T>
void launch_oe_invert(const T* Dc, T* Dinv, const OEGeom& oe, double mu_c, int* err, cudaStream_t st) {
  const int n = 2 * oe.nv;
  const size_t smem = (size_t)n * 2 * n * sizeof(cx<T>);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_oe_invert<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_oe_invert<T><<<oe.nhalf, 256, smem, st>>>(Dc, Dinv, oe, (T)mu_c, err);
}

// Generic odd-even stencil piece on sites of one parity (compact index k):
//   acc = pre + sgn * sum_{t=1..8} B_t(site) src(nb_t(site))   [src compact, other parity]
//   out = post ? Dinv(k) acc : acc
// pre: 0 (mode 0), (self + i mu_c G5c) v(site) with v compact (mode 1), or
// b(site) with b a full coarse vector (mode 2).
template <typename T>
struct OEArgs {
  const T* Dc;
  const T* Dinv;
  const T* src;   // compact, other parity
  const T* pre;   // mode 1: compact same parity; mode 2: full vector
  T* out;         // compact (or full when full_out)
  OEGeom oe;
  T mu_c;
  T sgn;
  int mode;
  int odd;        // target parity
  int post;       // multiply by Dinv (odd targets only)
  int full_out;   // write into a full coarse vector at the site
  // batch over right-hand sides (blockIdx.y): per-rhs strides in reals and an
  // optional mask of active right-hand sides
  long s_str, p_str, o_str;
  const int* active;
};

// Several right-hand sides per CTA: the CTA lists the active right-hand
// sides and takes group blockIdx.y of RB of them; it stages the group's
// source vectors at the site's 8 neighbours (and its own, mode 1) in shared
// memory, then thread (t, row) applies row `row` of block t to all RB of them,
// so every D_c entry it loads is used RB times and the vector reads are
// shared-memory broadcasts.
template <typename T, int RB>
__global__ void k_oe_stencil_mr(OEArgs<T> a, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nv = a.oe.nv, n = 2 * nv;
  cx<T>* xs = reinterpret_cast<cx<T>*>(smem_raw);      // [9][RB][n] sources
  cx<T>* part = xs + (size_t)9 * RB * n;                // [RB][9][n]
  cx<T>* accs = part + (size_t)RB * 9 * n;              // [RB][n]
  int* lst = reinterpret_cast<int*>(accs + (size_t)RB * n);  // [nrhs]
  __shared__ int nact;
  const int k = blockIdx.x;
  const int site = a.odd ? a.oe.odd_site[k] : a.oe.even_site[k];
  const int row = threadIdx.x % n, t = threadIdx.x / n;
  const cx<T>* B = reinterpret_cast<const cx<T>*>(a.Dc) + (long)site * 9 * n * n;
  if (threadIdx.x == 0) {
    int c = 0;
    for (int r = 0; r < nrhs; ++r)
      if (!a.active || a.active[r]) lst[c++] = r;
    nact = c;
  }
  __syncthreads();
  const int g0 = blockIdx.y * RB;
  if (g0 >= nact) return;  // uniform over the CTA
  const int gn = min(RB, nact - g0);
  // stage the sources
  for (int e = threadIdx.x; e < 9 * gn * n; e += blockDim.x) {
    const int tt = e / (gn * n), q = (e / n) % gn, col = e % n;
    const int r = lst[g0 + q];
    cx<T> v{0, 0};
    if (tt == 0) {
      if (a.mode == 1) v = reinterpret_cast<const cx<T>*>(a.pre + r * a.p_str)[(long)k * n + col];
    } else {
      const int nb = coarse_nb(a.oe.gc, site, tt);
      v = reinterpret_cast<const cx<T>*>(a.src + r * a.s_str)[(long)a.oe.cidx[nb] * n + col];
    }
    xs[((size_t)tt * RB + q) * n + col] = v;
  }
  __syncthreads();
  if (t < 9) {
    cx<T> acc[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) acc[q] = cx<T>{0, 0};
    const bool apply = t > 0 || a.mode == 1;
    if (apply) {
      const cx<T>* Bt = B + (long)t * n * n;
      const cx<T>* xt = xs + (size_t)t * RB * n;
#pragma unroll 8
      for (int col = 0; col < n; ++col) {
        const cx<T> bv = Bt[(long)col * n + row];
#pragma unroll
        for (int q = 0; q < RB; ++q)
          if (q < gn) cfma(acc[q], bv, xt[(size_t)q * n + col]);
      }
    }
    if (t == 0) {
      if (a.mode == 1) {
        const T sg = row < nv ? -a.mu_c : a.mu_c;  // i mu_c Gamma5_c
#pragma unroll
        for (int q = 0; q < RB; ++q)
          if (q < gn) {
            const cx<T> x = xs[(size_t)q * n + row];
            acc[q].r -= sg * x.i;
            acc[q].i += sg * x.r;
          }
      } else if (a.mode == 2) {
#pragma unroll
        for (int q = 0; q < RB; ++q)
          if (q < gn) acc[q] = reinterpret_cast<const cx<T>*>(a.pre + lst[g0 + q] * a.p_str)[(long)site * n + row];
      }
    } else {
#pragma unroll
      for (int q = 0; q < RB; ++q) acc[q] = a.sgn * acc[q];
    }
#pragma unroll
    for (int q = 0; q < RB; ++q)
      if (q < gn) part[((size_t)q * 9 + t) * n + row] = acc[q];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < gn * n; e += blockDim.x) {
    const int q = e / n, rr = e % n;
    cx<T> sum = part[((size_t)q * 9) * n + rr];
    for (int tt = 1; tt < 9; ++tt) sum = sum + part[((size_t)q * 9 + tt) * n + rr];
    accs[(size_t)q * n + rr] = sum;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < gn * n; e += blockDim.x) {
    const int q = e / n, rr = e % n;
    cx<T> res = accs[(size_t)q * n + rr];
    if (a.post) {
      const cx<T>* Di = reinterpret_cast<const cx<T>*>(a.Dinv) + (long)k * n * n;
      res = cx<T>{0, 0};
#pragma unroll 8
      for (int col = 0; col < n; ++col) cfma(res, Di[(long)col * n + rr], accs[(size_t)q * n + col]);
    }
    cx<T>* out = reinterpret_cast<cx<T>*>(a.out + lst[g0 + q] * a.o_str);
    if (a.full_out)
      out[(long)site * n + rr] = res;
    else
      out[(long)k * n + rr] = res;
  }
}

template <typename T, int RB>
static void launch_oe_mr(const OEArgs<T>& a, cudaStream_t st, int nrhs) {
  const int n = 2 * a.oe.nv;
  const int threads = (9 * n + 31) / 32 * 32;
  const size_t smem = (size_t)RB * 19 * n * sizeof(cx<T>) + (size_t)nrhs * sizeof(int);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_oe_stencil_mr<T, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  dim3 grid(a.oe.nhalf, (nrhs + RB - 1) / RB);
  k_oe_stencil_mr<T, RB><<<grid, threads, smem, st>>>(a, nrhs);
}

// right-hand sides per CTA for batched launches (FP32 covers 12 point sources)
template <typename T>
constexpr int oe_batch_rb() { return sizeof(T) == 4 ? 12 : 4; }

template <typename T>
static void launch_oe_stencil(const OEArgs<T>& a, cudaStream_t st, int nrhs = 1) {
  if (nrhs == 1)
    launch_oe_mr<T, 1>(a, st, 1);
  else
    launch_oe_mr<T, oe_batch_rb<T>()>(a, st, nrhs);
}

template <typename T>
void launch_oe_hop_inv(const T* Dc, const T* Dinv, const T* ve, T* uo, const OEGeom& oe, cudaStream_t st) {
  OEArgs<T> a{Dc, Dinv, ve, nullptr, uo, oe, T(0), T(1), 0, 1, 1, 0, 0, 0, 0, nullptr};
  launch_oe_stencil(a, st);
}
template <typename T>
void launch_oe_even(const T* Dc, const T* ve, const T* uo, T* ye, const OEGeom& oe, double mu_c, int diag,
                    cudaStream_t st) {
  OEArgs<T> a{Dc, nullptr, uo, ve, ye, oe, (T)mu_c, T(-1), diag ? 1 : 0, 0, 0, 0, 0, 0, 0, nullptr};
  launch_oe_stencil(a, st);
}
template <typename T>
void launch_oe_rhs(const T* Dc, const T* b, const T* to, T* bh, const OEGeom& oe, cudaStream_t st) {
  OEArgs<T> a{Dc, nullptr, to, b, bh, oe, T(0), T(-1), 2, 0, 0, 0, 0, 0, 0, nullptr};
  launch_oe_stencil(a, st);
}

// t_o = Dinv b_o  (b full); CTA per odd site, thread per row
template <typename T>
__global__ void k_oe_inv_odd(const T* __restrict__ Dinv, const T* __restrict__ b, T* __restrict__ to, OEGeom oe) {
  const int n = 2 * oe.nv;
  const int k = blockIdx.x, row = threadIdx.x;
  if (row >= n) return;
  const int site = oe.odd_site[k];
  const cx<T>* bb = reinterpret_cast<const cx<T>*>(b) + (long)site * n;
  const cx<T>* Di = reinterpret_cast<const cx<T>*>(Dinv) + (long)k * n * n;
  cx<T> acc{0, 0};
#pragma unroll 8
  for (int col = 0; col < n; ++col) cfma(acc, Di[(long)col * n + row], bb[col]);
  reinterpret_cast<cx<T>*>(to)[(long)k * n + row] = acc;
}

template <typename T>
void launch_oe_inv_odd(const T* Dinv, const T* b, T* to, const OEGeom& oe, cudaStream_t st) {
  const int n = 2 * oe.nv;
  k_oe_inv_odd<T><<<oe.nhalf, (n + 31) / 32 * 32, 0, st>>>(Dinv, b, to, oe);
}

// scatter the compact even solution into the full vector
template <typename T>
__global__ void k_oe_scatter_even(const T* __restrict__ xe, T* __restrict__ x, OEGeom oe) {
  const int n = 2 * oe.nv;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)oe.nhalf * n) return;
  const int k = (int)(e / n), row = (int)(e % n);
  reinterpret_cast<cx<T>*>(x)[(long)oe.even_site[k] * n + row] = reinterpret_cast<const cx<T>*>(xe)[e];
}

template <typename T>
void launch_oe_reconstruct(const T* Dc, const T* Dinv, const T* b, const T* xe, T* x, const OEGeom& oe,
                           cudaStream_t st) {
  const int n = 2 * oe.nv;
  const long tot = (long)oe.nhalf * n;
  k_oe_scatter_even<T><<<(int)((tot + 255) / 256), 256, 0, st>>>(xe, x, oe);
  OEArgs<T> a{Dc, Dinv, xe, b, x, oe, T(0), T(-1), 2, 1, 1, 1, 0, 0, 0, nullptr};
  launch_oe_stencil(a, st);
}

// ---- batched odd-even pieces (one launch for nrhs right-hand sides) -------
template <typename T>
__global__ void k_oe_inv_odd_b(const T* __restrict__ Dinv, const T* __restrict__ b, T* __restrict__ to, OEGeom oe,
                               long bstr, long tstr, const int* __restrict__ active) {
  const int n = 2 * oe.nv;
  const int k = blockIdx.x, row = threadIdx.x, r = blockIdx.y;
  if (row >= n || (active && !active[r])) return;
  const int site = oe.odd_site[k];
  const cx<T>* bb = reinterpret_cast<const cx<T>*>(b + r * bstr) + (long)site * n;
  const cx<T>* Di = reinterpret_cast<const cx<T>*>(Dinv) + (long)k * n * n;
  cx<T> acc{0, 0};
#pragma unroll 8
  for (int col = 0; col < n; ++col) cfma(acc, Di[(long)col * n + row], bb[col]);
  reinterpret_cast<cx<T>*>(to + r * tstr)[(long)k * n + row] = acc;
}

template <typename T>
__global__ void k_oe_scatter_even_b(const T* __restrict__ xe, T* __restrict__ x, OEGeom oe, long estr, long xstr,
                                    const int* __restrict__ active) {
  const int n = 2 * oe.nv, r = blockIdx.y;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)oe.nhalf * n || (active && !active[r])) return;
  const int k = (int)(e / n), row = (int)(e % n);
  reinterpret_cast<cx<T>*>(x + r * xstr)[(long)oe.even_site[k] * n + row] =
      reinterpret_cast<const cx<T>*>(xe + r * estr)[e];
}

template <typename T>
void launch_oe_schur_b(const T* Dc, const T* Dinv, const T* ve, T* uo, T* ye, const OEGeom& oe, double mu_c,
                       int nrhs, long vstr, long ustr, long ystr, const int* active, cudaStream_t st) {
  OEArgs<T> h1{Dc, Dinv, ve, nullptr, uo, oe, T(0), T(1), 0, 1, 1, 0, vstr, 0, ustr, active};
  launch_oe_stencil(h1, st, nrhs);
  OEArgs<T> h2{Dc, nullptr, uo, ve, ye, oe, (T)mu_c, T(-1), 1, 0, 0, 0, ustr, vstr, ystr, active};
  launch_oe_stencil(h2, st, nrhs);
}

template <typename T>
void launch_oe_prepare_b(const T* Dc, const T* Dinv, const T* b, T* to, T* bh, const OEGeom& oe, int nrhs,
                         long bstr, long cstr, cudaStream_t st) {
  const int n = 2 * oe.nv;
  dim3 g1(oe.nhalf, nrhs);
  k_oe_inv_odd_b<T><<<g1, (n + 31) / 32 * 32, 0, st>>>(Dinv, b, to, oe, bstr, cstr, nullptr);
  OEArgs<T> a{Dc, nullptr, to, b, bh, oe, T(0), T(-1), 2, 0, 0, 0, cstr, bstr, cstr, nullptr};
  launch_oe_stencil(a, st, nrhs);
}

template <typename T>
void launch_oe_reconstruct_b(const T* Dc, const T* Dinv, const T* b, const T* xe, T* x, const OEGeom& oe, int nrhs,
                             long bstr, long estr, cudaStream_t st) {
  const int n = 2 * oe.nv;
  const long tot = (long)oe.nhalf * n;
  dim3 g1((int)((tot + 255) / 256), nrhs);
  k_oe_scatter_even_b<T><<<g1, 256, 0, st>>>(xe, x, oe, estr, bstr, nullptr);
  OEArgs<T> a{Dc, Dinv, xe, b, x, oe, T(0), T(-1), 2, 1, 1, 1, estr, bstr, bstr, nullptr};
  launch_oe_stencil(a, st, nrhs);
}

#define TM_INST_B(T)                                                                                              \
  template void launch_oe_schur_b<T>(const T*, const T*, const T*, T*, T*, const OEGeom&, double, int, long, long, \
                                     long, const int*, cudaStream_t);                                             \
  template void launch_oe_prepare_b<T>(const T*, const T*, const T*, T*, T*, const OEGeom&, int, long, long,      \
                                       cudaStream_t);                                                             \
  template void launch_oe_reconstruct_b<T>(const T*, const T*, const T*, const T*, T*, const OEGeom&, int, long,  \
                                           long, cudaStream_t);
TM_INST_B(double)
TM_INST_B(float)
#undef TM_INST_B

#define TM_INST(T)                                                                                               \
  template void launch_orthonormalise<T>(T*, const AggGeom&, int*, cudaStream_t);                              \
  template void launch_restrict<T>(const T*, const T*, T*, const AggGeom&, int, cudaStream_t, const void*, int); \
  template void launch_prolong<T>(const T*, const T*, T*, const AggGeom&, int, bool, cudaStream_t, const void*,  \
                                  int);                                                                        \
  template void launch_coarse_build<T>(const T*, const T*, const T*, T*, const AggGeom&, double, cudaStream_t,   \
                                       BuildShape, double);                                                   \
  template void launch_coarse_apply<T>(const T*, const T*, T*, const Lat&, int, double, int, cudaStream_t,       \
                                       const void*, int);                                                       \
  template void launch_oe_invert<T>(const T*, T*, const OEGeom&, double, int*, cudaStream_t);                  \
  template void launch_oe_hop_inv<T>(const T*, const T*, const T*, T*, const OEGeom&, cudaStream_t);           \
  template void launch_oe_even<T>(const T*, const T*, const T*, T*, const OEGeom&, double, int, cudaStream_t); \
  template void launch_oe_inv_odd<T>(const T*, const T*, T*, const OEGeom&, cudaStream_t);                     \
  template void launch_oe_rhs<T>(const T*, const T*, const T*, T*, const OEGeom&, cudaStream_t);               \
  template void launch_oe_reconstruct<T>(const T*, const T*, const T*, const T*, T*, const OEGeom&, cudaStream_t);
TM_INST(double)
TM_INST(float)
#undef TM_INST

}  // namespace tmamg
