// D(mu) on FP32 input with an FP64-accurate result from pairs of FP32 numbers.
//
// The outer FGMRES applies D(mu) to the preconditioned vectors z_k = B(v_k),
// which the FP32 K-cycle produces; the Arnoldi relation D Z = V H needs that
// product to FP64 accuracy (an FP32 product would put a floor of ~1e-7 under
// the residual).  GB300 runs FP64 at 1/64 of its FP32 rate, so here every real
// is carried as an unevaluated sum h + l of two FP32 numbers (Dekker's
// "double-length" arithmetic, Numer. Math. 18 (1971) 224, with Knuth's
// two-sum): products a.h*b.h are made exact with an FMA, the cross terms and
// the rounding errors gather in l.  Links (all 18 reals, no third-row
// reconstruction) and clover blocks are stored as such pairs; the input is
// FP32 and therefore exact.  The relative error is about 2^-46 (a few 1e-14)
// times the cancellation of the sum, the output is FP64.
//
// Operator as in dirac.cu (Sec. 1: D(mu) = D_W + i mu Gamma5):
//   (D psi)(x) = A(x) psi(x) + i mu gamma5 psi(x)
//       - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu) ]
#include <type_traits>

#include "tm_kernels.h"
#include "tm_pair.cuh"

namespace tmamg {

namespace {

// exact difference / sum of two FP32 complex numbers as a pair
__device__ __forceinline__ cdf exact_sum(cx<float> a, cx<float> b) { return cdf{two_sum(a.r, b.r), two_sum(a.i, b.i)}; }
// the same for pair inputs (a pair sum)
__device__ __forceinline__ dfl pair_add(dfl a, dfl b) {
  const dfl s = two_sum(a.h, b.h);
  return dfl{s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ cdf exact_sum(cdf a, cdf b) { return cdf{pair_add(a.r, b.r), pair_add(a.i, b.i)}; }
__device__ __forceinline__ cx<float> negc(cx<float> z) { return cx<float>{-z.r, -z.i}; }
__device__ __forceinline__ cdf negc(cdf z) { return cdf{neg(z.r), neg(z.i)}; }
// acc += a * b for an input component b that is an exact FP32 number or a pair
__device__ __forceinline__ void fma_px(dfl& acc, dfl a, float b) { fma_pf(acc, a, b); }
__device__ __forceinline__ void fma_px(dfl& acc, dfl a, dfl b) { fma_pp(acc, a, b); }
__device__ __forceinline__ void cfma_px(cdf& acc, cdf u, cx<float> x) { cfma_pf(acc, u, x); }
__device__ __forceinline__ void cfma_px(cdf& acc, cdf u, cdf x) { cfma_pp(acc, u, x); }
__device__ __forceinline__ void cfmac_px(cdf& acc, cdf u, cx<float> x) { cfmac_pf(acc, u, x); }
__device__ __forceinline__ void cfmac_px(cdf& acc, cdf u, cdf x) { cfmac_pp(acc, u, x); }

// link entry e = 3 a + b of direction mu at site s: float4 (re.h, im.h, re.l, im.l)
__device__ __forceinline__ cdf ld_link_entry(const float4* __restrict__ gdf, long V, int mu, int e, long s) {
  const float4 v = __ldg(gdf + ((long)mu * 9 + e) * V + s);
  return cdf{dfl{v.x, v.z}, dfl{v.y, v.w}};
}

// multiply by the phase i^q, q runtime (exact; branch-free selects)
__device__ __forceinline__ cdf mulp_sel(cdf z, int q);
__device__ __forceinline__ cx<float> mulph_sel(cx<float> z, int q) {
  const bool sw = q & 1;
  const float sr = (q == 1 || q == 2) ? -1.f : 1.f, si = q >= 2 ? -1.f : 1.f;
  return cx<float>{sr * (sw ? z.i : z.r), si * (sw ? z.r : z.i)};
}
__device__ __forceinline__ cdf mulph_sel(cdf z, int q) { return mulp_sel(z, q); }
__device__ __forceinline__ cdf mulp_sel(cdf z, int q) {
  const bool sw = q & 1;
  const float sr = (q == 1 || q == 2) ? -1.f : 1.f, si = q >= 2 ? -1.f : 1.f;
  const dfl a = sw ? z.i : z.r, b = sw ? z.r : z.i;
  return cdf{dfl{sr * a.h, sr * a.l}, dfl{si * b.h, si * b.l}};
}
__device__ __forceinline__ int gphase_rt(int mu, int r) {
  return mu == 0 ? 2 : mu == 1 ? (r == 0 ? 3 : 1) : mu == 2 ? (r == 0 ? 2 : 0) : 3;
}

// acc += sign (1 -+ gamma_mu) U^(+) p for hop direction mu (runtime) and
// orientation fwd (U = U_mu(x), psi(x + mu), projector 1 - gamma) or backward
// (U^dagger of U_mu(x - mu), psi(x - mu), projector 1 + gamma); link site sl.
// One copy of the code serves all eight hops, so the kernel's loop over them
// stays in the instruction cache.
template <typename PT>  // input spinor components: exact FP32 (cx<float>) or pairs (cdf)
__device__ __forceinline__ void hop_df_rt(const PT (&p)[12], const float4* __restrict__ gdf, long V, long sl, int mu,
                                          bool fwd, float sign, cdf (&acc)[12]) {
  const bool sw = mu >= 2;  // A_mu's row r holds its entry in column r (T, Z) or 1 - r (Y, X)
  cdf h[2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const PT dn = (sw != (r == 1)) ? p[9 + k] : p[6 + k];  // spin 2 + perm(r)
      const PT lo = mulph_sel(dn, gphase_rt(mu, r));
      const PT up = p[3 * r + k];
      // (1 - gamma): h = up - A dn; (1 + gamma): h = up + A dn  (exact as pairs for FP32 input)
      cdf t = exact_sum(up, fwd ? negc(lo) : lo);
      t = cdf{dfl{sign * t.r.h, sign * t.r.l}, dfl{sign * t.i.h, sign * t.i.l}};
      h[r][k] = t;
    }
  cdf w[2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int a = 0; a < 3; ++a) w[r][a] = cdf{{0.f, 0.f}, {0.f, 0.f}};
  const float cj = fwd ? 1.f : -1.f;  // backward hops take conj(U[b][a])
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cdf u = ld_link_entry(gdf, V, mu, fwd ? 3 * a + b : 3 * b + a, sl);
      u.i = dfl{cj * u.i.h, cj * u.i.l};
#pragma unroll
      for (int r = 0; r < 2; ++r) cfma_pp(w[r][a], u, h[r][b]);
    }
  cdf lw[2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      add_to(acc[3 * r + k].r, w[r][k].r);
      add_to(acc[3 * r + k].i, w[r][k].i);
      // lower components: -+ A^dagger w, (A^dagger w)[perm r] = conj(phase r) w[r]
      cdf l = mulp_sel(w[r][k], conjph(gphase_rt(mu, r)));
      if (fwd) l = cdf{neg(l.r), neg(l.i)};
      lw[r][k] = l;
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const cdf l2 = sw ? lw[1][k] : lw[0][k], l3 = sw ? lw[0][k] : lw[1][k];
    add_to(acc[6 + k].r, l2.r);
    add_to(acc[6 + k].i, l2.i);
    add_to(acc[9 + k].r, l3.r);
    add_to(acc[9 + k].i, l3.i);
  }
}

struct DfArgs {
  const float4* gdf;
  const float4* cdf4;
  const void* in;     // FP32 (exact in pairs) or FP64 (split into pairs) spinors
  const double* sub;  // if set: out = sub - D in
  double* out;
  Lat g;
  dfl mu, mu_odd;  // twisted mass on even and on odd sites
  float bc;
  int nrhs;
};

// clover chunk j of site s: float4 (r[2j].h, r[2j+1].h, r[2j].l, r[2j+1].l)
__device__ __forceinline__ void ld_clover_pair(const float4* __restrict__ c4, long V, int j, long s, dfl& a, dfl& b) {
  const float4 v = __ldg(c4 + (long)j * V + s);
  a = dfl{v.x, v.z};
  b = dfl{v.y, v.w};
}

// input spinor of site s as exact FP32 components or as pairs split from FP64
__device__ __forceinline__ void ld_in(const float* in, long V, long s, cx<float> (&p)[12]) { ld_cx<float, 12>(in, V, s, p); }
__device__ __forceinline__ void ld_in(const double* in, long V, long s, cdf (&p)[12]) {
  const double2* q = reinterpret_cast<const double2*>(in);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double2 v0 = __ldg(q + 2 * (k * V + s)), v1 = __ldg(q + 2 * (k * V + s) + 1);
    p[2 * k] = cx2pair(v0.x, v0.y);
    p[2 * k + 1] = cx2pair(v1.x, v1.y);
  }
}

template <typename IN>
__global__ void __launch_bounds__(128) k_dslash_df(DfArgs a) {
  using PT = typename std::conditional<std::is_same<IN, float>::value, cx<float>, cdf>::type;
  const int rhs = a.nrhs == 1 ? 0 : (int)(blockIdx.x % a.nrhs);
  const int s = (a.nrhs == 1 ? blockIdx.x : blockIdx.x / a.nrhs) * blockDim.x + threadIdx.x;
  if (s >= a.g.V) return;
  const long off = (long)rhs * NR_SPINOR * a.g.V;
  const IN* in = static_cast<const IN*>(a.in) + off;
  int c[4];
  site_coords(a.g, s, c);
  cdf acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cdf{{0.f, 0.f}, {0.f, 0.f}};
  // the eight hops through one copy of the hop code (direction and orientation at run time)
#pragma unroll 1
  for (int hop = 0; hop < 8; ++hop) {
    const int mu = hop >> 1;
    const bool fwd = (hop & 1) == 0;
    const int cm = mu == 0 ? c[0] : mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
    const int Lm = mu == 0 ? a.g.L[0] : mu == 1 ? a.g.L[1] : mu == 2 ? a.g.L[2] : a.g.L[3];
    const int stm = mu == 0 ? a.g.st[0] : mu == 1 ? a.g.st[1] : mu == 2 ? a.g.st[2] : a.g.st[3];
    const int sn = fwd ? (cm + 1 < Lm ? s + stm : s - (Lm - 1) * stm) : (cm > 0 ? s - stm : s + (Lm - 1) * stm);
    const float sign = (mu == 0 && cm == (fwd ? Lm - 1 : 0)) ? a.bc : 1.f;
    PT p[12];
    ld_in(in, a.g.V, sn, p);
    hop_df_rt(p, a.gdf, a.g.V, fwd ? s : sn, mu, fwd, sign, acc);
  }
  PT p[12];
  ld_in(in, a.g.V, s, p);
  // y = A p + i mu gamma5 p - acc / 2
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    cdf y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      y[i].r = dfl{-0.5f * acc[6 * h + i].r.h, -0.5f * acc[6 * h + i].r.l};
      y[i].i = dfl{-0.5f * acc[6 * h + i].i.h, -0.5f * acc[6 * h + i].i.l};
    }
    // diagonal reals (chunks 18 h + 0..2 hold reals 36 h + 0..5)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      dfl d0, d1;
      ld_clover_pair(a.cdf4, a.g.V, 18 * h + j, s, d0, d1);
      fma_px(y[2 * j].r, d0, p[6 * h + 2 * j].r);
      fma_px(y[2 * j].i, d0, p[6 * h + 2 * j].i);
      fma_px(y[2 * j + 1].r, d1, p[6 * h + 2 * j + 1].r);
      fma_px(y[2 * j + 1].i, d1, p[6 * h + 2 * j + 1].i);
    }
    // upper triangle (0,1),(0,2),...,(4,5): complex entry q at reals 6 + 2q, 7 + 2q = chunk 3 + q
    int q = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i + 1; j < 6; ++j) {
        cdf u;
        ld_clover_pair(a.cdf4, a.g.V, 18 * h + 3 + q, s, u.r, u.i);
        ++q;
        cfma_px(y[i], u, p[6 * h + j]);
        cfmac_px(y[j], u, p[6 * h + i]);
      }
    // i mu gamma5 p, gamma5 = -1 on spins 0, 1 (h = 0), +1 on spins 2, 3
    const dfl mus = ((c[0] + c[1] + c[2] + c[3]) & 1) ? a.mu_odd : a.mu;
    const dfl m = h == 0 ? neg(mus) : mus;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      fma_px(y[i].r, neg(m), p[6 * h + i].i);
      fma_px(y[i].i, m, p[6 * h + i].r);
    }
    // FP64 output: h + l (or sub - (h + l))
    double2* o = reinterpret_cast<double2*>(a.out + off);
    const double2* sb = a.sub ? reinterpret_cast<const double2*>(a.sub + off) : nullptr;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int chunk = 3 * h + k;  // complex numbers 6 h + 2 k, 6 h + 2 k + 1
      const long i0 = 2 * ((long)chunk * a.g.V + s);
      double2 v0 = make_double2(pair2d(y[2 * k].r), pair2d(y[2 * k].i));
      double2 v1 = make_double2(pair2d(y[2 * k + 1].r), pair2d(y[2 * k + 1].i));
      if (sb) {
        const double2 b0 = sb[i0], b1 = sb[i0 + 1];
        v0 = make_double2(b0.x - v0.x, b0.y - v0.y);
        v1 = make_double2(b1.x - v1.x, b1.y - v1.y);
      }
      o[i0] = v0;
      o[i0 + 1] = v1;
    }
  }
}

__device__ __forceinline__ float2 split(double x) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}

// natural gauge [V][4][3][3] complex128 -> [4][9][V] float4 pairs
__global__ void k_pack_gauge_df(const double* __restrict__ nat, float4* __restrict__ gdf, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  if (s >= V) return;
  const double2* p = reinterpret_cast<const double2*>(nat) + ((long)s * 4 + mu) * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const double2 v = p[e];
    const float2 re = split(v.x), im = split(v.y);
    gdf[((long)mu * 9 + e) * V + s] = make_float4(re.x, im.x, re.y, im.y);
  }
}

// packed FP64 clover [18 chunks][V] (4 reals each) -> [36][V] float4 pairs
__global__ void k_clover_df(const double* __restrict__ c64, float4* __restrict__ c4, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  double r[72];
  ld_re<double, 72>(c64, V, s, r);
#pragma unroll
  for (int j = 0; j < 36; ++j) {
    const float2 a = split(r[2 * j]), b = split(r[2 * j + 1]);
    c4[(long)j * V + s] = make_float4(a.x, b.x, a.y, b.y);
  }
}

}  // namespace

void launch_pack_gauge_df(const double* nat, void* gdf, const Lat& g, cudaStream_t st) {
  dim3 grid((g.V + 127) / 128, 4);
  k_pack_gauge_df<<<grid, 128, 0, st>>>(nat, static_cast<float4*>(gdf), g.V);
}

void launch_clover_df(const double* c64, void* cdf, const Lat& g, cudaStream_t st) {
  k_clover_df<<<(g.V + 127) / 128, 128, 0, st>>>(c64, static_cast<float4*>(cdf), g.V);
}

DfArgs df_args(const void* gdf, const void* cdf, const void* in, const double* sub, double* out, const Lat& g,
               double mu, double bc_t, int nrhs, double rho) {
  const double muo = mu + rho;
  const float mh = (float)mu, moh = (float)muo;
  return DfArgs{static_cast<const float4*>(gdf), static_cast<const float4*>(cdf), in, sub, out, g,
                dfl{mh, (float)(mu - (double)mh)}, dfl{moh, (float)(muo - (double)moh)}, (float)bc_t, nrhs};
}

void launch_dslash_df(const void* gdf, const void* cdf, const float* in, double* out, const Lat& g, double mu,
                      double bc_t, int nrhs, cudaStream_t st, double rho) {
  dim3 grid((unsigned)((g.V + 127) / 128) * (unsigned)nrhs);
  k_dslash_df<float><<<grid, 128, 0, st>>>(df_args(gdf, cdf, in, nullptr, out, g, mu, bc_t, nrhs, rho));
}

void launch_residual_df(const void* gdf, const void* cdf, const double* x, const double* b, double* r, const Lat& g,
                        double mu, double bc_t, int nrhs, cudaStream_t st, double rho) {
  dim3 grid((unsigned)((g.V + 127) / 128) * (unsigned)nrhs);
  k_dslash_df<double><<<grid, 128, 0, st>>>(df_args(gdf, cdf, x, b, r, g, mu, bc_t, nrhs, rho));
}

}  // namespace tmamg
