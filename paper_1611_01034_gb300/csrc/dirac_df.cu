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
#include "tm_kernels.h"
#include "tm_pair.cuh"

namespace tmamg {

namespace {

// multiply by a phase from {+1, +i, -1, -i} (exact)
__device__ __forceinline__ cdf mulp(cdf z, int p) {
  switch (p & 3) {
    case 0: return z;
    case 1: return cdf{neg(z.i), z.r};
    case 2: return cdf{neg(z.r), neg(z.i)};
    default: return cdf{z.i, neg(z.r)};
  }
}

// multiply an FP32 complex number by a phase from {+1, +i, -1, -i} (exact)
__device__ __forceinline__ cx<float> mulph_rt(cx<float> z, int p) {
  switch (p & 3) {
    case 0: return z;
    case 1: return cx<float>{-z.i, z.r};
    case 2: return cx<float>{-z.r, -z.i};
    default: return cx<float>{z.i, -z.r};
  }
}

// exact difference / sum of two FP32 complex numbers as a pair
__device__ __forceinline__ cdf exact_sum(cx<float> a, cx<float> b) { return cdf{two_sum(a.r, b.r), two_sum(a.i, b.i)}; }

// link entry e = 3 a + b of direction mu at site s: float4 (re.h, im.h, re.l, im.l)
__device__ __forceinline__ cdf ld_link_entry(const float4* __restrict__ gdf, long V, int mu, int e, long s) {
  const float4 v = __ldg(gdf + ((long)mu * 9 + e) * V + s);
  return cdf{dfl{v.x, v.z}, dfl{v.y, v.w}};
}

// acc += sign (1 -+ gamma_MU) U^(+) p for one hop (FWD: U = U_MU(x), psi(x + MU), projector 1 - gamma;
// backward: U^dagger of U_MU(x - MU), psi(x - MU), projector 1 + gamma); link site sl
template <int MU, bool FWD>
__device__ __forceinline__ void hop_df(const cx<float> (&p)[12], const float4* __restrict__ gdf, long V, long sl,
                                       float sign, cdf (&acc)[12]) {
  cdf h[2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const cx<float> lo = mulph_rt(p[3 * (2 + gperm(MU, r)) + k], gphase(MU, r));
      const cx<float> up = p[3 * r + k];
      // (1 - gamma): h = up - A dn; (1 + gamma): h = up + A dn  (exact as pairs)
      cdf t = FWD ? exact_sum(up, cx<float>{-lo.r, -lo.i}) : exact_sum(up, lo);
      if (sign < 0) t = cdf{neg(t.r), neg(t.i)};
      h[r][k] = t;
    }
  cdf w[2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int a = 0; a < 3; ++a) w[r][a] = cdf{{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // forward: w[a] += U[a][b] h[b]; backward: w[a] += conj(U[b][a]) h[b]
      const cdf u = FWD ? ld_link_entry(gdf, V, MU, 3 * a + b, sl) : ld_link_entry(gdf, V, MU, 3 * b + a, sl);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (FWD)
          cfma_pp(w[r][a], u, h[r][b]);
        else
          cfmac_pp(w[r][a], u, h[r][b]);
      }
    }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      add_to(acc[3 * r + k].r, w[r][k].r);
      add_to(acc[3 * r + k].i, w[r][k].i);
      // lower components: -+ A^dagger w, (A^dagger w)[perm r] = conj(phase r) w[r]
      cdf lw = mulp(w[r][k], conjph(gphase(MU, r)));
      if (FWD) lw = cdf{neg(lw.r), neg(lw.i)};
      add_to(acc[3 * (2 + gperm(MU, r)) + k].r, lw.r);
      add_to(acc[3 * (2 + gperm(MU, r)) + k].i, lw.i);
    }
}

template <int MU>
__device__ __forceinline__ void hops_df(const float* __restrict__ in, const float4* __restrict__ gdf, const Lat& g,
                                        int s, const int c[4], float bc, cdf (&acc)[12]) {
  {
    cx<float> p[12];
    ld_cx<float, 12>(in, g.V, nb_fwd(g, s, c, MU), p);
    const float sign = (MU == 0 && c[0] == g.L[0] - 1) ? bc : 1.f;
    hop_df<MU, true>(p, gdf, g.V, s, sign, acc);
  }
  {
    const int sb = nb_bwd(g, s, c, MU);
    cx<float> p[12];
    ld_cx<float, 12>(in, g.V, sb, p);
    const float sign = (MU == 0 && c[0] == 0) ? bc : 1.f;
    hop_df<MU, false>(p, gdf, g.V, sb, sign, acc);
  }
}

struct DfArgs {
  const float4* gdf;
  const float4* cdf4;
  const float* in;
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

__global__ void __launch_bounds__(128) k_dslash_df(DfArgs a) {
  const int rhs = a.nrhs == 1 ? 0 : (int)(blockIdx.x % a.nrhs);
  const int s = (a.nrhs == 1 ? blockIdx.x : blockIdx.x / a.nrhs) * blockDim.x + threadIdx.x;
  if (s >= a.g.V) return;
  const long off = (long)rhs * NR_SPINOR * a.g.V;
  const float* in = a.in + off;
  int c[4];
  site_coords(a.g, s, c);
  cdf acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cdf{{0.f, 0.f}, {0.f, 0.f}};
  hops_df<0>(in, a.gdf, a.g, s, c, a.bc, acc);
  hops_df<1>(in, a.gdf, a.g, s, c, a.bc, acc);
  hops_df<2>(in, a.gdf, a.g, s, c, a.bc, acc);
  hops_df<3>(in, a.gdf, a.g, s, c, a.bc, acc);
  cx<float> p[12];
  ld_cx<float, 12>(in, a.g.V, s, p);
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
      fma_pf(y[2 * j].r, d0, p[6 * h + 2 * j].r);
      fma_pf(y[2 * j].i, d0, p[6 * h + 2 * j].i);
      fma_pf(y[2 * j + 1].r, d1, p[6 * h + 2 * j + 1].r);
      fma_pf(y[2 * j + 1].i, d1, p[6 * h + 2 * j + 1].i);
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
        cfma_pf(y[i], u, p[6 * h + j]);
        cfmac_pf(y[j], u, p[6 * h + i]);
      }
    // i mu gamma5 p, gamma5 = -1 on spins 0, 1 (h = 0), +1 on spins 2, 3
    const dfl mus = ((c[0] + c[1] + c[2] + c[3]) & 1) ? a.mu_odd : a.mu;
    const dfl m = h == 0 ? neg(mus) : mus;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      fma_pf(y[i].r, neg(m), p[6 * h + i].i);
      fma_pf(y[i].i, m, p[6 * h + i].r);
    }
    // FP64 output: h + l
    double2* o = reinterpret_cast<double2*>(a.out + off);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int chunk = 3 * h + k;  // complex numbers 6 h + 2 k, 6 h + 2 k + 1
      o[2 * ((long)chunk * a.g.V + s)] = make_double2(f2d_bits(y[2 * k].r.h) + f2d_bits(y[2 * k].r.l),
                                                      f2d_bits(y[2 * k].i.h) + f2d_bits(y[2 * k].i.l));
      o[2 * ((long)chunk * a.g.V + s) + 1] = make_double2(f2d_bits(y[2 * k + 1].r.h) + f2d_bits(y[2 * k + 1].r.l),
                                                          f2d_bits(y[2 * k + 1].i.h) + f2d_bits(y[2 * k + 1].i.l));
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

void launch_dslash_df(const void* gdf, const void* cdf, const float* in, double* out, const Lat& g, double mu,
                      double bc_t, int nrhs, cudaStream_t st, double rho) {
  const double muo = mu + rho;
  const float mh = (float)mu, moh = (float)muo;
  DfArgs a{static_cast<const float4*>(gdf), static_cast<const float4*>(cdf), in, out, g,
           dfl{mh, (float)(mu - (double)mh)}, dfl{moh, (float)(muo - (double)moh)}, (float)bc_t, nrhs};
  dim3 grid((unsigned)((g.V + 127) / 128) * (unsigned)nrhs);
  k_dslash_df<<<grid, 128, 0, st>>>(a);
}

}  // namespace tmamg
