// Odd-even reduced operator and the CG kernels of the oeCG comparison solver
// (Sec. 1, Fig. 1: DD-alphaAMG against CG on the odd-even preconditioned
// operator; Sec. 3: the odd-site Schur complement).
//
// Half-lattice fields hold one parity: the site with full index s (X even)
// has compact index s >> 1 within its parity, and a half field is the
// chunked SoA layout of a full field with V/2 in place of V.  With
// H psi(x) = sum_mu [(1 - gamma_mu) U_mu(x) psi(x + mu) + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu)]
// the off-diagonal blocks are D_eo = D_oe = -H / 2 restricted to the target
// parity, and
//   D^ x_o = D_oo x_o - D_oe D_ee^-1 D_eo x_o
// is two launches of one kernel:
//   mode 0:  out_p = [D_pp^-1 or its adjoint] (c H hin + din)
//   mode 1:  out_p = g5 [ D_pp(mu') (g5 din) + c H hin ]   (D_pp = 1 without clover)
// with D^dagger = G^5 D^(-mu) G^5 from the adjoint of the stored inverse and
// the sign-flipped twisted mass (Gamma5-hermiticity).
#include "tm_kernels.h"
#include "tm_stencil.cuh"

namespace tmamg {

namespace {

template <typename T>
struct OeArgs {
  const T* gauge;
  const T* clover;
  const T* dinv;
  const T* hin;  // other parity, or null (no hop term)
  const T* din;  // target parity, or null
  T* out;
  Lat g;
  int parity;
  T c_hop;
  T mu;  // mode 1: twisted mass of the target parity in D_pp
  T bc;
  int g5;   // mode 0: Gamma5 on hin; mode 1: Gamma5 on din and on the result
  int dag;  // mode 0: adjoint of the stored inverse
  int mode;
};

template <typename T>
__device__ __forceinline__ void g5_flip(cx<T> (&p)[12]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = cx<T>{-p[k].r, -p[k].i};  // gamma5 = -1 on spins 0, 1
}

// acc = H hin at site s (neighbours from the half field of the other parity)
template <typename T, int MU>
__device__ __forceinline__ void half_hops(const T* __restrict__ in, const T* __restrict__ gauge, const Lat& g, long Vh,
                                          int s, const int c[4], T bc, bool g5, cx<T> (&acc)[12]) {
  {
    const int sf = nb_fwd(g, s, c, MU);
    cx<T> p[12];
    ld_cx<T, 12>(in, Vh, sf >> 1, p);
    if (g5) g5_flip(p);
    const T sign = (MU == 0 && c[0] == g.L[0] - 1) ? bc : T(1);
    hop_fwd_p<T, MU>(p, gauge, g.V, s, sign, acc);
  }
  {
    const int sb = nb_bwd(g, s, c, MU);
    cx<T> p[12];
    ld_cx<T, 12>(in, Vh, sb >> 1, p);
    if (g5) g5_flip(p);
    const T sign = (MU == 0 && c[0] == 0) ? bc : T(1);
    hop_bwd_p<T, MU>(p, gauge, g.V, sb, sign, acc);
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_oe_apply(OeArgs<T> a) {
  const long Vh = a.g.V / 2;
  const long so = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (so >= Vh) return;
  const Lat& g = a.g;
  const long row = so / (g.L[3] / 2);
  const int xh = (int)(so % (g.L[3] / 2));
  int c[4];
  c[2] = (int)(row % g.L[2]);
  c[1] = (int)((row / g.L[2]) % g.L[1]);
  c[0] = (int)(row / ((long)g.L[2] * g.L[1]));
  c[3] = 2 * xh + (((c[0] + c[1] + c[2]) & 1) ^ a.parity);
  const int s = ((c[0] * g.L[1] + c[1]) * g.L[2] + c[2]) * g.L[3] + c[3];
  cx<T> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cx<T>{0, 0};
  if (a.hin) {
    const bool gh = a.mode == 0 && a.g5;
    half_hops<T, 0>(a.hin, a.gauge, g, Vh, s, c, a.bc, gh, acc);
    half_hops<T, 1>(a.hin, a.gauge, g, Vh, s, c, a.bc, gh, acc);
    half_hops<T, 2>(a.hin, a.gauge, g, Vh, s, c, a.bc, gh, acc);
    half_hops<T, 3>(a.hin, a.gauge, g, Vh, s, c, a.bc, gh, acc);
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = a.c_hop * acc[k];
  }
  cx<T> v[12];
  if (a.din) {
    ld_cx<T, 12>(a.din, Vh, so, v);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = cx<T>{0, 0};
  }
  cx<T> y[12];
  if (a.mode == 0) {
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = v[k] + acc[k];
    // y = M v or M^dagger v per chiral 6x6 block; row i of block h: 6 complex at chunk row (6 h + i)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int i = 0; i < 6; ++i) y[6 * h + i] = cx<T>{0, 0};
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        cx<T> m[6];
        ld_cx<T, 6>(a.dinv + (long)(h * 6 + i) * 12 * Vh, Vh, so, m);
        if (a.dag) {
#pragma unroll
          for (int j = 0; j < 6; ++j) cfmac(y[6 * h + j], m[j], v[6 * h + i]);  // (M^dagger)_{ji} = conj(M_ij)
        } else {
#pragma unroll
          for (int j = 0; j < 6; ++j) cfma(y[6 * h + i], m[j], v[6 * h + j]);
        }
      }
    }
  } else {
    if (a.g5) g5_flip(v);
    if (a.clover) {
      site_diag<T>(a.clover, g.V, s, a.mu, v, y);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) y[k] = v[k];
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) y[k] = y[k] + acc[k];
    if (a.g5) g5_flip(y);
  }
  st_cx<T, 12>(a.out, Vh, so, y);
}

// half field of one parity <-> full packed field
template <typename T>
__global__ void k_parity_copy(const T* __restrict__ src, T* __restrict__ dst, Lat g, int parity, int to_full) {
  const long Vh = g.V / 2;
  const long so = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (so >= Vh) return;
  const long row = so / (g.L[3] / 2);
  const int xh = (int)(so % (g.L[3] / 2));
  const int c2 = (int)(row % g.L[2]);
  const int c1 = (int)((row / g.L[2]) % g.L[1]);
  const int c0 = (int)(row / ((long)g.L[2] * g.L[1]));
  const long s = row * g.L[3] + 2 * xh + (((c0 + c1 + c2) & 1) ^ parity);
  cx<T> p[12];
  if (to_full) {
    ld_cx<T, 12>(src, Vh, so, p);
    st_cx<T, 12>(dst, g.V, s, p);
  } else {
    ld_cx<T, 12>(src, g.V, s, p);
    st_cx<T, 12>(dst, Vh, so, p);
  }
}

// CG updates with the scalars on the device (sc: FP64 reductions)
//   x += alpha p, r -= alpha q, alpha = sc[ig] / sc[iq]
template <typename T>
__global__ void k_cg_xr(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ q,
                        const double* __restrict__ sc, int ig, int iq, long n) {
  const double den = sc[iq];
  const T alpha = (T)(den > 0 ? sc[ig] / den : 0.0);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
  }
}
//   p = s + beta p, beta = sc[inew] / sc[iold]
template <typename T>
__global__ void k_cg_p(T* __restrict__ p, const T* __restrict__ s, const double* __restrict__ sc, int inew, int iold,
                       long n) {
  const double den = sc[iold];
  const T beta = (T)(den > 0 ? sc[inew] / den : 0.0);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], s[i]);
}

__global__ void k_acc_f32(const float* __restrict__ e, double* __restrict__ x, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    x[i] += (double)e[i];
}

int stream_grid(long n) {
  long b = (n + 255) / 256;
  if (b > 152L * 8) b = 152L * 8;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

template <typename T>
void launch_oe_apply(const T* gauge, const T* clover, const T* dinv, const T* hin, const T* din, T* out, const Lat& g,
                     int parity, double c_hop, double mu, double bc_t, int g5, int dag, int mode, cudaStream_t st) {
  OeArgs<T> a{gauge, clover, dinv, hin, din, out, g, parity, (T)c_hop, (T)mu, (T)bc_t, g5, dag, mode};
  const long Vh = g.V / 2;
  k_oe_apply<T><<<(unsigned)((Vh + 127) / 128), 128, 0, st>>>(a);
}

template <typename T>
void launch_parity_copy(const T* src, T* dst, const Lat& g, int parity, bool to_full, cudaStream_t st) {
  const long Vh = g.V / 2;
  k_parity_copy<T><<<(unsigned)((Vh + 127) / 128), 128, 0, st>>>(src, dst, g, parity, to_full ? 1 : 0);
}

template <typename T>
void launch_cg_xr(T* x, T* r, const T* p, const T* q, const double* sc, int ig, int iq, long n_reals,
                  cudaStream_t st) {
  k_cg_xr<T><<<stream_grid(n_reals), 256, 0, st>>>(x, r, p, q, sc, ig, iq, n_reals);
}

template <typename T>
void launch_cg_p(T* p, const T* s, const double* sc, int inew, int iold, long n_reals, cudaStream_t st) {
  k_cg_p<T><<<stream_grid(n_reals), 256, 0, st>>>(p, s, sc, inew, iold, n_reals);
}

void launch_acc_f32(const float* e, double* x, long n_reals, cudaStream_t st) {
  k_acc_f32<<<stream_grid(n_reals), 256, 0, st>>>(e, x, n_reals);
}

#define TM_INST_OE(T)                                                                                           \
  template void launch_oe_apply<T>(const T*, const T*, const T*, const T*, const T*, T*, const Lat&, int, double, \
                                   double, double, int, int, int, cudaStream_t);                                \
  template void launch_parity_copy<T>(const T*, T*, const Lat&, int, bool, cudaStream_t);                        \
  template void launch_cg_xr<T>(T*, T*, const T*, const T*, const double*, int, int, long, cudaStream_t);        \
  template void launch_cg_p<T>(T*, const T*, const double*, int, int, long, cudaStream_t);
TM_INST_OE(double)
TM_INST_OE(float)
#undef TM_INST_OE

}  // namespace tmamg
