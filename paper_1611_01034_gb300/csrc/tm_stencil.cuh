// Device pieces of the D(mu) stencil shared by the full-lattice apply
// (dirac.cu) and the SAP block solver (sap.cu).
//
// Spin projection in the chiral basis: with gamma_mu = [[0, A], [A^dagger, 0]]
// and A^dagger A = 1,
//   (1 - gamma_mu) psi = [h; -A^dagger h],  h = psi_up - A psi_dn,
//   (1 + gamma_mu) psi = [h;  A^dagger h],  h = psi_up + A psi_dn,
// so each hop multiplies only two colour vectors by the link.
#pragma once

#include "tm_internal.cuh"

namespace tmamg {

template <typename T>
__device__ __forceinline__ cx<T> mulp(cx<T> z, int p) {
  switch (p & 3) {
    case 0: return z;
    case 1: return cx<T>{-z.i, z.r};
    case 2: return cx<T>{-z.r, -z.i};
    default: return cx<T>{z.i, -z.r};
  }
}

// acc += sign (1 - gamma_MU) U p, p = psi(x + MU), U = U_MU(x) at link site sl
// (links stored as T, or in 16 bits for S = ST_F16 / ST_BF16)
template <typename T, int MU, int S = ST_NATIVE>
__device__ __forceinline__ void hop_fwd_p(const cx<T> (&p)[12], const void* __restrict__ gauge, int V, int sl,
                                          T sign, cx<T> (&acc)[12]) {
  cx<T> h[2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) h[r][k] = sign * (p[3 * r + k] - mulp(p[3 * (2 + gperm(MU, r)) + k], gphase(MU, r)));
  Link<T> U;
  ld_link_s<T, S>(gauge, V, MU, sl, U);
  cx<T> w[2][3];
  su3_mul(U, h[0], w[0]);
  su3_mul(U, h[1], w[1]);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc[3 * r + k] = acc[3 * r + k] + w[r][k];
      // lower = -A^dagger w, (A^dagger w)[perm r] = conj(phase r) w[r]
      acc[3 * (2 + gperm(MU, r)) + k] = acc[3 * (2 + gperm(MU, r)) + k] - mulp(w[r][k], conjph(gphase(MU, r)));
    }
}

// acc += sign (1 + gamma_MU) U^dagger p, p = psi(x - MU), U = U_MU(x - MU) at link site sl
template <typename T, int MU, int S = ST_NATIVE>
__device__ __forceinline__ void hop_bwd_p(const cx<T> (&p)[12], const void* __restrict__ gauge, int V, int sl,
                                          T sign, cx<T> (&acc)[12]) {
  cx<T> h[2][3];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) h[r][k] = sign * (p[3 * r + k] + mulp(p[3 * (2 + gperm(MU, r)) + k], gphase(MU, r)));
  Link<T> U;
  ld_link_s<T, S>(gauge, V, MU, sl, U);
  cx<T> w[2][3];
  su3_dag_mul(U, h[0], w[0]);
  su3_dag_mul(U, h[1], w[1]);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc[3 * r + k] = acc[3 * r + k] + w[r][k];
      acc[3 * (2 + gperm(MU, r)) + k] = acc[3 * (2 + gperm(MU, r)) + k] + mulp(w[r][k], conjph(gphase(MU, r)));
    }
}

// acc += both hops in direction MU with neighbours read from global memory
template <typename T, int MU, int S = ST_NATIVE>
__device__ __forceinline__ void hops_global(const T* __restrict__ in, const void* __restrict__ gauge, const Lat& g,
                                            int s, const int c[4], T bc, cx<T> (&acc)[12]) {
  const int sf = nb_fwd(g, s, c, MU);
  const int sb = nb_bwd(g, s, c, MU);
  {
    cx<T> p[12];
    ld_cx<T, 12>(in, g.V, sf, p);
    const T sign = (MU == 0 && c[0] == g.L[0] - 1) ? bc : T(1);
    hop_fwd_p<T, MU, S>(p, gauge, g.V, s, sign, acc);
  }
  {
    cx<T> p[12];
    ld_cx<T, 12>(in, g.V, sb, p);
    const T sign = (MU == 0 && c[0] == 0) ? bc : T(1);
    hop_bwd_p<T, MU, S>(p, gauge, g.V, sb, sign, acc);
  }
}

// sum over all 8 hops (without the -1/2) with global neighbours
template <typename T, int S = ST_NATIVE>
__device__ __forceinline__ void all_hops_global(const T* __restrict__ in, const void* __restrict__ gauge,
                                                const Lat& g, int s, const int c[4], T bc, cx<T> (&acc)[12]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cx<T>{0, 0};
  hops_global<T, 0, S>(in, gauge, g, s, c, bc, acc);
  hops_global<T, 1, S>(in, gauge, g, s, c, bc, acc);
  hops_global<T, 2, S>(in, gauge, g, s, c, bc, acc);
  hops_global<T, 3, S>(in, gauge, g, s, c, bc, acc);
}

// y = A(x) p + i mu gamma5 p at site s
template <typename T, int S = ST_NATIVE>
__device__ __forceinline__ void site_diag(const void* __restrict__ clover, int V, int s, T mu, const cx<T> (&p)[12],
                                          cx<T> (&y)[12]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    T m[36];
    if constexpr (S == ST_NATIVE)
      ld_re<T, 36>(static_cast<const T*>(clover) + (long)h * 36 * V, V, s, m);
    else
      ld_re_s<T, S, 36>(static_cast<const unsigned short*>(clover) + (long)h * 36 * V, V, s, m);
    herm6_mul(m, p + 6 * h, y + 6 * h);
    const T sg = h == 0 ? -mu : mu;  // gamma5 = -1 on spins 0, 1
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      y[6 * h + i].r -= sg * p[6 * h + i].i;
      y[6 * h + i].i += sg * p[6 * h + i].r;
    }
  }
}

}  // namespace tmamg
