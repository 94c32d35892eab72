// Fine-lattice operator: field packing, SU(3) link packing, clover term and
// the twisted-mass Wilson-clover stencil D(mu) = D_W + i mu Gamma5.
//
//   (D(mu) psi)(x) = A(x) psi(x) + i mu gamma5 psi(x)
//       - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                     + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu) ]
//
// (Sec. 1 of the paper: D(+-mu) = D_W +- i Gamma5 mu with D_W the Wilson
// clover operator; Sec. 2, eq. (2): gamma5 = diag(-1,-1,1,1), site order
// TZYX.)  A(x) = (m0 + 4) - (c_sw/32) sum_{mu,nu} gamma_mu gamma_nu (x)
// (Q_mu_nu - Q_nu_mu) is block diagonal in chirality because gamma_mu gamma_nu
// is; it is stored as two Hermitian 6x6 blocks.  Hops across the T boundary
// carry the factor bc_t.
#include "tm_kernels.h"
#include "tm_stencil.cuh"

namespace tmamg {

// ===========================================================================
// packing
// ===========================================================================
template <typename T>
__global__ void k_pack_spinor(const double* __restrict__ nat, T* __restrict__ field, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (s >= V) return;
  const double2* p = reinterpret_cast<const double2*>(nat) + ((long)r * V + s) * 12;
  cx<T> z[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 v = p[k];
    z[k] = cx<T>{(T)v.x, (T)v.y};
  }
  st_cx<T, 12>(field + (long)r * NR_SPINOR * V, V, s, z);
}

template <typename T>
__global__ void k_unpack_spinor(const T* __restrict__ field, double* __restrict__ nat, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (s >= V) return;
  cx<T> z[12];
  ld_cx<T, 12>(field + (long)r * NR_SPINOR * V, V, s, z);
  double2* p = reinterpret_cast<double2*>(nat) + ((long)r * V + s) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) p[k] = make_double2((double)z[k].r, (double)z[k].i);
}

template <typename T>
void launch_pack_spinor(const double* nat, T* field, const Lat& g, int nrhs, cudaStream_t st) {
  dim3 grid((g.V + 127) / 128, nrhs);
  k_pack_spinor<T><<<grid, 128, 0, st>>>(nat, field, g.V);
}
template <typename T>
void launch_unpack_spinor(const T* field, double* nat, const Lat& g, int nrhs, cudaStream_t st) {
  dim3 grid((g.V + 127) / 128, nrhs);
  k_unpack_spinor<T><<<grid, 128, 0, st>>>(field, nat, g.V);
}
template void launch_pack_spinor<double>(const double*, double*, const Lat&, int, cudaStream_t);
template void launch_pack_spinor<float>(const double*, float*, const Lat&, int, cudaStream_t);
template void launch_unpack_spinor<double>(const double*, double*, const Lat&, int, cudaStream_t);
template void launch_unpack_spinor<float>(const float*, double*, const Lat&, int, cudaStream_t);

// out = Gamma5 in on natural spinors: gamma5 = diag(-1,-1,+1,+1) negates the
// first six complex components (spins 0, 1) of every site
__global__ void k_gamma5_nat(const double* __restrict__ in, double* __restrict__ out, long nsites) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nsites * 24; i += (long)gridDim.x * blockDim.x)
    out[i] = (i % 24) < 12 ? -in[i] : in[i];
}

// zero the sites of one parity ((t + z + y + x) mod 2) of natural spinor arrays
__global__ void k_zero_parity_nat(double* __restrict__ nat, Lat g, int parity, int nrhs) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;  // site of one rhs
  if (i >= (long)g.V * nrhs) return;
  const int s = (int)(i % g.V);
  int c[4];
  site_coords(g, s, c);
  if (((c[0] + c[1] + c[2] + c[3]) & 1) != parity) return;
  double2* p = reinterpret_cast<double2*>(nat) + i * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) p[k] = make_double2(0.0, 0.0);
}

void launch_zero_parity_nat(double* nat, const Lat& g, int parity, int nrhs, cudaStream_t st) {
  const long n = (long)g.V * nrhs;
  k_zero_parity_nat<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nat, g, parity, nrhs);
}

void launch_gamma5_nat(const double* in, double* out, long nsites, cudaStream_t st) {
  long blocks = (nsites * 24 + 255) / 256;
  if (blocks > 152L * 16) blocks = 152L * 16;
  k_gamma5_nat<<<(int)blocks, 256, 0, st>>>(in, out, nsites);
}

// ===========================================================================
// 3x3 matrices for the gauge-field kernels (FP64, setup only)
// ===========================================================================
struct M3 {
  cx<double> m[3][3];
};

__device__ __forceinline__ M3 ld_nat_link(const double* __restrict__ nat, int s, int mu) {
  const double2* p = reinterpret_cast<const double2*>(nat) + ((long)s * 4 + mu) * 9;
  M3 U;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double2 v = p[a * 3 + b];
      U.m[a][b] = cx<double>{v.x, v.y};
    }
  return U;
}
__device__ __forceinline__ M3 mm(const M3& A, const M3& B) {
  M3 C;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cx<double> acc = A.m[a][0] * B.m[0][b];
      cfma(acc, A.m[a][1], B.m[1][b]);
      cfma(acc, A.m[a][2], B.m[2][b]);
      C.m[a][b] = acc;
    }
  return C;
}
__device__ __forceinline__ M3 dag(const M3& A) {
  M3 C;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) C.m[a][b] = conj(A.m[b][a]);
  return C;
}

// site index of coordinates c shifted by (dmu along mu, dnu along nu), periodic
__device__ __forceinline__ int shifted(const Lat& g, const int c[4], int mu, int dmu, int nu, int dnu) {
  int q[4] = {c[0], c[1], c[2], c[3]};
  q[mu] = (q[mu] + dmu + g.L[mu]) % g.L[mu];
  q[nu] = (q[nu] + dnu + g.L[nu]) % g.L[nu];
  return ((q[0] * g.L[1] + q[1]) * g.L[2] + q[2]) * g.L[3] + q[3];
}

// ===========================================================================
// gauge packing with SU(3) validation
// ===========================================================================
__global__ void k_pack_gauge(const double* __restrict__ nat, double* __restrict__ g64, float* __restrict__ g32,
                             int V, double tol, int* err) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  if (s >= V) return;
  M3 U = ld_nat_link(nat, s, mu);
  // unitarity and det = 1
  double dev = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cx<double> acc{0, 0};
      for (int k = 0; k < 3; ++k) cfmac(acc, U.m[b][k], U.m[a][k]);  // (U U^dagger)_{ab}
      acc.r -= (a == b) ? 1.0 : 0.0;
      dev = fmax(dev, sqrt(norm2(acc)));
    }
  cx<double> det = U.m[0][0] * (U.m[1][1] * U.m[2][2] - U.m[1][2] * U.m[2][1]) -
                   U.m[0][1] * (U.m[1][0] * U.m[2][2] - U.m[1][2] * U.m[2][0]) +
                   U.m[0][2] * (U.m[1][0] * U.m[2][1] - U.m[1][1] * U.m[2][0]);
  det.r -= 1.0;
  dev = fmax(dev, sqrt(norm2(det)));
  if (!(dev <= tol)) atomicOr(err, ERRF_NOT_SU3);
  cx<double> z[6];
  for (int k = 0; k < 3; ++k) {
    z[k] = U.m[0][k];
    z[3 + k] = U.m[1][k];
  }
  st_cx<double, 6>(g64 + (long)mu * NR_LINK * V, V, s, z);
  cx<float> zf[6];
  for (int k = 0; k < 6; ++k) zf[k] = cx<float>{(float)z[k].r, (float)z[k].i};
  st_cx<float, 6>(g32 + (long)mu * NR_LINK * V, V, s, zf);
}

void launch_pack_gauge(const double* nat, double* g64, float* g32, const Lat& g, double tol, int* err,
                       cudaStream_t st) {
  dim3 grid((g.V + 127) / 128, 4);
  k_pack_gauge<<<grid, 128, 0, st>>>(nat, g64, g32, g.V, tol, err);
}

// ===========================================================================
// clover term
// ===========================================================================
// 2x2 spin matrix A_mu of gamma_mu = [[0, A_mu], [A_mu^dagger, 0]]
__device__ __forceinline__ void amat(int mu, cx<double> (&A)[2][2]) {
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) A[r][c] = cx<double>{0, 0};
  for (int r = 0; r < 2; ++r) {
    int p = gphase(mu, r);
    cx<double> ph = p == 0 ? cx<double>{1, 0} : p == 1 ? cx<double>{0, 1} : p == 2 ? cx<double>{-1, 0}
                                                                                     : cx<double>{0, -1};
    A[r][gperm(mu, r)] = ph;
  }
}

__global__ void k_clover(const double* __restrict__ nat, double* __restrict__ c64, float* __restrict__ c32,
                         Lat g, double m0, double c_sw) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  cx<double> M[2][6][6];
  for (int h = 0; h < 2; ++h)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) M[h][i][j] = cx<double>{0, 0};

  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu) {
      // four leaves of the mu-nu plane through x, all with the same orientation
      M3 l1 = mm(mm(ld_nat_link(nat, s, mu), ld_nat_link(nat, shifted(g, c, mu, 1, nu, 0), nu)),
                 mm(dag(ld_nat_link(nat, shifted(g, c, mu, 0, nu, 1), mu)), dag(ld_nat_link(nat, s, nu))));
      M3 l2 = mm(mm(ld_nat_link(nat, s, nu), dag(ld_nat_link(nat, shifted(g, c, mu, -1, nu, 1), mu))),
                 mm(dag(ld_nat_link(nat, shifted(g, c, mu, -1, nu, 0), nu)),
                    ld_nat_link(nat, shifted(g, c, mu, -1, nu, 0), mu)));
      M3 l3 = mm(mm(dag(ld_nat_link(nat, shifted(g, c, mu, -1, nu, 0), mu)),
                    dag(ld_nat_link(nat, shifted(g, c, mu, -1, nu, -1), nu))),
                 mm(ld_nat_link(nat, shifted(g, c, mu, -1, nu, -1), mu),
                    ld_nat_link(nat, shifted(g, c, mu, 0, nu, -1), nu)));
      M3 l4 = mm(mm(dag(ld_nat_link(nat, shifted(g, c, mu, 0, nu, -1), nu)),
                    ld_nat_link(nat, shifted(g, c, mu, 0, nu, -1), mu)),
                 mm(ld_nat_link(nat, shifted(g, c, mu, 1, nu, -1), nu), dag(ld_nat_link(nat, s, mu))));
      M3 F;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          cx<double> q = l1.m[a][b] + l2.m[a][b] + l3.m[a][b] + l4.m[a][b];
          cx<double> qt = conj(l1.m[b][a] + l2.m[b][a] + l3.m[b][a] + l4.m[b][a]);
          F.m[a][b] = q - qt;
        }
      // gamma_mu gamma_nu = diag(A_mu A_nu^dagger, A_mu^dagger A_nu)
      cx<double> Am[2][2], An[2][2], G[2][2][2];
      amat(mu, Am);
      amat(nu, An);
      for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 2; ++q) {
          cx<double> g0{0, 0}, g1{0, 0};
          for (int k = 0; k < 2; ++k) {
            g0 = g0 + Am[r][k] * conj(An[q][k]);
            g1 = g1 + conj(Am[k][r]) * An[k][q];
          }
          G[0][r][q] = g0;
          G[1][r][q] = g1;
        }
      // sum over ordered pairs = 2 x sum over mu < nu
      for (int h = 0; h < 2; ++h)
        for (int r = 0; r < 2; ++r)
          for (int q = 0; q < 2; ++q)
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) {
                M[h][3 * r + a][3 * q + b] = M[h][3 * r + a][3 * q + b] + G[h][r][q] * F.m[a][b];
              }
    }
  double pk[72];
  const double scale = -c_sw / 16.0;
  for (int h = 0; h < 2; ++h) {
    double* o = pk + 36 * h;
    for (int i = 0; i < 6; ++i) o[i] = m0 + 4.0 + scale * M[h][i][i].r;
    int k = 6;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j) {
        o[k++] = scale * M[h][i][j].r;
        o[k++] = scale * M[h][i][j].i;
      }
  }
  st_re<double, 72>(c64, g.V, s, pk);
  float pf[72];
  for (int k = 0; k < 72; ++k) pf[k] = (float)pk[k];
  st_re<float, 72>(c32, g.V, s, pf);
}

void launch_clover(const double* nat, double* c64, float* c32, const Lat& g, double m0, double c_sw,
                   cudaStream_t st) {
  k_clover<<<(g.V + 63) / 64, 64, 0, st>>>(nat, c64, c32, g, m0, c_sw);
}

// ===========================================================================
// D(mu) stencil (hop helpers in tm_stencil.cuh)
// ===========================================================================
template <typename T>
struct DslashArgs {
  const T* gauge;
  const T* clover;
  const T* in;
  T* out;
  const T* b;
  Lat g;
  T mu;
  T bc;
  int nrhs;
  T rho;  // odd sites carry mu + rho (Sec. 2: a different twisted mass on even and odd sites)
};

// right-hand sides vary fastest over the CTAs so the links and clover of a site
// block are read from DRAM once and reused from L2 by the other right-hand sides
template <typename T, bool RES>
__global__ void __launch_bounds__(128) k_dslash(DslashArgs<T> a) {
  const int rhs = a.nrhs == 1 ? 0 : (int)(blockIdx.x % a.nrhs);
  const int s = (a.nrhs == 1 ? blockIdx.x : blockIdx.x / a.nrhs) * blockDim.x + threadIdx.x;
  if (s >= a.g.V) return;
  const long off = (long)rhs * NR_SPINOR * a.g.V;
  const T* in = a.in + off;
  int c[4];
  site_coords(a.g, s, c);
  cx<T> acc[12];
  all_hops_global<T>(in, a.gauge, a.g, s, c, a.bc, acc);
  cx<T> p[12], y[12];
  ld_cx<T, 12>(in, a.g.V, s, p);
  site_diag<T>(a.clover, a.g.V, s, ((c[0] + c[1] + c[2] + c[3]) & 1) ? a.mu + a.rho : a.mu, p, y);
  const T half = T(0.5);
#pragma unroll
  for (int k = 0; k < 12; ++k) y[k] = y[k] - half * acc[k];
  if constexpr (RES) {
    cx<T> bb[12];
    ld_cx<T, 12>(a.b + off, a.g.V, s, bb);
#pragma unroll
    for (int k = 0; k < 12; ++k) y[k] = bb[k] - y[k];
  }
  st_cx<T, 12>(a.out + off, a.g.V, s, y);
}

template <typename T>
void launch_dslash(const T* gauge, const T* clover, const T* in, T* out, const T* b, const Lat& g, double mu,
                   double bc_t, int nrhs, cudaStream_t st, double rho) {
  DslashArgs<T> a{gauge, clover, in, out, b, g, (T)mu, (T)bc_t, nrhs, (T)rho};
  dim3 grid((unsigned)((g.V + 127) / 128) * (unsigned)nrhs);
  if (b)
    k_dslash<T, true><<<grid, 128, 0, st>>>(a);
  else
    k_dslash<T, false><<<grid, 128, 0, st>>>(a);
}
template void launch_dslash<double>(const double*, const double*, const double*, double*, const double*,
                                    const Lat&, double, double, int, cudaStream_t, double);
template void launch_dslash<float>(const float*, const float*, const float*, float*, const float*, const Lat&,
                                   double, double, int, cudaStream_t, double);

}  // namespace tmamg
