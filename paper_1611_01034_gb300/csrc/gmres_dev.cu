// Device-side bookkeeping of a fixed-step GMRES cycle, so that a whole
// coarsest-level solve (Sec. 3: odd-even GMRES on the coarsest level) is a
// sequence of launches with no host decision in it and can be captured and
// replayed as one CUDA graph.
//
// Per right-hand side r, one thread keeps the least-squares state of GMRES:
// the Hessenberg columns H (rotated into upper-triangular R), the complex
// Givens rotations G_j = [[c_j, s_j], [-conj(s_j), c_j]] (c_j real) and the
// rotated right-hand side g = |b| e_1.  A right-hand side stops updating once
// the new Arnoldi vector vanishes or its residual estimate |g_{k+1}| reaches
// tol |b|; later steps of the graph then leave its state alone, and the
// solution update uses its first kk[r] basis vectors only.
#include "tm_kernels.h"

namespace tmamg {

namespace {

__device__ __forceinline__ void givens_dev(cx<double> a, double b, double& c, cx<double>& s, cx<double>& rho) {
  const double aa = sqrt(a.r * a.r + a.i * a.i);
  if (b == 0) {
    c = 1;
    s = cx<double>{0, 0};
    rho = a;
  } else if (aa == 0) {
    c = 0;
    s = cx<double>{1, 0};
    rho = cx<double>{b, 0};
  } else {
    const double nu = hypot(aa, b);
    c = aa / nu;
    const cx<double> ph{a.r / aa, a.i / aa};
    s = (b / nu) * ph;
    rho = nu * ph;
  }
}

__global__ void k_gmres_init(GmresDev st, const double* __restrict__ nrm, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const double bn = sqrt(nrm[r]);
  cx<double>* g = st.g + (long)r * (st.m + 1);
  for (int j = 0; j <= st.m; ++j) g[j] = cx<double>{0, 0};
  g[0] = cx<double>{bn, 0};
  st.bnorm[r] = bn;
  st.kk[r] = 0;
  st.done[r] = bn > 0 ? 0 : 1;
}

// step k: the Hessenberg column from the two CGS2 passes (d1, d2: k + 1 complex
// each at dd + r * ds) and |w|^2 (nrm), rotated, the new rotation, g updated
__global__ void k_gmres_step(GmresDev st, const double* __restrict__ dd, long ds, const double* __restrict__ nrm,
                             int k, int nrhs, double tol) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs || st.done[r]) return;
  const int m = st.m;
  const double* d1 = dd + (long)r * ds;
  const double* d2 = d1 + 2 * (k + 1);
  cx<double>* H = st.H + (long)r * (m + 1) * m;
  cx<double>* g = st.g + (long)r * (m + 1);
  double* cs = st.cs + (long)r * m;
  cx<double>* sn = st.sn + (long)r * m;
  for (int j = 0; j <= k; ++j) H[(long)j * m + k] = cx<double>{d1[2 * j] + d2[2 * j], d1[2 * j + 1] + d2[2 * j + 1]};
  const double hn = sqrt(nrm[r]);
  for (int j = 0; j < k; ++j) {
    const cx<double> a = H[(long)j * m + k], b = H[(long)(j + 1) * m + k];
    H[(long)j * m + k] = cs[j] * a + sn[j] * b;
    H[(long)(j + 1) * m + k] = cs[j] * b - cmulc(sn[j], a);
  }
  double c;
  cx<double> s, rho;
  givens_dev(H[(long)k * m + k], hn, c, s, rho);
  cs[k] = c;
  sn[k] = s;
  H[(long)k * m + k] = rho;
  g[k + 1] = -cmulc(s, g[k]);
  g[k] = c * g[k];
  st.kk[r] = k + 1;
  const double res = sqrt(g[k + 1].r * g[k + 1].r + g[k + 1].i * g[k + 1].i);
  if (hn == 0 || res <= tol * st.bnorm[r]) st.done[r] = 1;
}

// y = R^-1 g over the first kk[r] steps, written as the coefficients of the
// solution update (dd + r * ds, complex); coefficients up to kmax are zeroed
__global__ void k_gmres_solve(GmresDev st, double* __restrict__ dd, long ds, int kmax, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const int m = st.m, k = st.kk[r];
  const cx<double>* H = st.H + (long)r * (m + 1) * m;
  const cx<double>* g = st.g + (long)r * (m + 1);
  double* y = dd + (long)r * ds;
  for (int i = k; i < kmax; ++i) y[2 * i] = y[2 * i + 1] = 0;
  for (int i = k - 1; i >= 0; --i) {
    cx<double> acc = g[i];
    for (int j = i + 1; j < k; ++j) acc = acc - H[(long)i * m + j] * cx<double>{y[2 * j], y[2 * j + 1]};
    const cx<double> d = H[(long)i * m + i];
    const double dn = d.r * d.r + d.i * d.i;
    const cx<double> q = dn > 0 ? cx<double>{(acc.r * d.r + acc.i * d.i) / dn, (acc.i * d.r - acc.r * d.i) / dn}
                                : cx<double>{0, 0};
    y[2 * i] = q.r;
    y[2 * i + 1] = q.i;
  }
}

}  // namespace

void launch_gmres_init(const GmresDev& st, const double* nrm, int nrhs, cudaStream_t s) {
  k_gmres_init<<<(nrhs + 31) / 32, 32, 0, s>>>(st, nrm, nrhs);
}
void launch_gmres_step(const GmresDev& st, const double* dd, long ds, const double* nrm, int k, int nrhs, double tol,
                       cudaStream_t s) {
  k_gmres_step<<<(nrhs + 31) / 32, 32, 0, s>>>(st, dd, ds, nrm, k, nrhs, tol);
}
void launch_gmres_solve(const GmresDev& st, double* dd, long ds, int kmax, int nrhs, cudaStream_t s) {
  k_gmres_solve<<<(nrhs + 31) / 32, 32, 0, s>>>(st, dd, ds, kmax, nrhs);
}

}  // namespace tmamg
