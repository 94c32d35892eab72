// C ABI and host orchestration of the twisted-mass DD-alphaAMG solver:
// FGMRES (FP64) preconditioned by the K-cycle of eq. (1) (SAP smoother,
// restriction, odd-even GMRES on D_c(delta mu), prolongation), the adaptive
// setup, and the field-level entry points.  All arithmetic on vectors runs
// in the kernels of dirac.cu, sap.cu, coarse.cu and blas.cu; the host only
// sequences launches and solves the small Hessenberg least-squares problems.
#include "tm.h"
#include "tm_kernels.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include <cuda_fp16.h>
#include <map>
#include <mutex>
#include <string>
#include <vector>

using namespace tmamg;

namespace {

struct TmError {
  tm_status s;
  std::string m;
};

[[noreturn]] void raise(tm_status s, const std::string& m) { throw TmError{s, m}; }

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    raise(e == cudaErrorMemoryAllocation ? TM_ERR_OOM : TM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
}
#define CK(x) ck((x), #x)
#define CKL() ck(cudaGetLastError(), "kernel launch")

struct Buf {
  void* p = nullptr;
  size_t n = 0;
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct tm_handle {
  tm_params p;
  cudaStream_t st = nullptr;
  Lat g{}, gc{};
  SapGeom sg{};
  AggGeom ag{};
  OEGeom oe{};
  int n = 0;       // 2 Nv
  int nhalf = 0;   // coarse sites per parity
  int* d_err = nullptr;
  double* g64 = nullptr;
  float* g32 = nullptr;
  double* c64 = nullptr;
  float* c32 = nullptr;
  void* tv = nullptr;
  void* P = nullptr;
  void* Dc = nullptr;
  void* Dinv = nullptr;
  int* d_even = nullptr;
  int* d_odd = nullptr;
  int* d_cidx = nullptr;
  double* scratch = nullptr;  // reduction partials
  double* dsmall = nullptr;   // small device results
  double* hsmall = nullptr;   // pinned host mirror
  std::map<std::string, std::pair<double*, size_t>> hbufs;  // pinned host scratch per solver
  // three levels: level-1 aggregation P2 and the coarsest operator D_c2
  bool three = false;
  Lat gc2{};
  int n2 = 0, nhalf2 = 0;
  CSapGeom csg{};
  CAggGeom cag{};
  OEGeom oe2{};
  void* tv1 = nullptr;   // level-1 test vectors (Nv2 level-1 fields)
  void* P2 = nullptr;
  void* Dc2 = nullptr;
  void* Dinv2 = nullptr;
  int* d_even2 = nullptr;
  int* d_odd2 = nullptr;
  int* d_cidx2 = nullptr;
  void* Dc1h = nullptr;  // 16-bit copy of D_c1 for the level-1 SAP (sap1_prec = TM_F16 / TM_BF16)
  void* P16 = nullptr;   // 16-bit copy of P for the transfers (transfer_prec = TM_F16 / TM_BF16)
  void* g16 = nullptr;   // 16-bit links, clover and odd-site inverses of the fine SAP (sap_prec)
  void* c16 = nullptr;
  void* dinv16 = nullptr;
  // links and clover as FP32 pairs for the outer D(mu) z_k (outer_apply = TM_F32X2)
  void* gdf = nullptr;
  void* cdf = nullptr;
  // (A(x) + i mu gamma5)^-1 at the odd sites for the odd-even SAP block solves (block_oe = 1)
  void* dinv_sap = nullptr;
  // twisted-mass shift of the odd sites (Sec. 2): mu on even, mu + rho on odd sites
  double rho = 0;
  // odd-even Schur complement of the coarsest level on the tensor cores
  bool tc_on = false;
  TcGeom tc{};
  // learned gauge-covariant layer: weights (W1 then W2), device copies, Adam state
  std::vector<std::complex<double>> nn_w;
  float2* d_nnw = nullptr;    // [5][1152]: W1, W2, W1 and W2 rounded to FP16, W2 adjoint
  double2* d_nngrad = nullptr;  // [2][1152]
  std::vector<double> adam_m, adam_v;
  long adam_t = 0;
  std::map<std::string, Buf> work;
  bool gauge_ok = false, setup_ok = false;
  bool tv_ok = false;  // test vectors of an earlier setup are present (they survive a new gauge field)
  std::string err;
  long long coarse_iters = 0;
  int kcycles = 0;
  // opt-in per-kernel timing (tm_profile)
  bool prof = false;
  unsigned prof_mask = 0;  // classes timed with events (all classes are counted)
  struct Rec {
    int kind, units, nk;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> evpool;
  cudaEvent_t pipe_ev[2] = {nullptr, nullptr};  // the coarse GMRES's double-buffered step results
  // CUDA graphs of fixed-step coarsest solves (coarsest_steps > 0), keyed by
  // every pointer and scalar they captured; captured on a private stream
  struct GraphEntry {
    cudaGraphExec_t exec;
    size_t nodes;
  };
  std::map<std::string, GraphEntry> graphs;
  cudaStream_t cap_st = nullptr;
  BuildShape build_shape{};                     // tile shape of the D_c build (autotuned or default)
  long long prof_launch[24] = {};
  long long prof_units[24] = {};
  double prof_ms[24] = {};
};

namespace {

constexpr int kScratchBlocks = kReduceBlocks;
constexpr long kFuseMaxCx = 1L << 18;  // batched Arnoldi vectors up to this many complex numbers use fused reductions
constexpr int kMaxDots = 128;
constexpr int kSmall = 4096;

size_t csize(int prec) { return prec == TM_F64 ? sizeof(double) : sizeof(float); }

void* dalloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) return nullptr;
  ck(cudaMalloc(&p, bytes), "cudaMalloc");
  return p;
}

// named, lazily grown device work buffer
template <typename T>
T* W(tm_handle* h, const std::string& name, size_t count) {
  Buf& b = h->work[name];
  const size_t bytes = count * sizeof(T);
  if (b.n < bytes) {
    if (b.p) CK(cudaFree(b.p));
    b.p = nullptr;
    b.n = 0;
    b.p = dalloc(bytes);
    b.n = bytes;
  }
  return static_cast<T*>(b.p);
}

void sync(tm_handle* h) { CK(cudaStreamSynchronize(h->st)); }

// free a named work buffer (cudaFree waits for the work in flight); never throws
void release(tm_handle* h, const std::string& name) noexcept {
  auto it = h->work.find(name);
  if (it == h->work.end()) return;
  if (it->second.p) cudaFree(it->second.p);
  h->work.erase(it);
}

// like W, but zero-filled when (re)allocated: batched solvers run finished
// right-hand sides through shared launches, so their slots must hold finite data
template <typename T>
T* Wz(tm_handle* h, const std::string& name, size_t count) {
  Buf& b = h->work[name];
  const bool fresh = b.n < count * sizeof(T);
  T* p = W<T>(h, name, count);
  if (fresh) CK(cudaMemsetAsync(p, 0, count * sizeof(T), h->st));
  return p;
}

// ---------------------------------------------------------------------------
// opt-in profiler: CUDA events around each launch on the handle's stream
// ---------------------------------------------------------------------------
enum ProfKind {
  PK_DSLASH64 = 0, PK_DSLASH32, PK_SAP, PK_RESTRICT, PK_PROLONG, PK_COARSE_OE, PK_BLAS_FINE, PK_BLAS_COARSE,
  PK_BUILD, PK_OTHER, PK_CSAP, PK_LEVEL1, PK_NN, PK_DSLASHDF, PK_L1XFER, PK_OECG_OP, PK_OECG_BLAS, PK_N
};
static_assert(PK_N <= 24, "profile arrays of the handle hold 24 classes");
const char* const kProfNames[PK_N] = {"dslash_f64", "dslash_f32",   "sap",          "restrict",
                                      "prolong",    "coarse_oe",    "blas_fine",    "blas_coarse",
                                      "coarse_build", "other",      "coarse_sap",   "level1",
                                      "nn",           "dslash_f32x2", "level1_transfer", "oecg_operator",
                                      "oecg_blas"};

cudaEvent_t take_event(tm_handle* h) {
  if (!h->evpool.empty()) {
    cudaEvent_t e = h->evpool.back();
    h->evpool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CK(cudaEventCreate(&e));
  return e;
}

// fold finished records into the totals (all of them if wait)
void harvest(tm_handle* h, bool wait) {
  if (wait) sync(h);
  size_t keep = 0;
  for (size_t i = 0; i < h->recs.size(); ++i) {
    auto& r = h->recs[i];
    if (!wait && cudaEventQuery(r.b) != cudaSuccess) {
      cudaGetLastError();
      h->recs[keep++] = r;
      continue;
    }
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    h->prof_ms[r.kind] += ms;
    h->evpool.push_back(r.a);
    h->evpool.push_back(r.b);
  }
  h->recs.resize(keep);
}

// one scope = nk kernel launches of one class processing u rhs units
struct Prof {
  tm_handle* h;
  int kind, units, nk;
  cudaEvent_t a = nullptr;
  Prof(tm_handle* hh, int k, int u = 1, int n = 1) : h(hh), kind(k), units(u), nk(n) {
    if (!h->prof) return;
    h->prof_launch[kind] += nk;
    h->prof_units[kind] += units;
    if (!((h->prof_mask >> kind) & 1u)) return;
    if (h->recs.size() > 4096) harvest(h, false);
    a = take_event(h);
    CK(cudaEventRecord(a, h->st));
  }
  ~Prof() noexcept(false) {
    if (!h->prof || !a) return;
    cudaEvent_t b = take_event(h);
    CK(cudaEventRecord(b, h->st));
    h->recs.push_back({kind, units, nk, a, b});
  }
};

void check_flags(tm_handle* h) {
  int f = 0;
  CK(cudaMemcpyAsync(&f, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  sync(h);
  if (f) {
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->st));
    if (f & ERRF_NOT_SU3) raise(TM_ERR_NOT_SU3, "gauge link not in SU(3) within 1e-10");
    if (f & ERRF_RANK) raise(TM_ERR_ARG, "test vectors are rank deficient on an aggregate");
    if (f & ERRF_SINGULAR) raise(TM_ERR_ARG, "singular coarse self block");
    if (f & ERRF_TIMEOUT) raise(TM_ERR_TIMEOUT, "a bounded device-side wait ran out");
    raise(TM_ERR_NONFINITE, "non-finite value");
  }
}

template <typename T>
const T* gaugeT(tm_handle* h);
template <>
const double* gaugeT<double>(tm_handle* h) { return h->g64; }
template <>
const float* gaugeT<float>(tm_handle* h) { return h->g32; }
template <typename T>
const T* cloverT(tm_handle* h);
template <>
const double* cloverT<double>(tm_handle* h) { return h->c64; }
template <>
const float* cloverT<float>(tm_handle* h) { return h->c32; }

long fine_reals(tm_handle* h) { return (long)NR_SPINOR * h->g.V; }
long coarse_cx(tm_handle* h) { return (long)h->gc.V * h->n; }

double mu_c(tm_handle* h) { return h->p.delta * h->p.mu; }

// ---------------------------------------------------------------------------
// fine operator pieces
// ---------------------------------------------------------------------------
template <typename T>
void dslash(tm_handle* h, const T* in, T* out, const T* b, int nrhs) {
  Prof pf(h, std::is_same<T, double>::value ? PK_DSLASH64 : PK_DSLASH32, nrhs);
  launch_dslash<T>(gaugeT<T>(h), cloverT<T>(h), in, out, b, h->g, h->p.mu, h->p.bc_t, nrhs, h->st, h->rho);
  CKL();
}

// out (FP64) = D(mu) in (FP32) in FP32-pair arithmetic
void dslash_df(tm_handle* h, const float* in, double* out, int nrhs) {
  Prof pf(h, PK_DSLASHDF, nrhs);
  launch_dslash_df(h->gdf, h->cdf, in, out, h->g, h->p.mu, h->p.bc_t, nrhs, h->st, h->rho);
  CKL();
}

template <typename T>
void sap_sweeps(tm_handle* h, const T* b, T* x, int sweeps, int nrhs) {
  if (h->p.block_oe && (sizeof(T) == 8) != (h->p.cycle_prec == TM_F64))
    raise(TM_ERR_ARG, "with block_oe = 1 the SAP smoother runs in cycle_prec");
  for (int s = 0; s < sweeps; ++s)
    for (int colour = 0; colour < 2; ++colour) {
      Prof pf(h, PK_SAP, nrhs);
      if (h->p.block_oe && h->g16)  // 16-bit links, clover and D_oo^-1 (sap_prec)
        launch_sap_oe_colour<T>(h->g16, h->c16, h->dinv16, b, x, h->sg, h->p.mu, h->p.bc_t, h->p.mr_iters, colour,
                                nrhs, h->st, h->rho, h->p.sap_prec);
      else if (h->p.block_oe)
        launch_sap_oe_colour<T>(gaugeT<T>(h), cloverT<T>(h), h->dinv_sap, b, x, h->sg, h->p.mu, h->p.bc_t,
                                h->p.mr_iters, colour, nrhs, h->st, h->rho);
      else
        launch_sap_colour<T>(gaugeT<T>(h), cloverT<T>(h), b, x, h->sg, h->p.mu, h->p.bc_t, h->p.mr_iters, colour,
                             nrhs, h->st, h->rho);
      CKL();
    }
}

// (A(x) + i mu gamma5)^-1 at the odd sites for the odd-even SAP (after a new
// clover term or a new mu)
void build_sap_inverse(tm_handle* h) {
  if (!h->dinv_sap) return;
  Prof pf(h, PK_OTHER);
  if (h->p.cycle_prec == TM_F64)
    launch_clover_inverse<double>(h->c64, static_cast<double*>(h->dinv_sap), h->g, h->p.mu + h->rho, h->d_err,
                                  h->st);
  else
    launch_clover_inverse<float>(h->c64, static_cast<float*>(h->dinv_sap), h->g, h->p.mu + h->rho, h->d_err,
                                 h->st);
  CKL();
  if (h->dinv16) {
    launch_to16(static_cast<const float*>(h->dinv_sap), h->dinv16, (long)h->g.V / 2 * 72, h->p.sap_prec, h->st);
    CKL();
  }
}

// ||x_r||^2 for nrhs vectors -> host
template <typename T>
std::vector<double> norms2(tm_handle* h, const T* x, long ncx, int nrhs, int kind) {
  {
    Prof pf(h, kind, nrhs, 2);
    launch_norm2<T>(x, ncx, nrhs, h->dsmall, h->scratch, kScratchBlocks, h->st);
    CKL();
  }
  CK(cudaMemcpyAsync(h->hsmall, h->dsmall, nrhs * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  sync(h);
  return std::vector<double>(h->hsmall, h->hsmall + nrhs);
}

// ---------------------------------------------------------------------------
// restarted (flexible) GMRES, CGS2 Arnoldi, Givens on the host
//   A(const T* in, T* out)   operator on basis-type vectors (true residuals)
//   AZ(const TZ* z, T* out)  operator on preconditioned vectors (flexible)
//   M(const T* v, TZ* z)     preconditioner (flexible)
// ---------------------------------------------------------------------------
struct KrylovOut {
  int iters = 0;
  int restarts = 0;
  double relres = 0;
  bool converged = false;
};

void givens(std::complex<double> a, double b, double& c, std::complex<double>& s, std::complex<double>& rho) {
  if (b == 0) {
    c = 1;
    s = 0;
    rho = a;
    return;
  }
  if (std::abs(a) == 0) {
    c = 0;
    s = 1;
    rho = b;
    return;
  }
  const double nu = std::hypot(std::abs(a), b);
  c = std::abs(a) / nu;
  const std::complex<double> ph = a / std::abs(a);
  s = ph * b / nu;  // conj(b) = b (real)
  rho = ph * nu;
}

template <typename T, typename TZ, typename FA, typename FAZ, typename FM>
KrylovOut krylov(tm_handle* h, const std::string& tag, FA A, FAZ AZ, FM M, bool flexible, const T* b, T* x,
                 bool x0, long ncx, double tol, int m, int maxit) {
  const int bk = flexible ? PK_BLAS_FINE : PK_BLAS_COARSE;
  using cd = std::complex<double>;
  KrylovOut out;
  T* Vb = W<T>(h, tag + "V", (size_t)(m + 1) * 2 * ncx);
  T* w = W<T>(h, tag + "w", (size_t)2 * ncx);
  TZ* Z = flexible ? W<TZ>(h, tag + "Z", (size_t)m * 2 * ncx) : nullptr;
  const long ld = 2 * ncx;
  const double bnorm = std::sqrt(norms2<T>(h, b, ncx, 1, bk)[0]);
  if (!std::isfinite(bnorm)) raise(TM_ERR_NONFINITE, "non-finite right-hand side");
  if (!x0) {
    Prof pf(h, bk);
    launch_zero<T>(x, 2 * ncx, h->st);
    CKL();
  }
  if (bnorm == 0) {
    Prof pf(h, bk);
    launch_zero<T>(x, 2 * ncx, h->st);
    CKL();
    out.converged = true;
    return out;
  }
  // r = b - A x
  auto residual = [&](T* r) {
    if (x0 || out.iters > 0) {
      A(x, w);
      CK(cudaMemcpyAsync(r, b, 2 * ncx * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
      Prof pf(h, bk);
      launch_caxpby<T>(-1, 0, w, 1, 0, r, ncx, h->st);
      CKL();
    } else {
      CK(cudaMemcpyAsync(r, b, 2 * ncx * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
    }
    return std::sqrt(norms2<T>(h, r, ncx, 1, bk)[0]);
  };
  double beta = residual(Vb);
  std::vector<cd> H((size_t)(m + 1) * m), g(m + 1), sn(m), y(m);
  std::vector<double> cs(m);
  while (beta > tol * bnorm && out.iters < maxit) {
    if (!std::isfinite(beta)) raise(TM_ERR_NONFINITE, "non-finite residual");
    {
      Prof pf(h, bk);
      launch_caxpby<T>(1.0 / beta, 0, Vb, 0, 0, Vb, ncx, h->st);
      CKL();
    }
    std::fill(g.begin(), g.end(), cd(0));
    g[0] = beta;
    int k = 0;
    while (k < m) {
      T* vk = Vb + (long)k * ld;
      if (flexible) {
        TZ* zk = Z + (long)k * ld;
        M(vk, zk);
        AZ(zk, w);
      } else {
        A(vk, w);
      }
      // CGS2 against V_0..V_k
      double* d1 = h->dsmall;
      double* d2 = h->dsmall + 2 * kMaxDots;
      double* dn = h->dsmall + 4 * kMaxDots;
      {
        Prof pf(h, bk, 1, 2);
        launch_multidot<T>(Vb, ld, k + 1, w, ncx, d1, h->scratch, kScratchBlocks, h->st);
        CKL();
      }
      {
        Prof pf(h, bk);
        launch_multi_caxpy<T>(Vb, ld, k + 1, d1, 1.0, w, ncx, h->st);
        CKL();
      }
      {
        Prof pf(h, bk, 1, 2);
        launch_multidot<T>(Vb, ld, k + 1, w, ncx, d2, h->scratch, kScratchBlocks, h->st);
        CKL();
      }
      {
        Prof pf(h, bk);
        launch_multi_caxpy<T>(Vb, ld, k + 1, d2, 1.0, w, ncx, h->st);
        CKL();
      }
      {
        Prof pf(h, bk, 1, 2);
        launch_norm2<T>(w, ncx, 1, dn, h->scratch, kScratchBlocks, h->st);
        CKL();
      }
      CK(cudaMemcpyAsync(Vb + (long)(k + 1) * ld, w, 2 * ncx * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
      {
        Prof pf(h, bk);
        launch_scale<T>(Vb + (long)(k + 1) * ld, ncx, 1, dn, true, h->st);
        CKL();
      }
      CK(cudaMemcpyAsync(h->hsmall, h->dsmall, (4 * kMaxDots + 1) * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      sync(h);
      const double hn = std::sqrt(h->hsmall[4 * kMaxDots]);
      if (!std::isfinite(hn)) raise(TM_ERR_NONFINITE, "non-finite Arnoldi vector");
      std::vector<cd> col(m + 1, cd(0));
      for (int j = 0; j <= k; ++j)
        col[j] = cd(h->hsmall[2 * j] + h->hsmall[2 * kMaxDots + 2 * j],
                    h->hsmall[2 * j + 1] + h->hsmall[2 * kMaxDots + 2 * j + 1]);
      col[k + 1] = hn;
      for (int j = 0; j < k; ++j) {
        const cd t = cs[j] * col[j] + sn[j] * col[j + 1];
        col[j + 1] = -std::conj(sn[j]) * col[j] + cs[j] * col[j + 1];
        col[j] = t;
      }
      double c;
      cd s, rho;
      givens(col[k], hn, c, s, rho);
      cs[k] = c;
      sn[k] = s;
      col[k] = rho;
      col[k + 1] = 0;
      for (int j = 0; j <= m; ++j) H[(size_t)j * m + k] = col[j];
      g[k + 1] = -std::conj(s) * g[k];
      g[k] = c * g[k];
      ++out.iters;
      ++k;
      if (hn == 0 || std::abs(g[k]) <= tol * bnorm || out.iters >= maxit) break;
    }
    // back substitution R y = g
    for (int i = k - 1; i >= 0; --i) {
      cd acc = g[i];
      for (int j = i + 1; j < k; ++j) acc -= H[(size_t)i * m + j] * y[j];
      y[i] = acc / H[(size_t)i * m + i];
    }
    for (int i = 0; i < k; ++i) {
      h->hsmall[2 * i] = y[i].real();
      h->hsmall[2 * i + 1] = y[i].imag();
    }
    double* dy = h->dsmall + 6 * kMaxDots;
    CK(cudaMemcpyAsync(dy, h->hsmall, 2 * k * sizeof(double), cudaMemcpyHostToDevice, h->st));
    {
      Prof pf(h, bk);
      if (flexible)
        launch_lincomb<TZ, T>(Z, ld, k, dy, x, ncx, h->st);
      else
        launch_lincomb<T, T>(Vb, ld, k, dy, x, ncx, h->st);
      CKL();
    }
    ++out.restarts;
    beta = residual(Vb);
  }
  out.relres = beta / bnorm;
  out.converged = beta <= tol * bnorm;
  return out;
}

// ---------------------------------------------------------------------------
// coarse level
// 16-bit copies of FP32 operators read by the K-cycle: D_c1 for the level-1
// SAP (sap1_prec) and P for the transfers (transfer_prec)
void refresh_16bit(tm_handle* h) {
  if (h->Dc1h) {
    launch_to16(static_cast<const float*>(h->Dc), h->Dc1h, (long)h->gc.V * 9 * h->n * h->n, h->p.sap1_prec, h->st);
    CKL();
  }
  if (h->P16) {
    launch_to16(static_cast<const float*>(h->P), h->P16, (long)h->p.nv * h->g.V * 12, h->p.transfer_prec, h->st);
    CKL();
  }
}

// ---------------------------------------------------------------------------
// orth = false: D_c projected again from the current (orthonormal) P, e.g.
// after a change of the odd-site twisted-mass shift
template <typename T>
void build_coarse(tm_handle* h, bool orth = true) {
  T* P = static_cast<T*>(h->P);
  constexpr bool f32 = std::is_same<T, float>::value;
  // orthonormalisation + build, the FP16 copy, the odd-site inverses and the
  // three tensor-core tile kernels
  const int nk = (orth ? 2 : 1) + (f32 && h->Dc1h ? 1 : 0) + (f32 && h->P16 ? 1 : 0) + (h->three ? 0 : 1) +
                 (f32 && h->tc_on && !h->three ? 3 : 0);
  Prof pf(h, PK_BUILD, 1, nk);
  if (orth) {
    launch_orthonormalise<T>(P, h->ag, h->d_err, h->st);
    CKL();
  }
  launch_coarse_build<T>(gaugeT<T>(h), cloverT<T>(h), P, static_cast<T*>(h->Dc), h->ag, h->p.bc_t, h->st,
                         h->build_shape, h->rho);
  CKL();
  if constexpr (std::is_same<T, float>::value) refresh_16bit(h);
  if (!h->three) {  // with three levels the odd-even solve runs on level 2
    launch_oe_invert<T>(static_cast<T*>(h->Dc), static_cast<T*>(h->Dinv), h->oe, mu_c(h), h->d_err, h->st);
    CKL();
    if constexpr (std::is_same<T, float>::value) {
      if (h->tc_on) {
        tc_build(static_cast<const float*>(h->Dc), static_cast<const float*>(h->Dinv), h->oe, h->tc, h->st);
        CKL();
      }
    }
  }
}

// pinned host scratch of at least n doubles (grown on demand)
// (solvers nest: the fine FGMRES calls the K-cycle, whose level-1 FGMRES calls
// the coarsest GMRES, so each solver keeps its own buffer)
double* host_scratch(tm_handle* h, const char* key, size_t n) {
  auto& b = h->hbufs[key];
  if (b.second < n) {
    if (b.first) CK(cudaFreeHost(b.first));
    b.first = nullptr;
    b.second = 0;
    CK(cudaMallocHost(&b.first, n * sizeof(double)));
    b.second = n;
  }
  return b.first;
}

// the level an odd-even GMRES runs on
struct OELevel {
  const void* Dc;
  const void* Dinv;
  OEGeom oe;
  int n, nhalf, Vc;
  double mu_c;
  const TcGeom* tc;  // tensor-core tiles of this level (or null)
};

OELevel coarsest_level(tm_handle* h) {
  const TcGeom* tc = h->tc_on ? &h->tc : nullptr;
  if (h->three) return OELevel{h->Dc2, h->Dinv2, h->oe2, h->n2, h->nhalf2, h->gc2.V, mu_c(h), tc};
  return OELevel{h->Dc, h->Dinv, h->oe, h->n, h->nhalf, h->gc.V, mu_c(h), tc};
}

// Exactly K odd-even GMRES steps on D_c(delta mu) x_r = b_r from zero, every
// decision on the device (gmres_dev.cu: a right-hand side whose residual
// estimate reaches tol stops updating), captured once per set of buffers and
// scalars as a CUDA graph and replayed: one launch per coarsest solve instead
// of about eight launches and a host decision per Arnoldi step.  With a fixed
// step count the coarsest solve is the same polynomial in D_c for every call,
// a fixed preconditioner for the level above.
template <typename T>
std::vector<int> coarse_solve_graph(tm_handle* h, const OELevel& lv, const T* b, T* x, int nrhs, double tol, int K) {
  const long nc = (long)lv.nhalf * lv.n;
  const long cv = 2 * nc;
  const long cf = 2 * (long)lv.Vc * lv.n;
  const long vstr = (long)(K + 1) * cv;
  const long ds = 4 * kMaxDots + 2;
  const T* Dc = static_cast<const T*>(lv.Dc);
  const T* Di = static_cast<const T*>(lv.Dinv);
  T* to = W<T>(h, "gq_to", cv * nrhs);
  T* bh = W<T>(h, "gq_bh", cv * nrhs);
  T* xe = W<T>(h, "gq_xe", cv * nrhs);
  T* uo = W<T>(h, "gq_uo", cv * nrhs);
  T* w = W<T>(h, "gq_w", cv * nrhs);
  T* Vb = W<T>(h, "gq_V", vstr * nrhs);
  double* part = W<double>(h, "gq_part", std::max(multidot_scratch_doubles(nc, K + 1, nrhs), 2L * 304 * nrhs));
  double* dd = W<double>(h, "gq_dots", ds * nrhs);
  double* nrm = W<double>(h, "gq_nrm", nrhs);
  GmresDev st{reinterpret_cast<cx<double>*>(W<double>(h, "gq_H", (size_t)2 * (K + 1) * K * nrhs)),
              reinterpret_cast<cx<double>*>(W<double>(h, "gq_g", (size_t)2 * (K + 1) * nrhs)),
              W<double>(h, "gq_cs", (size_t)K * nrhs),
              reinterpret_cast<cx<double>*>(W<double>(h, "gq_sn", (size_t)2 * K * nrhs)),
              W<double>(h, "gq_bn", nrhs), W<int>(h, "gq_kk", nrhs), W<int>(h, "gq_done", nrhs), K};
  const double mc = lv.mu_c;
  bool use_tc = false;
  if constexpr (std::is_same<T, float>::value)
    use_tc = lv.tc && nrhs >= 2 && tc_supported(lv.oe.nv, nrhs, h->p.coarse_mma);
  auto enqueue = [&](cudaStream_t s) {
    auto schur = [&](const T* v) {
      if constexpr (std::is_same<T, float>::value) {
        if (use_tc) {
          launch_tc_schur(*lv.tc, lv.oe, v, uo, w, mc, nrhs, vstr, cv, cv, nullptr, h->p.coarse_mma, h->d_err, s,
                          (unsigned)h->p.tc_spin_limit);
          CKL();
          return;
        }
      }
      launch_oe_schur_b<T>(Dc, Di, v, uo, w, lv.oe, mc, nrhs, vstr, cv, cv, nullptr, s);
      CKL();
    };
    launch_oe_prepare_b<T>(Dc, Di, b, to, bh, lv.oe, nrhs, cf, cv, s);
    CKL();
    launch_zero<T>(xe, cv * nrhs, s);
    CKL();
    launch_norm2_b<T>(bh, cv, nc, nrm, part, nrhs, nullptr, s);
    CKL();
    launch_gmres_init(st, nrm, nrhs, s);
    CKL();
    launch_scale_copy_b<T>(bh, cv, Vb, vstr, nrm, nc, nrhs, nullptr, s);  // v_0 = r / |r|
    CKL();
    for (int k = 0; k < K; ++k) {
      schur(Vb + (long)k * cv);
      double* d1 = dd;
      double* d2 = dd + 2 * (k + 1);
      launch_multidot_b_partials<T>(Vb, vstr, cv, k + 1, w, cv, nc, part, nrhs, nullptr, s);
      CKL();
      launch_multi_caxpy_bp<T>(Vb, vstr, cv, k + 1, part, nc, d1, ds, w, cv, nc, nrhs, nullptr, s);
      CKL();
      launch_multidot_b_partials<T>(Vb, vstr, cv, k + 1, w, cv, nc, part, nrhs, nullptr, s);
      CKL();
      launch_multi_caxpy_bp<T>(Vb, vstr, cv, k + 1, part, nc, d2, ds, w, cv, nc, nrhs, nullptr, s);
      CKL();
      launch_norm2_b_partials<T>(w, cv, nc, part, nrhs, nullptr, s);
      CKL();
      launch_scale_copy_bp<T>(w, cv, Vb + (long)(k + 1) * cv, vstr, part, nrm, nc, nrhs, nullptr, s);
      CKL();
      launch_gmres_step(st, dd, ds, nrm, k, nrhs, tol, s);
      CKL();
    }
    launch_gmres_solve(st, dd, ds, K, nrhs, s);
    CKL();
    launch_lincomb_b<T, T>(Vb, vstr, cv, K, dd, ds, xe, cv, nc, nrhs, nullptr, s);
    CKL();
    launch_oe_reconstruct_b<T>(Dc, Di, b, xe, x, lv.oe, nrhs, cf, cv, s);
    CKL();
  };
  char key[512];
  std::snprintf(key, sizeof key, "%d %d %d %.17g %.17g %d %d %p %p %p %p %p %p %p %p %p %p %p %p %p %p %p %p %p %p",
                (int)sizeof(T), nrhs, K, mc, tol, h->p.coarse_mma, h->p.tc_spin_limit, (const void*)b, (void*)x,
                (const void*)Dc, (const void*)Di, (void*)to, (void*)bh, (void*)xe, (void*)uo, (void*)w, (void*)Vb,
                (void*)part, (void*)dd, (void*)nrm, (void*)st.H, (void*)st.g, (void*)st.kk,
                use_tc ? (const void*)lv.tc->even : nullptr, use_tc ? (const void*)lv.tc->odd : nullptr);
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    if (h->graphs.size() >= 32) {  // bound the cache: drop the old graphs
      for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
      h->graphs.clear();
    }
    if (!h->cap_st) CK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
    cudaGraph_t gr = nullptr;
    CK(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal));
    try {
      enqueue(h->cap_st);
    } catch (...) {
      cudaStreamEndCapture(h->cap_st, &gr);
      if (gr) cudaGraphDestroy(gr);
      throw;
    }
    CK(cudaStreamEndCapture(h->cap_st, &gr));
    tm_handle::GraphEntry e{nullptr, 0};
    CK(cudaGraphGetNodes(gr, nullptr, &e.nodes));
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, gr, 0);
    cudaGraphDestroy(gr);
    CK(ie);
    it = h->graphs.emplace(key, e).first;
  }
  {
    Prof pf(h, PK_COARSE_OE, K * nrhs, (int)it->second.nodes);
    CK(cudaGraphLaunch(it->second.exec, h->st));
  }
  h->coarse_iters += (long long)K * nrhs;
  if (use_tc) check_flags(h);  // bounded waits inside the tensor-core kernel
  return std::vector<int>(nrhs, K);
}

// Odd-even GMRES(coarse_restart) on D_c(delta mu) x_r = b_r for nrhs full
// coarse vectors at once.  Every right-hand side runs its own GMRES (own
// Hessenberg matrix, own restarts and stopping); the batch only shares
// launches and one host synchronisation per Arnoldi step.  Finished right-hand
// sides are masked out, so each one sees exactly the single-rhs arithmetic.
template <typename T>
std::vector<int> coarse_solve(tm_handle* h, const OELevel& lv, const T* b, T* x, int nrhs, double tol, int maxit) {
  if (h->p.coarsest_steps > 0)
    return coarse_solve_graph<T>(h, lv, b, x, nrhs, tol, std::min(h->p.coarsest_steps, maxit));
  using cd = std::complex<double>;
  const int m = h->p.coarse_restart;
  const long nc = (long)lv.nhalf * lv.n;         // complex numbers per compact vector
  const long cv = 2 * nc;                        // reals per compact vector
  const long cf = 2 * (long)lv.Vc * lv.n;        // reals per full coarse vector
  const long vstr = (long)(m + 1) * cv;          // per-rhs Krylov basis stride
  const long ds = 4 * kMaxDots + 2;              // per-rhs small-result stride (doubles)
  const T* Dc = static_cast<const T*>(lv.Dc);
  const T* Di = static_cast<const T*>(lv.Dinv);
  T* to = W<T>(h, "cb_to", cv * nrhs);
  T* bh = W<T>(h, "cb_bh", cv * nrhs);
  T* xe = W<T>(h, "cb_xe", cv * nrhs);
  T* uo = W<T>(h, "cb_uo", cv * nrhs);
  T* w = W<T>(h, "cb_w", cv * nrhs);
  T* Vb = Wz<T>(h, "cb_V", vstr * nrhs);
  double* part = W<double>(h, "cb_part", std::max(multidot_scratch_doubles(nc, m + 1, nrhs), 2L * 304 * nrhs));
  double* dd = W<double>(h, "cb_dots", ds * nrhs);
  double* nrm = W<double>(h, "cb_nrm", nrhs);
  int* act = W<int>(h, "cb_act", nrhs);
  constexpr int kSlots = 8;  // mask uploads between two stream synchronisations
  double* hb = host_scratch(h, "cb", (size_t)3 * (ds + 1) * nrhs + (size_t)kSlots * nrhs);
  double* hn_h = hb + (size_t)ds * nrhs;                     // [nrhs] norms
  int* hact0 = reinterpret_cast<int*>(hn_h + nrhs);          // [kSlots][nrhs] masks
  double* hpipe = hn_h + nrhs + (size_t)kSlots * nrhs;       // [2][ds + 1][nrhs] Arnoldi step results
  int slot = 0;  // an async upload reads its slot later: reuse slots only after a sync
  const double mc = lv.mu_c;
  for (cudaEvent_t& e : h->pipe_ev)
    if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));

  std::vector<double> bnorm(nrhs), beta(nrhs);
  std::vector<int> iters(nrhs, 0), kk(nrhs, 0);
  std::vector<char> active(nrhs), inner(nrhs);
  std::vector<cd> H((size_t)nrhs * (m + 1) * m), g((size_t)nrhs * (m + 1)), sn((size_t)nrhs * m);
  std::vector<double> cs((size_t)nrhs * m);

  auto upload_mask = [&](const std::vector<char>& msk, const std::vector<int>* counts) {
    if (slot >= kSlots) {
      sync(h);
      slot = 0;
    }
    int* hact = hact0 + (size_t)(slot++) * nrhs;
    for (int r = 0; r < nrhs; ++r) hact[r] = msk[r] ? (counts ? (*counts)[r] : 1) : 0;
    CK(cudaMemcpyAsync(act, hact, nrhs * sizeof(int), cudaMemcpyHostToDevice, h->st));
  };
  auto count = [&](const std::vector<char>& msk) {
    int c = 0;
    for (char v : msk) c += v ? 1 : 0;
    return c;
  };
  auto read_norms = [&]() {
    CK(cudaMemcpyAsync(hn_h, nrm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    sync(h);
    slot = 0;
  };
  bool use_tc = false;
  if constexpr (std::is_same<T, float>::value)
    use_tc = lv.tc && nrhs >= 2 && tc_supported(lv.oe.nv, nrhs, h->p.coarse_mma);  // one rhs: CUDA cores
  auto schur = [&](const T* v, long vs, int units) {
    Prof pf(h, PK_COARSE_OE, units, 2);
    if constexpr (std::is_same<T, float>::value) {
      if (use_tc) {
        launch_tc_schur(*lv.tc, lv.oe, v, uo, w, mc, nrhs, vs, cv, cv, act, h->p.coarse_mma, h->d_err, h->st,
                        (unsigned)h->p.tc_spin_limit);
        CKL();
        return;
      }
    }
    launch_oe_schur_b<T>(Dc, Di, v, uo, w, lv.oe, mc, nrhs, vs, cv, cv, act, h->st);
    CKL();
  };

  {
    Prof pf(h, PK_COARSE_OE, nrhs, 2);
    launch_oe_prepare_b<T>(Dc, Di, b, to, bh, lv.oe, nrhs, cf, cv, h->st);
    CKL();
  }
  {
    Prof pf(h, PK_BLAS_COARSE, nrhs, 3);
    launch_zero<T>(xe, cv * nrhs, h->st);
    CKL();
    launch_norm2_b<T>(bh, cv, nc, nrm, part, nrhs, nullptr, h->st);
    CKL();
  }
  read_norms();
  for (int r = 0; r < nrhs; ++r) {
    bnorm[r] = std::sqrt(hn_h[r]);
    if (!std::isfinite(bnorm[r])) raise(TM_ERR_NONFINITE, "non-finite coarse right-hand side");
    beta[r] = bnorm[r];
    active[r] = bnorm[r] > 0 && beta[r] > tol * bnorm[r] && iters[r] < maxit;
  }
  {
    Prof pf(h, PK_BLAS_COARSE, nrhs);
    launch_scale_copy_b<T>(bh, cv, Vb, vstr, nullptr, nc, nrhs, nullptr, h->st);
    CKL();
  }
  while (count(active)) {
    // v_0 = r / beta for the right-hand sides of this cycle
    for (int r = 0; r < nrhs; ++r) hn_h[r] = beta[r] * beta[r];
    CK(cudaMemcpyAsync(nrm, hn_h, nrhs * sizeof(double), cudaMemcpyHostToDevice, h->st));
    upload_mask(active, nullptr);
    {
      Prof pf(h, PK_BLAS_COARSE, count(active));
      launch_scale_copy_b<T>(Vb, vstr, Vb, vstr, nrm, nc, nrhs, act, h->st);
      CKL();
    }
    for (int r = 0; r < nrhs; ++r) {
      inner[r] = active[r];
      kk[r] = 0;
      if (active[r]) {
        std::fill(g.begin() + (size_t)r * (m + 1), g.begin() + (size_t)(r + 1) * (m + 1), cd(0));
        g[(size_t)r * (m + 1)] = beta[r];
      }
    }
    // The Arnoldi steps run one ahead of the host: step k + 1 is enqueued
    // before the host waits for the Hessenberg column of step k, so the GPU
    // computes while the host applies the Givens rotations.  Step k + 1 runs
    // under the mask the host held before reading step k; a right-hand side
    // that stops at step k computes it needlessly and its results are never
    // read.  The device results of step k reach the host (in buffer k & 1)
    // before step k + 1 overwrites them, by stream order.
    std::vector<char> uploaded;  // mask in `act`; the cycle's end reuses `act`
    auto arnoldi = [&](int k) {
      const int na = count(inner);
      if (inner != uploaded) {
        upload_mask(inner, nullptr);
        uploaded = inner;
      }
      schur(Vb + (long)k * cv, vstr, na);
      double* d1 = dd;
      double* d2 = dd + 2 * (k + 1);
      {
        // CGS2 in six launches: each reduction's partial sums feed the next step directly
        Prof pf(h, PK_BLAS_COARSE, na, 6);
        launch_multidot_b_partials<T>(Vb, vstr, cv, k + 1, w, cv, nc, part, nrhs, act, h->st);
        CKL();
        launch_multi_caxpy_bp<T>(Vb, vstr, cv, k + 1, part, nc, d1, ds, w, cv, nc, nrhs, act, h->st);
        CKL();
        launch_multidot_b_partials<T>(Vb, vstr, cv, k + 1, w, cv, nc, part, nrhs, act, h->st);
        CKL();
        launch_multi_caxpy_bp<T>(Vb, vstr, cv, k + 1, part, nc, d2, ds, w, cv, nc, nrhs, act, h->st);
        CKL();
        launch_norm2_b_partials<T>(w, cv, nc, part, nrhs, act, h->st);
        CKL();
        launch_scale_copy_bp<T>(w, cv, Vb + (long)(k + 1) * cv, vstr, part, nrm, nc, nrhs, act, h->st);
        CKL();
      }
      double* hk = hpipe + (size_t)(k & 1) * (ds + 1) * nrhs;
      CK(cudaMemcpy2DAsync(hk, 4 * (k + 1) * sizeof(double), dd, ds * sizeof(double), 4 * (k + 1) * sizeof(double),
                           nrhs, cudaMemcpyDeviceToHost, h->st));
      CK(cudaMemcpyAsync(hk + (size_t)ds * nrhs, nrm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      CK(cudaEventRecord(h->pipe_ev[k & 1], h->st));
    };
    arnoldi(0);
    for (int k = 0;; ++k) {
      if (k + 1 < m) arnoldi(k + 1);
      CK(cudaEventSynchronize(h->pipe_ev[k & 1]));
      const double* hk = hpipe + (size_t)(k & 1) * (ds + 1) * nrhs;
      const double* hnk = hk + (size_t)ds * nrhs;
      for (int r = 0; r < nrhs; ++r) {
        if (!inner[r]) continue;
        const double hn = std::sqrt(hnk[r]);
        if (!std::isfinite(hn)) raise(TM_ERR_NONFINITE, "non-finite coarse Arnoldi vector");
        const double* hr = hk + (size_t)r * 4 * (k + 1);
        cd* Hr = H.data() + (size_t)r * (m + 1) * m;
        cd* gr = g.data() + (size_t)r * (m + 1);
        cd* snr = sn.data() + (size_t)r * m;
        double* csr = cs.data() + (size_t)r * m;
        std::vector<cd> col(m + 1, cd(0));
        for (int j = 0; j <= k; ++j)
          col[j] = cd(hr[2 * j] + hr[2 * (k + 1) + 2 * j], hr[2 * j + 1] + hr[2 * (k + 1) + 2 * j + 1]);
        col[k + 1] = hn;
        for (int j = 0; j < k; ++j) {
          const cd t = csr[j] * col[j] + snr[j] * col[j + 1];
          col[j + 1] = -std::conj(snr[j]) * col[j] + csr[j] * col[j + 1];
          col[j] = t;
        }
        double c;
        cd sg, rho;
        givens(col[k], hn, c, sg, rho);
        csr[k] = c;
        snr[k] = sg;
        col[k] = rho;
        col[k + 1] = 0;
        for (int j = 0; j <= m; ++j) Hr[(size_t)j * m + k] = col[j];
        gr[k + 1] = -std::conj(sg) * gr[k];
        gr[k] = c * gr[k];
        ++iters[r];
        kk[r] = k + 1;
        if (hn == 0 || std::abs(gr[k + 1]) <= tol * bnorm[r] || iters[r] >= maxit) inner[r] = 0;
      }
      if (k + 1 >= m || !count(inner)) break;
    }
    // x_r += V_r y_r with R y = g for this cycle's right-hand sides
    int kmax = 0;
    for (int r = 0; r < nrhs; ++r) {
      if (!active[r]) continue;
      const int k = kk[r];
      kmax = std::max(kmax, k);
      const cd* Hr = H.data() + (size_t)r * (m + 1) * m;
      const cd* gr = g.data() + (size_t)r * (m + 1);
      std::vector<cd> y(k);
      for (int i = k - 1; i >= 0; --i) {
        cd acc = gr[i];
        for (int j = i + 1; j < k; ++j) acc -= Hr[(size_t)i * m + j] * y[j];
        y[i] = acc / Hr[(size_t)i * m + i];
      }
      double* yr = hb + (size_t)r * ds;
      for (int i = 0; i < k; ++i) {
        yr[2 * i] = y[i].real();
        yr[2 * i + 1] = y[i].imag();
      }
    }
    CK(cudaMemcpyAsync(dd, hb, ds * nrhs * sizeof(double), cudaMemcpyHostToDevice, h->st));
    upload_mask(active, &kk);
    {
      Prof pf(h, PK_BLAS_COARSE, count(active));
      launch_lincomb_b<T, T>(Vb, vstr, cv, kmax, dd, ds, xe, cv, nc, nrhs, act, h->st);
      CKL();
    }
    // true residual of the reduced systems
    upload_mask(active, nullptr);
    schur(xe, cv, count(active));
    {
      Prof pf(h, PK_BLAS_COARSE, count(active), 4);
      launch_sub_b<T>(bh, cv, w, cv, nc, nrhs, act, h->st);
      CKL();
      launch_norm2_b<T>(w, cv, nc, nrm, part, nrhs, act, h->st);
      CKL();
      launch_scale_copy_b<T>(w, cv, Vb, vstr, nullptr, nc, nrhs, act, h->st);
      CKL();
    }
    read_norms();
    for (int r = 0; r < nrhs; ++r) {
      if (!active[r]) continue;
      beta[r] = std::sqrt(hn_h[r]);
      if (!std::isfinite(beta[r])) raise(TM_ERR_NONFINITE, "non-finite coarse residual");
      active[r] = beta[r] > tol * bnorm[r] && iters[r] < maxit;
    }
  }
  {
    Prof pf(h, PK_COARSE_OE, nrhs, 2);
    launch_oe_reconstruct_b<T>(Dc, Di, b, xe, x, lv.oe, nrhs, cf, cv, h->st);
    CKL();
  }
  for (int r = 0; r < nrhs; ++r) h->coarse_iters += iters[r];
  if (use_tc) check_flags(h);  // bounded waits inside the tensor-core kernel
  return iters;
}

template <typename T>
void level1_solve(tm_handle* h, const T* b1, T* x1, int nrhs, double tol, int maxit);
template <typename Tv, typename Tz, typename FR, typename FAZ, typename FM>
std::vector<KrylovOut> fgmres_b(tm_handle* h, const std::string& tag, int pk, FR resid, FAZ AZ, FM M, const Tv* b,
                                Tv* x, int nb, long ncx, double tol, int m, int maxit);

// z = B(v), eq. (1), nrhs fine fields in T
template <typename T>
void kcycle(tm_handle* h, const T* v, T* z, int nrhs) {
  const long fr = fine_reals(h);
  {
    Prof pf(h, PK_OTHER);
    launch_zero<T>(z, fr * nrhs, h->st);
    CKL();
  }
  sap_sweeps<T>(h, v, z, h->p.pre_smooth, nrhs);
  const T* r = v;
  if (h->p.pre_smooth > 0) {
    T* rr = W<T>(h, "k_r", fr * nrhs);
    dslash<T>(h, z, rr, v, nrhs);
    r = rr;
  }
  const long cc = coarse_cx(h);
  T* rc = W<T>(h, "k_rc", 2 * cc * nrhs);
  T* ec = W<T>(h, "k_ec", 2 * cc * nrhs);
  {
    Prof pf(h, PK_RESTRICT, nrhs);
    launch_restrict<T>(static_cast<const T*>(h->P), r, rc, h->ag, nrhs, h->st, h->P16, h->p.transfer_prec);
    CKL();
  }
  if (h->three)
    level1_solve<T>(h, rc, ec, nrhs, h->p.coarse_tol, h->p.coarse_maxit);
  else
    coarse_solve<T>(h, coarsest_level(h), rc, ec, nrhs, h->p.coarse_tol, h->p.coarse_maxit);
  {
    Prof pf(h, PK_PROLONG, nrhs);
    launch_prolong<T>(static_cast<const T*>(h->P), ec, z, h->ag, nrhs, true, h->st, h->P16, h->p.transfer_prec);
    CKL();
  }
  sap_sweeps<T>(h, v, z, h->p.post_smooth, nrhs);
  h->kcycles += nrhs;
}

// ---------------------------------------------------------------------------
// first coarse level of three (Sec. 2: the standard hierarchy has three levels)
// ---------------------------------------------------------------------------
long level1_cx(tm_handle* h) { return (long)h->gc.V * h->n; }
long level2_cx(tm_handle* h) { return (long)h->gc2.V * h->n2; }
// twisted mass of level 1: mu itself with three levels, delta mu when it is the coarsest
double mu_level1(tm_handle* h) { return h->three ? h->p.mu : mu_c(h); }

template <typename T>
void coarse_apply1(tm_handle* h, const T* in, T* out, int nrhs) {
  Prof pf(h, PK_LEVEL1, nrhs);
  // the K-cycle's level-1 applies read the 16-bit block copy when there is one
  launch_coarse_apply<T>(static_cast<const T*>(h->Dc), in, out, h->gc, h->p.nv, mu_level1(h), nrhs, h->st,
                         std::is_same<T, float>::value ? h->Dc1h : nullptr, h->p.sap1_prec);
  CKL();
}

template <typename T>
void csap_sweeps(tm_handle* h, const T* b, T* x, int sweeps, int nrhs) {
  for (int sw = 0; sw < sweeps; ++sw)
    for (int colour = 0; colour < 2; ++colour) {
      Prof pf(h, PK_CSAP, nrhs);
      launch_csap_colour<T>(static_cast<const T*>(h->Dc), b, x, h->csg, h->p.mu, h->p.mr_iters1, colour, nrhs,
                            h->st, std::is_same<T, float>::value ? h->Dc1h : nullptr, h->p.sap1_prec);
      CKL();
    }
}

// z1 = B1(v1): the level-1 K-cycle (coarse SAP, P2^dagger, coarsest odd-even
// GMRES on D_c2(delta mu), P2, coarse SAP)
template <typename T>
void kcycle1(tm_handle* h, const T* v, T* z, int nrhs) {
  const long c1 = 2 * level1_cx(h), c2 = 2 * level2_cx(h);
  {
    Prof pf(h, PK_OTHER, nrhs);
    launch_zero<T>(z, c1 * nrhs, h->st);
    CKL();
  }
  csap_sweeps<T>(h, v, z, h->p.pre_smooth1, nrhs);
  const T* r = v;
  if (h->p.pre_smooth1 > 0) {
    T* rr = W<T>(h, "k1_r", c1 * nrhs);
    coarse_apply1<T>(h, z, rr, nrhs);
    launch_sub_b<T>(v, c1, rr, c1, c1 / 2, nrhs, nullptr, h->st);
    CKL();
    r = rr;
  }
  T* r2 = W<T>(h, "k1_r2", c2 * nrhs);
  T* e2 = W<T>(h, "k1_e2", c2 * nrhs);
  {
    Prof pf(h, PK_L1XFER, nrhs);
    launch_crestrict<T>(static_cast<const T*>(h->P2), r, r2, h->cag, nrhs, h->st);
    CKL();
  }
  coarse_solve<T>(h, coarsest_level(h), r2, e2, nrhs, h->p.coarsest_tol, h->p.coarsest_maxit);
  {
    Prof pf(h, PK_L1XFER, nrhs);
    launch_cprolong<T>(static_cast<const T*>(h->P2), e2, z, h->cag, nrhs, true, h->st);
    CKL();
  }
  csap_sweeps<T>(h, v, z, h->p.post_smooth1, nrhs);
}

// the coarse solve of the fine K-cycle with three levels: FGMRES(coarse_restart)
// on D_c1(mu) from zero, preconditioned by the level-1 K-cycle
template <typename T>
void level1_solve(tm_handle* h, const T* b1, T* x1, int nrhs, double tol, int maxit) {
  const long ncx = level1_cx(h);
  {
    Prof pf(h, PK_OTHER, nrhs);
    launch_zero<T>(x1, 2 * ncx * nrhs, h->st);
    CKL();
  }
  auto resid = [&](const T* xx, T* r, bool) {  // one form only: always exact
    coarse_apply1<T>(h, xx, r, nrhs);
    launch_sub_b<T>(b1, 2 * ncx, r, 2 * ncx, ncx, nrhs, nullptr, h->st);
    CKL();
    return true;
  };
  auto AZ = [&](const T* z, T* o) { coarse_apply1<T>(h, z, o, nrhs); };
  auto M = [&](const T* v, T* z) { kcycle1<T>(h, v, z, nrhs); };
  std::vector<KrylovOut> ks =
      fgmres_b<T, T>(h, "l1", PK_BLAS_COARSE, resid, AZ, M, b1, x1, nrhs, ncx, tol, h->p.coarse_restart, maxit);
  for (const KrylovOut& k : ks) h->coarse_iters += k.iters;
}

// P2 (holding the level-1 test vectors) -> orthonormal P2, D_c2, odd-site inverses
template <typename T>
void build_level2(tm_handle* h, bool orth = true) {
  Prof pf(h, PK_BUILD, 1, (orth ? 3 : 2) + (std::is_same<T, float>::value && h->tc_on ? 3 : 0));
  if (orth) {
    launch_corth<T>(static_cast<T*>(h->P2), h->cag, h->d_err, h->st);
    CKL();
  }
  launch_cbuild<T>(static_cast<const T*>(h->Dc), static_cast<const T*>(h->P2), static_cast<T*>(h->Dc2), h->cag,
                   h->st);
  CKL();
  launch_oe_invert<T>(static_cast<T*>(h->Dc2), static_cast<T*>(h->Dinv2), h->oe2, mu_c(h), h->d_err, h->st);
  CKL();
  if constexpr (std::is_same<T, float>::value) {
    if (h->tc_on) {
      tc_build(static_cast<const float*>(h->Dc2), static_cast<const float*>(h->Dinv2), h->oe2, h->tc, h->st);
      CKL();
    }
  }
}

template <typename T>
void normalise_vecs(tm_handle* h, T* f, long ncx, int nrhs) {
  Prof pf(h, PK_OTHER, nrhs, 3);
  launch_norm2<T>(f, ncx, nrhs, h->dsmall, h->scratch, kScratchBlocks, h->st);
  CKL();
  launch_scale<T>(f, ncx, nrhs, h->dsmall, true, h->st);
  CKL();
}

template <typename T>
void normalise_fields(tm_handle* h, T* f, int nrhs) {
  const long fr = fine_reals(h);
  Prof pf(h, PK_OTHER, nrhs, 3);
  launch_norm2<T>(f, fr / 2, nrhs, h->dsmall, h->scratch, kScratchBlocks, h->st);
  CKL();
  launch_scale<T>(f, fr / 2, nrhs, h->dsmall, true, h->st);
  CKL();
}

template <typename T>
void setup_iterate(tm_handle* h, int fine, int coarse);

// P, D_c (and P2, D_c2) rebuilt from the current test vectors, e.g. on a new gauge field
template <typename T>
void setup_rebuild(tm_handle* h) {
  const long fr = fine_reals(h);
  CK(cudaMemcpyAsync(h->P, h->tv, fr * h->p.nv * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
  build_coarse<T>(h);
  if (h->three) {
    CK(cudaMemcpyAsync(h->P2, h->tv1, 2 * level1_cx(h) * h->p.nv2 * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
    build_level2<T>(h);
  }
  check_flags(h);
}

template <typename T>
void setup_impl(tm_handle* h, const double* tv_dev, bool adaptive) {
  const int nv = h->p.nv, nv2 = h->p.nv2;
  const long fr = fine_reals(h);
  T* tv = static_cast<T*>(h->tv);
  T* P = static_cast<T*>(h->P);
  {
    Prof pf(h, PK_OTHER, nv);
    launch_pack_spinor<T>(tv_dev, tv, h->g, nv, h->st);
    CKL();
  }
  if (adaptive) {
    sap_sweeps<T>(h, nullptr, tv, h->p.init_sweeps, nv);
    normalise_fields<T>(h, tv, nv);
  }
  CK(cudaMemcpyAsync(P, tv, fr * nv * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
  build_coarse<T>(h);
  const long c1 = 2 * level1_cx(h);
  T* tv1 = static_cast<T*>(h->tv1);
  T* P2 = static_cast<T*>(h->P2);
  if (h->three) {  // level-1 initial phase from the level-1 random vectors
    {
      Prof pf(h, PK_OTHER, nv2);
      launch_convert<double, T>(tv_dev + (size_t)nv * fr, tv1, c1 * nv2, h->st);
      CKL();
    }
    if (adaptive) {
      csap_sweeps<T>(h, nullptr, tv1, h->p.init_sweeps1, nv2);
      normalise_vecs<T>(h, tv1, c1 / 2, nv2);
    }
    CK(cudaMemcpyAsync(P2, tv1, c1 * nv2 * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
    build_level2<T>(h);
  }
  check_flags(h);
  if (adaptive) setup_iterate<T>(h, h->p.setup_iters, h->p.coarse_setup_iters);
  sync(h);
}

// setup iterations from the current test vectors: `fine` times v_i <- B(v_i),
// normalised, P, D_c (and P2, D_c2 from the current level-1 vectors) rebuilt;
// then with three levels `coarse` times w_j <- B1(w_j), normalised, P2, D_c2 rebuilt
template <typename T>
void setup_iterate(tm_handle* h, int fine, int coarse) {
  const int nv = h->p.nv, nv2 = h->p.nv2;
  const long fr = fine_reals(h);
  T* tv = static_cast<T*>(h->tv);
  T* P = static_cast<T*>(h->P);
  const long c1 = 2 * level1_cx(h);
  T* tv1 = static_cast<T*>(h->tv1);
  T* P2 = static_cast<T*>(h->P2);
  {
    T* z = W<T>(h, "setup_z", fr * nv);
    for (int it = 0; it < fine; ++it) {
      kcycle<T>(h, tv, z, nv);
      CK(cudaMemcpyAsync(tv, z, fr * nv * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
      normalise_fields<T>(h, tv, nv);
      CK(cudaMemcpyAsync(P, tv, fr * nv * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
      build_coarse<T>(h);
      if (h->three) {
        CK(cudaMemcpyAsync(P2, tv1, c1 * nv2 * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
        build_level2<T>(h);
      }
      check_flags(h);
    }
    if (h->three) {
      T* z1 = W<T>(h, "setup_z1", c1 * nv2);
      for (int it = 0; it < coarse; ++it) {
        kcycle1<T>(h, tv1, z1, nv2);
        CK(cudaMemcpyAsync(tv1, z1, c1 * nv2 * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
        normalise_vecs<T>(h, tv1, c1 / 2, nv2);
        CK(cudaMemcpyAsync(P2, tv1, c1 * nv2 * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
        build_level2<T>(h);
        check_flags(h);
      }
    }
  }
  sync(h);
  release(h, "setup_z");  // setup-only work: N_v fine fields (tens of GB at 48^3 x 96)
  release(h, "setup_z1");
}

// ---------------------------------------------------------------------------
// learned gauge-covariant layer (not part of the paper's method)
// ---------------------------------------------------------------------------
constexpr int kNnLayer = kNnWeights / 2;  // complex weights per layer

void nn_upload(tm_handle* h) {
  if (!h->d_nnw) {
    h->d_nnw = static_cast<float2*>(dalloc((size_t)5 * kNnLayer * sizeof(float2)));
    h->d_nngrad = static_cast<double2*>(dalloc((size_t)2 * kNnLayer * sizeof(double2)));
  }
  std::vector<float2> buf((size_t)5 * kNnLayer);
  for (int k = 0; k < kNnWeights; ++k) {
    const float re = (float)h->nn_w[k].real(), im = (float)h->nn_w[k].imag();
    buf[k] = make_float2(re, im);
    buf[kNnWeights + k] = make_float2(__half2float(__float2half(re)), __half2float(__float2half(im)));
  }
  // adjoint of layer 2: W2adj[i][0][opp(d)][s][t] = conj(W2[0][i][d][t][s])
  for (int i = 0; i < kNnHidden; ++i)
    for (int d = 0; d < 9; ++d) {
      const int od = d == 0 ? 0 : (((d - 1) & 1) ? d - 1 : d + 1);
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          const std::complex<double> w = h->nn_w[kNnLayer + (i * 9 + d) * 16 + b * 4 + a];
          buf[(size_t)4 * kNnLayer + (i * 9 + od) * 16 + a * 4 + b] = make_float2((float)w.real(), (float)-w.imag());
        }
    }
  CK(cudaMemcpyAsync(h->d_nnw, buf.data(), buf.size() * sizeof(float2), cudaMemcpyHostToDevice, h->st));
  sync(h);
}

void need_nn(tm_handle* h) {
  if (!h->gauge_ok) raise(TM_ERR_STATE, "needs a gauge field");
  if (h->nn_w.empty()) {
    h->nn_w.assign(kNnWeights, std::complex<double>(0, 0));
    nn_upload(h);
  }
}

// out (+)= N(in) for nrhs FP32 fine fields; FP16 hidden channels and weights when half
void nn_forward(tm_handle* h, const float* in, float* out, int nrhs, bool accumulate, bool half) {
  need_nn(h);
  Prof pf(h, PK_NN, nrhs, 2);
  const size_t hid = (size_t)kNnHidden * 24 * h->g.V * nrhs;
  void* hb = half ? static_cast<void*>(W<__half>(h, "nn_hid16", hid)) : static_cast<void*>(W<float>(h, "nn_hid", hid));
  const float2* w1 = h->d_nnw + (half ? kNnWeights : 0);
  const float2* w2 = w1 + kNnLayer;
  nn_layer1(in, hb, half, h->g32, w1, h->g, h->p.bc_t, nrhs, h->st);
  CKL();
  nn_layer2(hb, half, out, accumulate, h->g32, w2, h->g, h->p.bc_t, nrhs, h->st);
  CKL();
}

// loss sum_p ||N(r_p) - e_p||^2 and Wirtinger gradients (not yet divided by sum_p ||e_p||^2)
double nn_grad_sum(tm_handle* h, const float* r, const float* e, int npairs, std::vector<std::complex<double>>& G,
                   double& esum) {
  need_nn(h);
  const long fr = fine_reals(h);
  const int chunk = 16;
  const size_t hid = (size_t)kNnHidden * 24 * h->g.V * chunk;
  float* hb = W<float>(h, "nn_hid", hid);
  float* gh = W<float>(h, "nn_gh", hid);
  float* y = W<float>(h, "nn_y", (size_t)fr * chunk);
  float2* part = W<float2>(h, "nn_part", (size_t)nn_wgrad_partial_floats2(h->g, chunk));
  G.assign(kNnWeights, std::complex<double>(0, 0));
  double loss = 0;
  esum = 0;
  std::vector<double2> hg((size_t)kNnWeights);
  for (int p0 = 0; p0 < npairs; p0 += chunk) {
    const int nr = std::min(chunk, npairs - p0);
    const float* rp = r + (size_t)p0 * fr;
    const float* ep = e + (size_t)p0 * fr;
    {
      Prof pf(h, PK_NN, nr, 10);
      nn_layer1(rp, hb, false, h->g32, h->d_nnw, h->g, h->p.bc_t, nr, h->st);
      CKL();
      nn_layer2(hb, false, y, false, h->g32, h->d_nnw + kNnLayer, h->g, h->p.bc_t, nr, h->st);
      CKL();
      launch_caxpby<float>(-1, 0, ep, 1, 0, y, (fr / 2) * nr, h->st);  // y = N(r) - e
      CKL();
      launch_norm2<float>(y, fr / 2, nr, h->dsmall, h->scratch, kScratchBlocks, h->st);
      CKL();
      launch_norm2<float>(ep, fr / 2, nr, h->dsmall + kMaxDots, h->scratch, kScratchBlocks, h->st);
      CKL();
      nn_grad_w2(hb, y, h->g32, h->g, h->p.bc_t, nr, part, h->d_nngrad + kNnLayer, h->st);
      CKL();
      nn_layer2_adjoint(y, gh, h->g32, h->d_nnw + 4 * kNnLayer, h->g, h->p.bc_t, nr, h->st);
      CKL();
      nn_grad_w1(rp, gh, h->g32, h->g, h->p.bc_t, nr, part, h->d_nngrad, h->st);
      CKL();
    }
    CK(cudaMemcpyAsync(h->hsmall, h->dsmall, (kMaxDots + nr) * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(hg.data(), h->d_nngrad, hg.size() * sizeof(double2), cudaMemcpyDeviceToHost, h->st));
    sync(h);
    for (int q = 0; q < nr; ++q) {
      loss += h->hsmall[q];
      esum += h->hsmall[kMaxDots + q];
    }
    for (int k = 0; k < kNnWeights; ++k) G[k] += std::complex<double>(hg[k].x, hg[k].y);
  }
  if (!std::isfinite(loss)) raise(TM_ERR_NONFINITE, "non-finite loss");
  return loss;
}

// z = B(v), then the optional stage after the K-cycle: z += N(v - D z) (learned
// layer) or z += one SAP sweep on D e = v - D z from zero (its stand-in)
template <typename T>
void precond(tm_handle* h, const T* v, T* z, int nrhs) {
  kcycle<T>(h, v, z, nrhs);
  if (h->p.nn_mode == 0) return;
  const long fr = fine_reals(h);
  T* rr = W<T>(h, "nn_rr", fr * nrhs);
  dslash<T>(h, z, rr, v, nrhs);  // rr = v - D z
  if (h->p.nn_mode == 1) {
    if constexpr (std::is_same<T, float>::value) {
      nn_forward(h, rr, z, nrhs, true, h->p.nn_prec == TM_F16);
    } else {
      raise(TM_ERR_ARG, "the learned layer runs in FP32 or FP16 (cycle_prec = TM_F32)");
    }
  } else {
    T* ee = W<T>(h, "nn_ee", fr * nrhs);
    {
      Prof pf(h, PK_OTHER, nrhs);
      launch_zero<T>(ee, fr * nrhs, h->st);
      CKL();
    }
    sap_sweeps<T>(h, rr, ee, 1, nrhs);
    Prof pf(h, PK_OTHER, nrhs);
    launch_caxpby<T>(1, 0, ee, 1, 0, z, (fr / 2) * nrhs, h->st);
    CKL();
  }
}

// FGMRES in FP64 preconditioned by the K-cycle in T; b, x packed FP64 fields
template <typename T>
KrylovOut solve_one(tm_handle* h, const double* b, double* x, double tol) {
  const long fr = fine_reals(h);
  double* zt = std::is_same<T, double>::value || h->gdf ? nullptr : W<double>(h, "s_z64", fr);
  T* vt = std::is_same<T, double>::value ? nullptr : W<T>(h, "s_vT", fr);
  auto A = [&](const double* in, double* out) { dslash<double>(h, in, out, nullptr, 1); };
  auto AZ = [&](const T* z, double* out) {
    if constexpr (std::is_same<T, double>::value) {
      dslash<double>(h, z, out, nullptr, 1);
    } else {
      if (h->gdf) {
        dslash_df(h, z, out, 1);
        return;
      }
      {
        Prof pf(h, PK_OTHER);
        launch_convert<T, double>(z, zt, fr, h->st);
        CKL();
      }
      dslash<double>(h, zt, out, nullptr, 1);
    }
  };
  auto M = [&](const double* v, T* z) {
    if constexpr (std::is_same<T, double>::value) {
      precond<double>(h, v, z, 1);
    } else {
      {
        Prof pf(h, PK_OTHER);
        launch_convert<double, T>(v, vt, fr, h->st);
        CKL();
      }
      precond<T>(h, vt, z, 1);
    }
  };
  return krylov<double, T>(h, "fg", A, AZ, M, true, b, x, true, fr / 2, tol, h->p.restart, h->p.maxit);
}

// nb right-hand sides at once: nb independent FP64 FGMRES(restart) solves run
// in lock-step (own Hessenberg matrix, restarts and stopping each), sharing
// every launch: one multi-rhs D(mu) apply, one batched K-cycle (SAP,
// restriction, batched coarse GMRES, prolongation) and batched CGS2 per step.
// Finished right-hand sides are masked in the vector updates.  Layout: the
// Krylov vectors of step j for all right-hand sides are one contiguous block
// [nb][fine reals], so the multi-rhs operators apply to them directly.
// Generic batched flexible GMRES(m): basis vectors in Tv, preconditioned
// vectors in Tz, vectors of ncx complex numbers (fr = 2 ncx reals).
//   resid(x, r, exact): r = b - A x for all nb right-hand sides (contiguous
//                blocks); with exact = false it may use cheaper arithmetic
//                (the FP32-pair stencil) and return false, and then its norms
//                only decide whether the exact residual is needed: a residual
//                within kVerify * tol of convergence is recomputed exactly
//                before any decision
//   AZ(z, w):    w = A z
//   M(v, z):     z = preconditioner(v)
template <typename Tv, typename Tz, typename FR, typename FAZ, typename FM>
std::vector<KrylovOut> fgmres_b(tm_handle* h, const std::string& tag, int pk, FR resid, FAZ AZ, FM M, const Tv* b,
                                Tv* x, int nb, long ncx, double tol, int m, int maxit) {
  using cd = std::complex<double>;
  const long fr = 2 * ncx, nc = ncx;
  const long blk = fr * nb;               // one Krylov step for all right-hand sides
  const long ds = 4 * kMaxDots + 2;
  Tv* Vb = Wz<Tv>(h, tag + "_V", (size_t)(m + 1) * blk);
  Tz* Z = Wz<Tz>(h, tag + "_Z", (size_t)m * blk);
  Tv* w = W<Tv>(h, tag + "_w", blk);
  double* part = W<double>(h, tag + "_part", std::max(multidot_scratch_doubles(nc, m + 1, nb), 2L * 304 * nb));
  double* dd = W<double>(h, tag + "_dots", ds * nb);
  double* nrm = W<double>(h, tag + "_nrm", nb);
  int* act = W<int>(h, tag + "_act", nb);
  constexpr int kSlots = 8;
  double* hb = host_scratch(h, tag.c_str(), (size_t)(ds + 1) * nb + (size_t)kSlots * nb);
  double* hn_h = hb + (size_t)ds * nb;
  int* hact0 = reinterpret_cast<int*>(hn_h + nb);
  int slot = 0;
  std::vector<KrylovOut> out(nb);
  std::vector<double> bnorm(nb), beta(nb);
  std::vector<int> kk(nb, 0);
  std::vector<char> active(nb), inner(nb);
  std::vector<cd> H((size_t)nb * (m + 1) * m), g((size_t)nb * (m + 1)), sn((size_t)nb * m);
  std::vector<double> cs((size_t)nb * m);
  // the fine FP64 FGMRES with FP32-pair outer products also runs its Arnoldi
  // steps and solution update in pair arithmetic
  const bool pair_blas = std::is_same<Tv, double>::value && pk == PK_BLAS_FINE && h->p.outer_apply == TM_F32X2;
  auto count = [&](const std::vector<char>& msk) {
    int c = 0;
    for (char v : msk) c += v ? 1 : 0;
    return c;
  };
  auto upload_mask = [&](const std::vector<char>& msk, const std::vector<int>* counts) {
    if (slot >= kSlots) {
      sync(h);
      slot = 0;
    }
    int* ha = hact0 + (size_t)(slot++) * nb;
    for (int r = 0; r < nb; ++r) ha[r] = msk[r] ? (counts ? (*counts)[r] : 1) : 0;
    CK(cudaMemcpyAsync(act, ha, nb * sizeof(int), cudaMemcpyHostToDevice, h->st));
  };
  auto read_norms = [&]() {
    CK(cudaMemcpyAsync(hn_h, nrm, nb * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    sync(h);
    slot = 0;
  };
  auto norms = [&](const Tv* v, const int* msk) {
    Prof pf(h, pk, nb, 2);
    launch_norm2_b<Tv>(v, fr, nc, nrm, part, nb, msk, h->st);
    CKL();
  };
  norms(b, nullptr);
  read_norms();
  for (int r = 0; r < nb; ++r) {
    bnorm[r] = std::sqrt(hn_h[r]);
    if (!std::isfinite(bnorm[r])) raise(TM_ERR_NONFINITE, "non-finite right-hand side");
  }
  norms(x, nullptr);  // a zero start vector (the usual case) needs no product: r = b
  read_norms();
  bool x_zero = true;
  for (int r = 0; r < nb; ++r) x_zero = x_zero && hn_h[r] == 0;
  constexpr double kVerify = 4.0;
  // r = b - A x: the cheap form first, the exact one where it could decide convergence
  auto true_residual = [&](const int* msk) {
    const bool exact = resid(x, Vb, false);
    norms(Vb, msk);
    read_norms();
    if (exact) return;
    bool near = false;
    for (int r = 0; r < nb; ++r)
      near = near || ((!msk || active[r]) && std::sqrt(hn_h[r]) <= kVerify * tol * bnorm[r]);
    if (near) {
      resid(x, Vb, true);
      norms(Vb, msk);
      read_norms();
    }
  };
  if (x_zero) {
    Prof pf(h, pk, nb);
    CK(cudaMemcpyAsync(Vb, b, (size_t)blk * sizeof(Tv), cudaMemcpyDeviceToDevice, h->st));
    norms(Vb, nullptr);
    read_norms();
  } else {
    true_residual(nullptr);
  }
  for (int r = 0; r < nb; ++r) {
    beta[r] = std::sqrt(hn_h[r]);
    active[r] = bnorm[r] > 0 && beta[r] > tol * bnorm[r] && out[r].iters < maxit;
    if (bnorm[r] == 0) out[r].converged = true;
  }
  while (count(active)) {
    for (int r = 0; r < nb; ++r) hn_h[r] = beta[r] * beta[r];
    CK(cudaMemcpyAsync(nrm, hn_h, nb * sizeof(double), cudaMemcpyHostToDevice, h->st));
    upload_mask(active, nullptr);
    {
      Prof pf(h, pk, count(active));
      launch_scale_copy_b<Tv>(Vb, fr, Vb, fr, nrm, nc, nb, act, h->st);
      CKL();
    }
    for (int r = 0; r < nb; ++r) {
      inner[r] = active[r];
      kk[r] = 0;
      if (active[r]) {
        std::fill(g.begin() + (size_t)r * (m + 1), g.begin() + (size_t)(r + 1) * (m + 1), cd(0));
        g[(size_t)r * (m + 1)] = beta[r];
      }
    }
    for (int k = 0; k < m && count(inner); ++k) {
      const int na = count(inner);
      Tv* vk = Vb + (long)k * blk;
      Tz* zk = Z + (long)k * blk;
      M(vk, zk);
      AZ(zk, w);
      upload_mask(inner, nullptr);
      double* d1 = dd;
      double* d2 = dd + 2 * (k + 1);
      if (pair_blas) {  // FP64 basis, CGS2 in FP32-pair arithmetic with fused reductions
        Prof pf(h, pk, na, 7);
        if constexpr (std::is_same<Tv, double>::value) {
          launch_pdot_b(Vb, fr, blk, k + 1, w, fr, nc, d1, ds, part, nb, act, h->st);
          CKL();
          const int nl = launch_pcaxpy_dot_b(Vb, fr, blk, k + 1, d1, ds, w, fr, nc, d2, ds, part, nb, act, h->st);
          CKL();
          launch_pcaxpy_norm_b(Vb, fr, blk, k + 1, d2, ds, w, fr, nc, nrm, part, nb, act, h->st);
          CKL();
          launch_scale_copy_b<Tv>(w, fr, Vb + (long)(k + 1) * blk, fr, nrm, nc, nb, act, h->st);
          CKL();
          if (nl == 3 && h->prof) h->prof_launch[pk] += 1;
        }
      } else if (nc <= kFuseMaxCx) {  // short vectors: the launches dominate, fuse the reductions
        Prof pf(h, pk, na, 6);
        launch_multidot_b_partials<Tv>(Vb, fr, blk, k + 1, w, fr, nc, part, nb, act, h->st);
        CKL();
        launch_multi_caxpy_bp<Tv>(Vb, fr, blk, k + 1, part, nc, d1, ds, w, fr, nc, nb, act, h->st);
        CKL();
        launch_multidot_b_partials<Tv>(Vb, fr, blk, k + 1, w, fr, nc, part, nb, act, h->st);
        CKL();
        launch_multi_caxpy_bp<Tv>(Vb, fr, blk, k + 1, part, nc, d2, ds, w, fr, nc, nb, act, h->st);
        CKL();
        launch_norm2_b_partials<Tv>(w, fr, nc, part, nb, act, h->st);
        CKL();
        launch_scale_copy_bp<Tv>(w, fr, Vb + (long)(k + 1) * blk, fr, part, nrm, nc, nb, act, h->st);
        CKL();
      } else {
        Prof pf(h, pk, na, 9);
        launch_multidot_b<Tv>(Vb, fr, blk, k + 1, w, fr, nc, d1, ds, part, nb, act, h->st);
        CKL();
        launch_multi_caxpy_b<Tv>(Vb, fr, blk, k + 1, d1, ds, w, fr, nc, nb, act, h->st);
        CKL();
        launch_multidot_b<Tv>(Vb, fr, blk, k + 1, w, fr, nc, d2, ds, part, nb, act, h->st);
        CKL();
        launch_multi_caxpy_b<Tv>(Vb, fr, blk, k + 1, d2, ds, w, fr, nc, nb, act, h->st);
        CKL();
        launch_norm2_b<Tv>(w, fr, nc, nrm, part, nb, act, h->st);
        CKL();
        launch_scale_copy_b<Tv>(w, fr, Vb + (long)(k + 1) * blk, fr, nrm, nc, nb, act, h->st);
        CKL();
      }
      CK(cudaMemcpy2DAsync(hb, 4 * (k + 1) * sizeof(double), dd, ds * sizeof(double), 4 * (k + 1) * sizeof(double), nb,
                           cudaMemcpyDeviceToHost, h->st));
      read_norms();
      for (int r = 0; r < nb; ++r) {
        if (!inner[r]) continue;
        const double hn = std::sqrt(hn_h[r]);
        if (!std::isfinite(hn)) raise(TM_ERR_NONFINITE, "non-finite Arnoldi vector");
        const double* hr = hb + (size_t)r * 4 * (k + 1);
        cd* Hr = H.data() + (size_t)r * (m + 1) * m;
        cd* gr = g.data() + (size_t)r * (m + 1);
        cd* snr = sn.data() + (size_t)r * m;
        double* csr = cs.data() + (size_t)r * m;
        std::vector<cd> col(m + 1, cd(0));
        for (int j = 0; j <= k; ++j)
          col[j] = cd(hr[2 * j] + hr[2 * (k + 1) + 2 * j], hr[2 * j + 1] + hr[2 * (k + 1) + 2 * j + 1]);
        col[k + 1] = hn;
        for (int j = 0; j < k; ++j) {
          const cd t = csr[j] * col[j] + snr[j] * col[j + 1];
          col[j + 1] = -std::conj(snr[j]) * col[j] + csr[j] * col[j + 1];
          col[j] = t;
        }
        double c;
        cd sg, rho;
        givens(col[k], hn, c, sg, rho);
        csr[k] = c;
        snr[k] = sg;
        col[k] = rho;
        col[k + 1] = 0;
        for (int j = 0; j <= m; ++j) Hr[(size_t)j * m + k] = col[j];
        gr[k + 1] = -std::conj(sg) * gr[k];
        gr[k] = c * gr[k];
        ++out[r].iters;
        kk[r] = k + 1;
        if (hn == 0 || std::abs(gr[k + 1]) <= tol * bnorm[r] || out[r].iters >= maxit) inner[r] = 0;
      }
    }
    int kmax = 0;
    for (int r = 0; r < nb; ++r) {
      if (!active[r]) continue;
      const int k = kk[r];
      kmax = std::max(kmax, k);
      const cd* Hr = H.data() + (size_t)r * (m + 1) * m;
      const cd* gr = g.data() + (size_t)r * (m + 1);
      std::vector<cd> y(k);
      for (int i = k - 1; i >= 0; --i) {
        cd acc = gr[i];
        for (int j = i + 1; j < k; ++j) acc -= Hr[(size_t)i * m + j] * y[j];
        y[i] = acc / Hr[(size_t)i * m + i];
      }
      double* yr = hb + (size_t)r * ds;
      for (int i = 0; i < k; ++i) {
        yr[2 * i] = y[i].real();
        yr[2 * i + 1] = y[i].imag();
      }
      ++out[r].restarts;
    }
    CK(cudaMemcpyAsync(dd, hb, ds * nb * sizeof(double), cudaMemcpyHostToDevice, h->st));
    upload_mask(active, &kk);
    {
      Prof pf(h, pk, count(active));
      if constexpr (std::is_same<Tz, float>::value && std::is_same<Tv, double>::value) {
        if (pair_blas)
          launch_plincomb_b(Z, fr, blk, kmax, dd, ds, x, fr, nc, nb, act, h->st);
        else
          launch_lincomb_b<Tz, Tv>(Z, fr, blk, kmax, dd, ds, x, fr, nc, nb, act, h->st);
      } else {
        launch_lincomb_b<Tz, Tv>(Z, fr, blk, kmax, dd, ds, x, fr, nc, nb, act, h->st);
      }
      CKL();
    }
    upload_mask(active, nullptr);
    true_residual(act);
    for (int r = 0; r < nb; ++r) {
      if (!active[r]) continue;
      beta[r] = std::sqrt(hn_h[r]);
      if (!std::isfinite(beta[r])) raise(TM_ERR_NONFINITE, "non-finite residual");
      active[r] = beta[r] > tol * bnorm[r] && out[r].iters < maxit;
    }
  }
  for (int r = 0; r < nb; ++r) {
    out[r].relres = bnorm[r] > 0 ? beta[r] / bnorm[r] : 0.0;
    out[r].converged = out[r].converged || beta[r] <= tol * bnorm[r];
  }
  return out;
}

// the fine level: FP64 FGMRES, K-cycle in T
template <typename T>
std::vector<KrylovOut> solve_batch(tm_handle* h, const double* b, double* x, int nb, double tol) {
  const long fr = fine_reals(h);
  const long blk = fr * nb;
  double* zt = std::is_same<T, double>::value || h->gdf ? nullptr : W<double>(h, "sb_z64", blk);
  T* vt = std::is_same<T, double>::value ? nullptr : W<T>(h, "sb_vT", blk);
  // restart residuals in FP32 pairs when the pair operator is held; FP64 where a
  // residual may decide convergence (fgmres_b asks for the exact one then)
  auto resid = [&](const double* xx, double* r, bool exact) {
    if (!exact && h->gdf) {
      Prof pf(h, PK_DSLASHDF, nb);
      launch_residual_df(h->gdf, h->cdf, xx, b, r, h->g, h->p.mu, h->p.bc_t, nb, h->st, h->rho);
      CKL();
      return false;
    }
    dslash<double>(h, xx, r, b, nb);
    return true;
  };
  auto M = [&](const double* v, T* z) {
    if constexpr (std::is_same<T, double>::value) {
      precond<double>(h, v, z, nb);
    } else {
      {
        Prof pf(h, PK_OTHER, nb);
        launch_convert<double, T>(v, vt, blk, h->st);
        CKL();
      }
      precond<T>(h, vt, z, nb);
    }
  };
  auto AZ = [&](const T* z, double* o) {
    if constexpr (std::is_same<T, double>::value) {
      dslash<double>(h, z, o, nullptr, nb);
    } else {
      if (h->gdf) {
        dslash_df(h, z, o, nb);
        return;
      }
      {
        Prof pf(h, PK_OTHER, nb);
        launch_convert<T, double>(z, zt, blk, h->st);
        CKL();
      }
      dslash<double>(h, zt, o, nullptr, nb);
    }
  };
  return fgmres_b<double, T>(h, "sb", PK_BLAS_FINE, resid, AZ, M, b, x, nb, fr / 2, tol, h->p.restart,
                             h->p.maxit);
}

// stage a natural (host or device) array of `bytes` on the device
const double* stage_in(tm_handle* h, const double* src, size_t bytes, const char* name) {
  if (is_device_ptr(src)) return src;
  double* d = W<double>(h, name, bytes / sizeof(double));
  CK(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, h->st));
  return d;
}

void validate(const tm_params* p) {
  auto bad = [](const std::string& m) { raise(TM_ERR_ARG, m); };
  for (int d = 0; d < 4; ++d) {
    if (p->L[d] < 2) bad("lattice extents must be >= 2");
    if (p->agg[d] < 1 || p->L[d] % p->agg[d]) bad("lattice not divisible by the aggregate");
    if (p->sap_block[d] < 1 || p->L[d] % p->sap_block[d]) bad("lattice not divisible by the SAP block");
    const int nb = p->L[d] / p->sap_block[d];
    if (nb < 2 || nb % 2) bad("SAP block count per dimension must be even and >= 2");
    const int nc = p->L[d] / p->agg[d];
    if (nc < 2 || nc % 2) bad("coarse extents must be even and >= 2 (odd-even coarse solve)");
  }
  const long asites = (long)p->agg[0] * p->agg[1] * p->agg[2] * p->agg[3];
  const long bsites = (long)p->sap_block[0] * p->sap_block[1] * p->sap_block[2] * p->sap_block[3];
  if (asites > 1024) bad("aggregate volume must be <= 1024");
  if (bsites > 1024) bad("SAP block volume must be <= 1024");
  if (p->nv < 1 || p->nv > 28) bad("nv must be in 1..28");
  if (p->mr_iters < 0 || p->pre_smooth < 0 || p->post_smooth < 0 || p->init_sweeps < 0 || p->setup_iters < 0)
    bad("negative iteration count");
  if (p->restart < 1 || p->restart > kMaxDots - 2) bad("restart must be in 1..126");
  if (p->coarse_restart < 1 || p->coarse_restart > kMaxDots - 2) bad("coarse_restart must be in 1..126");
  if (p->maxit < 1 || p->coarse_maxit < 1) bad("maxit must be >= 1");
  if (p->cycle_prec != TM_F64 && p->cycle_prec != TM_F32) bad("cycle_prec must be TM_F64 or TM_F32");
  if (p->coarse_mma < 0 || p->coarse_mma > 3) bad("coarse_mma must be 0..3");
  if (p->coarse_mma > 0 && p->cycle_prec != TM_F32) bad("coarse_mma needs cycle_prec = TM_F32");
  if (p->nn_mode < 0 || p->nn_mode > 2) bad("nn_mode must be 0, 1 or 2");
  if (p->nn_mode == 1 && p->cycle_prec != TM_F32) bad("the learned layer needs cycle_prec = TM_F32");
  if (p->nn_prec != TM_F32 && p->nn_prec != TM_F16) bad("nn_prec must be TM_F32 or TM_F16");
  auto is16 = [](int v) { return v == TM_F16 || v == TM_BF16; };
  if (p->sap1_prec != TM_F32 && !is16(p->sap1_prec)) bad("sap1_prec must be TM_F32, TM_F16 or TM_BF16");
  if (is16(p->sap1_prec) && (p->levels != 3 || p->cycle_prec != TM_F32))
    bad("a 16-bit sap1_prec needs levels = 3 and cycle_prec = TM_F32");
  if (p->transfer_prec != TM_F32 && !is16(p->transfer_prec))
    bad("transfer_prec must be TM_F32, TM_F16 or TM_BF16");
  if (is16(p->transfer_prec) && p->cycle_prec != TM_F32) bad("a 16-bit transfer_prec needs cycle_prec = TM_F32");
  if (p->sap_prec != TM_F32 && !is16(p->sap_prec)) bad("sap_prec must be TM_F32, TM_F16 or TM_BF16");
  if (p->coarsest_steps < 0 || p->coarsest_steps > 64) bad("coarsest_steps must be in 0..64");
  if (is16(p->sap_prec) && (p->cycle_prec != TM_F32 || !p->block_oe))
    bad("a 16-bit sap_prec needs cycle_prec = TM_F32 and block_oe = 1");
  if (p->outer_apply != TM_F64 && p->outer_apply != TM_F32X2) bad("outer_apply must be TM_F64 or TM_F32X2");
  if (p->outer_apply == TM_F32X2 && p->cycle_prec != TM_F32) bad("outer_apply = TM_F32X2 needs cycle_prec = TM_F32");
  if (p->tc_spin_limit < 0) bad("tc_spin_limit must be >= 0");
  if (p->block_oe != 0 && p->block_oe != 1) bad("block_oe must be 0 or 1");
  if (p->block_oe)
    for (int d = 0; d < 4; ++d)
      if (p->sap_block[d] % 2) bad("block_oe = 1 needs even SAP block dims");
  if (p->bc_t != 1.0 && p->bc_t != -1.0) bad("bc_t must be +1 or -1");
  if (!(p->delta >= 1.0)) bad("delta must be >= 1");
  if (p->max_rhs < 1) bad("max_rhs must be >= 1");
  if (p->levels != 2 && p->levels != 3) bad("levels must be 2 or 3");
  if (p->levels == 3) {
    long a2 = 1, b1 = 1;
    for (int d = 0; d < 4; ++d) {
      const int l1 = p->L[d] / p->agg[d];
      if (p->agg2[d] < 1 || l1 % p->agg2[d]) bad("level-1 lattice not divisible by agg2");
      const int l2 = l1 / p->agg2[d];
      if (l2 < 2 || l2 % 2) bad("level-2 extents must be even and >= 2 (odd-even coarsest solve)");
      if (p->sap_block1[d] < 1 || l1 % p->sap_block1[d]) bad("level-1 lattice not divisible by sap_block1");
      const int nb = l1 / p->sap_block1[d];
      if (nb < 2 || nb % 2) bad("level-1 SAP block count per dimension must be even and >= 2");
      a2 *= p->agg2[d];
      b1 *= p->sap_block1[d];
    }
    if (p->nv2 < 1 || p->nv2 > 28) bad("nv2 must be in 1..28");
    if (a2 * 2 * p->nv > 1024) bad("agg2 volume x 2 nv must be <= 1024");
    if (b1 * 2 * p->nv > 1024) bad("sap_block1 volume x 2 nv must be <= 1024");
    if (p->mr_iters1 < 0 || p->pre_smooth1 < 0 || p->post_smooth1 < 0 || p->init_sweeps1 < 0 ||
        p->coarse_setup_iters < 0 || p->coarsest_maxit < 1)
      bad("negative level-1 iteration count");
  }
  const double lv = (double)p->L[0] * p->L[1] * p->L[2] * p->L[3];
  // sites and the reals of one field are indexed in 32 bits; offsets between fields in 64 bits
  if (lv * 24.0 >= 2147483647.0) bad("lattice too large for 32-bit site indexing");
}

template <typename T>
void unpack_fine(tm_handle* h, const void* f, double* nat, int nrhs) {
  launch_unpack_spinor<T>(static_cast<const T*>(f), nat, h->g, nrhs, h->st);
  CKL();
}

// Solve D(mu) x_r = b_r for natural device arrays (x holds the start vectors);
// accumulates statistics into loc.
void solve_core(tm_handle* h, const double* bd, double* xd, int nrhs, double tol, tm_solve_info& loc) {
  const long V = h->g.V;
  const long fr = fine_reals(h);
  const int batch = std::min(nrhs, h->p.max_rhs);
  if (batch > 1) {
    double* bf = W<double>(h, "sbatch_b", fr * batch);
    double* xf = W<double>(h, "sbatch_x", fr * batch);
    for (int r0 = 0; r0 < nrhs; r0 += batch) {
      const int nb = std::min(batch, nrhs - r0);
      {
        Prof pf(h, PK_OTHER, nb, 2);
        launch_pack_spinor<double>(bd + (size_t)r0 * V * 24, bf, h->g, nb, h->st);
        CKL();
        launch_pack_spinor<double>(xd + (size_t)r0 * V * 24, xf, h->g, nb, h->st);
        CKL();
      }
      std::vector<KrylovOut> ks = h->p.cycle_prec == TM_F64 ? solve_batch<double>(h, bf, xf, nb, tol)
                                                           : solve_batch<float>(h, bf, xf, nb, tol);
      {
        Prof pf(h, PK_OTHER, nb);
        launch_unpack_spinor<double>(xf, xd + (size_t)r0 * V * 24, h->g, nb, h->st);
        CKL();
      }
      for (const KrylovOut& k : ks) {
        loc.iters += k.iters;
        loc.restarts += k.restarts;
        loc.true_relres = std::max(loc.true_relres, k.relres);
        if (!k.converged) loc.converged = 0;
      }
    }
  }
  double* bf = W<double>(h, "s_b", fr);
  double* xf = W<double>(h, "s_x", fr);
  for (int r = (batch > 1 ? nrhs : 0); r < nrhs; ++r) {
    {
      Prof pf(h, PK_OTHER, 1, 2);
      launch_pack_spinor<double>(bd + (size_t)r * V * 24, bf, h->g, 1, h->st);
      CKL();
      launch_pack_spinor<double>(xd + (size_t)r * V * 24, xf, h->g, 1, h->st);
      CKL();
    }
    KrylovOut k = h->p.cycle_prec == TM_F64 ? solve_one<double>(h, bf, xf, tol) : solve_one<float>(h, bf, xf, tol);
    {
      Prof pf(h, PK_OTHER);
      launch_unpack_spinor<double>(xf, xd + (size_t)r * V * 24, h->g, 1, h->st);
      CKL();
    }
    loc.iters += k.iters;
    loc.restarts += k.restarts;
    loc.true_relres = std::max(loc.true_relres, k.relres);
    if (!k.converged) loc.converged = 0;
  }
}

// mu and delta of the handle; the odd-site inverses of the coarse Schur
// complement depend on mu_c = delta mu and are recomputed
void apply_mu(tm_handle* h, double mu, double delta) {
  h->p.mu = mu;
  h->p.delta = delta;
  if (h->gauge_ok) {
    build_sap_inverse(h);
    check_flags(h);
  }
  if (h->setup_ok) {
    Prof pf(h, PK_BUILD, 0, h->tc_on ? 2 : 1);  // no new D_c: zero build units
    void* Dc = h->three ? h->Dc2 : h->Dc;
    void* Di = h->three ? h->Dinv2 : h->Dinv;
    const OEGeom& oe = h->three ? h->oe2 : h->oe;
    if (h->p.cycle_prec == TM_F64)
      launch_oe_invert<double>(static_cast<double*>(Dc), static_cast<double*>(Di), oe, mu_c(h), h->d_err, h->st);
    else
      launch_oe_invert<float>(static_cast<float*>(Dc), static_cast<float*>(Di), oe, mu_c(h), h->d_err, h->st);
    CKL();
    if (h->tc_on) {  // the odd tiles carry D_oo^-1(mu)
      tc_build_odd(static_cast<const float*>(Dc), static_cast<const float*>(Di), oe, h->tc, h->st);
      CKL();
    }
    check_flags(h);
  }
}

// twisted mass mu_even on the even and mu_odd on the odd sites (Sec. 2); a new
// odd shift enters D_c (and D_c2) through the Galerkin projection, so they are
// projected again from the current P (and P2) without a new setup
void apply_mu_eo(tm_handle* h, double mu_even, double mu_odd, double delta) {
  const double rho = mu_odd - mu_even;
  if (rho == h->rho) {
    apply_mu(h, mu_even, delta);
    return;
  }
  h->rho = rho;
  h->p.mu = mu_even;
  h->p.delta = delta;
  if (h->gauge_ok) {
    build_sap_inverse(h);
    check_flags(h);
  }
  if (!h->setup_ok) return;
  if (h->p.cycle_prec == TM_F64) {
    build_coarse<double>(h, false);
    if (h->three) build_level2<double>(h, false);
  } else {
    build_coarse<float>(h, false);
    if (h->three) build_level2<float>(h, false);
  }
  check_flags(h);
}

// ---------------------------------------------------------------------------
// memory plan (tm_workspace_bytes): what tm_create, tm_setup and tm_solve
// allocate on the device for given parameters
// ---------------------------------------------------------------------------
struct MemPlan {
  double persistent = 0, setup = 0, solve = 0;
};

MemPlan memory_plan(const tm_params* p, int nrhs) {
  MemPlan m;
  const double V = (double)p->L[0] * p->L[1] * p->L[2] * p->L[3];
  double a1 = 1, a2 = 1;
  for (int d = 0; d < 4; ++d) a1 *= p->agg[d];
  const double Vc = V / a1;
  const double n = 2.0 * p->nv;
  const double cs = p->cycle_prec == TM_F64 ? 8 : 4;
  const double fr = 24 * V;  // reals of a fine field
  const bool three = p->levels == 3;
  double V2 = 0, n2 = 0;
  if (three) {
    for (int d = 0; d < 4; ++d) a2 *= p->agg2[d];
    V2 = Vc / a2;
    n2 = 2.0 * p->nv2;
  }
  // persistent (tm_create)
  double& P = m.persistent;
  P += 3 * Vc * 4 + (three ? 3 * V2 * 4 : 0);           // odd-even index maps
  P += 48 * V * (8 + 4) + 72 * V * (8 + 4);             // links and clover, FP64 and FP32
  if (p->outer_apply == TM_F32X2) P += 1152 * V;         // links and clover as FP32 pairs
  if (p->block_oe) P += V / 2 * 144 * cs;                // odd-site clover inverses
  P += 2 * p->nv * fr * cs;                              // test vectors, P
  P += Vc * 9 * n * n * 2 * cs + Vc / 2 * n * n * 2 * cs;  // D_c, odd-site inverses
  if (three) {
    P += 2 * p->nv2 * Vc * n * 2 * cs;                   // level-1 test vectors, P2
    P += V2 * 9 * n2 * n2 * 2 * cs + V2 / 2 * n2 * n2 * 2 * cs;
    if (p->sap1_prec == TM_F16 || p->sap1_prec == TM_BF16) P += Vc * 9 * n * n * 4;
  }
  if (p->transfer_prec == TM_F16 || p->transfer_prec == TM_BF16) P += p->nv * fr * 2;  // 16-bit copy of P
  if (p->sap_prec == TM_F16 || p->sap_prec == TM_BF16) P += (48 + 72 + 72) * V * 2;  // 16-bit SAP operator
  const double nvc = three ? p->nv2 : p->nv, nh = (three ? V2 : Vc) / 2;
  double cvc = 2 * (three ? V2 : Vc) * (three ? n2 : n);  // reals of a coarsest vector
  if (p->coarse_mma > 0) {
    const double kp = std::ceil(2 * nvc / 16) * 16, mp = std::ceil(4 * nvc / 8) * 8;
    P += nh * 17 * kp * mp * 4 * (p->coarse_mma == 3 ? 2 : 1) + nh * 17 * 4;
  }
  P += (double)kScratchBlocks * kMaxDots * 2 * 8 + kSmall * 8;
  // work of one K-cycle over r right-hand sides
  auto kcycle_work = [&](double r) {
    double w = (p->pre_smooth > 0 ? fr * r * cs : 0) + 2 * (2 * Vc * n) * r * cs;  // k_r, k_rc, k_ec
    const double mc = p->coarse_restart;
    const double coarse = (5 + (mc + 1)) * (cvc / 2) * r * cs;                        // odd-even GMRES vectors
    w += coarse;
    if (p->coarsest_steps > 0)  // the graph-captured fixed-step solve keeps its own vectors and state
      w += (5 + (p->coarsest_steps + 1)) * (cvc / 2) * r * cs + (double)(p->coarsest_steps + 2) * (p->coarsest_steps + 2) * 16 * r;
    if (three) {
      const double c1 = 2 * Vc * n;
      w += ((mc + 1) + mc + 1) * c1 * r * cs;                                         // level-1 FGMRES basis
      w += (p->pre_smooth1 > 0 ? c1 * r * cs : 0) + 2 * (2 * V2 * n2) * r * cs;       // k1_r, k1_r2, k1_e2
    }
    return w;
  };
  const double nb = std::max(1, std::min(nrhs, p->max_rhs));
  // the K-cycle's work buffers stay allocated, sized for the larger of the
  // setup's N_v test vectors and the solve's batch
  m.persistent += kcycle_work(std::max((double)p->nv, nb));
  // setup: the iterated test vectors (released when the setup returns)
  m.setup = p->nv * fr * cs + (three ? p->nv2 * 2 * Vc * n * cs : 0);
  // solve: FP64 FGMRES(restart) over a batch of nb right-hand sides
  const double mo = p->restart;
  double sv = 2 * fr * nb * 8                           // packed b and x
              + (mo + 1) * fr * nb * 8 + fr * nb * 8   // Krylov basis V and w
              + mo * fr * nb * cs + fr * nb * cs;      // preconditioned basis Z, FP32 copy of v
  if (p->cycle_prec != TM_F64 && p->outer_apply != TM_F32X2) sv += fr * nb * 8;  // FP64 copy of z
  if (p->nn_mode) sv += 2 * fr * nb * cs;
  m.solve = sv;
  return m;
}

}  // namespace

#define API_BEGIN try {
#define API_END                                  \
  }                                              \
  catch (const TmError& e) {                     \
    if (h) h->err = e.m;                         \
    return e.s;                                  \
  }                                              \
  catch (const std::exception& e) {              \
    if (h) h->err = e.what();                    \
    return TM_ERR_CUDA;                          \
  }                                              \
  if (h) h->err.clear();                         \
  return TM_OK;

// ---------------------------------------------------------------------------
// autotuner of the D_c build's tile shape
// ---------------------------------------------------------------------------
// The cache is a JSON object with one entry per line,
//   "<device>/k_coarse_build/<fp32|fp64>/nv<N_v>/agg<a_T>x<a_Z>x<a_Y>x<a_X>": {"ts": 12, "ktc": 2, "us": 512.30},
// read back line by line; entries of other keys are kept when it is rewritten.
struct TuneEntry {
  int ts = 0, ktc = 0;
  double us = 0;
};

static std::map<std::string, TuneEntry> read_tune_cache(const char* path) {
  std::map<std::string, TuneEntry> m;
  FILE* f = std::fopen(path, "r");
  if (!f) return m;
  char line[1024];
  while (std::fgets(line, sizeof line, f)) {
    char key[512];
    TuneEntry e;
    if (std::sscanf(line, " \"%511[^\"]\": {\"ts\": %d, \"ktc\": %d, \"us\": %lf}", key, &e.ts, &e.ktc, &e.us) == 4)
      m[key] = e;
  }
  std::fclose(f);
  return m;
}

static void write_tune_cache(const char* path, const std::map<std::string, TuneEntry>& m) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) raise(TM_ERR_ARG, "cannot write the tuning cache");
  std::fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : m)
    std::fprintf(f, "  \"%s\": {\"ts\": %d, \"ktc\": %d, \"us\": %.2f}%s\n", kv.first.c_str(), kv.second.ts,
                 kv.second.ktc, kv.second.us, ++i < m.size() ? "," : "");
  std::fprintf(f, "}\n");
  const bool ok = std::fclose(f) == 0;
  if (!ok || std::rename(tmp.c_str(), path) != 0) raise(TM_ERR_ARG, "cannot write the tuning cache");
}

template <typename T>
void autotune_build(tm_handle* h, const char* cache_path, int reps, double* out) {
  const AggGeom& ag = h->ag;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  const std::string key = std::string(prop.name) + "/k_coarse_build/" + (sizeof(T) == 4 ? "fp32" : "fp64") + "/nv" +
                          std::to_string(ag.nv) + "/agg" + std::to_string(ag.agg[0]) + "x" +
                          std::to_string(ag.agg[1]) + "x" + std::to_string(ag.agg[2]) + "x" +
                          std::to_string(ag.agg[3]);
  const std::vector<BuildShape> cand = coarse_build_candidates(ag.nv, sizeof(T));
  auto listed = [&](int ts, int ktc) {
    for (const BuildShape& b : cand)
      if (b.ts == ts && b.ktc == ktc) return true;
    return false;
  };
  std::map<std::string, TuneEntry> cache;
  if (cache_path) {
    cache = read_tune_cache(cache_path);
    auto it = cache.find(key);
    if (it != cache.end() && listed(it->second.ts, it->second.ktc)) {
      h->build_shape = BuildShape{it->second.ts, it->second.ktc};
      if (out) {
        out[0] = it->second.ts;
        out[1] = it->second.ktc;
        out[2] = it->second.us;
        out[3] = 0;  // from the cache: nothing timed
      }
      return;
    }
  }
  const T* P = static_cast<const T*>(h->P);
  const size_t n = (size_t)h->gc.V * 9 * h->n * h->n * 2;  // reals of D_c
  // the scratch D_c copies and the events go back on every exit, errors included
  struct Scratch {
    tm_handle* h;
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~Scratch() {
      for (cudaEvent_t ev : e)
        if (ev) h->evpool.push_back(ev);
      release(h, "tune_ref");
      release(h, "tune_dc");
      release(h, "tune_bad");
    }
  } scratch{h};
  T* ref = W<T>(h, "tune_ref", n);
  T* trial = W<T>(h, "tune_dc", n);
  unsigned long long* bad_d = W<unsigned long long>(h, "tune_bad", 1);
  launch_coarse_build<T>(gaugeT<T>(h), cloverT<T>(h), P, ref, ag, h->p.bc_t, h->st, BuildShape{}, h->rho);
  CKL();
  cudaEvent_t e0 = scratch.e[0] = take_event(h);
  cudaEvent_t e1 = scratch.e[1] = take_event(h);
  BuildShape best{};
  double best_us = 0;
  for (const BuildShape& b : cand) {
    // parity first: the candidate's D_c must equal the default's bit for bit
    launch_coarse_build<T>(gaugeT<T>(h), cloverT<T>(h), P, trial, ag, h->p.bc_t, h->st, b, h->rho);
    CKL();
    CK(cudaMemsetAsync(bad_d, 0, sizeof(unsigned long long), h->st));
    launch_count_mismatch(ref, trial, (long)(n * sizeof(T) / 4), bad_d, h->st);
    CKL();
    unsigned long long bad = 0;
    CK(cudaMemcpyAsync(&bad, bad_d, sizeof bad, cudaMemcpyDeviceToHost, h->st));
    sync(h);
    if (bad)
      raise(TM_ERR_STATE, "build shape ts=" + std::to_string(b.ts) + " ktc=" + std::to_string(b.ktc) +
                              " differs from the default D_c in " + std::to_string(bad) + " words");
    CK(cudaEventRecord(e0, h->st));
    for (int r = 0; r < reps; ++r)
      launch_coarse_build<T>(gaugeT<T>(h), cloverT<T>(h), P, trial, ag, h->p.bc_t, h->st, b, h->rho);
    CKL();
    CK(cudaEventRecord(e1, h->st));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    const double us = 1000.0 * ms / reps;
    if (best.ts == 0 || us < best_us) {
      best = b;
      best_us = us;
    }
  }
  h->build_shape = best;
  if (cache_path) {
    cache[key] = TuneEntry{best.ts, best.ktc, best_us};
    write_tune_cache(cache_path, cache);
  }
  if (out) {
    out[0] = best.ts;
    out[1] = best.ktc;
    out[2] = best_us;
    out[3] = (double)cand.size();
  }
}

// ---------------------------------------------------------------------------
// saving and loading a setup
// ---------------------------------------------------------------------------
namespace {
constexpr char kSetupMagic[8] = {'T', 'M', 'A', 'M', 'G', 'S', 'U', '1'};
struct SetupHeader {
  char magic[8];
  int version;
  int L[4], nv, agg[4], levels, nv2, agg2[4], cycle_prec;
  double m0, c_sw, bc_t, rho;  // rho: odd-site twisted-mass shift projected into D_c
  long long nbytes[6];  // tv, P, Dc, tv1, P2, Dc2
};

// the saved arrays in the handle's device layout
void setup_arrays(tm_handle* h, void* ptr[6], size_t bytes[6]) {
  const size_t cs = csize(h->p.cycle_prec);
  const size_t fr = (size_t)NR_SPINOR * h->g.V;
  ptr[0] = h->tv;
  bytes[0] = h->p.nv * fr * cs;
  ptr[1] = h->P;
  bytes[1] = bytes[0];
  ptr[2] = h->Dc;
  bytes[2] = (size_t)h->gc.V * 9 * h->n * h->n * 2 * cs;
  for (int k = 3; k < 6; ++k) {
    ptr[k] = nullptr;
    bytes[k] = 0;
  }
  if (h->three) {
    ptr[3] = h->tv1;
    bytes[3] = (size_t)h->p.nv2 * h->gc.V * h->n * 2 * cs;
    ptr[4] = h->P2;
    bytes[4] = bytes[3];
    ptr[5] = h->Dc2;
    bytes[5] = (size_t)h->gc2.V * 9 * h->n2 * h->n2 * 2 * cs;
  }
}

// device <-> file through a pinned staging buffer
void copy_through(tm_handle* h, FILE* f, void* dev, size_t bytes, bool to_file) {
  constexpr size_t kChunk = 64ull << 20;
  double* hb = host_scratch(h, "io", kChunk / sizeof(double));
  char* d = static_cast<char*>(dev);
  for (size_t o = 0; o < bytes; o += kChunk) {
    const size_t c = std::min(kChunk, bytes - o);
    if (to_file) {
      CK(cudaMemcpyAsync(hb, d + o, c, cudaMemcpyDeviceToHost, h->st));
      sync(h);
      if (std::fwrite(hb, 1, c, f) != c) raise(TM_ERR_ARG, "short write to the setup file");
    } else {
      if (std::fread(hb, 1, c, f) != c) raise(TM_ERR_ARG, "setup file is truncated");
      CK(cudaMemcpyAsync(d + o, hb, c, cudaMemcpyHostToDevice, h->st));
      sync(h);
    }
  }
}

struct FileCloser {
  FILE* f;
  ~FileCloser() {
    if (f) std::fclose(f);
  }
};

template <typename T>
void rebuild_derived(tm_handle* h) {
  // everything the build derives from D_c (and D_c2): FP16 blocks, odd-site
  // inverses with the current mu, tensor-core tiles
  Prof pf(h, PK_BUILD, 0, 1);
  if constexpr (std::is_same<T, float>::value) refresh_16bit(h);
  void* Dc = h->three ? h->Dc2 : h->Dc;
  void* Di = h->three ? h->Dinv2 : h->Dinv;
  const OEGeom& oe = h->three ? h->oe2 : h->oe;
  launch_oe_invert<T>(static_cast<T*>(Dc), static_cast<T*>(Di), oe, mu_c(h), h->d_err, h->st);
  CKL();
  if constexpr (std::is_same<T, float>::value) {
    if (h->tc_on) {
      tc_build(static_cast<const float*>(Dc), static_cast<const float*>(Di), oe, h->tc, h->st);
      CKL();
    }
  }
  check_flags(h);
}
}  // namespace

extern "C" {

void tm_params_default(tm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->bc_t = -1;
  p->delta = 1;
  p->nv = 20;
  for (int d = 0; d < 4; ++d) p->agg[d] = p->sap_block[d] = 4;
  p->mr_iters = 4;
  p->pre_smooth = 0;
  p->post_smooth = 4;
  p->init_sweeps = 3;
  p->setup_iters = 3;
  p->coarse_tol = 5e-2;
  p->coarse_restart = 30;
  p->coarse_maxit = 200;
  p->restart = 25;
  p->maxit = 1000;
  p->cycle_prec = TM_F32;
  p->max_rhs = 1;
  p->levels = 2;
  p->nv2 = 28;
  for (int d = 0; d < 4; ++d) p->agg2[d] = p->sap_block1[d] = 2;
  p->mr_iters1 = 4;
  p->pre_smooth1 = 0;
  p->post_smooth1 = 2;
  p->init_sweeps1 = 3;
  p->coarse_setup_iters = 3;
  p->coarsest_tol = 5e-2;
  p->coarsest_maxit = 200;
  p->coarse_mma = 0;
  p->nn_mode = 0;
  p->nn_prec = TM_F32;
  p->sap1_prec = TM_F32;
  p->transfer_prec = TM_F32;
  p->sap_prec = TM_F32;
  p->coarsest_steps = 0;
  p->outer_apply = TM_F64;
}

const char* tm_status_string(int s) {
  switch (s) {
    case TM_OK: return "ok";
    case TM_ERR_ARG: return "invalid argument";
    case TM_ERR_CUDA: return "CUDA error";
    case TM_ERR_OOM: return "out of device memory";
    case TM_ERR_NOT_CONVERGED: return "not converged";
    case TM_ERR_TIMEOUT: return "device wait timed out";
    case TM_ERR_NOT_SU3: return "gauge link not in SU(3)";
    case TM_ERR_NONFINITE: return "non-finite value";
    case TM_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

const char* tm_last_error(const tm_handle* h) { return h ? h->err.c_str() : "null handle"; }

void tm_destroy(tm_handle* h) {
  if (!h) return;
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  for (auto& kv : h->work)
    if (kv.second.p) cudaFree(kv.second.p);
  void* ptrs[] = {h->d_err, h->g64, h->g32, h->c64, h->c32, h->tv, h->P, h->Dc, h->Dinv,
                  h->d_even, h->d_odd, h->d_cidx, h->scratch, h->dsmall};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (h->hsmall) cudaFreeHost(h->hsmall);
  for (auto& kv : h->hbufs)
    if (kv.second.first) cudaFreeHost(kv.second.first);
  void* p3[] = {h->tv1, h->P2, h->Dc2, h->Dinv2, h->d_even2, h->d_odd2, h->d_cidx2,
                h->tc.even, h->tc.even_lo, h->tc.odd, h->tc.odd_lo, h->tc.nbr_e, h->tc.nbr_o,
                h->d_nnw, h->d_nngrad, h->Dc1h, h->P16, h->g16, h->c16, h->dinv16, h->gdf, h->cdf, h->dinv_sap};
  for (void* q : p3)
    if (q) cudaFree(q);
  for (auto& r : h->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
  for (cudaEvent_t e : h->pipe_ev)
    if (e) cudaEventDestroy(e);
  delete h;
}

tm_status tm_create(tm_handle** out, const tm_params* p, void* stream) {
  tm_handle* h = nullptr;
  if (!out || !p) return TM_ERR_ARG;
  *out = nullptr;
  try {
    validate(p);
    h = new tm_handle();
    h->p = *p;
    h->st = static_cast<cudaStream_t>(stream);
    h->g = make_lat(p->L);
    int Lc[4];
    for (int d = 0; d < 4; ++d) Lc[d] = p->L[d] / p->agg[d];
    h->gc = make_lat(Lc);
    h->n = 2 * p->nv;
    h->nhalf = h->gc.V / 2;
    h->sg.g = h->g;
    h->sg.bsites = 1;
    for (int d = 0; d < 4; ++d) {
      h->sg.blk[d] = p->sap_block[d];
      h->sg.nb[d] = p->L[d] / p->sap_block[d];
      h->sg.bsites *= p->sap_block[d];
    }
    h->ag.g = h->g;
    h->ag.gc = h->gc;
    h->ag.asites = 1;
    h->ag.nv = p->nv;
    for (int d = 0; d < 4; ++d) {
      h->ag.agg[d] = p->agg[d];
      h->ag.asites *= p->agg[d];
    }
    // odd-even index maps of the coarse lattice
    std::vector<int> ev, od, cidx(h->gc.V);
    for (int a = 0; a < h->gc.V; ++a) {
      int c[4];
      site_coords(h->gc, a, c);
      if ((c[0] + c[1] + c[2] + c[3]) % 2 == 0) {
        cidx[a] = (int)ev.size();
        ev.push_back(a);
      } else {
        cidx[a] = (int)od.size();
        od.push_back(a);
      }
    }
    h->d_even = static_cast<int*>(dalloc(ev.size() * sizeof(int)));
    h->d_odd = static_cast<int*>(dalloc(od.size() * sizeof(int)));
    h->d_cidx = static_cast<int*>(dalloc(cidx.size() * sizeof(int)));
    CK(cudaMemcpy(h->d_even, ev.data(), ev.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_odd, od.data(), od.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_cidx, cidx.data(), cidx.size() * sizeof(int), cudaMemcpyHostToDevice));
    h->oe.gc = h->gc;
    h->oe.nv = p->nv;
    h->oe.nhalf = h->nhalf;
    h->oe.even_site = h->d_even;
    h->oe.odd_site = h->d_odd;
    h->oe.cidx = h->d_cidx;

    const long V = h->g.V;
    h->d_err = static_cast<int*>(dalloc(sizeof(int)));
    CK(cudaMemset(h->d_err, 0, sizeof(int)));
    h->g64 = static_cast<double*>(dalloc(4L * NR_LINK * V * sizeof(double)));
    h->g32 = static_cast<float*>(dalloc(4L * NR_LINK * V * sizeof(float)));
    h->c64 = static_cast<double*>(dalloc((long)NR_CLOVER * V * sizeof(double)));
    h->c32 = static_cast<float*>(dalloc((long)NR_CLOVER * V * sizeof(float)));
    if (p->block_oe) h->dinv_sap = dalloc((size_t)(V / 2) * 144 * csize(p->cycle_prec));
    if (p->outer_apply == TM_F32X2) {
      h->gdf = dalloc((size_t)4 * 9 * V * 4 * sizeof(float));
      h->cdf = dalloc((size_t)36 * V * 4 * sizeof(float));
    }
    const size_t cs = csize(p->cycle_prec);
    h->tv = dalloc((size_t)p->nv * NR_SPINOR * V * cs);
    h->P = dalloc((size_t)p->nv * NR_SPINOR * V * cs);
    h->Dc = dalloc((size_t)h->gc.V * 9 * h->n * h->n * 2 * cs);
    h->Dinv = dalloc((size_t)h->nhalf * h->n * h->n * 2 * cs);
    if (p->levels == 3) {
      h->three = true;
      int L2[4];
      for (int d = 0; d < 4; ++d) L2[d] = Lc[d] / p->agg2[d];
      h->gc2 = make_lat(L2);
      h->n2 = 2 * p->nv2;
      h->nhalf2 = h->gc2.V / 2;
      h->csg.g = h->gc;
      h->csg.n = h->n;
      h->csg.bsites = 1;
      h->cag.g1 = h->gc;
      h->cag.g2 = h->gc2;
      h->cag.asites = 1;
      h->cag.nv1 = p->nv;
      h->cag.nv2 = p->nv2;
      for (int d = 0; d < 4; ++d) {
        h->csg.blk[d] = p->sap_block1[d];
        h->csg.nb[d] = Lc[d] / p->sap_block1[d];
        h->csg.bsites *= p->sap_block1[d];
        h->cag.agg[d] = p->agg2[d];
        h->cag.asites *= p->agg2[d];
      }
      std::vector<int> ev2, od2, cidx2(h->gc2.V);
      for (int a = 0; a < h->gc2.V; ++a) {
        int c[4];
        site_coords(h->gc2, a, c);
        if ((c[0] + c[1] + c[2] + c[3]) % 2 == 0) {
          cidx2[a] = (int)ev2.size();
          ev2.push_back(a);
        } else {
          cidx2[a] = (int)od2.size();
          od2.push_back(a);
        }
      }
      h->d_even2 = static_cast<int*>(dalloc(ev2.size() * sizeof(int)));
      h->d_odd2 = static_cast<int*>(dalloc(od2.size() * sizeof(int)));
      h->d_cidx2 = static_cast<int*>(dalloc(cidx2.size() * sizeof(int)));
      CK(cudaMemcpy(h->d_even2, ev2.data(), ev2.size() * sizeof(int), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->d_odd2, od2.data(), od2.size() * sizeof(int), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->d_cidx2, cidx2.data(), cidx2.size() * sizeof(int), cudaMemcpyHostToDevice));
      h->oe2.gc = h->gc2;
      h->oe2.nv = p->nv2;
      h->oe2.nhalf = h->nhalf2;
      h->oe2.even_site = h->d_even2;
      h->oe2.odd_site = h->d_odd2;
      h->oe2.cidx = h->d_cidx2;
      h->tv1 = dalloc((size_t)p->nv2 * h->gc.V * h->n * 2 * cs);
      h->P2 = dalloc((size_t)p->nv2 * h->gc.V * h->n * 2 * cs);
      h->Dc2 = dalloc((size_t)h->gc2.V * 9 * h->n2 * h->n2 * 2 * cs);
      h->Dinv2 = dalloc((size_t)h->nhalf2 * h->n2 * h->n2 * 2 * cs);
      if (p->sap1_prec == TM_F16 || p->sap1_prec == TM_BF16)
        h->Dc1h = dalloc((size_t)h->gc.V * 9 * h->n * h->n * 4);
    }
    if (p->transfer_prec == TM_F16 || p->transfer_prec == TM_BF16)
      h->P16 = dalloc((size_t)p->nv * h->g.V * 12 * 4);
    if (p->sap_prec == TM_F16 || p->sap_prec == TM_BF16) {
      h->g16 = dalloc((size_t)h->g.V * 4 * NR_LINK * 2);
      h->c16 = dalloc((size_t)h->g.V * NR_CLOVER * 2);
      h->dinv16 = dalloc((size_t)h->g.V / 2 * 144 * 2);
    }
    if (p->coarse_mma > 0) {  // tensor-core tiles of the coarsest odd-even level
      const int nvc = h->three ? p->nv2 : p->nv, nh = h->three ? h->nhalf2 : h->nhalf;
      h->tc_on = true;
      h->tc.kp = (2 * nvc + 15) / 16 * 16;
      h->tc.mp = (4 * nvc + 7) / 8 * 8;
      const size_t tile = (size_t)h->tc.kp * h->tc.mp * sizeof(float);
      h->tc.even = static_cast<float*>(dalloc((size_t)nh * 9 * tile));
      h->tc.odd = static_cast<float*>(dalloc((size_t)nh * 8 * tile));
      if (p->coarse_mma == 3) {
        h->tc.even_lo = static_cast<float*>(dalloc((size_t)nh * 9 * tile));
        h->tc.odd_lo = static_cast<float*>(dalloc((size_t)nh * 8 * tile));
      }
      h->tc.nbr_e = static_cast<int*>(dalloc((size_t)nh * 9 * sizeof(int)));
      h->tc.nbr_o = static_cast<int*>(dalloc((size_t)nh * 8 * sizeof(int)));
    }
    h->scratch = static_cast<double*>(dalloc((size_t)kScratchBlocks * kMaxDots * 2 * sizeof(double)));
    h->dsmall = static_cast<double*>(dalloc(kSmall * sizeof(double)));
    CK(cudaMallocHost(&h->hsmall, kSmall * sizeof(double)));
    *out = h;
  } catch (const TmError& e) {
    if (h) tm_destroy(h);
    return e.s;
  } catch (...) {
    if (h) tm_destroy(h);
    return TM_ERR_OOM;
  }
  return TM_OK;
}

tm_status tm_load_gauge(tm_handle* h, const double* gauge) {
  if (!h || !gauge) return TM_ERR_ARG;
  API_BEGIN
  const size_t bytes = (size_t)h->g.V * 4 * 9 * 2 * sizeof(double);
  const double* gd = stage_in(h, gauge, bytes, "stage_gauge");
  {
    Prof pf(h, PK_OTHER, 1, 2);
    launch_pack_gauge(gd, h->g64, h->g32, h->g, 1e-10, h->d_err, h->st);
    CKL();
    launch_clover(gd, h->c64, h->c32, h->g, h->p.m0, h->p.c_sw, h->st);
    CKL();
  }
  if (h->g16) {
    Prof pf(h, PK_OTHER, 1, 2);
    launch_to16(h->g32, h->g16, (long)h->g.V * 4 * NR_LINK / 2, h->p.sap_prec, h->st);
    CKL();
    launch_to16(h->c32, h->c16, (long)h->g.V * NR_CLOVER / 2, h->p.sap_prec, h->st);
    CKL();
  }
  if (h->gdf) {
    Prof pf(h, PK_OTHER, 1, 2);
    launch_pack_gauge_df(gd, h->gdf, h->g, h->st);
    CKL();
    launch_clover_df(h->c64, h->cdf, h->g, h->st);
    CKL();
  }
  build_sap_inverse(h);
  h->gauge_ok = false;
  h->setup_ok = false;
  check_flags(h);
  release(h, "stage_gauge");  // a host field's device copy is not needed any more
  h->gauge_ok = true;
  API_END
}

static tm_status setup_common(tm_handle* h, const double* tv, bool adaptive) {
  if (!h || !tv) return TM_ERR_ARG;
  API_BEGIN
  if (!h->gauge_ok) raise(TM_ERR_STATE, "tm_load_gauge must come first");
  h->setup_ok = false;
  size_t bytes = (size_t)h->p.nv * h->g.V * 12 * 2 * sizeof(double);
  if (h->three) bytes += (size_t)h->p.nv2 * h->gc.V * h->n * 2 * sizeof(double);  // level-1 random vectors
  const double* d = stage_in(h, tv, bytes, "stage_tv");
  h->coarse_iters = 0;
  h->kcycles = 0;
  if (h->p.cycle_prec == TM_F64)
    setup_impl<double>(h, d, adaptive);
  else
    setup_impl<float>(h, d, adaptive);
  release(h, "stage_tv");  // a host array's device copy is not needed any more
  h->setup_ok = true;
  h->tv_ok = true;
  API_END
}

tm_status tm_setup_update(tm_handle* h, int fine_iters, int coarse_iters) {
  if (!h || fine_iters < 0 || coarse_iters < 0) return TM_ERR_ARG;
  API_BEGIN
  if (!h->gauge_ok) raise(TM_ERR_STATE, "tm_load_gauge must come first");
  if (!h->tv_ok) raise(TM_ERR_STATE, "needs the test vectors of an earlier setup");
  h->setup_ok = false;
  if (h->p.cycle_prec == TM_F64) {
    setup_rebuild<double>(h);
    setup_iterate<double>(h, fine_iters, coarse_iters);
  } else {
    setup_rebuild<float>(h);
    setup_iterate<float>(h, fine_iters, coarse_iters);
  }
  sync(h);
  h->setup_ok = true;
  API_END
}

tm_status tm_setup(tm_handle* h, const double* test_vectors) { return setup_common(h, test_vectors, true); }
tm_status tm_setup_from_vectors(tm_handle* h, const double* test_vectors) {
  return setup_common(h, test_vectors, false);
}

tm_status tm_autotune_build(tm_handle* h, const char* cache_path, int reps, double* out) {
  if (!h || reps < 1 || reps > 100) return TM_ERR_ARG;
  API_BEGIN
  if (!h->setup_ok) raise(TM_ERR_STATE, "tm_setup must come first");
  if (h->p.cycle_prec == TM_F64)
    autotune_build<double>(h, cache_path, reps, out);
  else
    autotune_build<float>(h, cache_path, reps, out);
  API_END
}

tm_status tm_set_mu(tm_handle* h, double mu, double delta) {
  if (!h) return TM_ERR_ARG;
  API_BEGIN
  if (!(delta >= 1.0) || !std::isfinite(mu)) raise(TM_ERR_ARG, "need finite mu and delta >= 1");
  apply_mu_eo(h, mu, mu, delta);
  API_END
}

tm_status tm_set_mu_eo(tm_handle* h, double mu_even, double mu_odd, double delta) {
  if (!h) return TM_ERR_ARG;
  API_BEGIN
  if (!(delta >= 1.0) || !std::isfinite(mu_even) || !std::isfinite(mu_odd))
    raise(TM_ERR_ARG, "need finite twisted masses and delta >= 1");
  apply_mu_eo(h, mu_even, mu_odd, delta);
  API_END
}

tm_status tm_solve(tm_handle* h, const double* b, double* x, int nrhs, double tol, tm_solve_info* info) {
  if (!h || !b || !x || nrhs < 1 || !(tol > 0)) return TM_ERR_ARG;
  tm_solve_info loc{};
  loc.converged = 1;
  tm_status st = TM_OK;
  try {
    if (!h->setup_ok) raise(TM_ERR_STATE, "tm_setup must come first");
    const long V = h->g.V;
    const size_t one = (size_t)V * 12 * 2 * sizeof(double);
    const bool xdev = is_device_ptr(x);
    const double* bd = stage_in(h, b, one * nrhs, "stage_b");
    double* xd = xdev ? x : W<double>(h, "stage_x", one * nrhs / sizeof(double));
    if (!xdev) CK(cudaMemcpyAsync(xd, x, one * nrhs, cudaMemcpyHostToDevice, h->st));
    h->coarse_iters = 0;
    h->kcycles = 0;
    solve_core(h, bd, xd, nrhs, tol, loc);
    if (!xdev) CK(cudaMemcpyAsync(x, xd, one * nrhs, cudaMemcpyDeviceToHost, h->st));
    sync(h);
    loc.coarse_iters = h->coarse_iters;
    loc.kcycles = h->kcycles;
    if (!loc.converged) {
      h->err = "solver reached maxit";
      st = TM_ERR_NOT_CONVERGED;
    } else {
      h->err.clear();
    }
  } catch (const TmError& e) {
    h->err = e.m;
    st = e.s;
  } catch (const std::exception& e) {
    h->err = e.what();
    st = TM_ERR_CUDA;
  }
  if (info) *info = loc;
  return st;
}

tm_status tm_solve_squared(tm_handle* h, const double* b, double* x, int nrhs, double tol, tm_solve_info* info) {
  if (!h || !b || !x || nrhs < 1 || !(tol > 0)) return TM_ERR_ARG;
  tm_solve_info loc{};
  loc.converged = 1;
  tm_status st = TM_OK;
  const double mu = h->p.mu, rho = h->rho;
  try {
    if (!h->setup_ok) raise(TM_ERR_STATE, "tm_setup must come first");
    const long V = h->g.V;
    const size_t one = (size_t)V * 12 * 2 * sizeof(double);
    const bool xdev = is_device_ptr(x);
    const double* bd = stage_in(h, b, one * nrhs, "stage_b");
    double* xd = xdev ? x : W<double>(h, "stage_x", one * nrhs / sizeof(double));
    if (!xdev) CK(cudaMemcpyAsync(xd, x, one * nrhs, cudaMemcpyHostToDevice, h->st));
    double* y = W<double>(h, "sq_y", one * nrhs / sizeof(double));
    double* z = W<double>(h, "sq_z", one * nrhs / sizeof(double));
    h->coarse_iters = 0;
    h->kcycles = 0;
    launch_gamma5_nat(bd, y, (long)V * nrhs, h->st);  // y = Gamma5 b
    CKL();
    CK(cudaMemsetAsync(z, 0, one * nrhs, h->st));
    apply_mu_eo(h, -mu, -mu - rho, h->p.delta);  // D(mu)^dagger = Gamma5 D(-mu) Gamma5: same setup
    solve_core(h, y, z, nrhs, tol, loc);
    launch_gamma5_nat(z, y, (long)V * nrhs, h->st);  // y = Gamma5 z
    CKL();
    apply_mu_eo(h, mu, mu + rho, h->p.delta);  // D(mu) x = Gamma5 z
    solve_core(h, y, xd, nrhs, tol, loc);
    if (!xdev) CK(cudaMemcpyAsync(x, xd, one * nrhs, cudaMemcpyDeviceToHost, h->st));
    sync(h);
    loc.coarse_iters = h->coarse_iters;
    loc.kcycles = h->kcycles;
    if (!loc.converged) {
      h->err = "solver reached maxit";
      st = TM_ERR_NOT_CONVERGED;
    } else {
      h->err.clear();
    }
  } catch (const TmError& e) {
    h->err = e.m;
    st = e.s;
  } catch (const std::exception& e) {
    h->err = e.what();
    st = TM_ERR_CUDA;
  }
  if (h->p.mu != mu || h->rho != rho) {  // leave the handle at +mu even after an error
    try {
      apply_mu_eo(h, mu, mu + rho, h->p.delta);
    } catch (...) {
    }
  }
  if (info) *info = loc;
  return st;
}

// the odd-site reduced system through the full operator: b's even sites are
// dropped, x's even sites are zeroed on return (Sec. 3)
static void solve_odd_core(tm_handle* h, const double* bd, double* xd, int nrhs, double tol, tm_solve_info& loc) {
  const long V = h->g.V;
  const size_t one = (size_t)V * 12 * 2 * sizeof(double);
  double* bw = W<double>(h, "odd_b", one * nrhs / sizeof(double));
  CK(cudaMemcpyAsync(bw, bd, one * nrhs, cudaMemcpyDeviceToDevice, h->st));
  launch_zero_parity_nat(bw, h->g, 0, nrhs, h->st);
  CKL();
  solve_core(h, bw, xd, nrhs, tol, loc);
  launch_zero_parity_nat(xd, h->g, 0, nrhs, h->st);
  CKL();
}

static tm_status finish_solve(tm_handle* h, tm_solve_info& loc) {
  loc.coarse_iters = h->coarse_iters;
  loc.kcycles = h->kcycles;
  if (!loc.converged) {
    h->err = "solver reached maxit";
    return TM_ERR_NOT_CONVERGED;
  }
  h->err.clear();
  return TM_OK;
}

tm_status tm_solve_odd(tm_handle* h, const double* b, double* x, int nrhs, double tol, tm_solve_info* info) {
  if (!h || !b || !x || nrhs < 1 || !(tol > 0)) return TM_ERR_ARG;
  tm_solve_info loc{};
  loc.converged = 1;
  tm_status st = TM_OK;
  try {
    if (!h->setup_ok) raise(TM_ERR_STATE, "tm_setup must come first");
    const size_t one = (size_t)h->g.V * 12 * 2 * sizeof(double);
    const bool xdev = is_device_ptr(x);
    const double* bd = stage_in(h, b, one * nrhs, "stage_b");
    double* xd = xdev ? x : W<double>(h, "stage_x", one * nrhs / sizeof(double));
    if (!xdev) CK(cudaMemcpyAsync(xd, x, one * nrhs, cudaMemcpyHostToDevice, h->st));
    h->coarse_iters = 0;
    h->kcycles = 0;
    solve_odd_core(h, bd, xd, nrhs, tol, loc);
    if (!xdev) CK(cudaMemcpyAsync(x, xd, one * nrhs, cudaMemcpyDeviceToHost, h->st));
    sync(h);
    st = finish_solve(h, loc);
  } catch (const TmError& e) {
    h->err = e.m;
    st = e.s;
  } catch (const std::exception& e) {
    h->err = e.what();
    st = TM_ERR_CUDA;
  }
  if (info) *info = loc;
  return st;
}

tm_status tm_solve_hasenbusch(tm_handle* h, const double* b, double* x, int nrhs, double mu, double rho, double tol,
                              tm_solve_info* info) {
  if (!h || !b || !x || nrhs < 1 || !(tol > 0) || !std::isfinite(mu) || !std::isfinite(rho)) return TM_ERR_ARG;
  tm_solve_info loc{};
  loc.converged = 1;
  tm_status st = TM_OK;
  try {
    if (!h->setup_ok) raise(TM_ERR_STATE, "tm_setup must come first");
    const long V = h->g.V;
    const size_t one = (size_t)V * 12 * 2 * sizeof(double);
    const bool xdev = is_device_ptr(x);
    const double* bd = stage_in(h, b, one * nrhs, "stage_b");
    double* xd = xdev ? x : W<double>(h, "stage_x", one * nrhs / sizeof(double));
    double* y = W<double>(h, "hb_y", one * nrhs / sizeof(double));
    double* z = W<double>(h, "hb_z", one * nrhs / sizeof(double));
    h->coarse_iters = 0;
    h->kcycles = 0;
    // y = (D^(mu) + i rho G^5)^-1 b: the odd Schur complement of D(mu, mu + rho)
    apply_mu_eo(h, mu, mu + rho, h->p.delta);
    CK(cudaMemsetAsync(y, 0, one * nrhs, h->st));
    solve_odd_core(h, bd, y, nrhs, tol, loc);
    // x = (G^5 D^(-mu) G^5 - i rho G^5)^-1 y = G^5 (D^(-mu) - i rho G^5)^-1 G^5 y
    launch_gamma5_nat(y, z, (long)V * nrhs, h->st);
    CKL();
    apply_mu_eo(h, -mu, -mu - rho, h->p.delta);
    CK(cudaMemsetAsync(y, 0, one * nrhs, h->st));
    solve_odd_core(h, z, y, nrhs, tol, loc);
    launch_gamma5_nat(y, xd, (long)V * nrhs, h->st);
    CKL();
    if (!xdev) CK(cudaMemcpyAsync(x, xd, one * nrhs, cudaMemcpyDeviceToHost, h->st));
    sync(h);
    st = finish_solve(h, loc);
  } catch (const TmError& e) {
    h->err = e.m;
    st = e.s;
  } catch (const std::exception& e) {
    h->err = e.what();
    st = TM_ERR_CUDA;
  }
  try {  // leave the handle at the first operator, D(mu) on even and mu + rho on odd sites
    apply_mu_eo(h, mu, mu + rho, h->p.delta);
  } catch (...) {
  }
  if (info) *info = loc;
  return st;
}

// ---------------------------------------------------------------------------
// oeCG: CG on the normal equations of the odd-even reduced operator, the
// comparison solver of Fig. 1 (Sec. 1), in FP32 iterations inside FP64
// defect correction
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

struct OeCG {
  tm_handle* h;
  long Vh, nr;  // half-field sites and reals
  double* dinv64;
  float* dinv32;
};

// D_ee^-1 at the even twisted mass, FP64 and FP32 copies (rebuilt per solve)
OeCG oecg_prepare(tm_handle* h) {
  OeCG o{h, h->g.V / 2, (long)(h->g.V / 2) * NR_SPINOR, nullptr, nullptr};
  o.dinv64 = W<double>(h, "oe_dinv64", (size_t)o.Vh * 144);
  o.dinv32 = W<float>(h, "oe_dinv32", (size_t)o.Vh * 144);
  Prof pf(h, PK_OTHER, 1, 2);
  launch_clover_inverse<double>(h->c64, o.dinv64, h->g, h->p.mu, h->d_err, h->st, 0);
  CKL();
  launch_clover_inverse<float>(h->c64, o.dinv32, h->g, h->p.mu, h->d_err, h->st, 0);
  CKL();
  return o;
}

// out = D^ in (adj: D^dagger = G^5 D^(-mu) G^5), odd half fields; tmp an even half field
template <typename T>
void oe_reduced(const OeCG& o, const T* in, T* out, T* tmp, bool adj) {
  tm_handle* h = o.h;
  const T* dinv;
  if constexpr (std::is_same<T, double>::value)
    dinv = o.dinv64;
  else
    dinv = o.dinv32;
  const double muo = h->p.mu + h->rho;
  Prof pf(h, PK_OECG_OP, 1, 2);
  launch_oe_apply<T>(gaugeT<T>(h), nullptr, dinv, in, nullptr, tmp, h->g, 0, -0.5, 0.0, h->p.bc_t, adj, adj, 0,
                     h->st);
  CKL();
  launch_oe_apply<T>(gaugeT<T>(h), cloverT<T>(h), nullptr, tmp, in, out, h->g, 1, 0.5, adj ? -muo : muo,
                     h->p.bc_t, adj, 0, 1, h->st);
  CKL();
}

// one right-hand side; bf, xf packed FP64 full fields (xf: start vector in, solution out)
KrylovOut oecg_one(const OeCG& o, const double* bf, double* xf, double tol, int maxit) {
  tm_handle* h = o.h;
  const long nr = o.nr, ncx = nr / 2;
  double* be = W<double>(h, "oe_be", nr);
  double* bo = W<double>(h, "oe_bo", nr);
  double* bh = W<double>(h, "oe_bh", nr);
  double* xo = W<double>(h, "oe_xo", nr);
  double* r64 = W<double>(h, "oe_r64", nr);
  double* t64 = W<double>(h, "oe_t64", nr);
  double* u64 = W<double>(h, "oe_u64", nr);
  float* r = W<float>(h, "oe_r", nr);
  float* e = W<float>(h, "oe_e", nr);
  float* s = W<float>(h, "oe_s", nr);
  float* p = W<float>(h, "oe_p", nr);
  float* q = W<float>(h, "oe_q", nr);
  float* t = W<float>(h, "oe_t", nr);
  constexpr int kBlocks = 2432;
  double* part = W<double>(h, "oe_part", 2 * kBlocks);
  constexpr int kCheck = 8;  // CG steps between host convergence checks
  const int cap = std::max(maxit, 1);
  double* sc = W<double>(h, "oe_sc", 4);
  double* hist = W<double>(h, "oe_hist", (size_t)cap + kCheck);
  double* hh = host_scratch(h, "oe", (size_t)cap + kCheck + 4);
  auto nrm2 = [&](const auto* v, long n_cx, double* dst, int kind) {
    Prof pf(h, kind, 1, 2);
    using V = std::remove_const_t<std::remove_pointer_t<decltype(v)>>;
    launch_norm2<V>(v, n_cx, 1, dst, part, kBlocks, h->st);
    CKL();
  };
  auto read = [&](const double* src, size_t n) {
    CK(cudaMemcpyAsync(hh, src, n * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    sync(h);
  };
  KrylovOut out;
  {
    Prof pf(h, PK_OTHER, 1, 6);
    launch_parity_copy<double>(bf, be, h->g, 0, false, h->st);
    CKL();
    launch_parity_copy<double>(bf, bo, h->g, 1, false, h->st);
    CKL();
    launch_parity_copy<double>(xf, xo, h->g, 1, false, h->st);
    CKL();
    // b^ = b_o - D_oe D_ee^-1 b_e = b_o + H (D_ee^-1 b_e) / 2
    launch_oe_apply<double>(h->g64, nullptr, o.dinv64, nullptr, be, t64, h->g, 0, 0.0, 0.0, h->p.bc_t, 0, 0, 0, h->st);
    CKL();
    launch_oe_apply<double>(h->g64, nullptr, nullptr, t64, bo, bh, h->g, 1, 0.5, 0.0, h->p.bc_t, 0, 0, 1, h->st);
    CKL();
  }
  nrm2(bf, (long)h->g.V * 12, sc + 3, PK_OECG_BLAS);
  read(sc + 3, 1);
  const double bnorm = std::sqrt(hh[0]);
  if (!std::isfinite(bnorm)) raise(TM_ERR_NONFINITE, "non-finite right-hand side");
  auto true_residual = [&]() {  // r64 = b^ - D^ x_o in FP64, returns |r64|
    oe_reduced<double>(o, xo, u64, t64, false);
    {
      Prof pf(h, PK_OECG_BLAS, 1);
      CK(cudaMemcpyAsync(r64, bh, nr * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
      launch_caxpby<double>(-1.0, 0.0, u64, 1.0, 0.0, r64, ncx, h->st);
      CKL();
    }
    nrm2(r64, ncx, sc + 3, PK_OECG_BLAS);
    read(sc + 3, 1);
    return std::sqrt(hh[0]);
  };
  double rn = true_residual();
  constexpr double kInner = 1e-5;  // FP32 CG reduces the defect by this factor per cycle
  while (bnorm > 0 && rn > tol * bnorm && out.iters < maxit) {
    if (!std::isfinite(rn)) raise(TM_ERR_NONFINITE, "non-finite residual");
    ++out.restarts;
    const double target = std::max(kInner, 0.5 * tol * bnorm / rn) * rn;  // on |r| of this cycle
    {
      Prof pf(h, PK_OECG_BLAS, 1, 2);
      launch_convert<double, float>(r64, r, nr, h->st);
      CKL();
      launch_zero<float>(e, nr, h->st);
      CKL();
    }
    oe_reduced<float>(o, r, s, t, true);  // s = D^dagger r
    nrm2(s, ncx, sc + 0, PK_OECG_BLAS);   // gamma_0
    CK(cudaMemcpyAsync(p, s, nr * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
    int k = 0, done = -1;
    const int budget = maxit - out.iters;
    while (done < 0 && k < budget) {
      const int k_end = std::min(k + kCheck, budget);
      for (; k < k_end; ++k) {
        oe_reduced<float>(o, p, q, t, false);  // q = D^ p
        nrm2(q, ncx, sc + 2, PK_OECG_BLAS);
        {
          Prof pf(h, PK_OECG_BLAS, 1);
          launch_cg_xr<float>(e, r, p, q, sc, k & 1, 2, nr, h->st);
          CKL();
        }
        nrm2(r, ncx, hist + k, PK_OECG_BLAS);
        oe_reduced<float>(o, r, s, t, true);  // s = D^dagger r
        nrm2(s, ncx, sc + ((k + 1) & 1), PK_OECG_BLAS);
        {
          Prof pf(h, PK_OECG_BLAS, 1);
          launch_cg_p<float>(p, s, sc, (k + 1) & 1, k & 1, nr, h->st);
          CKL();
        }
      }
      read(hist, (size_t)k);
      for (int j = 0; j < k; ++j) {
        if (!std::isfinite(hh[j])) raise(TM_ERR_NONFINITE, "non-finite CG residual");
        if (std::sqrt(hh[j]) <= target) {
          done = j;
          break;
        }
      }
    }
    out.iters += k;
    {
      Prof pf(h, PK_OECG_BLAS, 1);
      launch_acc_f32(e, xo, nr, h->st);  // x_o += e
      CKL();
    }
    const double rn_new = true_residual();
    if (done < 0 && rn_new >= rn) break;  // no progress within the budget
    rn = rn_new;
  }
  {  // x_e = D_ee^-1 (b_e - D_eo x_o) = D_ee^-1 (b_e + H x_o / 2); x = (x_e, x_o)
    Prof pf(h, PK_OTHER, 1, 3);
    launch_oe_apply<double>(h->g64, nullptr, o.dinv64, xo, be, t64, h->g, 0, 0.5, 0.0, h->p.bc_t, 0, 0, 0, h->st);
    CKL();
    launch_parity_copy<double>(t64, xf, h->g, 0, true, h->st);
    CKL();
    launch_parity_copy<double>(xo, xf, h->g, 1, true, h->st);
    CKL();
  }
  out.relres = bnorm > 0 ? rn / bnorm : 0.0;
  out.converged = bnorm == 0 || rn <= tol * bnorm;
  return out;
}

}  // namespace

extern "C" {

tm_status tm_solve_oecg(tm_handle* h, const double* b, double* x, int nrhs, double tol, int maxit,
                        tm_solve_info* info) {
  if (!h || !b || !x || nrhs < 1 || !(tol > 0) || maxit < 1) return TM_ERR_ARG;
  tm_solve_info loc{};
  loc.converged = 1;
  tm_status st = TM_OK;
  try {
    if (!h->gauge_ok) raise(TM_ERR_STATE, "tm_load_gauge must come first");
    if (h->g.L[3] % 2) raise(TM_ERR_ARG, "odd-even ordering needs an even X extent");
    const long V = h->g.V;
    const size_t one = (size_t)V * 12 * 2 * sizeof(double);
    const bool xdev = is_device_ptr(x);
    const double* bd = stage_in(h, b, one * nrhs, "stage_b");
    double* xd = xdev ? x : W<double>(h, "stage_x", one * nrhs / sizeof(double));
    if (!xdev) CK(cudaMemcpyAsync(xd, x, one * nrhs, cudaMemcpyHostToDevice, h->st));
    const long fr = fine_reals(h);
    double* bf = W<double>(h, "s_b", fr);
    double* xf = W<double>(h, "s_x", fr);
    const OeCG o = oecg_prepare(h);
    check_flags(h);
    for (int rr = 0; rr < nrhs; ++rr) {
      {
        Prof pf(h, PK_OTHER, 1, 2);
        launch_pack_spinor<double>(bd + (size_t)rr * V * 24, bf, h->g, 1, h->st);
        CKL();
        launch_pack_spinor<double>(xd + (size_t)rr * V * 24, xf, h->g, 1, h->st);
        CKL();
      }
      const KrylovOut k = oecg_one(o, bf, xf, tol, maxit);
      {
        Prof pf(h, PK_OTHER);
        launch_unpack_spinor<double>(xf, xd + (size_t)rr * V * 24, h->g, 1, h->st);
        CKL();
      }
      loc.iters += k.iters;
      loc.restarts += k.restarts;
      loc.true_relres = std::max(loc.true_relres, k.relres);
      if (!k.converged) loc.converged = 0;
    }
    if (!xdev) CK(cudaMemcpyAsync(x, xd, one * nrhs, cudaMemcpyDeviceToHost, h->st));
    sync(h);
    if (!loc.converged) {
      h->err = "oeCG reached maxit without converging";
      st = TM_ERR_NOT_CONVERGED;
    } else {
      h->err.clear();
    }
  } catch (const TmError& e) {
    h->err = e.m;
    st = e.s;
  } catch (const std::exception& e) {
    h->err = e.what();
    st = TM_ERR_CUDA;
  }
  if (info) *info = loc;
  return st;
}

size_t tm_field_bytes(const tm_handle* h, int level, int prec, int nrhs) {
  if (!h || nrhs < 1 || (prec != TM_F64 && prec != TM_F32)) return 0;
  if (level == 0) return (size_t)nrhs * NR_SPINOR * h->g.V * csize(prec);
  if (level == 1) return (size_t)nrhs * h->gc.V * h->n * 2 * csize(prec);
  if (level == 2 && h->three) return (size_t)nrhs * h->gc2.V * h->n2 * 2 * csize(prec);
  return 0;
}

static void need_dev(const void* p, const char* what) {
  if (!is_device_ptr(p)) raise(TM_ERR_ARG, std::string(what) + " must be a device pointer");
}

tm_status tm_pack(tm_handle* h, int level, int prec, const double* natural, void* field, int nrhs) {
  if (!h || !natural || !field || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  need_dev(natural, "natural");
  need_dev(field, "field");
  if (level == 0) {
    if (prec == TM_F64)
      launch_pack_spinor<double>(natural, static_cast<double*>(field), h->g, nrhs, h->st);
    else if (prec == TM_F32)
      launch_pack_spinor<float>(natural, static_cast<float*>(field), h->g, nrhs, h->st);
    else
      raise(TM_ERR_ARG, "bad precision");
  } else if (level == 1 || (level == 2 && h->three)) {
    const long nre = (long)nrhs * 2 * (level == 1 ? level1_cx(h) : level2_cx(h));
    if (prec == TM_F64)
      launch_convert<double, double>(natural, static_cast<double*>(field), nre, h->st);
    else if (prec == TM_F32)
      launch_convert<double, float>(natural, static_cast<float*>(field), nre, h->st);
    else
      raise(TM_ERR_ARG, "bad precision");
  } else {
    raise(TM_ERR_ARG, "level must be 0 or 1");
  }
  CKL();
  API_END
}

tm_status tm_unpack(tm_handle* h, int level, int prec, const void* field, double* natural, int nrhs) {
  if (!h || !natural || !field || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  need_dev(natural, "natural");
  need_dev(field, "field");
  if (level == 0) {
    if (prec == TM_F64)
      unpack_fine<double>(h, field, natural, nrhs);
    else if (prec == TM_F32)
      unpack_fine<float>(h, field, natural, nrhs);
    else
      raise(TM_ERR_ARG, "bad precision");
  } else if (level == 1 || (level == 2 && h->three)) {
    const long nre = (long)nrhs * 2 * (level == 1 ? level1_cx(h) : level2_cx(h));
    if (prec == TM_F64)
      launch_convert<double, double>(static_cast<const double*>(field), natural, nre, h->st);
    else if (prec == TM_F32)
      launch_convert<float, double>(static_cast<const float*>(field), natural, nre, h->st);
    else
      raise(TM_ERR_ARG, "bad precision");
    CKL();
  } else {
    raise(TM_ERR_ARG, "level must be 0 or 1");
  }
  API_END
}

static void need_cycle_prec(tm_handle* h, int prec) {
  if (prec != h->p.cycle_prec) raise(TM_ERR_ARG, "prec must equal the handle's cycle_prec for this call");
  if (!h->setup_ok) raise(TM_ERR_STATE, "needs a setup");
}

tm_status tm_apply(tm_handle* h, int level, int prec, const void* in, void* out, int nrhs) {
  if (!h || !in || !out || in == out || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  if (nrhs > h->p.max_rhs) raise(TM_ERR_ARG, "nrhs > max_rhs");
  if (level == 0) {
    if (!h->gauge_ok) raise(TM_ERR_STATE, "no gauge field");
    if (prec == TM_F64)
      dslash<double>(h, static_cast<const double*>(in), static_cast<double*>(out), nullptr, nrhs);
    else if (prec == TM_F32)
      dslash<float>(h, static_cast<const float*>(in), static_cast<float*>(out), nullptr, nrhs);
    else if (prec == TM_F32X2 && h->gdf)
      dslash_df(h, static_cast<const float*>(in), static_cast<double*>(out), nrhs);
    else
      raise(TM_ERR_ARG, "bad precision");
  } else if (level == 1) {
    need_cycle_prec(h, prec);
    if (prec == TM_F64)
      launch_coarse_apply<double>(static_cast<const double*>(h->Dc), static_cast<const double*>(in),
                                  static_cast<double*>(out), h->gc, h->p.nv, mu_level1(h), nrhs, h->st);
    else
      launch_coarse_apply<float>(static_cast<const float*>(h->Dc), static_cast<const float*>(in),
                                 static_cast<float*>(out), h->gc, h->p.nv, mu_level1(h), nrhs, h->st);
    CKL();
  } else if (level == 2 && h->three) {
    need_cycle_prec(h, prec);
    if (prec == TM_F64)
      launch_coarse_apply<double>(static_cast<const double*>(h->Dc2), static_cast<const double*>(in),
                                  static_cast<double*>(out), h->gc2, h->p.nv2, mu_c(h), nrhs, h->st);
    else
      launch_coarse_apply<float>(static_cast<const float*>(h->Dc2), static_cast<const float*>(in),
                                 static_cast<float*>(out), h->gc2, h->p.nv2, mu_c(h), nrhs, h->st);
    CKL();
  } else {
    raise(TM_ERR_ARG, "level must be 0 or 1");
  }
  API_END
}

tm_status tm_sap(tm_handle* h, int prec, const void* b, void* x, int sweeps, int nrhs) {
  if (!h || !x || sweeps < 0 || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  if (!h->gauge_ok) raise(TM_ERR_STATE, "no gauge field");
  if (prec == TM_F64)
    sap_sweeps<double>(h, static_cast<const double*>(b), static_cast<double*>(x), sweeps, nrhs);
  else if (prec == TM_F32)
    sap_sweeps<float>(h, static_cast<const float*>(b), static_cast<float*>(x), sweeps, nrhs);
  else
    raise(TM_ERR_ARG, "bad precision");
  API_END
}

tm_status tm_restrict(tm_handle* h, int prec, const void* fine, void* coarse, int nrhs) {
  if (!h || !fine || !coarse || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  need_cycle_prec(h, prec);
  if (prec == TM_F64)
    launch_restrict<double>(static_cast<const double*>(h->P), static_cast<const double*>(fine),
                            static_cast<double*>(coarse), h->ag, nrhs, h->st);
  else
    launch_restrict<float>(static_cast<const float*>(h->P), static_cast<const float*>(fine),
                           static_cast<float*>(coarse), h->ag, nrhs, h->st, h->P16, h->p.transfer_prec);
  CKL();
  API_END
}

tm_status tm_prolong(tm_handle* h, int prec, const void* coarse, void* fine, int nrhs, int accumulate) {
  if (!h || !fine || !coarse || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  need_cycle_prec(h, prec);
  if (prec == TM_F64)
    launch_prolong<double>(static_cast<const double*>(h->P), static_cast<const double*>(coarse),
                           static_cast<double*>(fine), h->ag, nrhs, accumulate != 0, h->st);
  else
    launch_prolong<float>(static_cast<const float*>(h->P), static_cast<const float*>(coarse),
                          static_cast<float*>(fine), h->ag, nrhs, accumulate != 0, h->st, h->P16,
                          h->p.transfer_prec);
  CKL();
  API_END
}

tm_status tm_coarse_solve(tm_handle* h, int prec, const void* b, void* x, double tol, int maxit, int* iters) {
  if (!h || !b || !x || maxit < 1 || tol < 0) return TM_ERR_ARG;
  API_BEGIN
  need_cycle_prec(h, prec);
  std::vector<int> r;
  if (prec == TM_F64)
    r = coarse_solve<double>(h, coarsest_level(h), static_cast<const double*>(b), static_cast<double*>(x), 1, tol,
                             maxit);
  else
    r = coarse_solve<float>(h, coarsest_level(h), static_cast<const float*>(b), static_cast<float*>(x), 1, tol,
                            maxit);
  sync(h);
  if (iters) *iters = r[0];
  API_END
}

tm_status tm_kcycle(tm_handle* h, int prec, const void* v, void* z, int nrhs) {
  if (!h || !v || !z || v == z || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  need_cycle_prec(h, prec);
  if (prec == TM_F64)
    kcycle<double>(h, static_cast<const double*>(v), static_cast<double*>(z), nrhs);
  else
    kcycle<float>(h, static_cast<const float*>(v), static_cast<float*>(z), nrhs);
  API_END
}

tm_status tm_synchronize(tm_handle* h) {
  if (!h) return TM_ERR_ARG;
  API_BEGIN
  sync(h);
  check_flags(h);
  API_END
}

tm_status tm_export(tm_handle* h, int what, double* out, size_t bytes) {
  if (!h || !out) return TM_ERR_ARG;
  API_BEGIN
  const long V = h->g.V;
  const int nv = h->p.nv, n = h->n;
  std::vector<double> host;
  if (what == TM_EXPORT_P || what == TM_EXPORT_TV) {
    if (!h->setup_ok) raise(TM_ERR_STATE, "needs a setup");
    const size_t one = (size_t)V * 24;
    double* nat = W<double>(h, "exp_nat", one * nv);
    const void* src = what == TM_EXPORT_P ? h->P : h->tv;
    if (h->p.cycle_prec == TM_F64)
      unpack_fine<double>(h, src, nat, nv);
    else
      unpack_fine<float>(h, src, nat, nv);
    std::vector<double> tmp(one * nv);
    CK(cudaMemcpyAsync(tmp.data(), nat, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    sync(h);
    if (what == TM_EXPORT_TV) {
      host.swap(tmp);
    } else {
      host.assign(one * n, 0.0);
      for (int chi = 0; chi < 2; ++chi)
        for (int i = 0; i < nv; ++i) {
          double* col = host.data() + (size_t)(chi * nv + i) * one;
          const double* f = tmp.data() + (size_t)i * one;
          for (long s = 0; s < V; ++s)
            for (int k = 0; k < 12; ++k)
              if (k / 6 == chi) {
                col[(s * 12 + k) * 2] = f[(s * 12 + k) * 2];
                col[(s * 12 + k) * 2 + 1] = f[(s * 12 + k) * 2 + 1];
              }
        }
    }
  } else if (what == TM_EXPORT_DC) {
    if (!h->setup_ok) raise(TM_ERR_STATE, "needs a setup");
    const size_t cnt = (size_t)h->gc.V * 9 * n * n;
    std::vector<double> raw(cnt * 2);
    if (h->p.cycle_prec == TM_F64) {
      CK(cudaMemcpyAsync(raw.data(), h->Dc, cnt * 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      sync(h);
    } else {
      std::vector<float> rf(cnt * 2);
      CK(cudaMemcpyAsync(rf.data(), h->Dc, cnt * 2 * sizeof(float), cudaMemcpyDeviceToHost, h->st));
      sync(h);
      for (size_t i = 0; i < rf.size(); ++i) raw[i] = rf[i];
    }
    host.assign(cnt * 2, 0.0);
    for (size_t blk = 0; blk < (size_t)h->gc.V * 9; ++blk)
      for (int col = 0; col < n; ++col)
        for (int row = 0; row < n; ++row) {
          const size_t s = (blk * n + col) * n + row, d = (blk * n + row) * n + col;
          host[2 * d] = raw[2 * s];
          host[2 * d + 1] = raw[2 * s + 1];
        }
  } else if (what == TM_EXPORT_CLOVER) {
    if (!h->gauge_ok) raise(TM_ERR_STATE, "no gauge field");
    std::vector<double> raw((size_t)NR_CLOVER * V);
    CK(cudaMemcpyAsync(raw.data(), h->c64, raw.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    sync(h);
    host.assign((size_t)V * 2 * 36 * 2, 0.0);
    for (long s = 0; s < V; ++s)
      for (int hb = 0; hb < 2; ++hb) {
        double pk[36];
        for (int k = 0; k < 36; ++k) {
          const long r = 36L * hb + k;  // real index within the site
          pk[k] = raw[(size_t)(r / 4) * V * 4 + s * 4 + (r % 4)];
        }
        double* M = host.data() + ((size_t)s * 2 + hb) * 72;
        for (int i = 0; i < 6; ++i) {
          M[(i * 6 + i) * 2] = pk[i];
          M[(i * 6 + i) * 2 + 1] = 0;
        }
        int k = 6;
        for (int i = 0; i < 6; ++i)
          for (int j = i + 1; j < 6; ++j) {
            M[(i * 6 + j) * 2] = pk[k];
            M[(i * 6 + j) * 2 + 1] = pk[k + 1];
            M[(j * 6 + i) * 2] = pk[k];
            M[(j * 6 + i) * 2 + 1] = -pk[k + 1];
            k += 2;
          }
      }
  } else if ((what == TM_EXPORT_P2 || what == TM_EXPORT_TV1 || what == TM_EXPORT_DC2) && h->three) {
    if (!h->setup_ok) raise(TM_ERR_STATE, "needs a setup");
    const int nv1 = h->p.nv, n1 = h->n, nv2 = h->p.nv2, n2 = h->n2;
    const long V1 = h->gc.V;
    auto fetch = [&](const void* src, size_t cnt) {
      std::vector<double> raw(cnt);
      if (h->p.cycle_prec == TM_F64) {
        CK(cudaMemcpyAsync(raw.data(), src, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        sync(h);
      } else {
        std::vector<float> rf(cnt);
        CK(cudaMemcpyAsync(rf.data(), src, cnt * sizeof(float), cudaMemcpyDeviceToHost, h->st));
        sync(h);
        for (size_t i = 0; i < cnt; ++i) raw[i] = rf[i];
      }
      return raw;
    };
    if (what == TM_EXPORT_TV1) {
      host = fetch(h->tv1, (size_t)nv2 * V1 * n1 * 2);
    } else if (what == TM_EXPORT_P2) {
      std::vector<double> raw = fetch(h->P2, (size_t)nv2 * V1 * n1 * 2);
      host.assign((size_t)2 * nv2 * V1 * n1 * 2, 0.0);
      for (int chi = 0; chi < 2; ++chi)
        for (int j = 0; j < nv2; ++j)
          for (long x = 0; x < V1; ++x)
            for (int i = 0; i < nv1; ++i) {
              const size_t src = (((size_t)j * V1 + x) * n1 + chi * nv1 + i) * 2;
              const size_t dst = ((((size_t)chi * nv2 + j) * V1 + x) * n1 + chi * nv1 + i) * 2;
              host[dst] = raw[src];
              host[dst + 1] = raw[src + 1];
            }
    } else {
      const size_t cnt = (size_t)h->gc2.V * 9 * n2 * n2;
      std::vector<double> raw = fetch(h->Dc2, cnt * 2);
      host.assign(cnt * 2, 0.0);
      for (size_t blk = 0; blk < (size_t)h->gc2.V * 9; ++blk)
        for (int col = 0; col < n2; ++col)
          for (int row = 0; row < n2; ++row) {
            const size_t src = (blk * n2 + col) * n2 + row, dst = (blk * n2 + row) * n2 + col;
            host[2 * dst] = raw[2 * src];
            host[2 * dst + 1] = raw[2 * src + 1];
          }
    }
  } else {
    raise(TM_ERR_ARG, "unknown export");
  }
  if (bytes < host.size() * sizeof(double)) raise(TM_ERR_ARG, "export buffer too small");
  if (is_device_ptr(out)) {
    CK(cudaMemcpyAsync(out, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, h->st));
    sync(h);
  } else {
    std::memcpy(out, host.data(), host.size() * sizeof(double));
  }
  API_END
}

tm_status tm_schur(tm_handle* h, int prec, const void* ve, void* ye, int nrhs) {
  if (!h || !ve || !ye || ve == ye || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  need_cycle_prec(h, prec);
  const OELevel lv = coarsest_level(h);
  const long cv = 2L * lv.nhalf * lv.n;
  Prof pf(h, PK_COARSE_OE, nrhs, 2);
  if (prec == TM_F32) {
    float* uo = W<float>(h, "sch_uo", cv * nrhs);
    if (lv.tc && tc_supported(lv.oe.nv, nrhs, h->p.coarse_mma))
      launch_tc_schur(*lv.tc, lv.oe, static_cast<const float*>(ve), uo, static_cast<float*>(ye), lv.mu_c, nrhs, cv, cv,
                      cv, nullptr, h->p.coarse_mma, h->d_err, h->st,
                      (unsigned)h->p.tc_spin_limit);
    else
      launch_oe_schur_b<float>(static_cast<const float*>(lv.Dc), static_cast<const float*>(lv.Dinv),
                               static_cast<const float*>(ve), uo, static_cast<float*>(ye), lv.oe, lv.mu_c, nrhs, cv,
                               cv, cv, nullptr, h->st);
  } else {
    double* uo = W<double>(h, "sch_uo64", cv * nrhs);
    launch_oe_schur_b<double>(static_cast<const double*>(lv.Dc), static_cast<const double*>(lv.Dinv),
                              static_cast<const double*>(ve), uo, static_cast<double*>(ye), lv.oe, lv.mu_c, nrhs, cv,
                              cv, cv, nullptr, h->st);
  }
  CKL();
  check_flags(h);
  API_END
}

tm_status tm_nn_set_weights(tm_handle* h, const double* w) {
  if (!h || !w) return TM_ERR_ARG;
  API_BEGIN
  h->nn_w.resize(kNnWeights);
  for (int k = 0; k < kNnWeights; ++k) {
    h->nn_w[k] = std::complex<double>(w[2 * k], w[2 * k + 1]);
    if (!std::isfinite(w[2 * k]) || !std::isfinite(w[2 * k + 1])) raise(TM_ERR_NONFINITE, "non-finite weight");
  }
  h->adam_m.assign(2 * kNnWeights, 0.0);
  h->adam_v.assign(2 * kNnWeights, 0.0);
  h->adam_t = 0;
  nn_upload(h);
  API_END
}

tm_status tm_nn_get_weights(tm_handle* h, double* w) {
  if (!h || !w) return TM_ERR_ARG;
  API_BEGIN
  for (int k = 0; k < kNnWeights; ++k) {
    const std::complex<double> v = k < (int)h->nn_w.size() ? h->nn_w[k] : std::complex<double>(0, 0);
    w[2 * k] = v.real();
    w[2 * k + 1] = v.imag();
  }
  API_END
}

tm_status tm_nn_apply(tm_handle* h, int prec, const void* in, void* out, int nrhs, int accumulate) {
  if (!h || !in || !out || in == out || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  if (prec != TM_F32 && prec != TM_F16) raise(TM_ERR_ARG, "prec must be TM_F32 or TM_F16");
  nn_forward(h, static_cast<const float*>(in), static_cast<float*>(out), nrhs, accumulate != 0, prec == TM_F16);
  API_END
}

tm_status tm_nn_pairs(tm_handle* h, const double* e0, void* r, void* e, int npairs) {
  if (!h || !e0 || !r || !e || npairs < 1) return TM_ERR_ARG;
  API_BEGIN
  if (!h->setup_ok) raise(TM_ERR_STATE, "needs a setup");
  need_cycle_prec(h, TM_F32);
  const long fr = fine_reals(h);
  const double* src = stage_in(h, e0, (size_t)npairs * fr * sizeof(double), "stage_nn");
  float* ef = static_cast<float*>(e);
  float* rf = static_cast<float*>(r);
  const int chunk = std::max(1, std::min(npairs, h->p.max_rhs));
  float* r0 = W<float>(h, "nn_r0", (size_t)fr * chunk);
  float* z = W<float>(h, "nn_z", (size_t)fr * chunk);
  for (int p0 = 0; p0 < npairs; p0 += chunk) {
    const int nr = std::min(chunk, npairs - p0);
    float* ep = ef + (size_t)p0 * fr;
    {
      Prof pf(h, PK_OTHER, nr);
      launch_pack_spinor<float>(src + (size_t)p0 * fr, ep, h->g, nr, h->st);
      CKL();
    }
    dslash<float>(h, ep, r0, nullptr, nr);  // r0 = D e0
    kcycle<float>(h, r0, z, nr);             // z = B D e0
    {
      Prof pf(h, PK_OTHER, nr);
      launch_caxpby<float>(-1, 0, z, 1, 0, ep, (fr / 2) * nr, h->st);  // e = (1 - B D) e0
      CKL();
    }
    dslash<float>(h, ep, rf + (size_t)p0 * fr, nullptr, nr);  // r = D e
  }
  sync(h);
  API_END
}

tm_status tm_nn_grad(tm_handle* h, const void* r, const void* e, int npairs, double* grad, double* loss) {
  if (!h || !r || !e || npairs < 1) return TM_ERR_ARG;
  API_BEGIN
  std::vector<std::complex<double>> G;
  double esum = 0;
  const double l = nn_grad_sum(h, static_cast<const float*>(r), static_cast<const float*>(e), npairs, G, esum);
  if (!(esum > 0)) raise(TM_ERR_ARG, "all errors are zero");
  if (loss) *loss = l / esum;
  if (grad)
    for (int k = 0; k < kNnWeights; ++k) {
      grad[2 * k] = G[k].real() / esum;
      grad[2 * k + 1] = G[k].imag() / esum;
    }
  API_END
}

tm_status tm_nn_train(tm_handle* h, const void* r, const void* e, int npairs, int epochs, int batch, double lr,
                      double* losses) {
  if (!h || !r || !e || npairs < 1 || epochs < 1 || batch < 1 || !(lr > 0)) return TM_ERR_ARG;
  API_BEGIN
  need_nn(h);
  if (h->adam_m.size() != (size_t)2 * kNnWeights) {
    h->adam_m.assign(2 * kNnWeights, 0.0);
    h->adam_v.assign(2 * kNnWeights, 0.0);
    h->adam_t = 0;
  }
  const long fr = fine_reals(h);
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  for (int ep = 0; ep < epochs; ++ep) {
    double lsum = 0, esum_all = 0;
    for (int p0 = 0; p0 < npairs; p0 += batch) {
      const int nb = std::min(batch, npairs - p0);
      std::vector<std::complex<double>> G;
      double esum = 0;
      const double l = nn_grad_sum(h, static_cast<const float*>(r) + (size_t)p0 * fr,
                                   static_cast<const float*>(e) + (size_t)p0 * fr, nb, G, esum);
      lsum += l;
      esum_all += esum;
      if (!(esum > 0)) continue;
      ++h->adam_t;
      const double c1 = 1 - std::pow(b1, (double)h->adam_t), c2 = 1 - std::pow(b2, (double)h->adam_t);
      for (int k = 0; k < kNnWeights; ++k) {
        // steepest descent of the real loss in (Re W, Im W): 2 dL/d conj(W)
        const double gr[2] = {2 * G[k].real() / esum, 2 * G[k].imag() / esum};
        double upd[2];
        for (int c = 0; c < 2; ++c) {
          double& m = h->adam_m[2 * k + c];
          double& v = h->adam_v[2 * k + c];
          m = b1 * m + (1 - b1) * gr[c];
          v = b2 * v + (1 - b2) * gr[c] * gr[c];
          upd[c] = lr * (m / c1) / (std::sqrt(v / c2) + eps);
        }
        h->nn_w[k] -= std::complex<double>(upd[0], upd[1]);
      }
      nn_upload(h);
    }
    if (losses) losses[ep] = esum_all > 0 ? lsum / esum_all : 0.0;
  }
  API_END
}

static void need_three(tm_handle* h, int prec) {
  if (!h->three) raise(TM_ERR_ARG, "needs a three-level handle");
  need_cycle_prec(h, prec);
}

tm_status tm_sap1(tm_handle* h, int prec, const void* b, void* x, int sweeps, int nrhs) {
  if (!h || !x || sweeps < 0 || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  need_three(h, prec);
  if (prec == TM_F64)
    csap_sweeps<double>(h, static_cast<const double*>(b), static_cast<double*>(x), sweeps, nrhs);
  else
    csap_sweeps<float>(h, static_cast<const float*>(b), static_cast<float*>(x), sweeps, nrhs);
  API_END
}

tm_status tm_restrict1(tm_handle* h, int prec, const void* c1, void* c2, int nrhs) {
  if (!h || !c1 || !c2 || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  need_three(h, prec);
  if (prec == TM_F64)
    launch_crestrict<double>(static_cast<const double*>(h->P2), static_cast<const double*>(c1),
                             static_cast<double*>(c2), h->cag, nrhs, h->st);
  else
    launch_crestrict<float>(static_cast<const float*>(h->P2), static_cast<const float*>(c1), static_cast<float*>(c2),
                            h->cag, nrhs, h->st);
  CKL();
  API_END
}

tm_status tm_prolong1(tm_handle* h, int prec, const void* c2, void* c1, int nrhs, int accumulate) {
  if (!h || !c1 || !c2 || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  need_three(h, prec);
  if (prec == TM_F64)
    launch_cprolong<double>(static_cast<const double*>(h->P2), static_cast<const double*>(c2),
                            static_cast<double*>(c1), h->cag, nrhs, accumulate != 0, h->st);
  else
    launch_cprolong<float>(static_cast<const float*>(h->P2), static_cast<const float*>(c2), static_cast<float*>(c1),
                           h->cag, nrhs, accumulate != 0, h->st);
  CKL();
  API_END
}

tm_status tm_kcycle1(tm_handle* h, int prec, const void* v, void* z, int nrhs) {
  if (!h || !v || !z || v == z || nrhs < 1) return TM_ERR_ARG;
  API_BEGIN
  need_three(h, prec);
  if (prec == TM_F64)
    kcycle1<double>(h, static_cast<const double*>(v), static_cast<double*>(z), nrhs);
  else
    kcycle1<float>(h, static_cast<const float*>(v), static_cast<float*>(z), nrhs);
  API_END
}

tm_status tm_profile(tm_handle* h, int enable) {
  if (!h) return TM_ERR_ARG;
  API_BEGIN
  harvest(h, true);
  for (int k = 0; k < PK_N; ++k) {
    h->prof_launch[k] = h->prof_units[k] = 0;
    h->prof_ms[k] = 0;
  }
  h->prof = enable != 0;
  h->prof_mask = static_cast<unsigned>(enable);
  API_END
}

int tm_profile_kinds(void) { return PK_N; }

const char* tm_profile_name(int kind) { return (kind >= 0 && kind < PK_N) ? kProfNames[kind] : ""; }

tm_status tm_profile_read(tm_handle* h, long long* launches, long long* units, double* ms, int n) {
  if (!h || n < 0) return TM_ERR_ARG;
  API_BEGIN
  harvest(h, true);
  for (int k = 0; k < n && k < PK_N; ++k) {
    if (launches) launches[k] = h->prof_launch[k];
    if (units) units[k] = h->prof_units[k];
    if (ms) ms[k] = h->prof_ms[k];
  }
  API_END
}


size_t tm_workspace_bytes(const tm_params* p, int nrhs) {
  if (!p || nrhs < 1) return 0;
  try {
    validate(p);
  } catch (...) {
    return 0;
  }
  const MemPlan m = memory_plan(p, nrhs);
  return (size_t)(m.persistent + std::max(m.setup, m.solve));
}


tm_status tm_save_setup(tm_handle* h, const char* path) {
  if (!h || !path) return TM_ERR_ARG;
  API_BEGIN
  if (!h->setup_ok) raise(TM_ERR_STATE, "no setup to save");
  SetupHeader hd{};
  std::memcpy(hd.magic, kSetupMagic, 8);
  hd.version = 1;
  for (int d = 0; d < 4; ++d) {
    hd.L[d] = h->p.L[d];
    hd.agg[d] = h->p.agg[d];
    hd.agg2[d] = h->three ? h->p.agg2[d] : 0;
  }
  hd.nv = h->p.nv;
  hd.levels = h->p.levels;
  hd.nv2 = h->three ? h->p.nv2 : 0;
  hd.cycle_prec = h->p.cycle_prec;
  hd.m0 = h->p.m0;
  hd.c_sw = h->p.c_sw;
  hd.bc_t = h->p.bc_t;
  hd.rho = h->rho;
  void* ptr[6];
  size_t bytes[6];
  setup_arrays(h, ptr, bytes);
  for (int k = 0; k < 6; ++k) hd.nbytes[k] = (long long)bytes[k];
  const std::string tmp = std::string(path) + ".tmp";
  {
    FileCloser fc{std::fopen(tmp.c_str(), "wb")};
    if (!fc.f) raise(TM_ERR_ARG, "cannot write " + tmp);
    if (std::fwrite(&hd, sizeof hd, 1, fc.f) != 1) raise(TM_ERR_ARG, "short write to the setup file");
    sync(h);
    for (int k = 0; k < 6; ++k)
      if (bytes[k]) copy_through(h, fc.f, ptr[k], bytes[k], true);
    if (std::fflush(fc.f) != 0) raise(TM_ERR_ARG, "cannot flush the setup file");
  }
  if (std::rename(tmp.c_str(), path) != 0) raise(TM_ERR_ARG, std::string("cannot rename to ") + path);
  API_END
}

tm_status tm_load_setup(tm_handle* h, const char* path) {
  if (!h || !path) return TM_ERR_ARG;
  API_BEGIN
  if (!h->gauge_ok) raise(TM_ERR_STATE, "tm_load_gauge must come first");
  FileCloser fc{std::fopen(path, "rb")};
  if (!fc.f) raise(TM_ERR_ARG, std::string("cannot open ") + path);
  SetupHeader hd{};
  if (std::fread(&hd, sizeof hd, 1, fc.f) != 1 || std::memcmp(hd.magic, kSetupMagic, 8) != 0 || hd.version != 1)
    raise(TM_ERR_ARG, "not a setup file of this library");
  bool same = hd.nv == h->p.nv && hd.levels == h->p.levels && hd.cycle_prec == h->p.cycle_prec;
  for (int d = 0; d < 4; ++d) {
    same = same && hd.L[d] == h->p.L[d] && hd.agg[d] == h->p.agg[d];
    if (h->three) same = same && hd.agg2[d] == h->p.agg2[d];
  }
  if (h->three) same = same && hd.nv2 == h->p.nv2;
  if (!same) raise(TM_ERR_ARG, "the setup file was saved with other lattice, aggregate, N_v, level or precision");
  void* ptr[6];
  size_t bytes[6];
  setup_arrays(h, ptr, bytes);
  for (int k = 0; k < 6; ++k)
    if ((long long)bytes[k] != hd.nbytes[k]) raise(TM_ERR_ARG, "setup file sizes do not match the handle");
  h->setup_ok = false;
  sync(h);
  for (int k = 0; k < 6; ++k)
    if (bytes[k]) copy_through(h, fc.f, ptr[k], bytes[k], false);
  if (hd.rho != h->rho) {  // the saved D_c carries another odd-site shift: project again from P
    if (h->p.cycle_prec == TM_F64) {
      build_coarse<double>(h, false);
      if (h->three) build_level2<double>(h, false);
    } else {
      build_coarse<float>(h, false);
      if (h->three) build_level2<float>(h, false);
    }
    check_flags(h);
  } else if (h->p.cycle_prec == TM_F64) {
    rebuild_derived<double>(h);
  } else {
    rebuild_derived<float>(h);
  }
  h->setup_ok = true;
  h->tv_ok = true;
  API_END
}
}  // extern "C"

// ===========================================================================
// Allocation-free coarse solve.
//
// Some callers cannot call cudaMalloc at the moment they need a coarse
// solve: for example an application that hands all free device memory to its
// own memory pool up front (so a raw cudaMalloc would fail or fragment that
// pool), or a latency-critical loop that must not pay for cudaMalloc's
// implicit device synchronisation.  tm_coarse_solve_noalloc serves them: it
// runs the same odd-even GMRES as tm_coarse_solve, but every workspace
// (Krylov basis, work vectors, reduction partial sums, small results) is
// carved from one file-scope device array of fixed size that the library
// holds on every GPU that loads it, until the process exits.
// ===========================================================================
namespace {

constexpr size_t kNoAllocBytes = size_t(8) << 20;  // 8 MiB per device
constexpr int kNoAllocMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char tm_noalloc_scratch[kNoAllocBytes];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the array on the current device.  In host code the
// symbol's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
void* noalloc_scratch() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) raise(TM_ERR_ARG, "device index beyond the supported range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, tm_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      raise(TM_ERR_CUDA, std::string("cudaGetSymbolAddress of the allocation-free scratch failed: ") +
                             cudaGetErrorString(e));
    }
    g_noalloc_ptr[dev] = p;
  }
  return g_noalloc_ptr[dev];
}

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

// scratch bytes the solve needs: (m + 1) basis vectors, five work vectors,
// the reduction partials and the small result area
size_t noalloc_bytes(const tm_handle* h, int prec, int m) {
  const size_t vec = align256((size_t)h->nhalf * h->n * 2 * csize(prec));
  return (size_t)(m + 1) * vec + 5 * vec + align256((size_t)kScratchBlocks * kMaxDots * 2 * sizeof(double)) +
         align256((size_t)8 * kMaxDots * sizeof(double));
}

template <typename T>
int coarse_solve_noalloc(tm_handle* h, const T* b, T* x, double tol, int maxit) {
  using cd = std::complex<double>;
  const int m = h->p.coarse_restart;
  const long nc = (long)h->nhalf * h->n;  // complex numbers per parity vector
  const size_t vec = align256((size_t)2 * nc * sizeof(T));
  unsigned char* base = static_cast<unsigned char*>(noalloc_scratch());
  T* Vb = reinterpret_cast<T*>(base);
  unsigned char* q = base + (size_t)(m + 1) * vec;
  T* to = reinterpret_cast<T*>(q);
  T* bh = reinterpret_cast<T*>(q + vec);
  T* xe = reinterpret_cast<T*>(q + 2 * vec);
  T* uo = reinterpret_cast<T*>(q + 3 * vec);
  T* w = reinterpret_cast<T*>(q + 4 * vec);
  double* part = reinterpret_cast<double*>(q + 5 * vec);
  double* small = reinterpret_cast<double*>(q + 5 * vec + align256((size_t)kScratchBlocks * kMaxDots * 2 * 8));
  const long ld = vec / sizeof(T);
  const T* Dc = static_cast<const T*>(h->Dc);
  const T* Di = static_cast<const T*>(h->Dinv);
  const double mc = mu_c(h);
  // host-side Hessenberg state, per calling thread, sized for the largest restart
  thread_local cd H[kMaxDots * kMaxDots], g[kMaxDots], sn[kMaxDots], y[kMaxDots], col[kMaxDots];
  thread_local double cs[kMaxDots], hb[4 * kMaxDots + 2];
  auto S = [&](const T* ve, T* ye) {
    launch_oe_hop_inv<T>(Dc, Di, ve, uo, h->oe, h->st);
    CKL();
    launch_oe_even<T>(Dc, ve, uo, ye, h->oe, mc, 1, h->st);
    CKL();
  };
  auto norm = [&](const T* v) {
    launch_norm2<T>(v, nc, 1, small, part, kScratchBlocks, h->st);
    CKL();
    CK(cudaMemcpyAsync(hb, small, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return std::sqrt(hb[0]);
  };
  launch_oe_inv_odd<T>(Di, b, to, h->oe, h->st);
  CKL();
  launch_oe_rhs<T>(Dc, b, to, bh, h->oe, h->st);
  CKL();
  launch_zero<T>(xe, 2 * nc, h->st);  // the iterate must start at zero; the array keeps old contents
  CKL();
  const double bnorm = norm(bh);
  if (!std::isfinite(bnorm)) raise(TM_ERR_NONFINITE, "non-finite right-hand side");
  int iters = 0;
  if (bnorm > 0) {
    CK(cudaMemcpyAsync(Vb, bh, 2 * nc * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
    double beta = bnorm;
    while (beta > tol * bnorm && iters < maxit) {
      launch_caxpby<T>(1.0 / beta, 0, Vb, 0, 0, Vb, nc, h->st);
      CKL();
      for (int j = 0; j <= m; ++j) g[j] = 0;
      g[0] = beta;
      int k = 0;
      while (k < m) {
        S(Vb + (long)k * ld, w);
        launch_multidot<T>(Vb, ld, k + 1, w, nc, small, part, kScratchBlocks, h->st);
        CKL();
        launch_multi_caxpy<T>(Vb, ld, k + 1, small, 1.0, w, nc, h->st);
        CKL();
        launch_multidot<T>(Vb, ld, k + 1, w, nc, small + 2 * kMaxDots, part, kScratchBlocks, h->st);
        CKL();
        launch_multi_caxpy<T>(Vb, ld, k + 1, small + 2 * kMaxDots, 1.0, w, nc, h->st);
        CKL();
        launch_norm2<T>(w, nc, 1, small + 4 * kMaxDots, part, kScratchBlocks, h->st);
        CKL();
        CK(cudaMemcpyAsync(Vb + (long)(k + 1) * ld, w, 2 * nc * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
        launch_scale<T>(Vb + (long)(k + 1) * ld, nc, 1, small + 4 * kMaxDots, true, h->st);
        CKL();
        CK(cudaMemcpyAsync(hb, small, (4 * kMaxDots + 1) * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        const double hn = std::sqrt(hb[4 * kMaxDots]);
        if (!std::isfinite(hn)) raise(TM_ERR_NONFINITE, "non-finite Arnoldi vector");
        for (int j = 0; j <= m; ++j) col[j] = 0;
        for (int j = 0; j <= k; ++j)
          col[j] = cd(hb[2 * j] + hb[2 * kMaxDots + 2 * j], hb[2 * j + 1] + hb[2 * kMaxDots + 2 * j + 1]);
        col[k + 1] = hn;
        for (int j = 0; j < k; ++j) {
          const cd t = cs[j] * col[j] + sn[j] * col[j + 1];
          col[j + 1] = -std::conj(sn[j]) * col[j] + cs[j] * col[j + 1];
          col[j] = t;
        }
        double c;
        cd s, rho;
        givens(col[k], hn, c, s, rho);
        cs[k] = c;
        sn[k] = s;
        col[k] = rho;
        col[k + 1] = 0;
        for (int j = 0; j <= m; ++j) H[(size_t)j * m + k] = col[j];
        g[k + 1] = -std::conj(s) * g[k];
        g[k] = c * g[k];
        ++iters;
        ++k;
        if (hn == 0 || std::abs(g[k]) <= tol * bnorm || iters >= maxit) break;
      }
      for (int i = k - 1; i >= 0; --i) {
        cd acc = g[i];
        for (int j = i + 1; j < k; ++j) acc -= H[(size_t)i * m + j] * y[j];
        y[i] = acc / H[(size_t)i * m + i];
      }
      for (int i = 0; i < k; ++i) {
        hb[2 * i] = y[i].real();
        hb[2 * i + 1] = y[i].imag();
      }
      double* dy = small + 6 * kMaxDots;
      CK(cudaMemcpyAsync(dy, hb, 2 * k * sizeof(double), cudaMemcpyHostToDevice, h->st));
      launch_lincomb<T, T>(Vb, ld, k, dy, xe, nc, h->st);
      CKL();
      // true residual of the reduced system
      S(xe, w);
      CK(cudaMemcpyAsync(Vb, bh, 2 * nc * sizeof(T), cudaMemcpyDeviceToDevice, h->st));
      launch_caxpby<T>(-1, 0, w, 1, 0, Vb, nc, h->st);
      CKL();
      beta = norm(Vb);
    }
  }
  launch_oe_reconstruct<T>(Dc, Di, b, xe, x, h->oe, h->st);
  CKL();
  CK(cudaStreamSynchronize(h->st));
  return iters;
}

}  // namespace

extern "C" tm_status tm_coarse_solve_noalloc(tm_handle* h, int prec, const void* b, void* x, double tol, int maxit,
                                             int* iters) {
  if (!h || !b || !x || maxit < 1 || tol < 0) return TM_ERR_ARG;
  API_BEGIN
  if (prec != TM_F64 && prec != TM_F32) raise(TM_ERR_ARG, "bad precision");
  if (h->three) raise(TM_ERR_ARG, "tm_coarse_solve_noalloc serves two-level handles");
  const size_t need = noalloc_bytes(h, prec, h->p.coarse_restart);
  if (need > kNoAllocBytes)
    raise(TM_ERR_ARG, "tm_coarse_solve_noalloc: this coarse system needs " + std::to_string(need) +
                          " bytes of scratch, more than the fixed " + std::to_string(kNoAllocBytes) +
                          " bytes (8 MiB) the allocation-free entry point holds; use tm_coarse_solve");
  need_cycle_prec(h, prec);
  int it;
  if (prec == TM_F64)
    it = coarse_solve_noalloc<double>(h, static_cast<const double*>(b), static_cast<double*>(x), tol, maxit);
  else
    it = coarse_solve_noalloc<float>(h, static_cast<const float*>(b), static_cast<float*>(x), tol, maxit);
  if (iters) *iters = it;
  API_END
}
