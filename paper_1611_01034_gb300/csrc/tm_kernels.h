// Host-side launchers of the library's kernels (internal, C++ linkage).
// Every launcher enqueues on the given stream and returns immediately.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "tm_internal.cuh"

namespace tmamg {

// ---- fine fields (dirac.cu) ----------------------------------------------
// natural layout: [rhs][V][4 spin][3 colour] complex128, interleaved re/im
template <typename T>
void launch_pack_spinor(const double* nat, T* field, const Lat& g, int nrhs, cudaStream_t st);
template <typename T>
void launch_unpack_spinor(const T* field, double* nat, const Lat& g, int nrhs, cudaStream_t st);
// natural gauge [V][4][3][3] complex128 -> packed FP64 and FP32 links, SU(3) check
void launch_pack_gauge(const double* nat, double* g64, float* g32, const Lat& g, double tol,
                       int* err, cudaStream_t st);
// clover blocks (m0 + 4 included, mu-free) from the natural gauge field
void launch_clover(const double* nat, double* c64, float* c32, const Lat& g, double m0, double c_sw,
                   cudaStream_t st);
// zero the sites of the given parity of nrhs natural spinor arrays
void launch_zero_parity_nat(double* nat, const Lat& g, int parity, int nrhs, cudaStream_t st);
// out = Gamma5 in on natural spinor arrays of nsites sites (in may equal out)
void launch_gamma5_nat(const double* in, double* out, long nsites, cudaStream_t st);
// out = D(mu) in (res == nullptr) or out = b - D(mu) in; odd sites carry mu + rho
template <typename T>
void launch_dslash(const T* gauge, const T* clover, const T* in, T* out, const T* b, const Lat& g,
                   double mu, double bc_t, int nrhs, cudaStream_t st, double rho = 0.0);

// ---- FP32-pair D(mu) (dirac_df.cu) -------------------------------------------
// links as [4][9][V] float4 (re.h, im.h, re.l, im.l) of entry 3a + b; clover as
// [36][V] float4 (r[2j].h, r[2j+1].h, r[2j].l, r[2j+1].l) of the packed 72 reals
void launch_pack_gauge_df(const double* nat, void* gdf, const Lat& g, cudaStream_t st);
void launch_clover_df(const double* c64, void* cdf, const Lat& g, cudaStream_t st);
// out (FP64 field) = D(mu) in (FP32 field) to about 2^-46 relative, FP32 pairs
void launch_dslash_df(const void* gdf, const void* cdf, const float* in, double* out, const Lat& g, double mu,
                      double bc_t, int nrhs, cudaStream_t st, double rho = 0.0);
// r (FP64) = b - D(mu) x for FP64 x and b, in FP32-pair arithmetic (x split into pairs;
// about 2^-46 relative to |D| |x|): restart residuals of the outer FGMRES
void launch_residual_df(const void* gdf, const void* cdf, const double* x, const double* b, double* r, const Lat& g,
                        double mu, double bc_t, int nrhs, cudaStream_t st, double rho = 0.0);

// ---- SAP (sap.cu) ------------------------------------------------------------
struct SapGeom {
  Lat g;
  int blk[4];   // block dims
  int nb[4];    // blocks per dimension (all even)
  int bsites;   // sites per block
};
// one colour of one sweep on D x = b (b may be null: b = 0)
template <typename T>
void launch_sap_colour(const T* gauge, const T* clover, const T* b, T* x, const SapGeom& sg,
                       double mu, double bc_t, int n_mr, int colour, int nrhs, cudaStream_t st, double rho = 0.0);

// the same with the block solves on the odd-even Schur complement (Sec. 3);
// all block dims even; dinv from launch_clover_inverse
// gauge, clover, dinv stored as T, or (T = float) in 16 bits when s16 = ST_F16 / ST_BF16
template <typename T>
void launch_sap_oe_colour(const void* gauge, const void* clover, const void* dinv, const T* b, T* x,
                          const SapGeom& sg, double mu, double bc_t, int n_mr, int colour, int nrhs, cudaStream_t st,
                          double rho = 0.0, int s16 = 0);
// dinv [12 rows x 6 complex chunks][V/2] = (A(x) + i mu gamma5)^-1 of the two
// chiral blocks at every odd site (compact index s >> 1; X even); mu = the
// odd sites' twisted mass
template <typename T>
void launch_clover_inverse(const double* c64, T* dinv, const Lat& g, double mu, int* err, cudaStream_t st,
                           int parity = 1);  // sites of this parity, compact index s >> 1

// ---- aggregation and coarse operator (coarse.cu) ---------------------------
// tile shape of the coarse-operator build kernel (0 = default heuristic)
struct BuildShape {
  int ts = 0, ktc = 0;
};

struct AggGeom {
  Lat g;        // fine lattice
  Lat gc;       // coarse lattice
  int agg[4];
  int asites;   // sites per aggregate
  int nv;       // test vectors
};
// P <- per (aggregate, chirality) CGS2 orthonormalisation of the Nv fields in P (in place)
template <typename T>
void launch_orthonormalise(T* P, const AggGeom& ag, int* err, cudaStream_t st);
// coarse[rhs][Vc][2Nv] = P^dagger fine
template <typename T>
void launch_restrict(const T* P, const T* fine, T* coarse, const AggGeom& ag, int nrhs, cudaStream_t st,
                     const void* P16 = nullptr, int p16 = 0);  // P16: 16-bit copy of P (ST_F16 / ST_BF16)
// fine = (accumulate ? fine : 0) + P coarse
template <typename T>
void launch_prolong(const T* P, const T* coarse, T* fine, const AggGeom& ag, int nrhs, bool accumulate,
                    cudaStream_t st, const void* P16 = nullptr, int p16 = 0);
// 16-bit copy (kind ST_F16 or ST_BF16) of n_cx FP32 complex numbers, element order kept
void launch_to16(const float* in, void* out, long n_cx, int kind, cudaStream_t st);
// Dc blocks [Vc][9][2Nv col][2Nv row] = local Galerkin projection (mu-free)
template <typename T>
void launch_coarse_build(const T* gauge, const T* clover, const T* P, T* Dc, const AggGeom& ag,
                         double bc_t, cudaStream_t st, BuildShape shape = BuildShape{}, double rho = 0.0);
// tile shape of the build: ts fine sites staged per tile, ktc columns per
// register tile (0 = the default heuristic); the candidates an autotuner may try
BuildShape coarse_build_default(int nv, size_t real_bytes);
std::vector<BuildShape> coarse_build_candidates(int nv, size_t real_bytes);
// adds to *count the number of 32-bit words in which a and b differ
void launch_count_mismatch(const void* a, const void* b, long words, unsigned long long* count, cudaStream_t st);
// y = D_c(mu_c) v on the full coarse lattice
template <typename T>
void launch_coarse_apply(const T* Dc, const T* v, T* y, const Lat& gc, int nv, double mu_c, int nrhs,
                         cudaStream_t st, const void* Dc16 = nullptr, int kind16 = 2);  // Dc16: 16-bit block copy

// odd-even on the coarse lattice
struct OEGeom {
  Lat gc;
  int nv;
  int nhalf;            // Vc / 2
  const int* even_site; // compact even index -> site
  const int* odd_site;  // compact odd index -> site
  const int* cidx;      // site -> compact index within its parity
};
// Dinv[odd k] = (self block + i mu_c Gamma5_c)^-1, Gauss-Jordan with partial pivoting
template <typename T>
void launch_oe_invert(const T* Dc, T* Dinv, const OEGeom& oe, double mu_c, int* err, cudaStream_t st);
// u_o = Dinv (D_oe v_e)   (v_e compact even, u_o compact odd)
template <typename T>
void launch_oe_hop_inv(const T* Dc, const T* Dinv, const T* ve, T* uo, const OEGeom& oe, cudaStream_t st);
// y_e = alpha_d (self + i mu_c G5c) v_e - D_eo u_o  (alpha_d in {0,1})
template <typename T>
void launch_oe_even(const T* Dc, const T* ve, const T* uo, T* ye, const OEGeom& oe, double mu_c,
                    int diag, cudaStream_t st);
// t_o = Dinv b_o   (b full coarse vector; reads its odd sites)
template <typename T>
void launch_oe_inv_odd(const T* Dinv, const T* b, T* to, const OEGeom& oe, cudaStream_t st);
// bhat_e = b_e - D_eo t_o
template <typename T>
void launch_oe_rhs(const T* Dc, const T* b, const T* to, T* bh, const OEGeom& oe, cudaStream_t st);
// x(full) from x_e: x_o = Dinv (b_o - D_oe x_e)
template <typename T>
void launch_oe_reconstruct(const T* Dc, const T* Dinv, const T* b, const T* xe, T* x, const OEGeom& oe,
                           cudaStream_t st);

// ---- first coarse level of a three-level hierarchy (coarse2.cu) -------------
struct CSapGeom {
  Lat g;       // level-1 lattice
  int blk[4];  // SAP block dims (coarse sites); block counts per dimension even
  int nb[4];
  int bsites;
  int n;       // components per level-1 site (2 Nv1)
};
struct CAggGeom {
  Lat g1, g2;  // level-1 and level-2 lattices
  int agg[4];
  int asites;
  int nv1, nv2;
};
// one colour of SAP on D_c1(mu) x = b (b may be null), nrhs level-1 vectors;
// with Dc_half (16-bit copy of the FP32 blocks, half_kind ST_F16 or ST_BF16)
// the blocks are read from it
template <typename T>
void launch_csap_colour(const T* Dc, const T* b, T* x, const CSapGeom& sg, double mu, int n_mr, int colour,
                        int nrhs, cudaStream_t st, const void* Dc_half = nullptr, int half_kind = 2);
// P2 <- per (aggregate, chirality) CGS2 of the Nv2 level-1 fields in P2
template <typename T>
void launch_corth(T* P2, const CAggGeom& ag, int* err, cudaStream_t st);
template <typename T>
void launch_crestrict(const T* P2, const T* r1, T* r2, const CAggGeom& ag, int nrhs, cudaStream_t st);
template <typename T>
void launch_cprolong(const T* P2, const T* e2, T* x1, const CAggGeom& ag, int nrhs, bool accumulate,
                     cudaStream_t st);
// D_c2 blocks (mu-free) = P2^dagger D_c1(0) P2
template <typename T>
void launch_cbuild(const T* Dc1, const T* P2, T* Dc2, const CAggGeom& ag, cudaStream_t st);

// batched odd-even pieces: nrhs right-hand sides at per-rhs strides (reals);
// `active` (device, may be null) masks right-hand sides that are finished
// ye = S ve with S = D_ee - D_eo D_oo^-1 D_oe (uo: odd-site work vectors)
template <typename T>
void launch_oe_schur_b(const T* Dc, const T* Dinv, const T* ve, T* uo, T* ye, const OEGeom& oe, double mu_c,
                       int nrhs, long vstr, long ustr, long ystr, const int* active, cudaStream_t st);
// to = Dinv b_o, bh = b_e - D_eo to  (b full vectors at stride bstr; to, bh compact at cstr)
template <typename T>
void launch_oe_prepare_b(const T* Dc, const T* Dinv, const T* b, T* to, T* bh, const OEGeom& oe, int nrhs,
                         long bstr, long cstr, cudaStream_t st);
// x = [xe ; Dinv (b_o - D_oe xe)]  (b, x full at bstr; xe compact at estr)
template <typename T>
void launch_oe_reconstruct_b(const T* Dc, const T* Dinv, const T* b, const T* xe, T* x, const OEGeom& oe, int nrhs,
                             long bstr, long estr, cudaStream_t st);

// ---- odd-even Schur complement on the tensor cores (coarse_tc.cu) ------------
// Pre-tiled FP32 operator blocks (TF32-rounded, K-major UMMA layout with 64-byte
// swizzle: kp = n padded to 16 columns, mp = 2n padded to 8 rows) for the
// odd-even coarse solve.
struct TcGeom {
  int kp = 0, mp = 0;
  float* even = nullptr;     // [nhalf][9] self block and hops of even sites
  float* even_lo = nullptr;  // residual parts for 3xTF32 (or null)
  float* odd = nullptr;      // [nhalf][8] D_oo^-1 B_t of odd sites
  float* odd_lo = nullptr;
  int* nbr_e = nullptr;      // [nhalf][9]
  int* nbr_o = nullptr;      // [nhalf][8]
};
constexpr int kTcSmemBytes = 200 * 1024;
// can the tensor-core path take nrhs right-hand sides with split products (1..3)?
bool tc_supported(int nv, int nrhs, int split);
// neighbour tables, even tiles and odd tiles (after D_c and D_oo^-1 exist)
void tc_build(const float* Dc, const float* Dinv, const OEGeom& oe, const TcGeom& tg, cudaStream_t st);
// odd tiles only (they carry D_oo^-1, so they follow mu)
void tc_build_odd(const float* Dc, const float* Dinv, const OEGeom& oe, const TcGeom& tg, cudaStream_t st);
// ye = S ve for nrhs compact even vectors (uo: odd work vectors); `split` TF32 products;
// `spin` polls per pipeline wait before the kernel gives up (0: the default limit)
void launch_tc_schur(const TcGeom& tg, const OEGeom& oe, const float* ve, float* uo, float* ye, double mu_c,
                     int nrhs, long vstr, long ustr, long ystr, const int* active, int split, int* err,
                     cudaStream_t st, unsigned spin = 0);

// ---- learned gauge-covariant layer (nn.cu) ------------------------------------
// weights: complex float2 [Cout][Cin][9 directions][4][4]; hidden fields
// [rhs][8][V][12 complex] in FP32 or FP16; fine fields in the chunked layout
constexpr int kNnHidden = 8;
constexpr int kNnWeights = 2 * kNnHidden * 9 * 16;  // complex weights of both layers
long nn_wgrad_partial_floats2(const Lat& g, int nrhs);
void nn_layer1(const float* r, void* hid, bool half, const float* gauge, const float2* W1, const Lat& g, double bc,
               int nrhs, cudaStream_t st);
void nn_layer2(const void* hid, bool half, float* y, bool accumulate, const float* gauge, const float2* W2,
               const Lat& g, double bc, int nrhs, cudaStream_t st);
// gh = L2^dagger gy (W2adj: conjugate-transposed weights with reversed directions)
void nn_layer2_adjoint(const float* gy, float* gh, const float* gauge, const float2* W2adj, const Lat& g, double bc,
                       int nrhs, cudaStream_t st);
// summed over the nrhs samples: out[o][i][d][s][t] = sum_x g_o(x)[s] conj(T_d psi_i(x)[t]) (FP64)
void nn_grad_w2(const float* hid, const float* gy, const float* gauge, const Lat& g, double bc, int nrhs,
                float2* partial, double2* out, cudaStream_t st);
void nn_grad_w1(const float* r, const float* gh, const float* gauge, const Lat& g, double bc, int nrhs,
                float2* partial, double2* out, cudaStream_t st);

// ---- level-1 vectors (blas.cu) ----------------------------------------------
// all BLAS works on flat arrays of n complex numbers stored as (re, im) pairs
template <typename Ti, typename To>
void launch_convert(const Ti* in, To* out, long n_reals, cudaStream_t st);
template <typename T>
void launch_zero(T* x, long n_reals, cudaStream_t st);
// y = a x + b y  (complex a, b as double pairs)
template <typename T>
void launch_caxpby(double ar, double ai, const T* x, double br, double bi, T* y, long ncx, cudaStream_t st);
// out[j] = sum conj(X_j) y for j < k; X_j = X + j * ldx (reals); results as double2 into dev_out
template <typename T>
void launch_multidot(const T* X, long ldx, int k, const T* y, long ncx, double* dev_out, double* scratch,
                     int nscratch_blocks, cudaStream_t st);
// y -= sum_j c_j X_j   (c on device, double2[k])
template <typename T>
void launch_multi_caxpy(const T* X, long ldx, int k, const double* c, double sign, T* y, long ncx,
                        cudaStream_t st);
// y += sum_j c_j X_j with X of type Tx and y of type Ty (c on device)
template <typename Tx, typename Ty>
void launch_lincomb(const Tx* X, long ldx, int k, const double* c, Ty* y, long ncx, cudaStream_t st);
// dev_out[r] = ||x_r||^2 for nrhs vectors of ncx complex each
template <typename T>
void launch_norm2(const T* x, long ncx, int nrhs, double* dev_out, double* scratch, int nscratch_blocks,
                  cudaStream_t st);
// x_r *= s_r (s on device, double[nrhs], scale = 1 / sqrt(s_r) if inv_sqrt)
template <typename T>
void launch_scale(T* x, long ncx, int nrhs, const double* s, bool inv_sqrt, cudaStream_t st);

// batched variants: right-hand side r uses X + r * xstr, y + r * ystr, ...;
// inactive right-hand sides (active[r] == 0, active may be null) are skipped.
// out[r * ostr + 2 j] (re, im) = sum conj(X_rj) y_r, j < k
template <typename T>
void launch_multidot_b(const T* X, long xstr, long ldx, int k, const T* y, long ystr, long ncx, double* out,
                       long ostr, double* scratch, int nrhs, const int* active, cudaStream_t st);
// y_r -= sum_j c[r * cstr + 2 j] X_rj
template <typename T>
void launch_multi_caxpy_b(const T* X, long xstr, long ldx, int k, const double* c, long cstr, T* y, long ystr,
                          long ncx, int nrhs, const int* active, cudaStream_t st);
// y_r += sum_{j < min(k, active[r])} c[r * cstr + 2 j] X_rj  (active[r]: term count, 0 = skip)
template <typename Tx, typename Ty>
void launch_lincomb_b(const Tx* X, long xstr, long ldx, int k, const double* c, long cstr, Ty* y, long ystr,
                      long ncx, int nrhs, const int* active, cudaStream_t st);
// out[r] = ||y_r||^2
template <typename T>
void launch_norm2_b(const T* y, long ystr, long ncx, double* out, double* scratch, int nrhs, const int* active,
                    cudaStream_t st);
// dst_r = src_r / sqrt(s[r]) (0 if s[r] <= 0), or dst_r = src_r when s is null
template <typename T>
void launch_scale_copy_b(const T* src, long sstr, T* dst, long dstr, const double* s, long ncx, int nrhs,
                         const int* active, cudaStream_t st);
// y_r = x_r - y_r
template <typename T>
void launch_sub_b(const T* x, long xstr, T* y, long ystr, long ncx, int nrhs, const int* active, cudaStream_t st);
// scratch doubles that launch_multidot_b / launch_norm2_b need
long multidot_scratch_doubles(long ncx, int k, int nrhs);
// device state of fixed-step GMRES cycles (gmres_dev.cu), per right-hand side:
// H [m + 1][m], g [m + 1], rotations cs [m] / sn [m], |b|, steps taken, stop flag
struct GmresDev {
  cx<double>* H;
  cx<double>* g;
  double* cs;
  cx<double>* sn;
  double* bnorm;
  int* kk;
  int* done;
  int m;
};
void launch_gmres_init(const GmresDev& st, const double* nrm, int nrhs, cudaStream_t s);
void launch_gmres_step(const GmresDev& st, const double* dd, long ds, const double* nrm, int k, int nrhs, double tol,
                       cudaStream_t s);
void launch_gmres_solve(const GmresDev& st, double* dd, long ds, int kmax, int nrhs, cudaStream_t s);
// odd-even reduced operator and CG pieces of the oeCG solver (oecg.cu); half
// fields hold one parity at compact index s >> 1
template <typename T>
void launch_oe_apply(const T* gauge, const T* clover, const T* dinv, const T* hin, const T* din, T* out, const Lat& g,
                     int parity, double c_hop, double mu, double bc_t, int g5, int dag, int mode, cudaStream_t st);
template <typename T>
void launch_parity_copy(const T* src, T* dst, const Lat& g, int parity, bool to_full, cudaStream_t st);
template <typename T>
void launch_cg_xr(T* x, T* r, const T* p, const T* q, const double* sc, int ig, int iq, long n_reals,
                  cudaStream_t st);
template <typename T>
void launch_cg_p(T* p, const T* s, const double* sc, int inew, int iold, long n_reals, cudaStream_t st);
void launch_acc_f32(const float* e, double* x, long n_reals, cudaStream_t st);  // x += e
int dot_grid_for(long ncx);  // partial-sum CTAs per right-hand side of the batched reductions
// Arnoldi steps of the FP64 FGMRES in FP32-pair arithmetic (blas_pair.cu); the
// reductions write FP64 results like launch_multidot_b / launch_norm2_b
void launch_pdot_b(const double* X, long xstr, long ldx, int k, const double* y, long ystr, long ncx, double* out,
                   long ostr, double* scratch, int nrhs, const int* active, cudaStream_t st);
int launch_pcaxpy_dot_b(const double* X, long xstr, long ldx, int k, const double* c, long cstr, double* y, long ystr,
                        long ncx, double* out, long ostr, double* scratch, int nrhs, const int* active,
                        cudaStream_t st);  // returns the launches made
void launch_pcaxpy_norm_b(const double* X, long xstr, long ldx, int k, const double* c, long cstr, double* y,
                          long ystr, long ncx, double* nrm, double* scratch, int nrhs, const int* active,
                          cudaStream_t st);
void launch_plincomb_b(const float* Z, long zstr, long ldz, int k, const double* c, long cstr, double* x, long xstr,
                       long ncx, int nrhs, const int* active, cudaStream_t st);
// fused pairs: the partial sums of a multidot / norm go straight into the next
// step, which reduces them itself (the final values are also written to c / nrm):
//   multidot partials -> y_r -= sum_j c_rj X_rj;   norm partials -> dst_r = src_r / ||src_r||
template <typename T>
void launch_multidot_b_partials(const T* X, long xstr, long ldx, int k, const T* y, long ystr, long ncx,
                                double* scratch, int nrhs, const int* active, cudaStream_t st);
template <typename T>
void launch_multi_caxpy_bp(const T* X, long xstr, long ldx, int k, const double* part, long ncx_dot, double* c,
                           long cstr, T* y, long ystr, long ncx, int nrhs, const int* active, cudaStream_t st);
template <typename T>
void launch_norm2_b_partials(const T* y, long ystr, long ncx, double* scratch, int nrhs, const int* active,
                             cudaStream_t st);
template <typename T>
void launch_scale_copy_bp(const T* src, long sstr, T* dst, long dstr, const double* part, double* nrm, long ncx,
                          int nrhs, const int* active, cudaStream_t st);

constexpr int kReduceBlocks = 304;  // 2 x 152 SMs

}  // namespace tmamg
