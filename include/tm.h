/*
 * tm.h -- C ABI of the GB300 twisted-mass DD-alphaAMG library.
 *
 * The library solves D(mu) x = b for the twisted-mass Wilson-clover operator
 * D(mu) = D_W + i mu Gamma5 (Bacchio et al., "DDalphaAMG for Twisted Mass
 * Fermions", Sec. 1) with flexible GMRES preconditioned at every step by the
 * multigrid error propagation of eq. (1):
 *     eps <- (I - M D)^k (I - P D_c^-1 P^dagger D) (I - M D)^j eps,
 * M the SAP smoother, P the Gamma5-compatible aggregation interpolation,
 * D_c = P^dagger D_W P + i delta mu Gamma5_c the coarse operator with the
 * coarse twisted mass shifted by delta >= 1 (Sec. 1).  Everything runs on one
 * GPU in hand-written sm_103a kernels; there is no CPU fallback.
 *
 * Conventions (Sec. 2 of the paper fixes gamma5 = diag(-1,-1,+1,+1) and the
 * lexicographic site order TZYX; everything else below is this library's):
 *   - Lattice extents L = {T, Z, Y, X}, X fastest.  Direction index 0..3 is
 *     T, Z, Y, X and carries gamma_4, gamma_3, gamma_2, gamma_1 of the chiral
 *     basis gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = [[0,-1],[-1,0]].
 *   - D_W has (m0 + 4) plus the clover term c_sw on the diagonal and the hops
 *     -1/2 [(1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu)];
 *     hops across the T boundary are multiplied by bc_t.
 *   - "Natural" arrays are complex128 with interleaved re/im:
 *       gauge  [T][Z][Y][X][mu=4][3][3]   (links U_mu(x), rows x columns)
 *       spinor [nrhs][T][Z][Y][X][spin 4][colour 3]
 *       coarse [nrhs][Tc][Zc][Yc][Xc][2 Nv]   (chirality -1 first, then +1)
 *   - "Fields" are the library's internal device layout (tm_field_bytes).
 *
 * Ownership: the caller owns every buffer it passes; the handle owns its
 * internal storage (packed gauge, clover, P, D_c, workspaces) and frees it in
 * tm_destroy.  Pointers marked "host or device" may be either; the library
 * copies host data itself.  Pointers marked "device" must be device memory.
 *
 * Errors: no call aborts or throws; each returns a tm_status and keeps a
 * message readable with tm_last_error().  Kernels never trap: device-side
 * checks set a flag that the host turns into a status.
 *
 * Streams: every call enqueues on the stream given to tm_create.  Calls that
 * return results to the host (tm_solve, tm_setup, tm_load_gauge,
 * tm_coarse_solve, tm_export) synchronise that stream before returning;
 * tm_apply, tm_sap, tm_restrict, tm_prolong, tm_kcycle, tm_pack and
 * tm_unpack are asynchronous.
 */
#ifndef TM_H
#define TM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tm_handle tm_handle;

typedef enum {
  TM_OK = 0,
  TM_ERR_ARG = -1,           /* invalid argument or parameter combination */
  TM_ERR_CUDA = -2,          /* a CUDA runtime call or kernel launch failed */
  TM_ERR_OOM = -3,           /* device allocation failed */
  TM_ERR_NOT_CONVERGED = -4, /* solve hit maxit; x holds the best iterate */
  TM_ERR_TIMEOUT = -5,       /* a bounded device-side wait ran out (tensor-core kernels) */
  TM_ERR_NOT_SU3 = -6,       /* a link is not unitary with det 1 (tolerance 1e-10) */
  TM_ERR_NONFINITE = -7,     /* NaN or Inf in an input or a reduction */
  TM_ERR_STATE = -8          /* call out of order (e.g. solve before setup) */
} tm_status;

/* storage/arithmetic precision of a field.  TM_F16 and TM_BF16 are storage
   formats of operators read by the FP32 K-cycle (arithmetic stays FP32): the
   interpolation P of the restriction and prolongation (tm_params.transfer_prec),
   the level-1 SAP blocks (sap1_prec), and FP16 for learned-layer inference.
   TM_F32X2: FP32 storage of the input, arithmetic in pairs of FP32 numbers (an
   unevaluated sum hi + lo, about 2^-46 relative) with an FP64 result; see
   tm_params.outer_apply and tm_apply. */
enum { TM_F64 = 0, TM_F32 = 1, TM_F16 = 2, TM_BF16 = 3, TM_F32X2 = 4 };

/* what tm_export copies out */
enum {
  TM_EXPORT_P = 0,       /* P columns as fine fields, natural [2Nv][T][Z][Y][X][4][3] */
  TM_EXPORT_DC = 1,      /* D_c blocks, [Tc][Zc][Yc][Xc][9][2Nv row][2Nv col], mu-free;
                            block 0 self, 1 + 2 mu forward (to x+mu), 2 + 2 mu backward */
  TM_EXPORT_CLOVER = 2,  /* A(x) chiral blocks incl. (m0+4), [T][Z][Y][X][2][6][6] */
  TM_EXPORT_TV = 3,      /* current test vectors, natural [Nv][T][Z][Y][X][4][3] */
  /* three-level handles only (levels = 3), after a setup; level-1 vectors
     are natural [Tc][Zc][Yc][Xc][2Nv] complex128 */
  TM_EXPORT_P2 = 4,      /* P2 columns as level-1 vectors, [2Nv2][level-1 vector] */
  TM_EXPORT_DC2 = 5,     /* D_c2 blocks, [T2][Z2][Y2][X2][9][2Nv2 row][2Nv2 col], mu-free */
  TM_EXPORT_TV1 = 6      /* level-1 test vectors, [Nv2][level-1 vector] */
};

typedef struct {
  int L[4];             /* T, Z, Y, X; each divisible by agg and sap_block */
  double m0;            /* bare mass (kappa = 1 / (2 (m0 + 4))) */
  double c_sw;          /* clover coefficient */
  double mu;            /* twisted mass of D(mu) (Sec. 1) */
  double delta;         /* coarse twisted mass mu_c = delta * mu, delta >= 1 (Sec. 1) */
  double bc_t;          /* -1 antiperiodic (default) or +1 periodic in T */
  int nv;               /* number of test vectors N_v (Sec. 1, O(20)) */
  int agg[4];           /* aggregate dims; coarse extents must be even */
  int sap_block[4];     /* SAP block dims; block counts per dimension even */
  int mr_iters;         /* minimal-residual steps per block solve */
  int pre_smooth;       /* j of eq. (1) */
  int post_smooth;      /* k of eq. (1) */
  int init_sweeps;      /* SAP sweeps on D v = 0 applied to the random vectors */
  int setup_iters;      /* adaptive setup iterations (Fig. 1: 3 few rhs, 5 many) */
  double coarse_tol;    /* coarse GMRES tolerance, relative to the reduced rhs */
  int coarse_restart;   /* coarse GMRES restart length */
  int coarse_maxit;     /* coarse GMRES iteration cap */
  int restart;          /* outer FGMRES restart length */
  int maxit;            /* outer FGMRES iteration cap */
  int cycle_prec;       /* TM_F64 or TM_F32: precision of smoother, P, D_c, coarse solve */
  int max_rhs;          /* largest nrhs passed to field-level calls */
  /* Third level (Sec. 2: DD-alphaAMG recurses; the paper runs three levels
     on its large lattices).  levels = 2 ignores everything below. */
  int levels;           /* 2 or 3 */
  int nv2;              /* level-1 test vectors (1..28) */
  int agg2[4];          /* level-2 aggregate dims in coarse sites; level-2 extents even */
  int sap_block1[4];    /* level-1 SAP block dims; block counts per dimension even */
  int mr_iters1;        /* MR steps per level-1 block solve */
  int pre_smooth1;      /* level-1 j of eq. (1) */
  int post_smooth1;     /* level-1 k of eq. (1) */
  int init_sweeps1;     /* level-1 SAP sweeps on D_c1 w = 0 applied to the random w */
  int coarse_setup_iters; /* level-1 adaptive passes inside each fine setup iteration */
  double coarsest_tol;  /* level-2 GMRES tolerance */
  int coarsest_maxit;   /* level-2 GMRES iteration cap */
  /* Odd-even Schur complement of the coarsest level (Sec. 3) on the tensor
     cores: 0 = CUDA cores (FP32/FP64), 1 = TF32 products, 2 = TF32 with the
     vectors split in two TF32 parts, 3 = 3xTF32 (operator split as well, about
     FP32 accuracy).  1..3 need cycle_prec = TM_F32; FP32 accumulation. */
  int coarse_mma;
  /* Stage after the K-cycle in the solve's preconditioner (not in the paper):
     0 = none, 1 = learned layer z = B(v) + N(v - D B(v)) (tm_nn_*), 2 = one SAP
     sweep in place of N (the stand-in the learned layer is compared with).
     nn_prec: TM_F32, or TM_F16 for FP16 hidden channels and weights. */
  int nn_mode;
  int nn_prec;
  /* Storage of the level-1 operator blocks read by the K-cycle's level-1 SAP
     smoother and level-1 Krylov solve (three levels, cycle_prec = TM_F32):
     TM_F32, or TM_F16 / TM_BF16 for a 16-bit copy (half the bytes; FP32
     arithmetic).  tm_apply at level 1 keeps the FP32 blocks. */
  int sap1_prec;
  /* Arithmetic of the outer FGMRES's products w = D(mu) z_k with the
     preconditioned vectors z_k (which the FP32 K-cycle returns in FP32):
     TM_F64 (z_k converted to FP64, FP64 stencil) or TM_F32X2 (FP32 pairs on
     the FP32 z_k, FP64 result, about 2^-46 relative; GB300's FP64 rate is
     1/64 of its FP32 rate).  TM_F32X2 needs cycle_prec = TM_F32 and keeps
     the links and the clover term once more as FP32 pairs (288 B per site
     each).  The true residual b - D x stays FP64 either way. */
  int outer_apply;
  /* SAP block solves (Sec. 3: odd-even preconditioning in the smoother):
     0 = mr_iters MR steps on the block operator D_B; 1 = mr_iters MR steps on
     the block's odd-even Schur complement D_ee - D_eo D_oo^-1 D_oe over its
     even sites, odd sites recovered afterwards.  1 needs even sap_block dims
     and keeps (A(x) + i mu gamma5)^-1 of every odd site (144 reals per odd
     site in cycle_prec); SAP then runs in cycle_prec only. */
  int block_oe;
  /* Polls of each pipeline mbarrier wait in the tensor-core kernel before it
     gives up (0 = the default, 2^22).  On a timeout the kernel drains its
     copies and MMAs, frees its tensor memory and the call returns
     TM_ERR_TIMEOUT; the context stays usable.  Small values exist to test that
     path. */
  int tc_spin_limit;
  /* Storage of P as read by the K-cycle's restriction P^dagger r and
     prolongation P e between the fine and the first coarse level
     (cycle_prec = TM_F32): TM_F32 (P itself), or TM_F16 / TM_BF16 for a 16-bit
     copy made after every build of P (half the bytes of the largest operand
     of both transfers; FP32 arithmetic and FP32 vectors).  The coarse
     operator is built from the full-precision P.  tm_restrict / tm_prolong
     with prec = TM_F32 use the same copy. */
  int transfer_prec;
  /* Storage of the links, the clover term and the odd-site inverses D_oo^-1
     read by the fine SAP smoother with odd-even block solves (block_oe = 1,
     cycle_prec = TM_F32): TM_F32, or TM_F16 / TM_BF16 for 16-bit copies made
     with every gauge field and twisted mass (FP32 arithmetic and FP32
     vectors; the smoother then works with the rounded operator, which the
     flexible outer solver tolerates).  The outer D(mu), the coarse build and
     the FP32 D apply keep the full-precision operator. */
  int sap_prec;
  /* Coarsest-level solve: 0 = GMRES(coarse_restart) on the odd-even Schur
     complement to coarse_tol / coarsest_tol with the host deciding each step;
     k in 1..64 = exactly k GMRES steps (a right-hand side whose residual
     estimate reaches the tolerance stops updating), all bookkeeping on the
     device, captured once as a CUDA graph and replayed for every later
     coarsest solve with the same buffers and twisted mass. */
  int coarsest_steps;
} tm_params;

typedef struct {
  int iters;              /* outer FGMRES iterations (summed over rhs) */
  int restarts;           /* restart cycles (summed over rhs) */
  int converged;          /* 1 if every rhs reached tol */
  double true_relres;     /* max over rhs of ||b - D x|| / ||b||, FP64 on the GPU */
  long long coarse_iters; /* coarse GMRES iterations in the solve */
  int kcycles;            /* preconditioner applications */
} tm_solve_info;

/* Fill p with the defaults: bc_t = -1, delta = 1, nv = 20, agg = sap_block
 * = 4^4, mr_iters = 4, pre = 0, post = 4, init_sweeps = 3, setup_iters = 3,
 * coarse_tol = 5e-2, coarse_restart = 30, coarse_maxit = 200, restart = 25,
 * maxit = 1000, cycle_prec = TM_F32, max_rhs = 1, levels = 2, nv2 = 28,
 * agg2 = sap_block1 = 2^4, mr_iters1 = 4, pre_smooth1 = 0, post_smooth1 = 2,
 * init_sweeps1 = 3, coarse_setup_iters = 3, coarsest_tol = 5e-2,
 * coarsest_maxit = 200, coarse_mma = 0, nn_mode = 0, nn_prec = TM_F32,
 * sap1_prec = TM_F32, outer_apply = TM_F64, block_oe = 0, tc_spin_limit = 0,
 * transfer_prec = sap_prec = TM_F32, coarsest_steps = 0.
 * L, m0, c_sw, mu are 0. */
void tm_params_default(tm_params* p);

/* Validate p and allocate a handle bound to a CUDA stream (cudaStream_t,
 * may be NULL for the legacy default stream) on the current device.
 * Errors: TM_ERR_ARG (divisibility, even block/coarse counts, nv in 1..28,
 * aggregate and block volume <= 1024), TM_ERR_OOM, TM_ERR_CUDA. */
tm_status tm_create(tm_handle** h, const tm_params* p, void* stream);

/* Free everything the handle owns.  NULL is ignored. */
void tm_destroy(tm_handle* h);

/* Static text of a status code. */
const char* tm_status_string(int status);

/* Message of the last failing call on h (empty string if none). */
const char* tm_last_error(const tm_handle* h);

/* A0: take the gauge field (natural layout, host or device, complex128),
 * check every link is SU(3) to 1e-10 (TM_ERR_NOT_SU3 otherwise), pack the
 * links as 12 reals in FP64 and FP32 and build the clover term A(x) =
 * (m0+4) - (c_sw/32) sum_{mu,nu} gamma_mu gamma_nu (Q_mu_nu - Q_nu_mu)
 * as two Hermitian 6x6 blocks (D_W of Sec. 1).  Invalidates any setup. */
tm_status tm_load_gauge(tm_handle* h, const double* gauge);

/* A8: adaptive setup (Sec. 1; Fig. 1 setup iterations).  test_vectors
 * (natural, [nv] spinors, host or device) are the random starting vectors.
 * Each gets init_sweeps SAP sweeps on D v = 0 and is normalised; P
 * (per aggregate and chirality thin QR, Gamma5 P = P Gamma5_c) and
 * D_c(delta mu) are built; then setup_iters times every v_i <- B(v_i) with
 * the current K-cycle B, normalised, and P, D_c rebuilt.
 * Three levels (levels = 3): test_vectors continues with nv2 level-1 random
 * vectors (natural [nv2][Tc][Zc][Yc][Xc][2Nv]); after P, D_c1 they get
 * init_sweeps1 level-1 SAP sweeps on D_c1(mu) w = 0, are normalised and give
 * P2, D_c2; each fine iteration then also rebuilds P2, D_c2 from the current
 * w_j, and finally coarse_setup_iters times every w_j <- B1(w_j) with the
 * level-1 K-cycle, normalised, P2 and D_c2 rebuilt (Sec. 3: the fine and the
 * coarse setup iteration counts).
 * The setup's own work buffers (N_v fine fields for the iterated vectors) are
 * freed before it returns.
 * Errors: TM_ERR_STATE (no gauge), TM_ERR_ARG (rank-deficient aggregate),
 * TM_ERR_NONFINITE. */
tm_status tm_setup(tm_handle* h, const double* test_vectors);

/* Build P and D_c directly from the given vectors (no smoothing, no
 * iterations): the interpolation of Sec. 1 for a fixed set of v_i (with three
 * levels also P2, D_c2 from the appended level-1 vectors, as in tm_setup). */
tm_status tm_setup_from_vectors(tm_handle* h, const double* test_vectors);

/* Setup update after the gauge field changed (Sec. 3: during an HMC
 * trajectory the setup is updated by one fine and three first-coarse-grid
 * iterations instead of rebuilt).  Call after tm_load_gauge with the new
 * field: P and D_c (and P2, D_c2) are rebuilt from the test vectors of the
 * last setup, then fine_iters times v_i <- B(v_i) and, with three levels,
 * coarse_iters times w_j <- B1(w_j), as in tm_setup.  Errors: TM_ERR_STATE
 * (no gauge field, or no earlier setup on this handle). */
tm_status tm_setup_update(tm_handle* h, int fine_iters, int coarse_iters);

/* Autotune the tile shape of the D_c build (the Galerkin projection
 * P^dagger D P of Sec. 1) for this handle's N_v, aggregate and cycle
 * precision.  Each candidate (sites staged per tile, columns per register
 * tile) first rebuilds D_c into a scratch buffer that must equal the default
 * shape's D_c bit for bit (every shape sums each entry in the same order),
 * then is timed with CUDA events over `reps` (1..100) builds; the fastest is
 * kept for the handle's later builds.  cache_path (may be NULL): a JSON file
 * of earlier choices keyed by device name, kernel, precision, N_v and
 * aggregate; a hit takes the stored shape without timing, a miss adds the
 * new choice (the file is rewritten through a temporary file beside it).
 * out (may be NULL): 4 doubles = sites per tile, columns per register tile,
 * microseconds per build, candidates timed (0 for a cache hit).  The D_c in
 * use is unchanged; timing takes two D_c-sized scratch buffers, released
 * before the call returns (on errors too).  Synchronises the handle's
 * stream.  Errors: TM_ERR_STATE (no setup, or a candidate whose D_c
 * differs), TM_ERR_ARG (reps out of range, cache not writable). */
tm_status tm_autotune_build(tm_handle* h, const char* cache_path, int reps, double* out);

/* Change mu and delta without a new setup (Sec. 1: D_c(mu) = D_c +
 * i mu Gamma5_c, so only the diagonal shift and the odd-site inverses of the
 * coarse Schur complement change; one setup serves D(+mu) and D(-mu)).  The
 * twisted mass becomes mu on all sites (see tm_set_mu_eo). */
tm_status tm_set_mu(tm_handle* h, double mu, double delta);

/* A different twisted mass on the even and the odd sites (Sec. 2, needed for
 * Hasenbusch preconditioning with odd-even preconditioning): D = D_W +
 * i Gamma5 mu(x), mu(x) = mu_even on sites with (t+z+y+x) even, mu_odd on odd
 * ones.  The coarse operators are the Galerkin projections of
 * D_W + i (mu_odd - mu_even) Pi_odd Gamma5 plus i mu_even Gamma5_c (times
 * delta on the coarsest level): a change of mu_odd - mu_even projects D_c
 * (and D_c2) again from the current P (and P2), without a new setup.
 * Errors: TM_ERR_ARG (non-finite masses, delta < 1). */
tm_status tm_set_mu_eo(tm_handle* h, double mu_even, double mu_odd, double delta);

/* The odd-even reduced system D^ x_o = b_o, D^ = D_oo - D_oe D_ee^-1 D_eo on
 * the odd sites of the handle's current operator, solved through the full
 * operator (Sec. 3: DD-alphaAMG inverts the full operator even when the
 * reduced one is wanted): D x = (0 on even sites, b_o on odd sites) to tol,
 * x_o the odd part.  b, x natural spinors (host or device) of which only the
 * odd sites count; x holds a start vector and returns x_o with zeros on the
 * even sites.  info as tm_solve (the residual is that of the full system). */
tm_status tm_solve_odd(tm_handle* h, const double* b, double* x, int nrhs, double tol, tm_solve_info* info);

/* The two inversions of a Hasenbusch-preconditioned HMC force term (Sec. 3),
 * in the order the paper lists them, on the odd sites:
 *   y = (D^(mu) + i rho G^5)^-1 b,   x = (G^5 D^(-mu) G^5 - i rho G^5)^-1 y,
 * G^5 = Gamma5 on the odd sites, with one setup.  The first operator is the
 * odd Schur complement of D(mu on even, mu + rho on odd sites); the second is
 * its adjoint, inverted as G^5 (D^(-mu) - i rho G^5)^-1 G^5 with D(-mu,
 * -mu - rho): x = (A A^dagger)^-1 b, A = D^(mu) + i rho G^5.  b, x as
 * tm_solve_odd (x is overwritten, no start vector); info sums both solves.
 * The handle is left at mu on even and mu + rho on odd sites. */
tm_status tm_solve_hasenbusch(tm_handle* h, const double* b, double* x, int nrhs, double mu, double rho, double tol,
                              tm_solve_info* info);

/* f4: the comparison solver of Fig. 1 (Sec. 1): oeCG, conjugate gradient on
 * D^dagger D^ x_o = D^dagger b^ for the odd-even reduced operator
 * D^ = D_oo - D_oe D_ee^-1 D_eo of Sec. 3 (twisted mass mu on even and
 * mu + rho on odd sites as set by tm_set_mu / tm_set_mu_eo), with
 * b^ = b_o - D_oe D_ee^-1 b_e and x_e = D_ee^-1 (b_e - D_eo x_o) afterwards.
 * CG iterates in FP32 (CGLS form, scalars on the device) inside FP64 defect
 * correction: after each inner solve, which reduces the defect by 1e-5 or to
 * the target, the reduced residual is recomputed in FP64 and the solve stops
 * once |b^ - D^ x_o| = |b - D x| <= tol |b|.  Right-hand sides are solved
 * one after another.  Needs tm_load_gauge only (no setup).  b, x as tm_solve
 * (x holds the start vector; its odd sites are used).  maxit bounds the CG
 * iterations per right-hand side.  info->iters = CG iterations in all,
 * ->restarts = defect-correction cycles, ->true_relres = max FP64 relative
 * residual, coarse_iters = kcycles = 0.  Errors: TM_ERR_STATE (no gauge
 * field), TM_ERR_ARG (odd X extent), TM_ERR_NOT_CONVERGED. */
tm_status tm_solve_oecg(tm_handle* h, const double* b, double* x, int nrhs, double tol, int maxit,
                        tm_solve_info* info);

/* A7: solve D(mu) x_r = b_r for nrhs right-hand sides to ||b - D x|| <=
 * tol ||b|| by FGMRES(restart) preconditioned with the K-cycle of eq. (1).
 * b, x natural spinors (host or device); x holds the start vector on entry
 * and the solution on return.  The outer vectors and every residual that
 * decides convergence are FP64 (with outer_apply = TM_F32X2 the products
 * D(mu) z_k, the CGS2 arithmetic and the restart residuals far from
 * convergence use FP32 pairs, about 2^-46 relative); the K-cycle runs in
 * cycle_prec.  A zero start vector skips the first residual product.
 * info may be NULL.
 * Errors: TM_ERR_STATE (no setup), TM_ERR_NOT_CONVERGED (x = best iterate,
 * info filled), TM_ERR_NONFINITE. */
tm_status tm_solve(tm_handle* h, const double* b, double* x, int nrhs, double tol, tm_solve_info* info);

/* Squared-operator solve with one setup (Sec. 1: the same setup serves
 * D(+mu) and D(-mu); Sec. 3: the squared operator is inverted by two solves
 * of the non-squared operator): x = (D(mu)^dagger D(mu))^-1 b computed as
 * D(mu)^-1 Gamma5 D(-mu)^-1 Gamma5 b, using D(mu)^dagger = Gamma5 D(-mu) Gamma5
 * (with an odd-site shift the adjoint flips it too: D(-mu, -mu - rho)).
 * The D(-mu) solve starts from zero, the D(mu) solve from x; both run to tol.
 * Arguments, layouts and errors as tm_solve; info sums both solves.  The
 * handle is left at +mu. */
tm_status tm_solve_squared(tm_handle* h, const double* b, double* x, int nrhs, double tol, tm_solve_info* info);

/* Device memory a handle with parameters p needs, in bytes: what tm_create
 * allocates, plus the larger of the adaptive setup's work (with device
 * test vectors) and the work of tm_solve with nrhs right-hand sides (batched
 * up to max_rhs).  For planning before anything is allocated (a 48^3 x 96
 * three-level handle needs well over 100 GB); inputs passed as host arrays
 * add a device copy of their size.  0 for invalid parameters. */
size_t tm_workspace_bytes(const tm_params* p, int nrhs);

/* Save the setup of a handle (test vectors, P and D_c; with three levels also
 * the level-1 test vectors, P2 and D_c2, in the handle's device layout and
 * cycle precision) to a file, with a header of the lattice, aggregates, N_v,
 * levels and precision; the file is written through `path`.tmp and renamed.
 * Sec. 3: one setup serves many inversions and, updated, the next gauge
 * fields of an HMC trajectory.  Errors: TM_ERR_STATE (no setup), TM_ERR_ARG
 * (file not writable). */
tm_status tm_save_setup(tm_handle* h, const char* path);

/* Load a saved setup into a handle created with the same lattice, aggregates,
 * N_v (N_v2, agg2) and cycle_prec, after tm_load_gauge.  The odd-site
 * inverses (current mu and delta), the FP16 level-1 blocks and the
 * tensor-core tiles are rebuilt from the loaded D_c.  A solve after loading
 * reproduces a solve with the saved handle's setup bit for bit on the same
 * gauge field; with another field follow with tm_setup_update.  Errors:
 * TM_ERR_STATE (no gauge field), TM_ERR_ARG (unreadable or foreign file,
 * other sizes). */
tm_status tm_load_setup(tm_handle* h, const char* path);

/* Bytes of one field of nrhs vectors: level 0 = fine spinors, level 1 =
 * coarse vectors; prec TM_F64 or TM_F32.  0 for invalid arguments. */
size_t tm_field_bytes(const tm_handle* h, int level, int prec, int nrhs);

/* Convert natural complex128 vectors (device) to a field of the given
 * level and precision (device), and back.  Level 1 is a plain cast. */
tm_status tm_pack(tm_handle* h, int level, int prec, const double* natural, void* field, int nrhs);
tm_status tm_unpack(tm_handle* h, int level, int prec, const void* field, double* natural, int nrhs);

/* A1 (level 0): out = D(mu) in, fine fields, prec TM_F64 or TM_F32; with
 * prec TM_F32X2 (handles created with outer_apply = TM_F32X2) in is an FP32
 * field and out an FP64 field, computed in FP32-pair arithmetic.
 * A4 (level 1): out = D_c(delta mu) in, coarse fields, prec = cycle_prec,
 * after a setup.  in and out are distinct device fields of nrhs vectors. */
tm_status tm_apply(tm_handle* h, int level, int prec, const void* in, void* out, int nrhs);

/* A2: sweeps SAP sweeps (red blocks, then black) on D x = b with mr_iters MR
 * steps per block solve (Sec. 1: the smoother M; with block_oe = 1 on the
 * block's odd-even Schur complement, Sec. 3).  b may be NULL (b = 0).
 * Fine fields, prec TM_F64 or TM_F32 (cycle_prec with block_oe = 1); x is
 * updated in place. */
tm_status tm_sap(tm_handle* h, int prec, const void* b, void* x, int sweeps, int nrhs);

/* A3: coarse = P^dagger fine.  A6: fine = P coarse (accumulate = 0) or
 * fine += P coarse (accumulate = 1).  prec = cycle_prec, after a setup; with
 * a 16-bit transfer_prec the FP32 transfers read the 16-bit copy of P. */
tm_status tm_restrict(tm_handle* h, int prec, const void* fine, void* coarse, int nrhs);
tm_status tm_prolong(tm_handle* h, int prec, const void* coarse, void* fine, int nrhs, int accumulate);

/* A5: solve D_c(delta mu) x = b on the coarse lattice by GMRES(coarse_restart)
 * on the odd-even Schur complement (Sec. 3), from zero, to tol relative to
 * the reduced right-hand side or maxit steps.  One coarse field each (device,
 * cycle_prec).  *iters (may be NULL) receives the step count. */
tm_status tm_coarse_solve(tm_handle* h, int prec, const void* b, void* x, double tol, int maxit, int* iters);

/* y_e = S v_e with S = D_ee - D_eo D_oo^-1 D_oe the odd-even Schur
 * complement of the coarsest operator D_c(delta mu) (Sec. 3: the coarsest
 * level is solved on S by GMRES).  v_e, y_e: distinct device arrays of nrhs
 * compact even vectors [nrhs][Vc/2][2N_v] complex (even sites in lexicographic
 * order), prec = cycle_prec, after a setup.  With coarse_mma > 0 and nrhs <=
 * 32 this runs on the tensor cores; TM_ERR_TIMEOUT if a device wait ran out. */
tm_status tm_schur(tm_handle* h, int prec, const void* ve, void* ye, int nrhs);

/* Allocation-free variant of tm_coarse_solve (the paper has no counterpart;
 * this is a library convenience).  Some callers cannot call cudaMalloc when
 * they need a coarse solve, e.g. an application whose own memory pool has
 * already taken the free device memory, or a latency-critical loop that must
 * not pay for cudaMalloc's implicit synchronisation.  This call computes the
 * same odd-even GMRES as tm_coarse_solve (same arguments, same result) but
 * allocates nothing: every workspace lives in one fixed 8 MiB device array
 * that the library holds on each GPU that loads it until the process exits.
 * The handle's setup data (D_c, the odd-site inverses) must exist already.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress, with the device current) and caches it; make
 *     that first call before any stream capture.  Call with the handle's
 *     device current.
 *   - Coarse systems whose Krylov basis (coarse_restart + 1 vectors), five
 *     work vectors and reduction buffers exceed 8 MiB are rejected with
 *     TM_ERR_ARG and a message giving the size needed.
 *   - All calls share the array and it keeps the last call's contents; the
 *     call zeroes the iterate it keeps there and writes everything else
 *     before reading it.  Calls whose work overlaps on the GPU (other
 *     threads, other streams) race on the array: serialise them. */
tm_status tm_coarse_solve_noalloc(tm_handle* h, int prec, const void* b, void* x, double tol, int maxit,
                                  int* iters);

/* Three-level handles: the level-1 pieces of the recursive cycle (Sec. 2),
 * all on level-1 fields in cycle_prec after a setup; TM_ERR_ARG on a
 * two-level handle.  With three levels, level 1 of tm_apply applies
 * D_c1(mu) (the first coarse level keeps the fine twisted mass) and level 2
 * applies D_c2(delta mu); tm_coarse_solve solves on level 2.
 *   tm_sap1:      sweeps red/black SAP sweeps on D_c1(mu) x = b (b may be NULL)
 *                 with mr_iters1 MR steps per block, x updated in place.
 *   tm_restrict1: c2 = P2^dagger c1.   tm_prolong1: c1 (+)= P2 c2.
 *   tm_kcycle1:   z = B1(v): eq. (1) on level 1 with pre_smooth1 / post_smooth1
 *                 sweeps and a level-2 GMRES to coarsest_tol. */
tm_status tm_sap1(tm_handle* h, int prec, const void* b, void* x, int sweeps, int nrhs);
tm_status tm_restrict1(tm_handle* h, int prec, const void* c1, void* c2, int nrhs);
tm_status tm_prolong1(tm_handle* h, int prec, const void* c2, void* c1, int nrhs, int accumulate);
tm_status tm_kcycle1(tm_handle* h, int prec, const void* v, void* z, int nrhs);

/* Learned gauge-covariant layer (an addition; the paper has no learned parts).
 * N = L2 o L1, L1: 1 -> 8 and L2: 8 -> 1 spinor channels, no nonlinearity:
 *   y_o(x) = sum_i sum_d W[o][i][d] (T_d psi_i)(x), d = self, then +T, -T, +Z,
 *   -Z, +Y, -Y, +X, -X; (T_{+mu} psi)(x) = U_mu(x) psi(x + mu), (T_{-mu} psi)(x) =
 *   U_mu(x - mu)^dagger psi(x - mu) (boundary factor bc_t across T); W[o][i][d]
 *   a complex 4 x 4 spin matrix acting trivially on colour.
 * Weights: 2304 complex numbers as interleaved doubles (host memory), W1
 * [8][1][9][4][4] then W2 [1][8][9][4][4] (row index first).  Default: zero.
 *   tm_nn_set_weights / tm_nn_get_weights copy them in or out (set resets the
 *     optimiser state).
 *   tm_nn_apply: out = N(in) (accumulate = 0) or out += N(in); in, out
 *     distinct device arrays of nrhs FP32 fine fields (tm_field_bytes(h, 0,
 *     TM_F32, nrhs)); prec TM_F32 or TM_F16.  Needs a gauge field.
 *   tm_nn_pairs: training pairs from random errors e0 (natural spinors, host
 *     or device, npairs of them): e = (1 - B D) e0 with the current K-cycle B
 *     and r = D e, written as FP32 fine fields.  Needs a setup with cycle_prec
 *     = TM_F32.
 *   tm_nn_grad: loss L = sum_p ||N(r_p) - e_p||^2 / sum_p ||e_p||^2 and its
 *     Wirtinger gradient dL/d conj(W) (2304 complex, interleaved; either
 *     output may be NULL).
 *   tm_nn_train: `epochs` passes of Adam (beta 0.9, 0.999, eps 1e-8, step lr)
 *     over minibatches of `batch` pairs in order, FP32 forward and backward on
 *     the GPU; losses (may be NULL) receives the mean loss of each epoch. */
tm_status tm_nn_set_weights(tm_handle* h, const double* w);
tm_status tm_nn_get_weights(tm_handle* h, double* w);
tm_status tm_nn_apply(tm_handle* h, int prec, const void* in, void* out, int nrhs, int accumulate);
tm_status tm_nn_pairs(tm_handle* h, const double* e0, void* r, void* e, int npairs);
tm_status tm_nn_grad(tm_handle* h, const void* r, const void* e, int npairs, double* grad, double* loss);
tm_status tm_nn_train(tm_handle* h, const void* r, const void* e, int npairs, int epochs, int batch, double lr,
                      double* losses);

/* A7 preconditioner: z = B(v), one application of eq. (1) from a zero start
 * (pre SAP sweeps, coarse correction, post SAP sweeps).  Fine fields in
 * cycle_prec, nrhs vectors. */
tm_status tm_kcycle(tm_handle* h, int prec, const void* v, void* z, int nrhs);

/* Copy internal data out as natural complex128 (host or device pointer of
 * at least `bytes` bytes); see the TM_EXPORT_* layouts. */
tm_status tm_export(tm_handle* h, int what, double* out, size_t bytes);

/* Wait for all work queued on the handle's stream; reports asynchronous
 * kernel errors. */
tm_status tm_synchronize(tm_handle* h);

/* Opt-in per-kernel accounting.  Kernel launches fall into
 * tm_profile_kinds() classes (named by tm_profile_name: dslash_f64,
 * dslash_f32, sap, restrict, prolong, coarse_oe, blas_fine, blas_coarse,
 * coarse_build, other, coarse_sap (level-1 SAP), level1 (level-1 operator),
 * nn, dslash_f32x2 (FP32-pair products and restart residuals),
 * level1_transfer (P2 and P2^dagger), oecg_operator, oecg_blas; a
 * graph-captured coarsest solve counts as coarse_oe with its node count as
 * launches).  With enable != 0
 * every launch is counted (launches
 * and right-hand-side units) and the launches of class k are also bracketed
 * by a pair of CUDA events on the handle's stream when bit k of enable is set
 * (enable = -1 times every class).  tm_profile resets the totals;
 * tm_profile_read waits for the stream and copies, per class, the launches,
 * the units and the summed event time in milliseconds (arrays of n; any may
 * be NULL).  Not part of the method: measurement only. */
tm_status tm_profile(tm_handle* h, int enable);
int tm_profile_kinds(void);
const char* tm_profile_name(int kind);
tm_status tm_profile_read(tm_handle* h, long long* launches, long long* units, double* ms, int n);

#ifdef __cplusplus
}
#endif

#endif /* TM_H */
