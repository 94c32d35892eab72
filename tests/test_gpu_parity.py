"""GPU parity: every step of the hot path through the C ABI against the oracle.

Tolerances (relative L2): FP64 single operator applies <= 1e-12; FP64
composite fixed-count applications (SAP sweeps, coarse GMRES with a fixed
step count, one K-cycle) <= 1e-10; FP32 single applies <= 5e-6 (24-bit
mantissa, sums of <= 100 terms).  Shapes cover the 4^4 configuration, a
ragged 4x6x4x10 lattice (960 sites: the last 128-thread CTA is partial;
60-site aggregates and SAP blocks leave idle lanes in every warp) and 8^4.
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator, clover_blocks
from oracle.sap import SAP
from oracle.coarse import Interpolation, CoarseOperator, OddEvenCoarse
from oracle.krylov import gmres
from oracle.amg import TwoLevel, AMGParams

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1611_01034_gb300 as tm  # noqa: E402
from tests.gpu_helpers import GPU, rel  # noqa: E402

F64, F32 = tm.TM_F64, tm.TM_F32

KAPPA1 = 0.13
CASES = {
    # name: (L, eps, seed, m0, c_sw, mu, delta, nv, agg/sap block)
    "c1_4x4x4x4": ((4, 4, 4, 4), 0.3, 1, 1 / (2 * KAPPA1) - 4, 1.0, 0.01, 1.0, 8, (2, 2, 2, 2)),
    "ragged_4x6x4x10": ((4, 6, 4, 10), 0.5, 3, -0.3, 1.5, 0.02, 3.0, 6, (2, 3, 2, 5)),
    "8x8x8x8": ((8, 8, 8, 8), 0.5, 5, -0.4, 1.5, 0.005, 5.0, 8, (4, 4, 4, 4)),
}


def _case(name, prec=F64, **over):
    L, eps, seed, m0, csw, mu, delta, nv, blk = CASES[name]
    U = inputs.gauge_field(L, eps, seed)
    kw = dict(m0=m0, c_sw=csw, mu=mu, delta=delta, nv=nv, agg=blk, sap_block=blk, cycle_prec=prec,
              max_rhs=4)
    kw.update(over)
    g = GPU(U, **kw)
    op = Operator(U, m0, csw, mu)
    return U, g, op, seed


@pytest.mark.parametrize("name", list(CASES))
def test_clover_matches_oracle(name):
    U, g, op, _ = _case(name)
    assert rel(g.clover(), clover_blocks(op.A)) <= 1e-13


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,tol", [(F64, 1e-12), (F32, 5e-6)])
def test_dirac_apply(name, prec, tol):
    U, g, op, seed = _case(name)
    psi = inputs.gaussian_spinor(g.L, seed + 1000, nrhs=3)
    got = g.apply_fine(psi, prec, nrhs=3)
    assert rel(got, op.apply(psi)) <= tol
    for r in range(3):
        assert rel(got[r], op.apply(psi[r])) <= tol


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("bc_t", [-1.0, 1.0])
def test_dirac_apply_fp32_pairs(name, bc_t):
    """D(mu) on an FP32 field in FP32-pair arithmetic, FP64 result: against the
    oracle's FP64 D(mu) of the same FP32-rounded input within 1e-13 (pairs keep
    about 46 significant bits; the stencil's sums cancel by less than 2^6)."""
    L, eps, seed, m0, csw, mu, delta, nv, blk = CASES[name]
    U = inputs.gauge_field(L, eps, seed)
    g = GPU(U, m0=m0, c_sw=csw, mu=mu, delta=delta, nv=nv, agg=blk, sap_block=blk, cycle_prec=F32,
            max_rhs=3, bc_t=bc_t, outer_apply=tm.TM_F32X2)
    op = Operator(U, m0, csw, mu, bc_t=bc_t)
    psi = inputs.gaussian_spinor(L, seed + 1000, nrhs=3).astype(np.complex64).astype(np.complex128)
    fi = g.pack(0, F32, psi, 3)
    fo = g.field(0, F64, 3)
    tm.tm_apply(g.h, 0, tm.TM_F32X2, fi, fo, 3)
    got = g.unpack(0, F64, fo, psi.shape, 3)
    for r in range(3):
        assert rel(got[r], op.apply(psi[r])) <= 1e-13
    # the plain FP32 stencil is ~1e6 times further off
    assert rel(g.apply_fine(psi, F32, nrhs=3), op.apply(psi)) > 1e-9


def test_dirac_periodic_and_free_field():
    L = (4, 6, 4, 10)
    U = inputs.unit_gauge(L)
    g = GPU(U, m0=-0.2, c_sw=1.1, mu=0.3, nv=4, agg=(2, 3, 2, 5), sap_block=(2, 3, 2, 5), bc_t=1.0,
            cycle_prec=F64)
    op = Operator(U, -0.2, 1.1, 0.3, bc_t=1.0)
    psi = inputs.gaussian_spinor(L, 7)
    assert rel(g.apply_fine(psi, F64), op.apply(psi)) <= 1e-13


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,tol", [(F64, 1e-10), (F32, 5e-5)])
def test_sap_sweeps(name, prec, tol):
    U, g, op, seed = _case(name)
    blk = CASES[name][8]
    sap = SAP(op, blk, n_mr=4)
    b = inputs.gaussian_spinor(g.L, seed + 11)
    x0 = 0.1 * inputs.gaussian_spinor(g.L, seed + 12)
    expect = sap.smooth(b, x0, 2)
    got = g.sap(b, x0, 2, prec)
    assert rel(got, expect) <= tol
    # homogeneous system (b = 0), as in the setup's initial smoothing
    expect0 = sap.smooth(np.zeros_like(b), x0, 1)
    got0 = g.sap(None, x0, 1, prec)
    assert rel(got0, expect0) <= tol


OE_CASES = ["c1_4x4x4x4", "8x8x8x8"]  # even SAP block dims


@pytest.mark.parametrize("name", OE_CASES)
@pytest.mark.parametrize("prec,tol", [(F64, 1e-10), (F32, 5e-5)])
def test_sap_sweeps_odd_even_blocks(name, prec, tol):
    """SAP with the block solves on the odd-even Schur complement (Sec. 3)
    against the oracle's SAP.mr_oe; the handle's cycle precision is prec."""
    U, g, op, seed = _case(name, prec, block_oe=1)
    blk = CASES[name][8]
    sap = SAP(op, blk, n_mr=4, block_oe=True)
    b = inputs.gaussian_spinor(g.L, seed + 11)
    x0 = 0.1 * inputs.gaussian_spinor(g.L, seed + 12)
    assert rel(g.sap(b, x0, 2, prec), sap.smooth(b, x0, 2)) <= tol
    assert rel(g.sap(None, x0, 1, prec), sap.smooth(np.zeros_like(b), x0, 1)) <= tol
    # the sign of mu reaches the odd-site inverses (tm_set_mu rebuilds them)
    tm.tm_set_mu(g.h, -op.mu, g.p.delta)
    sapm = SAP(op.with_mu(-op.mu), blk, n_mr=4, block_oe=True)
    assert rel(g.sap(b, x0, 1, prec), sapm.smooth(b, x0, 1)) <= tol


def _from_vectors(name, prec=F64):
    U, g, op, seed = _case(name, prec)
    tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
    tm.tm_setup_from_vectors(g.h, tv)
    P = Interpolation(tv, g.p.agg)
    Dc = CoarseOperator.build(op, P, mu_c=g.p.delta * g.p.mu)
    return g, op, P, Dc, seed


@pytest.mark.parametrize("name", list(CASES))
def test_interpolation_and_coarse_operator(name):
    g, op, P, Dc, _ = _from_vectors(name)
    assert rel(g.P_columns(), P.columns()) <= 1e-12
    assert rel(g.Dc_blocks(), Dc.blocks) <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,tol", [(F64, 1e-12), (F32, 5e-6)])
def test_restrict_prolong_coarse_apply(name, prec, tol):
    g, op, P, Dc, seed = _from_vectors(name, prec)
    psi = inputs.gaussian_spinor(g.L, seed + 21, nrhs=2)
    fi = g.pack(0, prec, psi, 2)
    fc = g.field(1, prec, 2)
    tm.tm_restrict(g.h, prec, fi, fc, 2)
    rc = g.unpack(1, prec, fc, g.coarse_shape(2), 2)
    assert rel(rc, P.restrict(psi)) <= tol
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(g.coarse_shape(2)) + 1j * rng.standard_normal(g.coarse_shape(2))
    fv = g.pack(1, prec, v, 2)
    fo = g.pack(0, prec, psi, 2)
    tm.tm_prolong(g.h, prec, fv, fo, 2, 1)
    assert rel(g.unpack(0, prec, fo, psi.shape, 2), psi + P.prolong(v)) <= tol
    tm.tm_prolong(g.h, prec, fv, fo, 2, 0)
    assert rel(g.unpack(0, prec, fo, psi.shape, 2), P.prolong(v)) <= tol
    fy = g.field(1, prec, 2)
    tm.tm_apply(g.h, 1, prec, fv, fy, 2)
    assert rel(g.unpack(1, prec, fy, v.shape, 2), Dc.apply(v)) <= tol


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tp,tol", [(tm.TM_F16, 5e-3), (tm.TM_BF16, 3e-2)])
def test_restrict_prolong_with_16bit_interpolation(name, tp, tol):
    # the K-cycle's transfers read a 16-bit copy of P (11 / 8 significant bits,
    # FP32 arithmetic); the coarse operator stays the full-precision Galerkin product
    U, g, op, seed = _case(name, F32, transfer_prec=tp)
    tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
    tm.tm_setup_from_vectors(g.h, tv)
    P = Interpolation(tv, g.p.agg)
    Dc = CoarseOperator.build(op, P, mu_c=g.p.delta * g.p.mu)
    assert rel(g.Dc_blocks(), Dc.blocks) <= 5e-6
    psi = inputs.gaussian_spinor(g.L, seed + 21, nrhs=2)
    fc = g.field(1, F32, 2)
    tm.tm_restrict(g.h, F32, g.pack(0, F32, psi, 2), fc, 2)
    err_r = rel(g.unpack(1, F32, fc, g.coarse_shape(2), 2), P.restrict(psi))
    assert err_r <= tol
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(g.coarse_shape(2)) + 1j * rng.standard_normal(g.coarse_shape(2))
    fo = g.field(0, F32, 2)
    tm.tm_prolong(g.h, F32, g.pack(1, F32, v, 2), fo, 2, 0)
    err_p = rel(g.unpack(0, F32, fo, psi.shape, 2), P.prolong(v))
    assert err_p <= tol
    # the rounding is that of the 16-bit format, not more (and not the FP32 result)
    assert max(err_r, err_p) >= (1e-5 if tp == tm.TM_F16 else 1e-4)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,tol", [(F64, 1e-10), (F32, 1e-3)])
def test_coarse_solve_device_graph(name, prec, tol):
    # coarsest_steps = k: exactly k GMRES steps with the Givens bookkeeping on the
    # device, captured as a CUDA graph and replayed; the same iterate as the oracle's
    # GMRES after k steps, for every replay and after a change of mu
    for steps in (1, 7, 24):
        U, g, op, seed = _case(name, prec, coarsest_steps=steps)
        tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
        tm.tm_setup_from_vectors(g.h, tv)
        P = Interpolation(tv, g.p.agg)
        rng = np.random.default_rng(seed + 3)
        b = rng.standard_normal(g.coarse_shape()) + 1j * rng.standard_normal(g.coarse_shape())
        for mu in (g.p.mu, -2 * g.p.mu):
            if mu != g.p.mu:
                tm.tm_set_mu(g.h, mu, g.p.delta)
            oe = OddEvenCoarse(CoarseOperator.build(op.with_mu(mu), P, mu_c=g.p.delta * mu))
            res = gmres(oe.schur, oe.reduced_rhs(b), tol=0.0, restart=steps, maxit=steps)
            expect = oe.reconstruct(b, res.x)
            got = []
            for _ in range(2):
                fx = g.field(1, prec)
                it = tm.tm_coarse_solve(g.h, prec, g.pack(1, prec, b), fx, 0.0, steps)
                assert it == steps
                got.append(g.unpack(1, prec, fx, b.shape))
            assert rel(got[0], expect) <= tol
            assert np.array_equal(got[0], got[1])


@pytest.mark.parametrize("coarsest_steps", [12, 24])
def test_solve_with_device_graph_coarsest(coarsest_steps):
    # fixed-step coarsest solves as the preconditioner's coarse correction: the
    # outer solve still reaches the oracle's FP64 residual <= 1e-10
    name = "8x8x8x8"
    U, g, op, seed = _case(name, F32, setup_iters=2, coarsest_steps=coarsest_steps, coarse_mma=1, max_rhs=4)
    tm.tm_setup(g.h, inputs.random_test_vectors(g.L, g.nv, seed + 2000))
    b = inputs.gaussian_spinor(g.L, seed + 1000, nrhs=4)
    x = np.zeros_like(b)
    st, info = tm.tm_solve(g.h, b, x, 4, 1e-10)
    assert st == tm.TM_OK and info.converged
    for r in range(4):
        assert np.linalg.norm(b[r] - op.apply(x[r])) / np.linalg.norm(b[r]) <= 1e-10


@pytest.mark.parametrize("name", list(CASES))
def test_coarse_solve_fixed_steps(name):
    g, op, P, Dc, seed = _from_vectors(name)
    rng = np.random.default_rng(seed + 3)
    b = rng.standard_normal(g.coarse_shape()) + 1j * rng.standard_normal(g.coarse_shape())
    oe = OddEvenCoarse(Dc)
    for steps in (1, 7, 45):
        res = gmres(oe.schur, oe.reduced_rhs(b), tol=0.0, restart=g.p.coarse_restart, maxit=steps)
        expect = oe.reconstruct(b, res.x)
        fb = g.pack(1, F64, b)
        fx = g.field(1, F64)
        it = tm.tm_coarse_solve(g.h, F64, fb, fx, 0.0, steps)
        assert it == steps == res.iters
        assert rel(g.unpack(1, F64, fx, b.shape), expect) <= 1e-10


@pytest.mark.parametrize("name", list(CASES))
def test_coarse_solve_to_tolerance(name):
    g, op, P, Dc, seed = _from_vectors(name)
    rng = np.random.default_rng(seed + 4)
    b = rng.standard_normal(g.coarse_shape()) + 1j * rng.standard_normal(g.coarse_shape())
    fb = g.pack(1, F64, b)
    fx = g.field(1, F64)
    tm.tm_coarse_solve(g.h, F64, fb, fx, 1e-11, 400)
    x = g.unpack(1, F64, fx, b.shape)
    assert np.linalg.norm(Dc.apply(x) - b) / np.linalg.norm(b) <= 1e-9


def _oracle_two_level(g, U, name, **over):
    L, eps, seed, m0, csw, mu, delta, nv, blk = CASES[name]
    prm = AMGParams(m0=m0, c_sw=csw, mu=mu, delta=delta, nv=nv, agg=blk, sap_block=blk,
                    mr_iters=g.p.mr_iters, pre_smooth=g.p.pre_smooth, post_smooth=g.p.post_smooth,
                    init_sweeps=g.p.init_sweeps, setup_iters=g.p.setup_iters,
                    coarse_tol=g.p.coarse_tol, coarse_restart=g.p.coarse_restart,
                    coarse_maxit=g.p.coarse_maxit, restart=g.p.restart, maxit=g.p.maxit)
    for k, v in over.items():
        setattr(prm, k, v)
    return TwoLevel(U, prm)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("pre", [0, 1])
def test_kcycle_fixed_coarse_steps(name, pre):
    U, g, op, seed = _case(name, F64, coarse_tol=0.0, coarse_maxit=9, pre_smooth=pre, post_smooth=2)
    tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
    tm.tm_setup_from_vectors(g.h, tv)
    tl = _oracle_two_level(g, U, name)
    tl.build_coarse(tv)
    v = inputs.gaussian_spinor(g.L, seed + 31, nrhs=2)
    fv = g.pack(0, F64, v, 2)
    fz = g.field(0, F64, 2)
    tm.tm_kcycle(g.h, F64, fv, fz, 2)
    got = g.unpack(0, F64, fz, v.shape, 2)
    for r in range(2):
        assert rel(got[r], tl.kcycle(v[r])) <= 1e-10


@pytest.mark.parametrize("name", OE_CASES)
def test_kcycle_odd_even_smoother_fixed_coarse_steps(name):
    U, g, op, seed = _case(name, F64, coarse_tol=0.0, coarse_maxit=9, pre_smooth=1, post_smooth=2, block_oe=1)
    tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
    tm.tm_setup_from_vectors(g.h, tv)
    tl = _oracle_two_level(g, U, name, block_oe=True)
    tl.sap = SAP(tl.op, tl.prm.sap_block, tl.prm.mr_iters, True)
    tl.build_coarse(tv)
    v = inputs.gaussian_spinor(g.L, seed + 31, nrhs=2)
    fv = g.pack(0, F64, v, 2)
    fz = g.field(0, F64, 2)
    tm.tm_kcycle(g.h, F64, fv, fz, 2)
    got = g.unpack(0, F64, fz, v.shape, 2)
    for r in range(2):
        assert rel(got[r], tl.kcycle(v[r])) <= 1e-10


@pytest.mark.parametrize("name", OE_CASES)
def test_solve_with_odd_even_smoother(name):
    U, g, op, seed = _case(name, F32, setup_iters=2, block_oe=1)
    tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
    tm.tm_setup(g.h, tv)
    b = inputs.gaussian_spinor(g.L, seed + 1000, nrhs=2)
    x = np.zeros_like(b)
    st, info = tm.tm_solve(g.h, b, x, 2, 1e-10)
    assert st == tm.TM_OK and info.converged
    for r in range(2):
        assert np.linalg.norm(b[r] - op.apply(x[r])) / np.linalg.norm(b[r]) <= 1e-10


@pytest.mark.parametrize("name", ["c1_4x4x4x4", "ragged_4x6x4x10"])
def test_adaptive_setup_matches_oracle(name):
    U, g, op, seed = _case(name, F64, setup_iters=1)
    tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
    tm.tm_setup(g.h, tv)
    tl = _oracle_two_level(g, U, name)
    tl.setup(tv)
    assert rel(g.export(tm.TM_EXPORT_TV, (g.nv,) + g.L + (4, 3)), tl.test_vectors) <= 1e-9
    assert rel(g.P_columns(), tl.P.columns()) <= 1e-9
    assert rel(g.Dc_blocks(), tl.Dc.blocks) <= 1e-9


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [F64, F32])
def test_solve_true_residual(name, prec):
    U, g, op, seed = _case(name, prec, setup_iters=2)
    tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
    tm.tm_setup(g.h, tv)
    b = inputs.gaussian_spinor(g.L, seed + 1000, nrhs=2)
    x = np.zeros_like(b)
    st, info = tm.tm_solve(g.h, b, x, 2, 1e-10)
    assert st == tm.TM_OK and info.converged
    for r in range(2):
        assert np.linalg.norm(b[r] - op.apply(x[r])) / np.linalg.norm(b[r]) <= 1e-10
    assert info.true_relres <= 1e-10


@pytest.mark.parametrize("name", list(CASES))
def test_solve_with_fp32_pair_outer_apply(name):
    """FGMRES whose D(mu) z_k products run in FP32 pairs: same outer iteration
    count as the FP64 products (the two Arnoldi relations agree to ~1e-14) and
    the oracle's FP64 true residual of the solution <= 1e-10."""
    iters = {}
    for oa in (tm.TM_F64, tm.TM_F32X2):
        U, g, op, seed = _case(name, F32, setup_iters=2, outer_apply=oa)
        tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
        tm.tm_setup(g.h, tv)
        b = inputs.gaussian_spinor(g.L, seed + 1000, nrhs=2)
        x = np.zeros_like(b)
        st, info = tm.tm_solve(g.h, b, x, 2, 1e-10)
        assert st == tm.TM_OK and info.converged
        for r in range(2):
            assert np.linalg.norm(b[r] - op.apply(x[r])) / np.linalg.norm(b[r]) <= 1e-10
        iters[oa] = info.iters
    assert abs(iters[tm.TM_F64] - iters[tm.TM_F32X2]) <= 1, iters


@pytest.mark.parametrize("name", OE_CASES)
@pytest.mark.parametrize("sp,tol", [(tm.TM_F16, 5e-3), (tm.TM_BF16, 3e-2)])
def test_sap_odd_even_blocks_16bit_operator(name, sp, tol):
    # links, clover and D_oo^-1 of the smoother stored in 16 bits, FP32 arithmetic:
    # the sweeps follow the oracle's exact-operator SAP to the format's rounding
    U, g, op, seed = _case(name, F32, block_oe=1, sap_prec=sp)
    sap = SAP(op, CASES[name][8], n_mr=4, block_oe=True)
    b = inputs.gaussian_spinor(g.L, seed + 11)
    x0 = 0.1 * inputs.gaussian_spinor(g.L, seed + 12)
    err = rel(g.sap(b, x0, 2, F32), sap.smooth(b, x0, 2))
    assert err <= tol
    assert err >= (1e-5 if sp == tm.TM_F16 else 1e-4)  # the 16-bit copy is the one read
    # a new twisted mass reaches the 16-bit inverses
    tm.tm_set_mu(g.h, -op.mu, g.p.delta)
    sapm = SAP(op.with_mu(-op.mu), CASES[name][8], n_mr=4, block_oe=True)
    assert rel(g.sap(b, x0, 1, F32), sapm.smooth(b, x0, 1)) <= tol


@pytest.mark.parametrize("opts", [dict(sap_prec=tm.TM_F16, transfer_prec=tm.TM_F16),
                                  dict(sap_prec=tm.TM_BF16, transfer_prec=tm.TM_BF16)])
def test_solve_with_16bit_preconditioner_operators(opts):
    # 16-bit operator copies inside the K-cycle change the preconditioner, not
    # the accuracy: the oracle's FP64 residual of the solution stays <= 1e-10
    name = "8x8x8x8"
    U, g, op, seed = _case(name, F32, setup_iters=2, block_oe=1, outer_apply=tm.TM_F32X2, **opts)
    tm.tm_setup(g.h, inputs.random_test_vectors(g.L, g.nv, seed + 2000))
    b = inputs.gaussian_spinor(g.L, seed + 1000, nrhs=2)
    x = np.zeros_like(b)
    st, info = tm.tm_solve(g.h, b, x, 2, 1e-10)
    assert st == tm.TM_OK and info.converged
    for r in range(2):
        assert np.linalg.norm(b[r] - op.apply(x[r])) / np.linalg.norm(b[r]) <= 1e-10


def test_solve_iterations_match_oracle_fp64():
    name = "c1_4x4x4x4"
    U, g, op, seed = _case(name, F64, setup_iters=2)
    tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
    tm.tm_setup(g.h, tv)
    tl = _oracle_two_level(g, U, name)
    tl.setup(tv)
    b = inputs.gaussian_spinor(g.L, seed + 1000)
    res = tl.solve(b, tol=1e-10)
    x = np.zeros_like(b)
    st, info = tm.tm_solve(g.h, b, x, 1, 1e-10)
    assert st == tm.TM_OK
    assert abs(info.iters - res.iters) <= max(1, int(0.1 * res.iters))
    assert rel(x, res.x) <= 1e-8


def test_device_pointers_and_mu_change():
    name = "8x8x8x8"
    U, g, op, seed = _case(name, F32, setup_iters=1)
    tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
    from tests.gpu_helpers import dev, host
    tm.tm_setup(g.h, dev(tv))
    b = inputs.gaussian_spinor(g.L, seed + 1000)
    for mu in (op.mu, -op.mu):  # one setup serves D(+mu) and D(-mu)
        tm.tm_set_mu(g.h, mu, g.p.delta)
        xd = dev(np.zeros_like(b))
        st, info = tm.tm_solve(g.h, dev(b), xd, 1, 1e-10)
        assert st == tm.TM_OK
        x = host(xd)
        opm = op.with_mu(mu)
        assert np.linalg.norm(b - opm.apply(x)) / np.linalg.norm(b) <= 1e-10


@pytest.mark.parametrize("name", list(CASES))
def test_kcycle_fp32_against_fp64_oracle(name):
    """The FP32 K-cycle (FP32 SAP, P, D_c, coarse GMRES) stays within FP32
    rounding (amplified by the nonlinear MR and GMRES steps) of the FP64
    oracle; the input arrives as an FP64 field, as in the solve."""
    U, g, op, seed = _case(name, F32, coarse_tol=0.0, coarse_maxit=9, post_smooth=2)
    tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
    tm.tm_setup_from_vectors(g.h, tv)
    tl = _oracle_two_level(g, U, name)
    tl.build_coarse(tv)
    v = inputs.gaussian_spinor(g.L, seed + 31)
    fv = g.pack(0, F32, v)
    fz = g.field(0, F32)
    tm.tm_kcycle(g.h, F32, fv, fz, 1)
    assert rel(g.unpack(0, F32, fz, v.shape), tl.kcycle(v)) <= 1e-4


@pytest.mark.parametrize("name", list(CASES))
def test_coarse_solve_fp32_fixed_steps(name):
    g, op, P, Dc, seed = _from_vectors(name, F32)
    rng = np.random.default_rng(seed + 3)
    b = rng.standard_normal(g.coarse_shape()) + 1j * rng.standard_normal(g.coarse_shape())
    oe = OddEvenCoarse(Dc)
    res = gmres(oe.schur, oe.reduced_rhs(b), tol=0.0, restart=g.p.coarse_restart, maxit=12)
    fb = g.pack(1, F32, b)
    fx = g.field(1, F32)
    assert tm.tm_coarse_solve(g.h, F32, fb, fx, 0.0, 12) == 12
    assert rel(g.unpack(1, F32, fx, b.shape), oe.reconstruct(b, res.x)) <= 1e-4


def test_mixed_precision_cycle_iterations():
    """FP32 cycle inside FP64 FGMRES needs about as many outer steps as the FP64 cycle."""
    L = (8, 8, 8, 8)
    U = inputs.gauge_field(L, 0.5, 5)
    b = inputs.gaussian_spinor(L, 1005)
    tv = inputs.random_test_vectors(L, 8, 2005)
    iters = {}
    for prec in (F64, F32):
        g = GPU(U, m0=-0.4, c_sw=1.5, mu=0.005, delta=5.0, nv=8, agg=(4, 4, 4, 4),
                sap_block=(4, 4, 4, 4), setup_iters=3, cycle_prec=prec)
        tm.tm_setup(g.h, tv)
        x = np.zeros_like(b)
        st, info = tm.tm_solve(g.h, b, x, 1, 1e-10)
        assert st == tm.TM_OK
        iters[prec] = info.iters
        g.close()
    assert iters[F32] <= 1.25 * iters[F64] + 2, iters


@pytest.mark.parametrize("prec", [F64, F32])
def test_batched_solve_matches_single_rhs_solves(prec):
    """nrhs independent FGMRES solves run in lock-step give each rhs what a
    single-rhs solve gives (up to rounding of the shared launches)."""
    name = "8x8x8x8"
    U, g, op, seed = _case(name, prec, setup_iters=1, max_rhs=12)
    tm.tm_setup(g.h, inputs.random_test_vectors(g.L, g.nv, seed + 2000))
    b = inputs.gaussian_spinor(g.L, seed + 1000, nrhs=3)
    xb = np.zeros_like(b)
    st, info = tm.tm_solve(g.h, b, xb, 3, 1e-10)
    assert st == tm.TM_OK and info.converged
    single_iters = 0
    for r in range(3):
        x = np.zeros_like(b[r])
        st1, i1 = tm.tm_solve(g.h, b[r], x, 1, 1e-10)
        assert st1 == tm.TM_OK
        single_iters += i1.iters
        assert rel(xb[r], x) <= 1e-8
        assert np.linalg.norm(b[r] - op.apply(xb[r])) / np.linalg.norm(b[r]) <= 1e-10
    assert abs(info.iters - single_iters) <= 3


def test_twelve_point_sources_batched():
    """The 12 spin-colour point sources at one site, solved in one batch."""
    name = "8x8x8x8"
    U, g, op, seed = _case(name, F32, setup_iters=2, max_rhs=12)
    tm.tm_setup(g.h, inputs.random_test_vectors(g.L, g.nv, seed + 2000))
    b, x0 = inputs.point_sources(g.L, seed + 1000)
    x = np.zeros_like(b)
    st, info = tm.tm_solve(g.h, b, x, 12, 1e-10)
    assert st == tm.TM_OK and info.converged
    for r in range(12):
        assert np.linalg.norm(b[r] - op.apply(x[r])) / np.linalg.norm(b[r]) <= 1e-10
