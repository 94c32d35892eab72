"""GPU parity of the even/odd twisted mass and the Hasenbusch solves (Sec. 2
and Sec. 3) against oracle.dirac (Operator with the odd shift rho) and
oracle.evenodd.

Tolerances: FP64 applies 1e-12, FP32 5e-6, FP32 pairs 1e-13, FP64 SAP
sweeps and coarse blocks 1e-12 / 1e-10 as elsewhere.  Reduced solves: the
full system is solved to 1e-10 and the reduced residual r_o - D_oe D_ee^-1
r_e is at most a few times that (1e-9); the Hasenbusch pair is checked by
A A^dagger x = b on the odd sites, whose error grows with the condition of A
(1e-7).
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator, site_parity
from oracle.sap import SAP
from oracle.coarse import Interpolation, CoarseOperator
from oracle.multilevel import ThreeLevel, ThreeLevelParams
from oracle import evenodd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1611_01034_gb300 as tm  # noqa: E402
from tests.gpu_helpers import GPU, rel  # noqa: E402

F64, F32 = tm.TM_F64, tm.TM_F32
CASES = {
    # name: (L, eps, seed, m0, c_sw, mu, rho, delta, nv, agg / sap block)
    "4x4x4x4": ((4, 4, 4, 4), 0.3, 1, -0.15, 1.0, 0.01, 0.07, 2.0, 8, (2, 2, 2, 2)),
    "8x8x8x8": ((8, 8, 8, 8), 0.5, 5, -0.4, 1.5, 0.005, 0.02, 5.0, 8, (4, 4, 4, 4)),
}


def _case(name, prec, **over):
    L, eps, seed, m0, csw, mu, rho, delta, nv, blk = CASES[name]
    U = inputs.gauge_field(L, eps, seed)
    kw = dict(m0=m0, c_sw=csw, mu=mu, delta=delta, nv=nv, agg=blk, sap_block=blk, cycle_prec=prec, max_rhs=2)
    kw.update(over)
    g = GPU(U, **kw)
    tm.tm_set_mu_eo(g.h, mu, mu + rho, delta)
    return U, g, Operator(U, m0, csw, mu, rho=rho), seed


@pytest.mark.parametrize("name", list(CASES))
def test_apply_with_odd_shift(name):
    for prec, tol, over in ((F64, 1e-12, {}), (F32, 5e-6, {}), (tm.TM_F32X2, 1e-13, {"outer_apply": tm.TM_F32X2})):
        U, g, op, seed = _case(name, F64 if prec == F64 else F32, **over)
        psi = inputs.gaussian_spinor(g.L, seed + 5, nrhs=2)
        if prec == tm.TM_F32X2:
            psi = psi.astype(np.complex64).astype(complex)
            fo = g.field(0, F64, 2)
            tm.tm_apply(g.h, 0, prec, g.pack(0, F32, psi, 2), fo, 2)
            got = g.unpack(0, F64, fo, psi.shape, 2)
        else:
            got = g.apply_fine(psi, prec, nrhs=2)
        for r in range(2):
            assert rel(got[r], op.apply(psi[r])) <= tol, prec
    # the shift only acts on odd sites: its contribution is i rho gamma5 psi there
    assert np.any(site_parity(g.L) == 1)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("block_oe", [0, 1])
def test_sap_with_odd_shift(name, block_oe):
    U, g, op, seed = _case(name, F64, block_oe=block_oe)
    sap = SAP(op, CASES[name][9], n_mr=4, block_oe=bool(block_oe))
    b = inputs.gaussian_spinor(g.L, seed + 11)
    x0 = 0.1 * inputs.gaussian_spinor(g.L, seed + 12)
    assert rel(g.sap(b, x0, 2, F64), sap.smooth(b, x0, 2)) <= 1e-10


@pytest.mark.parametrize("name", list(CASES))
def test_coarse_operator_with_odd_shift(name):
    U, g, op, seed = _case(name, F64)
    blk = CASES[name][9]
    tv = inputs.random_test_vectors(g.L, g.nv, seed + 2000)
    tm.tm_setup_from_vectors(g.h, tv)
    P = Interpolation(tv, blk)
    assert rel(g.Dc_blocks(), CoarseOperator.build(op, P, mu_c=0.0).blocks) <= 1e-12
    # another shift: D_c projected again from the same P
    mu = op.mu
    tm.tm_set_mu_eo(g.h, -mu, -mu - 0.03, g.p.delta)
    op2 = op.with_mu_eo(-mu, -mu - 0.03)
    assert rel(g.Dc_blocks(), CoarseOperator.build(op2, P, mu_c=0.0).blocks) <= 1e-12
    assert rel(g.apply_fine(inputs.gaussian_spinor(g.L, 3), F64), op2.apply(inputs.gaussian_spinor(g.L, 3))) <= 1e-12


def test_three_level_coarse_operators_with_odd_shift():
    L, agg, nv, agg2, nv2 = (8, 8, 8, 8), (2, 2, 2, 2), 6, (2, 2, 2, 2), 4
    U = inputs.gauge_field(L, 0.5, 5)
    mu, rho, delta = 0.005, 0.02, 5.0
    g = GPU(U, m0=-0.4, c_sw=1.5, mu=mu, delta=delta, nv=nv, agg=agg, sap_block=(4, 4, 4, 4), cycle_prec=F64,
            levels=3, nv2=nv2, agg2=agg2, sap_block1=(2, 2, 2, 2))
    tm.tm_set_mu_eo(g.h, mu, mu + rho, delta)
    Lc1 = tuple(L[d] // agg[d] for d in range(4))
    v0 = inputs.random_test_vectors(L, nv, 2005)
    w0 = inputs.random_coarse_vectors(Lc1, 2 * nv, nv2, 2006)
    tm.tm_setup_from_vectors(g.h, np.concatenate([v0.ravel(), w0.ravel()]))
    prm = ThreeLevelParams(m0=-0.4, c_sw=1.5, mu=mu, delta=delta, nv=nv, agg=agg, sap_block=(4, 4, 4, 4), nv2=nv2,
                           agg2=agg2, sap_block1=(2, 2, 2, 2), rho=rho)
    tl = ThreeLevel(U, prm)
    tl.build_level1(v0)
    tl.build_level2(w0)
    Lc2 = tuple(Lc1[d] // agg2[d] for d in range(4))
    assert rel(g.Dc_blocks(), tl.Dc1.blocks) <= 1e-12
    assert rel(g.export(tm.TM_EXPORT_DC2, Lc2 + (9, 2 * nv2, 2 * nv2)), tl.Dc2.blocks) <= 1e-12


def _reduced_residual(op, x, b):
    od = op.odd[..., None, None]
    return np.linalg.norm(evenodd.reduced_apply(op, x) - b * od) / np.linalg.norm(b * od)


@pytest.mark.parametrize("name", list(CASES))
def test_reduced_solve(name):
    U, g, op, seed = _case(name, F32, setup_iters=2, block_oe=1)
    tm.tm_setup(g.h, inputs.random_test_vectors(g.L, g.nv, seed + 2000))
    tm.tm_set_mu_eo(g.h, op.mu, op.mu + op.rho, g.p.delta)
    b = inputs.gaussian_spinor(g.L, seed + 1000, nrhs=2)
    x = np.zeros_like(b)
    st, info = tm.tm_solve_odd(g.h, b, x, 2, 1e-10)
    assert st == tm.TM_OK and info.converged
    for r in range(2):
        assert np.all(x[r][site_parity(g.L) == 0] == 0)
        assert _reduced_residual(op, x[r], b[r]) <= 1e-9


@pytest.mark.parametrize("name", list(CASES))
def test_hasenbusch_pair(name):
    U, g, op, seed = _case(name, F32, setup_iters=2)
    tm.tm_setup(g.h, inputs.random_test_vectors(g.L, g.nv, seed + 2000))
    mu, rho = op.mu, op.rho
    b = inputs.gaussian_spinor(g.L, seed + 1001, nrhs=2)
    x = np.zeros_like(b)
    st, info = tm.tm_solve_hasenbusch(g.h, b, x, 2, mu, rho, 1e-10)
    assert st == tm.TM_OK and info.converged
    op_p = op.with_mu_eo(mu, mu + rho)
    op_m = op.with_mu_eo(-mu, -mu - rho)

    def A(v):
        return evenodd.reduced_apply(op_p, v)

    def A_dag(v):
        return evenodd.gamma5(evenodd.reduced_apply(op_m, evenodd.gamma5(v)))

    for r in range(2):
        bo = evenodd.restrict_odd(op, b[r])
        assert np.linalg.norm(A(A_dag(x[r])) - bo) <= 1e-7 * np.linalg.norm(bo)
    # the handle is left at the first operator of the pair
    psi = inputs.gaussian_spinor(g.L, 9)
    assert rel(g.apply_fine(psi, F64), op_p.apply(psi)) <= 1e-12


def test_squared_solve_with_odd_shift():
    U, g, op, seed = _case("8x8x8x8", F32, setup_iters=2)
    tm.tm_setup(g.h, inputs.random_test_vectors(g.L, g.nv, seed + 2000))
    b = inputs.gaussian_spinor(g.L, seed + 1002)
    x = np.zeros_like(b)
    st, info = tm.tm_solve_squared(g.h, b, x, 1, 1e-11)
    assert st == tm.TM_OK
    Dx = op.apply(x)
    DdDx = evenodd.gamma5(op.with_mu_eo(-op.mu, -op.mu - op.rho).apply(evenodd.gamma5(Dx)))
    assert np.linalg.norm(DdDx - b) <= 1e-8 * np.linalg.norm(b)
