"""GPU parity at the benchmark's own operator shapes.

The benchmark runs N_v = 20 (two levels, 40 components per coarse site) and
N_v = 24 / N_v2 = 28 with 2^4 level-1 aggregates (three levels, 48 and 56
components, the coarsest Schur complement on the tensor cores at n = 56),
with 4^4 fine aggregates and SAP blocks.  These tests run exactly those
block sizes on small lattices the oracle handles in seconds:

* two levels, 16 x 8^3, N_v = 20: the K-cycle with a fixed coarse step count
  (FP64), the odd-even coarse GMRES with a fixed step count, the tensor-core
  Schur complement at n = 40 (1 and 12 right-hand sides), and a solve with
  the 16^3 x 32 benchmark's settings checked by the oracle's true residual;
* three levels, 16^4, N_v 24 / 28: P, D_c1, P2, D_c2 from given vectors,
  level-1 SAP (FP64 and FP16 blocks), the level-1 K-cycle with a fixed
  coarsest step count, the coarsest Schur complement at n = 56 on the tensor
  cores, and a four-point-source solve with the 48^3 x 96 benchmark's
  settings (FP32 pairs, odd-even SAP, FP16 level-1 blocks, TF32 coarsest,
  FGMRES(8)) checked by the oracle's true residual.

Tolerances as in the other GPU tests: FP64 single applies 1e-12, FP64
fixed-count composites 1e-10, FP16 level-1 blocks 5e-3, TF32 Schur 5e-3,
3xTF32 2e-5, solves 1e-10 by the oracle's FP64 residual.
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator
from oracle.coarse import Interpolation, CoarseOperator, OddEvenCoarse
from oracle.amg import TwoLevel, AMGParams
from oracle.multilevel import CoarseSAP, ThreeLevel, ThreeLevelParams
from oracle.krylov import gmres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1611_01034_gb300 as tm  # noqa: E402
from tests.gpu_helpers import GPU, dev, rel  # noqa: E402
from tests.test_gpu_tensor_core import _schur_case  # noqa: E402

F64, F32, F16 = tm.TM_F64, tm.TM_F32, tm.TM_F16

# two levels: the 16^3 x 32 benchmark's parameters on 16 x 8^3
L2 = (16, 8, 8, 8)
P2LVL = dict(m0=-0.4176881402499312, c_sw=1.5, mu=0.003, delta=5.0, nv=20, agg=(4, 4, 4, 4),
             sap_block=(4, 4, 4, 4))
SEED2 = 31


def _two(prec=F64, **over):
    U = inputs.gauge_field(L2, 0.5, SEED2)
    kw = dict(P2LVL, cycle_prec=prec, max_rhs=12)
    kw.update(over)
    g = GPU(U, **kw)
    tv = inputs.random_test_vectors(L2, 20, SEED2 + inputs.TV_SEED_OFFSET)
    return U, g, tv


def test_nv20_kcycle_fixed_coarse_steps():
    U, g, tv = _two(F64, coarse_tol=0.0, coarse_maxit=7, pre_smooth=1, post_smooth=2)
    tm.tm_setup_from_vectors(g.h, tv)
    prm = AMGParams(m0=P2LVL["m0"], c_sw=1.5, mu=0.003, delta=5.0, nv=20, agg=(4, 4, 4, 4),
                    sap_block=(4, 4, 4, 4), pre_smooth=1, post_smooth=2, coarse_tol=0.0, coarse_maxit=7)
    tl = TwoLevel(U, prm)
    tl.build_coarse(tv)
    v = inputs.gaussian_spinor(L2, SEED2 + 31, nrhs=2)
    fz = g.field(0, F64, 2)
    tm.tm_kcycle(g.h, F64, g.pack(0, F64, v, 2), fz, 2)
    got = g.unpack(0, F64, fz, v.shape, 2)
    for r in range(2):
        assert rel(got[r], tl.kcycle(v[r])) <= 1e-10
    # odd-even coarse GMRES with a fixed step count
    b = inputs.random_coarse_vectors(g.Lc, 40, 1, SEED2 + 41).reshape(g.Lc + (40,))
    res = gmres(tl.oe.schur, tl.oe.reduced_rhs(b), tol=0.0, restart=g.p.coarse_restart, maxit=12)
    fx = g.field(1, F64)
    assert tm.tm_coarse_solve(g.h, F64, g.pack(1, F64, b), fx, 0.0, 12) == 12
    assert rel(g.unpack(1, F64, fx, b.shape), tl.oe.reconstruct(b, res.x)) <= 1e-10


@pytest.mark.parametrize("mma,tol", [(1, 5e-3), (3, 2e-5)])
@pytest.mark.parametrize("nrhs", [1, 12])
def test_nv20_tensor_core_schur(mma, tol, nrhs):
    U, g, tv = _two(F32, coarse_mma=mma)
    tm.tm_setup_from_vectors(g.h, tv)
    op = Operator(U, P2LVL["m0"], 1.5, 0.003)
    oe = OddEvenCoarse(CoarseOperator.build(op, Interpolation(tv, (4, 4, 4, 4)), mu_c=5.0 * 0.003))
    got, expect = _schur_case(g, oe, g.Lc, 40, nrhs, SEED2 + 500 + nrhs)
    for r in range(nrhs):
        assert rel(got[r], expect[r]) <= tol


def test_nv20_solve_with_benchmark_settings():
    U, g, tv = _two(F32, coarse_mma=1, setup_iters=3)
    tm.tm_setup(g.h, tv)
    op = Operator(U, P2LVL["m0"], 1.5, 0.003)
    b = inputs.gaussian_spinor(L2, SEED2 + inputs.RHS_SEED_OFFSET, nrhs=2)
    x = np.zeros_like(b)
    st, info = tm.tm_solve(g.h, b, x, 2, 1e-10)
    assert st == tm.TM_OK and info.converged
    for r in range(2):
        assert np.linalg.norm(b[r] - op.apply(x[r])) / np.linalg.norm(b[r]) <= 1e-10


# ----------------------------------------------------------------------------
# three levels: the 48^3 x 96 benchmark's block sizes on 16^4
# ----------------------------------------------------------------------------
L3 = (16, 16, 16, 16)
SEED3 = 1
P3LVL = dict(m0=-0.5948514200964429, c_sw=1.57551, mu=0.0009, delta=5.0, nv=24, agg=(4, 4, 4, 4),
             sap_block=(4, 4, 4, 4), levels=3, nv2=28, agg2=(2, 2, 2, 2), sap_block1=(2, 2, 2, 2))
LC1 = (4, 4, 4, 4)
LC2 = (2, 2, 2, 2)


@pytest.fixture(scope="module")
def three():
    """Field, random vectors and the oracle hierarchy built from them (once)."""
    U = inputs.gauge_field(L3, 0.6, SEED3)
    v0 = inputs.random_test_vectors(L3, 24, SEED3 + inputs.TV_SEED_OFFSET)
    w0 = inputs.random_coarse_vectors(LC1, 48, 28, SEED3 + inputs.TV_SEED_OFFSET + 1)
    prm = ThreeLevelParams(m0=P3LVL["m0"], c_sw=1.57551, mu=0.0009, delta=5.0, nv=24, agg=(4, 4, 4, 4),
                           sap_block=(4, 4, 4, 4), nv2=28, agg2=(2, 2, 2, 2), sap_block1=(2, 2, 2, 2),
                           coarsest_tol=0.0, coarsest_maxit=5, pre_smooth1=1, post_smooth1=2)
    tl = ThreeLevel(U, prm)
    tl.build_level1(v0)
    tl.build_level2(w0)
    return U, v0, w0, tl


def _gpu3(U, prec, **over):
    kw = dict(P3LVL, cycle_prec=prec, max_rhs=12)
    kw.update(over)
    return GPU(U, **kw)


def test_nv24_28_hierarchy_from_vectors(three):
    U, v0, w0, tl = three
    g = _gpu3(U, F64)
    tm.tm_setup_from_vectors(g.h, np.concatenate([v0.ravel(), w0.ravel()]))
    assert rel(g.P_columns(), tl.P1.columns()) <= 1e-12
    assert rel(g.Dc_blocks(), tl.Dc1.blocks) <= 1e-12
    assert rel(g.export(tm.TM_EXPORT_P2, (56,) + LC1 + (48,)), tl.P2.columns()) <= 1e-12
    assert rel(g.export(tm.TM_EXPORT_DC2, LC2 + (9, 56, 56)), tl.Dc2.blocks) <= 1e-12
    # level-1 SAP on the 48-component stencil, FP64 and FP16 blocks
    b = inputs.random_coarse_vectors(LC1, 48, 1, 71).reshape(LC1 + (48,))
    x0 = 0.3 * inputs.random_coarse_vectors(LC1, 48, 1, 72).reshape(LC1 + (48,))
    expect = CoarseSAP(tl.Dc1, (2, 2, 2, 2), g.p.mr_iters1).smooth(b, x0, 2)
    fx = g.pack(1, F64, x0)
    tm.tm_sap1(g.h, F64, g.pack(1, F64, b), fx, 2, 1)
    assert rel(g.unpack(1, F64, fx, x0.shape), expect) <= 1e-12
    # level-1 K-cycle with a fixed coarsest step count
    g1 = _gpu3(U, F64, coarsest_tol=0.0, coarsest_maxit=5, pre_smooth1=1, post_smooth1=2)
    tm.tm_setup_from_vectors(g1.h, np.concatenate([v0.ravel(), w0.ravel()]))
    v = inputs.random_coarse_vectors(LC1, 48, 2, 73).reshape((2,) + LC1 + (48,))
    fz = g1.field(1, F64, 2)
    tm.tm_kcycle1(g1.h, F64, g1.pack(1, F64, v, 2), fz, 2)
    got = g1.unpack(1, F64, fz, v.shape, 2)
    for r in range(2):
        assert rel(got[r], tl.kcycle1(v[r])) <= 1e-10


def test_nv24_28_fp16_level1_blocks(three):
    U, v0, w0, tl = three
    g = _gpu3(U, F32, sap1_prec=F16)
    tm.tm_setup_from_vectors(g.h, np.concatenate([v0.ravel(), w0.ravel()]))
    b = inputs.random_coarse_vectors(LC1, 48, 1, 71).reshape(LC1 + (48,))
    x0 = 0.3 * inputs.random_coarse_vectors(LC1, 48, 1, 72).reshape(LC1 + (48,))
    fx = g.pack(1, F32, x0)
    tm.tm_sap1(g.h, F32, g.pack(1, F32, b), fx, 2, 1)
    expect = CoarseSAP(tl.Dc1, (2, 2, 2, 2), g.p.mr_iters1).smooth(b, x0, 2)
    assert rel(g.unpack(1, F32, fx, x0.shape), expect) <= 5e-3


@pytest.mark.parametrize("mma,tol", [(1, 5e-3), (3, 2e-5)])
@pytest.mark.parametrize("nrhs", [4, 12])
def test_nv28_tensor_core_schur_n56(three, mma, tol, nrhs):
    U, v0, w0, tl = three
    g = _gpu3(U, F32, coarse_mma=mma)
    tm.tm_setup_from_vectors(g.h, np.concatenate([v0.ravel(), w0.ravel()]))
    got, expect = _schur_case(g, tl.oe2, LC2, 56, nrhs, 900 + nrhs)
    for r in range(nrhs):
        assert rel(got[r], expect[r]) <= tol


def test_nv24_28_four_source_solve_with_benchmark_settings(three):
    U = three[0]
    g = _gpu3(U, F32, coarse_mma=1, sap1_prec=F16, outer_apply=tm.TM_F32X2, block_oe=1, restart=8,
              setup_iters=2, coarse_setup_iters=2, max_rhs=4)
    v0, w0 = three[1], three[2]
    tm.tm_setup(g.h, np.concatenate([v0.ravel(), w0.ravel()]))
    b, x0 = inputs.point_sources(L3, SEED3 + inputs.RHS_SEED_OFFSET)
    b = b[:4]
    xd = dev(np.zeros_like(b))
    st, info = tm.tm_solve(g.h, dev(b), xd, 4, 1e-10)
    assert st == tm.TM_OK and info.converged
    x = xd.cpu().numpy()
    op = Operator(U, P3LVL["m0"], 1.57551, 0.0009)
    for r in range(4):
        assert np.linalg.norm(b[r] - op.apply(x[r])) / np.linalg.norm(b[r]) <= 1e-10
