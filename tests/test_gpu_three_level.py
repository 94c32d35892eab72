"""GPU parity of the three-level hierarchy (Sec. 2) against ``oracle.multilevel``.

Every level-1 piece is called through the C ABI on the same seeded inputs as
the oracle: the level-1 aggregation P2 and D_c2, coarse SAP sweeps, P2 and
P2^dagger, D_c1(mu) and D_c2(delta mu) applies, the coarsest odd-even GMRES
with a fixed step count, the level-1 K-cycle and the fine K-cycle with fixed
inner step counts, the adaptive setup and full solves.

Tolerances (relative L2) as for two levels: FP64 single applies <= 1e-12,
fixed-count composites <= 1e-10, adaptive setup <= 1e-9.  The ragged case
has 3840 fine sites, 60-site fine aggregates, 5 and 3 test vectors (10 and 6
components per coarse site) and 2-site level-1 SAP blocks.
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator
from oracle.multilevel import CoarseSAP, ThreeLevel, ThreeLevelParams
from oracle.krylov import gmres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1611_01034_gb300 as tm  # noqa: E402
from tests.gpu_helpers import GPU, rel  # noqa: E402

F64, F32 = tm.TM_F64, tm.TM_F32

CASES = {
    # name: (L, eps, seed, m0, c_sw, mu, delta, nv, agg, sap_block, nv2, agg2, sap_block1)
    "8x4x4x4": ((8, 4, 4, 4), 0.5, 7, -0.3, 1.4, 0.05, 3.0, 6, (2, 2, 2, 2), (2, 2, 2, 2),
                4, (2, 1, 1, 1), (2, 1, 1, 1)),
    "ragged_8x6x4x20": ((8, 6, 4, 20), 0.5, 11, -0.35, 1.5, 0.02, 2.0, 5, (2, 3, 2, 5), (2, 3, 2, 5),
                        3, (2, 1, 1, 2), (1, 1, 1, 2)),
    "8x8x8x8": ((8, 8, 8, 8), 0.5, 5, -0.4, 1.5, 0.005, 5.0, 8, (2, 2, 2, 2), (4, 4, 4, 4),
                6, (2, 2, 2, 2), (2, 2, 2, 2)),
}


class Three:
    """GPU handle and oracle hierarchy on the same gauge field and parameters."""

    def __init__(self, name, prec=F64, **over):
        (L, eps, seed, m0, csw, mu, delta, nv, agg, blk, nv2, agg2, blk1) = CASES[name]
        self.seed = seed
        self.U = inputs.gauge_field(L, eps, seed)
        kw = dict(m0=m0, c_sw=csw, mu=mu, delta=delta, nv=nv, agg=agg, sap_block=blk, cycle_prec=prec,
                  max_rhs=4, levels=3, nv2=nv2, agg2=agg2, sap_block1=blk1)
        kw.update(over)
        self.g = GPU(self.U, **kw)
        p = self.g.p
        self.prm = ThreeLevelParams(
            m0=m0, c_sw=csw, mu=mu, delta=delta, nv=nv, agg=agg, sap_block=blk,
            mr_iters=p.mr_iters, pre_smooth=p.pre_smooth, post_smooth=p.post_smooth,
            init_sweeps=p.init_sweeps, setup_iters=p.setup_iters, coarse_tol=p.coarse_tol,
            coarse_restart=p.coarse_restart, coarse_maxit=p.coarse_maxit, restart=p.restart, maxit=p.maxit,
            nv2=nv2, agg2=agg2, sap_block1=blk1, mr_iters1=p.mr_iters1, pre_smooth1=p.pre_smooth1,
            post_smooth1=p.post_smooth1, init_sweeps1=p.init_sweeps1,
            coarse_setup_iters=p.coarse_setup_iters, coarsest_tol=p.coarsest_tol,
            coarsest_maxit=p.coarsest_maxit)
        self.tl = ThreeLevel(self.U, self.prm)
        self.L = tuple(L)
        self.Lc1 = tuple(L[d] // agg[d] for d in range(4))
        self.Lc2 = tuple(self.Lc1[d] // agg2[d] for d in range(4))
        self.n1, self.n2 = 2 * nv, 2 * nv2
        self.v0 = inputs.random_test_vectors(self.L, nv, seed + inputs.TV_SEED_OFFSET)
        self.w0 = inputs.random_coarse_vectors(self.Lc1, self.n1, nv2, seed + inputs.TV_SEED_OFFSET + 1)

    def vectors(self):
        return np.concatenate([self.v0.ravel(), self.w0.ravel()])

    def from_vectors(self):
        tm.tm_setup_from_vectors(self.g.h, self.vectors())
        self.tl.build_level1(self.v0)
        self.tl.build_level2(self.w0)

    def c1_shape(self, nrhs=None):
        s = self.Lc1 + (self.n1,)
        return s if nrhs is None else (nrhs,) + s

    def c2_shape(self, nrhs=None):
        s = self.Lc2 + (self.n2,)
        return s if nrhs is None else (nrhs,) + s

    def rand1(self, k, nrhs=None):
        return inputs.random_coarse_vectors(self.Lc1, self.n1, nrhs or 1, self.seed + 300 + k).reshape(
            self.c1_shape(nrhs))

    def rand2(self, k, nrhs=None):
        return inputs.random_coarse_vectors(self.Lc2, self.n2, nrhs or 1, self.seed + 400 + k).reshape(
            self.c2_shape(nrhs))


@pytest.mark.parametrize("name", list(CASES))
def test_level2_from_vectors(name):
    t = Three(name)
    t.from_vectors()
    g, tl = t.g, t.tl
    assert rel(g.P_columns(), tl.P1.columns()) <= 1e-12
    assert rel(g.Dc_blocks(), tl.Dc1.blocks) <= 1e-12
    assert rel(g.export(tm.TM_EXPORT_TV1, (g.p.nv2,) + t.c1_shape()), t.w0) <= 1e-15
    assert rel(g.export(tm.TM_EXPORT_P2, (t.n2,) + t.c1_shape()), tl.P2.columns()) <= 1e-12
    assert rel(g.export(tm.TM_EXPORT_DC2, t.Lc2 + (9, t.n2, t.n2)), tl.Dc2.blocks) <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("with_b", [True, False])
def test_coarse_sap_sweeps(name, with_b):
    t = Three(name)
    t.from_vectors()
    g = t.g
    b = t.rand1(1) if with_b else np.zeros(t.c1_shape(), dtype=complex)
    x0 = 0.3 * t.rand1(2)
    sap = CoarseSAP(t.tl.Dc1, g.p.sap_block1, g.p.mr_iters1)
    for sweeps in (1, 3):
        fx = g.pack(1, F64, x0)
        tm.tm_sap1(g.h, F64, g.pack(1, F64, b) if with_b else None, fx, sweeps, 1)
        assert rel(g.unpack(1, F64, fx, x0.shape), sap.smooth(b, x0, sweeps)) <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("sp,tol", [(tm.TM_F16, 5e-3), (tm.TM_BF16, 3e-2)])
def test_coarse_sap_16bit_blocks(name, sp, tol):
    # 16-bit copy of the level-1 blocks read by the smoother (FP16: 11, BF16: 8
    # significant bits; FP32 arithmetic)
    t = Three(name, F32, sap1_prec=sp)
    t.from_vectors()
    g = t.g
    b = t.rand1(1)
    x0 = 0.3 * t.rand1(2)
    sap = CoarseSAP(t.tl.Dc1, g.p.sap_block1, g.p.mr_iters1)
    fx = g.pack(1, F32, x0)
    tm.tm_sap1(g.h, F32, g.pack(1, F32, b), fx, 2, 1)
    assert rel(g.unpack(1, F32, fx, x0.shape), sap.smooth(b, x0, 2)) <= tol


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("sp", [tm.TM_F32, tm.TM_F16])
@pytest.mark.parametrize("nrhs", [3, 7])
def test_coarse_sap_batched_right_hand_sides(name, sp, nrhs):
    # several right-hand sides per CTA share the block-entry loads; each keeps
    # its own MR coefficients: the same sweeps as one right-hand side at a time
    t = Three(name, F32, sap1_prec=sp, max_rhs=8)
    t.from_vectors()
    g = t.g
    b = t.rand1(5, nrhs=nrhs)
    x0 = 0.3 * t.rand1(6, nrhs=nrhs)
    fx = g.pack(1, F32, x0, nrhs)
    tm.tm_sap1(g.h, F32, g.pack(1, F32, b, nrhs), fx, 2, nrhs)
    got = g.unpack(1, F32, fx, x0.shape, nrhs)
    sap = CoarseSAP(t.tl.Dc1, g.p.sap_block1, g.p.mr_iters1)
    tol = 5e-5 if sp == tm.TM_F32 else 5e-3
    for r in range(nrhs):
        fx1 = g.pack(1, F32, x0[r])
        tm.tm_sap1(g.h, F32, g.pack(1, F32, b[r]), fx1, 2, 1)
        one = g.unpack(1, F32, fx1, x0[r].shape)
        assert rel(got[r], one) <= 1e-6
        assert rel(got[r], sap.smooth(b[r], x0[r], 2)) <= tol


@pytest.mark.parametrize("name", list(CASES))
def test_level_transfers_and_applies(name):
    t = Three(name)
    t.from_vectors()
    g, tl = t.g, t.tl
    v1 = t.rand1(3, nrhs=2)
    v2 = t.rand2(4, nrhs=2)
    f1 = g.pack(1, F64, v1, 2)
    f2 = g.field(2, F64, 2)
    tm.tm_restrict1(g.h, F64, f1, f2, 2)
    got = g.unpack(2, F64, f2, v2.shape, 2)
    for r in range(2):
        assert rel(got[r], tl.P2.restrict(v1[r])) <= 1e-12
    f2 = g.pack(2, F64, v2, 2)
    tm.tm_prolong1(g.h, F64, f2, f1, 2, True)
    got = g.unpack(1, F64, f1, v1.shape, 2)
    for r in range(2):
        assert rel(got[r], v1[r] + tl.P2.prolong(v2[r])) <= 1e-12
    # level 1 keeps the fine twisted mass, level 2 carries delta mu
    f1 = g.pack(1, F64, v1, 2)
    o1 = g.field(1, F64, 2)
    tm.tm_apply(g.h, 1, F64, f1, o1, 2)
    got = g.unpack(1, F64, o1, v1.shape, 2)
    o2 = g.field(2, F64, 2)
    tm.tm_apply(g.h, 2, F64, f2, o2, 2)
    got2 = g.unpack(2, F64, o2, v2.shape, 2)
    for r in range(2):
        assert rel(got[r], tl.Dc1.apply(v1[r])) <= 1e-12
        assert rel(got2[r], tl.Dc2.apply(v2[r])) <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_coarsest_solve_fixed_steps(name):
    t = Three(name)
    t.from_vectors()
    g, tl = t.g, t.tl
    b = t.rand2(5)
    for steps in (1, 6, 40):
        res = gmres(tl.oe2.schur, tl.oe2.reduced_rhs(b), tol=0.0, restart=g.p.coarse_restart, maxit=steps)
        expect = tl.oe2.reconstruct(b, res.x)
        fx = g.field(2, F64)
        it = tm.tm_coarse_solve(g.h, F64, g.pack(2, F64, b), fx, 0.0, steps)
        assert it == steps == res.iters
        assert rel(g.unpack(2, F64, fx, b.shape), expect) <= 1e-10
    with pytest.raises(tm.TMError) as e:
        tm.tm_coarse_solve_noalloc(g.h, F64, g.pack(2, F64, b), g.field(2, F64), 1e-6, 10)
    assert e.value.status == tm.TM_ERR_ARG


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("pre1", [0, 1])
def test_level1_kcycle_fixed_steps(name, pre1):
    t = Three(name, coarsest_tol=0.0, coarsest_maxit=5, pre_smooth1=pre1, post_smooth1=2)
    t.from_vectors()
    g, tl = t.g, t.tl
    v = t.rand1(6, nrhs=2)
    fz = g.field(1, F64, 2)
    tm.tm_kcycle1(g.h, F64, g.pack(1, F64, v, 2), fz, 2)
    got = g.unpack(1, F64, fz, v.shape, 2)
    for r in range(2):
        assert rel(got[r], tl.kcycle1(v[r])) <= 1e-10


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("pre", [0, 1])
def test_fine_kcycle_fixed_steps(name, pre):
    t = Three(name, coarse_tol=0.0, coarse_maxit=3, coarsest_tol=0.0, coarsest_maxit=4, pre_smooth=pre,
              post_smooth=2)
    t.from_vectors()
    g, tl = t.g, t.tl
    v = inputs.gaussian_spinor(t.L, t.seed + 31, nrhs=2)
    fz = g.field(0, F64, 2)
    tm.tm_kcycle(g.h, F64, g.pack(0, F64, v, 2), fz, 2)
    got = g.unpack(0, F64, fz, v.shape, 2)
    for r in range(2):
        assert rel(got[r], tl.kcycle(v[r])) <= 1e-10


@pytest.mark.parametrize("name", ["8x4x4x4", "ragged_8x6x4x20"])
def test_three_level_adaptive_setup(name):
    t = Three(name, setup_iters=1, coarse_setup_iters=1)
    g, tl = t.g, t.tl
    tm.tm_setup(g.h, t.vectors())
    v, w = tl.setup(t.v0, t.w0)
    assert rel(g.export(tm.TM_EXPORT_TV, (g.p.nv,) + t.L + (4, 3)), v) <= 1e-9
    assert rel(g.export(tm.TM_EXPORT_TV1, (g.p.nv2,) + t.c1_shape()), w) <= 1e-9
    assert rel(g.export(tm.TM_EXPORT_P2, (t.n2,) + t.c1_shape()), tl.P2.columns()) <= 1e-9
    assert rel(g.export(tm.TM_EXPORT_DC2, t.Lc2 + (9, t.n2, t.n2)), tl.Dc2.blocks) <= 1e-9


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,sap1,tp", [(F64, 1, 1), (F32, 1, 1), (F32, 2, 1), (F32, 3, 2), (F32, 2, 3)])
def test_three_level_solve_true_residual(name, prec, sap1, tp):
    # 16-bit operator copies in the preconditioner do not limit the accuracy of the solution
    t = Three(name, prec, setup_iters=2, coarse_setup_iters=2, sap1_prec=sap1, transfer_prec=tp)
    g = t.g
    tm.tm_setup(g.h, t.vectors())
    op = Operator(t.U, t.prm.m0, t.prm.c_sw, t.prm.mu)
    b = inputs.gaussian_spinor(t.L, t.seed + inputs.RHS_SEED_OFFSET, nrhs=2)
    x = np.zeros_like(b)
    st, info = tm.tm_solve(g.h, b, x, 2, 1e-10)
    assert st == tm.TM_OK and info.converged and info.true_relres <= 1e-10
    for r in range(2):
        assert np.linalg.norm(b[r] - op.apply(x[r])) / np.linalg.norm(b[r]) <= 1e-10


def test_three_level_iterations_match_oracle_fp64():
    t = Three("8x4x4x4", F64, setup_iters=1, coarse_setup_iters=1)
    g, tl = t.g, t.tl
    tm.tm_setup(g.h, t.vectors())
    tl.setup(t.v0, t.w0)
    b = inputs.gaussian_spinor(t.L, t.seed + inputs.RHS_SEED_OFFSET)
    res = tl.solve(b, tol=1e-10)
    x = np.zeros_like(b)
    st, info = tm.tm_solve(g.h, b, x, 1, 1e-10)
    assert st == tm.TM_OK
    assert abs(info.iters - res.iters) <= max(1, int(0.1 * res.iters))
    assert rel(x, res.x) <= 1e-8


def test_three_level_batched_solve_and_mu_change():
    t = Three("8x8x8x8", F32, setup_iters=2, coarse_setup_iters=2, max_rhs=3)
    g = t.g
    tm.tm_setup(g.h, t.vectors())
    b = inputs.gaussian_spinor(t.L, t.seed + inputs.RHS_SEED_OFFSET, nrhs=3)
    for mu in (t.prm.mu, -t.prm.mu):
        tm.tm_set_mu(g.h, mu, t.prm.delta)
        op = Operator(t.U, t.prm.m0, t.prm.c_sw, mu)
        x = np.zeros_like(b)
        st, info = tm.tm_solve(g.h, b, x, 3, 1e-10)
        assert st == tm.TM_OK and info.converged
        for r in range(3):
            assert np.linalg.norm(b[r] - op.apply(x[r])) / np.linalg.norm(b[r]) <= 1e-10
