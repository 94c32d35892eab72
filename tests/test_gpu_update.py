"""GPU parity of the setup update after a gauge-field change (Sec. 3):
setup on U, tm_load_gauge(U'), tm_setup_update against the oracle's update
on U' from the same test vectors (FP64 cycle, composite tolerance 1e-9 as for
the adaptive setup), and a solve on U' after the update."""
import numpy as np
import pytest

import inputs
from oracle.amg import TwoLevel, AMGParams
from oracle.dirac import Operator
from oracle.multilevel import ThreeLevel, ThreeLevelParams

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1611_01034_gb300 as tm  # noqa: E402
from tests.gpu_helpers import GPU, dev, rel  # noqa: E402

F64, F32 = tm.TM_F64, tm.TM_F32


def test_two_level_update_matches_oracle():
    L = (4, 6, 4, 10)
    agg = (2, 3, 2, 5)
    U = inputs.gauge_field(L, 0.5, 3)
    U2 = inputs.evolve_gauge(U, 0.05, 91)
    g = GPU(U, m0=-0.3, c_sw=1.5, mu=0.02, delta=3.0, nv=6, agg=agg, sap_block=agg, cycle_prec=F64,
            setup_iters=1, max_rhs=2)
    tv = inputs.random_test_vectors(L, 6, 3 + inputs.TV_SEED_OFFSET)
    tm.tm_setup(g.h, tv)
    tm.tm_load_gauge(g.h, dev(U2))
    with pytest.raises(tm.TMError):
        tm.tm_solve(g.h, np.zeros((1,) + L + (4, 3), dtype=complex), np.zeros((1,) + L + (4, 3), dtype=complex),
                    1, 1e-10)
    tm.tm_setup_update(g.h, 1)
    prm = AMGParams(m0=-0.3, c_sw=1.5, mu=0.02, delta=3.0, nv=6, agg=agg, sap_block=agg,
                    mr_iters=g.p.mr_iters, pre_smooth=g.p.pre_smooth, post_smooth=g.p.post_smooth,
                    init_sweeps=g.p.init_sweeps, setup_iters=1, coarse_tol=g.p.coarse_tol,
                    coarse_restart=g.p.coarse_restart, coarse_maxit=g.p.coarse_maxit)
    a = TwoLevel(U, prm)
    a.setup(tv)
    b = TwoLevel(U2, prm)
    b.update(1, a.test_vectors)
    assert rel(g.export(tm.TM_EXPORT_TV, (6,) + L + (4, 3)), b.test_vectors) <= 1e-9
    assert rel(g.Dc_blocks(), b.Dc.blocks) <= 1e-9
    rhs = inputs.gaussian_spinor(L, 1003)[None]
    x = np.zeros_like(rhs)
    st, info = tm.tm_solve(g.h, rhs, x, 1, 1e-10)
    assert st == tm.TM_OK and info.converged
    op = Operator(U2, -0.3, 1.5, 0.02)
    assert np.linalg.norm(rhs[0] - op.apply(x[0])) / np.linalg.norm(rhs[0]) <= 1e-10


def test_three_level_update_matches_oracle():
    L, agg1, nv1, agg2, nv2 = (8, 4, 4, 4), (2, 2, 2, 2), 6, (2, 1, 1, 1), 4
    U = inputs.gauge_field(L, 0.5, 7)
    U2 = inputs.evolve_gauge(U, 0.05, 92)
    g = GPU(U, m0=-0.3, c_sw=1.4, mu=0.05, delta=3.0, nv=nv1, agg=agg1, sap_block=(2, 2, 2, 2), cycle_prec=F64,
            levels=3, nv2=nv2, agg2=agg2, sap_block1=(2, 1, 1, 1), setup_iters=1, coarse_setup_iters=1)
    Lc1 = tuple(L[d] // agg1[d] for d in range(4))
    v0 = inputs.random_test_vectors(L, nv1, 7 + inputs.TV_SEED_OFFSET)
    w0 = inputs.random_coarse_vectors(Lc1, 2 * nv1, nv2, 7 + inputs.TV_SEED_OFFSET + 1)
    tm.tm_setup(g.h, np.concatenate([v0.ravel(), w0.ravel()]))
    tm.tm_load_gauge(g.h, dev(U2))
    tm.tm_setup_update(g.h, 1, 3)
    p = g.p
    prm = ThreeLevelParams(m0=-0.3, c_sw=1.4, mu=0.05, delta=3.0, nv=nv1, agg=agg1, sap_block=(2, 2, 2, 2),
                           mr_iters=p.mr_iters, pre_smooth=p.pre_smooth, post_smooth=p.post_smooth,
                           init_sweeps=p.init_sweeps, setup_iters=1, coarse_tol=p.coarse_tol,
                           coarse_restart=p.coarse_restart, coarse_maxit=p.coarse_maxit, nv2=nv2, agg2=agg2,
                           sap_block1=(2, 1, 1, 1), coarse_setup_iters=1)
    a = ThreeLevel(U, prm)
    a.setup(v0, w0)
    b = ThreeLevel(U2, prm)
    b.update(1, 3, a.test_vectors, a.test_vectors1)
    assert rel(g.export(tm.TM_EXPORT_TV1, (nv2,) + Lc1 + (2 * nv1,)), b.test_vectors1) <= 1e-9
    Lc2 = tuple(Lc1[d] // agg2[d] for d in range(4))
    assert rel(g.export(tm.TM_EXPORT_DC2, Lc2 + (9, 2 * nv2, 2 * nv2)), b.Dc2.blocks) <= 1e-9


def test_update_needs_an_earlier_setup():
    L = (4, 4, 4, 4)
    g = GPU(inputs.gauge_field(L, 0.3, 1), m0=-0.2, c_sw=1.0, mu=0.01, nv=8, agg=(2, 2, 2, 2),
            sap_block=(2, 2, 2, 2))
    with pytest.raises(tm.TMError) as e:
        tm.tm_setup_update(g.h, 1)
    assert e.value.status == tm.TM_ERR_STATE
