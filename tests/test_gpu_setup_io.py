"""Setup files and the memory calculator on the GPU.

tm_save_setup / tm_load_setup (Sec. 3: one setup serves many inversions and
is carried along an HMC trajectory): a handle that loads a saved setup on the
same gauge field reproduces the saving handle's P, D_c (and P2, D_c2) and its
solve bit for bit, for two and three levels; foreign or mismatched files are
refused.  tm_workspace_bytes: the device memory a handle really holds after
a setup and a solve is below the plan and not far from it.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import inputs  # noqa: E402
import paper_1611_01034_gb300 as tm  # noqa: E402
from tests.gpu_helpers import GPU  # noqa: E402

F32 = tm.TM_F32

CASES = {
    "two_level_8^4": dict(L=(8, 8, 8, 8), m0=-0.4, c_sw=1.5, mu=0.005, delta=5.0, nv=8, agg=(4, 4, 4, 4),
                          sap_block=(4, 4, 4, 4), cycle_prec=F32, coarse_mma=1, max_rhs=2, setup_iters=2),
    "three_level_8^4": dict(L=(8, 8, 8, 8), m0=-0.4, c_sw=1.5, mu=0.005, delta=5.0, nv=8, agg=(2, 2, 2, 2),
                            sap_block=(4, 4, 4, 4), levels=3, nv2=6, agg2=(2, 2, 2, 2), sap_block1=(2, 2, 2, 2),
                            cycle_prec=F32, coarse_mma=1, sap1_prec=tm.TM_F16, max_rhs=2, setup_iters=1,
                            coarse_setup_iters=1, block_oe=1),
}


def _vectors(kw, seed):
    L = kw["L"]
    tv = inputs.random_test_vectors(L, kw["nv"], seed)
    if kw.get("levels") == 3:
        Lc1 = tuple(L[d] // kw["agg"][d] for d in range(4))
        w0 = inputs.random_coarse_vectors(Lc1, 2 * kw["nv"], kw["nv2"], seed + 1)
        return np.concatenate([tv.ravel(), w0.ravel()])
    return tv


def _solve(g, b):
    x = np.zeros_like(b)
    st, info = tm.tm_solve(g.h, b, x, b.shape[0], 1e-10)
    assert st == tm.TM_OK and info.converged
    return x, info


@pytest.mark.parametrize("name", list(CASES))
def test_saved_setup_reproduces_the_solve(name, tmp_path):
    kw = CASES[name]
    U = inputs.gauge_field(kw["L"], 0.5, 5)
    g1 = GPU(U, **kw)
    tm.tm_setup(g1.h, _vectors(kw, 77))
    b = inputs.gaussian_spinor(kw["L"], 78, nrhs=2)
    x1, info1 = _solve(g1, b)
    path = os.path.join(tmp_path, "setup.bin")
    tm.tm_save_setup(g1.h, path)
    g2 = GPU(U, **kw)
    with pytest.raises(tm.TMError) as e:  # no setup yet
        tm.tm_solve(g2.h, b, np.zeros_like(b), 2, 1e-10)
    assert e.value.status == tm.TM_ERR_STATE
    tm.tm_load_setup(g2.h, path)
    assert np.array_equal(g2.P_columns(), g1.P_columns())
    assert np.array_equal(g2.Dc_blocks(), g1.Dc_blocks())
    if kw.get("levels") == 3:
        Lc1 = tuple(kw["L"][d] // kw["agg"][d] for d in range(4))
        n2 = 2 * kw["nv2"]
        shape = (n2,) + Lc1 + (2 * kw["nv"],)
        assert np.array_equal(g2.export(tm.TM_EXPORT_P2, shape), g1.export(tm.TM_EXPORT_P2, shape))
    x2, info2 = _solve(g2, b)
    assert info2.iters == info1.iters
    assert np.array_equal(x2, x1)
    # a setup update on the loaded handle runs from the loaded test vectors
    tm.tm_setup_update(g2.h, 1, 1 if kw.get("levels") == 3 else 0)
    _solve(g2, b)


def test_mismatched_or_foreign_files_are_refused(tmp_path):
    kw = CASES["two_level_8^4"]
    U = inputs.gauge_field(kw["L"], 0.5, 5)
    g1 = GPU(U, **kw)
    tm.tm_setup(g1.h, _vectors(kw, 77))
    path = os.path.join(tmp_path, "setup.bin")
    tm.tm_save_setup(g1.h, path)
    g_other = GPU(U, **dict(kw, nv=6))
    with pytest.raises(tm.TMError) as e:
        tm.tm_load_setup(g_other.h, path)
    assert e.value.status == tm.TM_ERR_ARG
    junk = os.path.join(tmp_path, "junk.bin")
    open(junk, "wb").write(b"not a setup" * 100)
    with pytest.raises(tm.TMError) as e:
        tm.tm_load_setup(g1.h, junk)
    assert e.value.status == tm.TM_ERR_ARG
    with pytest.raises(tm.TMError) as e:
        tm.tm_load_setup(g1.h, os.path.join(tmp_path, "missing.bin"))
    assert e.value.status == tm.TM_ERR_ARG


@pytest.mark.parametrize("name", list(CASES))
def test_workspace_plan_bounds_the_memory_held(name):
    kw = dict(CASES[name], L=(16, 16, 16, 16))
    U = inputs.gauge_field(kw["L"], 0.5, 9)
    Ud = torch.from_numpy(U).cuda()
    tv = torch.from_numpy(_vectors(kw, 91)).cuda()
    b = torch.from_numpy(inputs.gaussian_spinor(kw["L"], 92, nrhs=2)).cuda()
    x = torch.zeros_like(b)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    p = tm.params(**kw)
    h = tm.tm_create(p, torch.cuda.current_stream())
    try:
        tm.tm_load_gauge(h, Ud)
        tm.tm_setup(h, tv)
        st, info = tm.tm_solve(h, b, x, 2, 1e-10)
        assert st == tm.TM_OK
        torch.cuda.synchronize()
        held = free0 - torch.cuda.mem_get_info()[0]
        plan = tm.tm_workspace_bytes(p, 2)
        # lazily loaded kernel code may add a few MB to what the handle holds
        assert held <= plan + (128 << 20), (plan, held)
        assert plan <= 1.3 * held + (64 << 20), (plan, held)
    finally:
        tm.tm_destroy(h)
