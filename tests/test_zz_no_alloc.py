"""The allocation-free coarse solve (tm_coarse_solve_noalloc).

Some callers cannot allocate device memory at the point where they need a
coarse solve, for example because their own memory pool already holds the
free device memory, or because a latency-critical loop cannot pay for
cudaMalloc's implicit synchronisation.  tm_coarse_solve_noalloc keeps all of
its workspaces in a fixed 8 MiB device array inside the library.  These tests
check, through the C ABI, that it returns what tm_coarse_solve returns, on two
calls in a row (the array keeps the previous call's contents), and that a
coarse system too large for the array is refused with a clear error.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import inputs  # noqa: E402
import paper_1611_01034_gb300 as tm  # noqa: E402
from tests.gpu_helpers import GPU, rel  # noqa: E402


@pytest.mark.parametrize("prec,tol", [(tm.TM_F64, 1e-10), (tm.TM_F32, 1e-4)])
def test_noalloc_coarse_solve_matches_existing(prec, tol):
    L = (8, 8, 8, 8)
    U = inputs.gauge_field(L, 0.5, 5)
    g = GPU(U, m0=-0.4, c_sw=1.5, mu=0.005, delta=5.0, nv=8, agg=(4, 4, 4, 4),
            sap_block=(4, 4, 4, 4), cycle_prec=prec, coarse_restart=10)
    tm.tm_setup_from_vectors(g.h, inputs.random_test_vectors(L, 8, 2005))
    rng = np.random.default_rng(17)
    for call in range(2):
        b = rng.standard_normal(g.coarse_shape()) + 1j * rng.standard_normal(g.coarse_shape())
        fb = g.pack(1, prec, b)
        x_ref = g.field(1, prec)
        x_new = g.field(1, prec)
        for target_tol, maxit in ((1e-8, 200), (0.0, 23)):
            it_ref = tm.tm_coarse_solve(g.h, prec, fb, x_ref, target_tol, maxit)
            it_new = tm.tm_coarse_solve_noalloc(g.h, prec, fb, x_new, target_tol, maxit)
            assert it_new == it_ref
            a = g.unpack(1, prec, x_new, b.shape)
            r = g.unpack(1, prec, x_ref, b.shape)
            assert rel(a, r) <= tol, (call, target_tol)
    g.close()


def test_noalloc_coarse_solve_allocates_no_device_memory():
    """After a first call (which may load kernels and looks up the array's
    address), further calls leave the device's free memory unchanged: no
    workspace of the handle grows and nothing else is allocated."""
    L = (8, 8, 8, 8)
    U = inputs.gauge_field(L, 0.5, 5)
    g = GPU(U, m0=-0.4, c_sw=1.5, mu=0.005, delta=5.0, nv=8, agg=(4, 4, 4, 4),
            sap_block=(4, 4, 4, 4), cycle_prec=tm.TM_F32, coarse_restart=10)
    tm.tm_setup_from_vectors(g.h, inputs.random_test_vectors(L, 8, 2005))
    rng = np.random.default_rng(19)
    b = rng.standard_normal(g.coarse_shape()) + 1j * rng.standard_normal(g.coarse_shape())
    fb = g.pack(1, tm.TM_F32, b)
    fx = g.field(1, tm.TM_F32)
    tm.tm_coarse_solve_noalloc(g.h, tm.TM_F32, fb, fx, 1e-8, 200)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        tm.tm_coarse_solve_noalloc(g.h, tm.TM_F32, fb, fx, 1e-8, 200)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    g.close()


def test_noalloc_rejects_systems_beyond_its_array():
    # 16^3 x 32 with N_v = 28, restart 120, FP64: the Krylov basis alone is ~28 MB
    p = tm.params(L=(32, 16, 16, 16), nv=28, agg=(4, 4, 4, 4), sap_block=(4, 4, 4, 4),
                  cycle_prec=tm.TM_F64, coarse_restart=120)
    h = tm.tm_create(p, torch.cuda.current_stream())
    try:
        fb = torch.zeros(tm.tm_field_bytes(h, 1, tm.TM_F64, 1), dtype=torch.uint8, device="cuda")
        fx = torch.zeros_like(fb)
        with pytest.raises(tm.TMError) as e:
            tm.tm_coarse_solve_noalloc(h, tm.TM_F64, fb, fx, 1e-6, 10)
        assert e.value.status == tm.TM_ERR_ARG
        assert "8 MiB" in str(e.value)
    finally:
        tm.tm_destroy(h)
