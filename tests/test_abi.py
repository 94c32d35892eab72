"""Host-side checks of the C ABI (no GPU needed).

The library must build for sm_103a, load, and export every entry point that
``include/tm.h`` declares; parameter validation runs before any device call,
so invalid parameters are rejected with TM_ERR_ARG even without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1611_01034_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_declares_exactly_the_header():
    from paper_1611_01034_gb300._binding import exported_symbols
    assert sorted(exported_symbols()) == _declared()


def test_defaults_and_status_strings(lib):
    import paper_1611_01034_gb300 as tm
    p = tm.tm_params_default()
    assert p.nv == 20 and list(p.agg) == [4, 4, 4, 4] and p.bc_t == -1.0
    assert p.cycle_prec == tm.TM_F32 and p.delta == 1.0
    assert p.levels == 2 and p.nv2 == 28 and list(p.agg2) == [2, 2, 2, 2] and list(p.sap_block1) == [2, 2, 2, 2]
    assert (p.pre_smooth1, p.post_smooth1, p.coarse_setup_iters, p.coarsest_maxit) == (0, 2, 3, 200)
    assert p.outer_apply == tm.TM_F64
    assert tm.tm_status_string(tm.TM_ERR_NOT_CONVERGED) == "not converged"
    assert tm.tm_status_string(12345) == "unknown status"


@pytest.mark.parametrize("bad", [
    dict(L=(4, 4, 4, 6), agg=(4, 4, 4, 4)),              # not divisible
    dict(L=(8, 8, 8, 12), agg=(2, 2, 2, 4)),             # odd coarse extent (3)
    dict(L=(8, 8, 8, 8), sap_block=(8, 4, 4, 4)),        # one SAP block in T
    dict(L=(8, 8, 8, 8), nv=40),                          # too many test vectors
    dict(L=(8, 8, 8, 8), delta=0.5),                      # delta < 1
    dict(L=(8, 8, 8, 8), cycle_prec=7),
    dict(L=(8, 8, 8, 8), bc_t=0.3),
    dict(L=(32, 32, 32, 32), agg=(8, 8, 8, 4)),          # aggregate volume > 1024
    dict(L=(8, 8, 8, 8), levels=4),
    dict(L=(8, 8, 8, 8), levels=3),                       # level-2 extents 1
    dict(L=(16, 16, 16, 16), levels=3, nv2=29),
    dict(L=(16, 16, 16, 16), levels=3, sap_block1=(4, 2, 2, 2)),  # one level-1 SAP block in T
    dict(L=(16, 16, 16, 16), levels=3, nv=20, agg2=(4, 2, 2, 2), sap_block1=(2, 2, 2, 2)),  # not divisible
    dict(L=(8, 8, 8, 8), coarse_mma=4),
    dict(L=(8, 8, 8, 8), coarse_mma=1, cycle_prec=0),     # tensor cores need the FP32 cycle
    dict(L=(8, 8, 8, 8), nn_mode=3),
    dict(L=(8, 8, 8, 8), nn_mode=1, cycle_prec=0),        # learned layer needs the FP32 cycle
    dict(L=(8, 8, 8, 8), nn_prec=7),
    dict(L=(8, 8, 8, 8), sap1_prec=2),                    # FP16 level-1 blocks need three levels
    dict(L=(8, 8, 8, 8), sap1_prec=3),                    # BF16 as well
    dict(L=(8, 8, 8, 8), transfer_prec=5),
    dict(L=(8, 8, 8, 8), transfer_prec=2, cycle_prec=0),  # 16-bit P copies need the FP32 cycle
    dict(L=(8, 8, 8, 8), sap_prec=2),                     # 16-bit SAP operator needs block_oe = 1
    dict(L=(8, 8, 8, 8), sap_prec=6, block_oe=1),
    dict(L=(8, 8, 8, 8), coarsest_steps=65),
    dict(L=(8, 8, 8, 8), coarsest_steps=-1),
    dict(L=(8, 8, 8, 8), restart=0),
    dict(L=(8, 8, 8, 8), restart=127),                    # Hessenberg column beyond the fixed bound
    dict(L=(8, 8, 8, 8), coarse_restart=200),
    dict(L=(8, 8, 8, 8), maxit=0),
    dict(L=(8, 8, 8, 8), max_rhs=0),
    dict(L=(8, 8, 8, 8), mr_iters=-1),
    dict(L=(8, 8, 8, 8), outer_apply=1),                  # only TM_F64 or TM_F32X2
    dict(L=(8, 8, 8, 8), outer_apply=4, cycle_prec=0),    # FP32 pairs need the FP32 cycle
    dict(L=(8, 8, 8, 8), block_oe=2),
    dict(L=(6, 6, 6, 6), agg=(3, 3, 3, 3), sap_block=(3, 3, 3, 3), block_oe=1),  # odd SAP block dims
])
def test_invalid_parameters_rejected_before_any_device_call(lib, bad):
    import paper_1611_01034_gb300 as tm
    kw = dict(L=(8, 8, 8, 8), agg=(4, 4, 4, 4), sap_block=(4, 4, 4, 4), nv=8)
    kw.update(bad)
    with pytest.raises(tm.TMError) as e:
        tm.tm_create(tm.params(**kw))
    assert e.value.status == tm.TM_ERR_ARG


def test_null_handle_calls_fail_cleanly(lib):
    import paper_1611_01034_gb300 as tm
    L = tm.lib()
    assert L.tm_solve(None, None, None, 1, 1e-10, None) == tm.TM_ERR_ARG
    assert L.tm_apply(None, 0, 0, None, None, 1) == tm.TM_ERR_ARG
    assert L.tm_synchronize(None) == tm.TM_ERR_ARG
    assert L.tm_autotune_build(None, None, 3, None) == tm.TM_ERR_ARG
    assert L.tm_set_mu(None, 0.01, 2.0) == tm.TM_ERR_ARG
    assert L.tm_setup_update(None, 1, 0) == tm.TM_ERR_ARG
    L.tm_destroy(None)


def test_names_the_tests_and_bench_use_exist():
    """Every ``tm.<name>`` that a test file or bench.py refers to is exported by
    the package (the GPU tests are skipped on a machine without a GPU, so a
    missing name would otherwise only show there)."""
    import glob
    import paper_1611_01034_gb300 as tm
    files = glob.glob(os.path.join(ROOT, "tests", "*.py")) + [os.path.join(ROOT, "bench.py"),
                                                           os.path.join(ROOT, "__graft_entry__.py")]
    missing = set()
    for f in files:
        for name in re.findall(r"\btm\.([A-Za-z_][A-Za-z0-9_]*)", open(f).read()):
            if name != "h" and not hasattr(tm, name):  # "tm.h" is the header
                missing.add((os.path.basename(f), name))
    assert not missing, sorted(missing)


def test_workspace_bytes_plan(lib):
    """The memory calculator needs no GPU: the 48^3 x 96 three-level benchmark
    handle with 4 right-hand sides per solve fits one GB300 (280 GB), one
    right-hand side needs less, more than max_rhs changes nothing, and
    invalid parameters give 0."""
    import paper_1611_01034_gb300 as tm
    kw = dict(L=(96, 48, 48, 48), m0=-0.59, c_sw=1.57551, mu=0.0009, delta=5.0, nv=24, agg=(4, 4, 4, 4),
              sap_block=(4, 4, 4, 4), levels=3, nv2=28, agg2=(2, 2, 2, 2), sap_block1=(2, 2, 2, 2), restart=8,
              max_rhs=4, coarse_mma=1, sap1_prec=tm.TM_F16, outer_apply=tm.TM_F32X2, block_oe=1,
              cycle_prec=tm.TM_F32)
    p = tm.params(**kw)
    b1, b4, b8 = (tm.tm_workspace_bytes(p, r) for r in (1, 4, 8))
    assert 100e9 < b1 < b4 <= 280e9
    assert b8 == b4
    # FP64 cycle: the smoother, P and D_c double
    assert tm.tm_workspace_bytes(tm.params(**dict(kw, cycle_prec=tm.TM_F64, coarse_mma=0, sap1_prec=tm.TM_F32,
                                                  outer_apply=tm.TM_F64)), 4) > b4
    # a 16-bit copy of P: nv fine fields of 4 bytes per complex number
    b16 = tm.tm_workspace_bytes(tm.params(**dict(kw, transfer_prec=tm.TM_BF16)), 4)
    assert b16 - b4 == 24 * 96 * 48 ** 3 * 12 * 4
    assert tm.tm_workspace_bytes(tm.params(**dict(kw, nv=40)), 1) == 0
    assert tm.tm_workspace_bytes(p, 0) == 0
