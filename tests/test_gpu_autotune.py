"""GPU checks of the build-shape autotuner: every candidate tile shape of the
D_c build must reproduce the default shape's blocks bit for bit (the tuner
refuses otherwise), the chosen shape is cached in JSON and taken from there
without timing, and a rebuild with the tuned shape gives the same D_c, which
still matches the oracle's Galerkin projection P^dagger D P (Sec. 1)."""
import json

import numpy as np
import pytest

import inputs
from oracle.coarse import CoarseOperator, Interpolation
from oracle.dirac import Operator

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1611_01034_gb300 as tm  # noqa: E402
from tests.gpu_helpers import GPU, rel  # noqa: E402


@pytest.mark.parametrize("prec", [tm.TM_F32, tm.TM_F64])
def test_autotune_build_parity_and_cache(tmp_path, prec):
    L, agg, nv = (8, 8, 8, 16), (4, 4, 4, 4), 12
    U = inputs.gauge_field(L, 0.5, 21)
    g = GPU(U, m0=-0.3, c_sw=1.5, mu=0.02, delta=3.0, nv=nv, agg=agg, sap_block=agg, cycle_prec=prec,
            max_rhs=1)
    tv = inputs.random_test_vectors(L, nv, 21 + inputs.TV_SEED_OFFSET)
    tm.tm_setup_from_vectors(g.h, tv)
    before = g.Dc_blocks()
    cache = tmp_path / "tune.json"
    first = tm.tm_autotune_build(g.h, str(cache), reps=2)
    assert first["timed"] >= 3 and first["us"] > 0
    assert 1 <= first["ts"] <= 16 and first["ktc"] in (2, 3, 4)
    entries = json.loads(cache.read_text())
    key = [k for k in entries if f"/k_coarse_build/{'fp32' if prec == tm.TM_F32 else 'fp64'}/nv{nv}/agg4x4x4x4" in k]
    assert len(key) == 1 and entries[key[0]]["ts"] == first["ts"] and entries[key[0]]["ktc"] == first["ktc"]
    # a second call takes the cached shape without timing
    again = tm.tm_autotune_build(g.h, str(cache), reps=2)
    assert again["timed"] == 0 and (again["ts"], again["ktc"]) == (first["ts"], first["ktc"])
    # the tuner leaves the D_c in use unchanged; a rebuild with the tuned shape is bit-identical
    assert np.array_equal(g.Dc_blocks(), before)
    tm.tm_setup_update(g.h, 0)
    assert np.array_equal(g.Dc_blocks(), before)
    # and it is still the oracle's projection of the same test vectors
    Dc = CoarseOperator.build(Operator(U, -0.3, 1.5, 0.02), Interpolation(tv, agg), mu_c=3.0 * 0.02)
    assert rel(g.Dc_blocks(), Dc.blocks) <= (1e-12 if prec == tm.TM_F64 else 5e-6)


def test_autotune_build_needs_setup_and_valid_reps():
    L = (8, 8, 8, 8)
    U = inputs.gauge_field(L, 0.5, 22)
    g = GPU(U, m0=-0.3, c_sw=1.5, mu=0.02, delta=3.0, nv=4, agg=(4, 4, 4, 4), sap_block=(4, 4, 4, 4))
    with pytest.raises(tm.TMError):
        tm.tm_autotune_build(g.h, None, reps=1)
    tv = inputs.random_test_vectors(L, 4, 22 + inputs.TV_SEED_OFFSET)
    tm.tm_setup(g.h, tv)
    with pytest.raises(tm.TMError):
        tm.tm_autotune_build(g.h, None, reps=0)
    res = tm.tm_autotune_build(g.h, None, reps=1)
    assert res["timed"] >= 1
