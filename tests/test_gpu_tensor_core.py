"""Tensor-core odd-even Schur complement (tcgen05, TF32 with FP32 accumulation).

y_e = (D_ee - D_eo D_oo^-1 D_oe) v_e of the coarsest level through tm_schur,
against the FP64 oracle (Sec. 3, the odd-even reduced coarse system), for
1..24 right-hand sides per launch, operator shapes n = 2 N_v from 8 to 48
(K padded to a multiple of 8, M = 2n padded to 128 inside the MMA) and
lattices with fewer targets than SMs.

Tolerances (relative L2 against the FP64 oracle; the GPU coarse operator is
built in FP32): CUDA-core FP32 path 2e-5; 3xTF32 (operator and vectors split
into two TF32 parts) 2e-5; TF32 with only the vectors split, and plain TF32,
5e-3 (TF32 keeps 11 significant bits: unit roundoff 2^-11 = 4.9e-4 per
product, sums of 9 n terms).  Solves with the tensor-core coarse solve reach a
true FP64 residual of 1e-10.
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator
from oracle.coarse import Interpolation, CoarseOperator, OddEvenCoarse
from oracle.multilevel import ThreeLevel, ThreeLevelParams

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1611_01034_gb300 as tm  # noqa: E402
from tests.gpu_helpers import GPU, dev, rel  # noqa: E402

F32 = tm.TM_F32

CASES = {
    # name: (L, eps, seed, m0, c_sw, mu, delta, nv, agg, sap_block)
    "8x8x8x8_nv24": ((8, 8, 8, 8), 0.5, 21, -0.4, 1.5, 0.003, 5.0, 24, (2, 2, 2, 2), (4, 4, 4, 4)),
    "16x8x8x8_nv12": ((16, 8, 8, 8), 0.5, 22, -0.35, 1.5, 0.01, 2.0, 12, (2, 2, 2, 2), (4, 4, 4, 4)),
    "ragged_4x6x4x10_nv6": ((4, 6, 4, 10), 0.5, 3, -0.3, 1.5, 0.02, 3.0, 6, (2, 3, 2, 5), (2, 3, 2, 5)),
}
TOL = {0: 2e-5, 1: 5e-3, 2: 5e-3, 3: 2e-5}


def _two_level(name, mma, **over):
    L, eps, seed, m0, csw, mu, delta, nv, agg, blk = CASES[name]
    U = inputs.gauge_field(L, eps, seed)
    kw = dict(m0=m0, c_sw=csw, mu=mu, delta=delta, nv=nv, agg=agg, sap_block=blk, cycle_prec=F32,
              coarse_mma=mma, max_rhs=24)
    kw.update(over)
    g = GPU(U, **kw)
    tv = inputs.random_test_vectors(L, nv, seed + inputs.TV_SEED_OFFSET)
    tm.tm_setup_from_vectors(g.h, tv)
    op = Operator(U, m0, csw, mu)
    Dc = CoarseOperator.build(op, Interpolation(tv, agg), mu_c=delta * mu)
    return g, U, op, tv, OddEvenCoarse(Dc), seed


def _even_sites(Lc):
    c = np.indices(Lc).reshape(4, -1)
    return np.flatnonzero(c.sum(axis=0) % 2 == 0)


def _schur_case(g, oe, Lc, n, nrhs, seed):
    ev = _even_sites(Lc)
    v = inputs.random_coarse_vectors((len(ev),), n, nrhs, seed)      # compact even vectors
    full = np.zeros((nrhs, int(np.prod(Lc)), n), dtype=complex)
    full[:, ev] = v
    expect = np.stack([oe.schur(full[r].reshape(Lc + (n,))).reshape(-1, n)[ev] for r in range(nrhs)])
    fv = dev(v.astype(np.complex64).view(np.float32))
    fy = torch.zeros_like(fv)
    tm.tm_schur(g.h, F32, fv, fy, nrhs)
    torch.cuda.synchronize()
    got = fy.cpu().numpy().view(np.complex64).reshape(v.shape).astype(complex)
    return got, expect


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mma", [0, 1, 2, 3])
@pytest.mark.parametrize("nrhs", [1, 3, 12])
def test_schur_against_oracle(name, mma, nrhs):
    g, U, op, tv, oe, seed = _two_level(name, mma)
    n = 2 * g.nv
    got, expect = _schur_case(g, oe, g.Lc, n, nrhs, seed + 500 + nrhs)
    for r in range(nrhs):
        assert rel(got[r], expect[r]) <= TOL[mma], (r, rel(got[r], expect[r]))


def test_schur_24_rhs_and_mu_change():
    g, U, op, tv, oe, seed = _two_level("8x8x8x8_nv24", 3)
    L, eps, seed, m0, csw, mu, delta, nv, agg, blk = CASES["8x8x8x8_nv24"]
    got, expect = _schur_case(g, oe, g.Lc, 2 * nv, 24, seed + 600)
    assert max(rel(got[r], expect[r]) for r in range(24)) <= TOL[3]
    # the odd tiles carry D_oo^-1(delta mu): rebuilt by tm_set_mu
    tm.tm_set_mu(g.h, -mu, delta)
    Dc = CoarseOperator.build(Operator(U, m0, csw, -mu), Interpolation(tv, agg), mu_c=-delta * mu)
    got, expect = _schur_case(g, OddEvenCoarse(Dc), g.Lc, 2 * nv, 5, seed + 601)
    assert max(rel(got[r], expect[r]) for r in range(5)) <= TOL[3]


def test_schur_three_level_coarsest():
    L, AGG1, NV1, AGG2, NV2 = (8, 4, 4, 4), (2, 2, 2, 2), 6, (2, 1, 1, 1), 4
    U = inputs.gauge_field(L, 0.5, 7)
    g = GPU(U, m0=-0.3, c_sw=1.4, mu=0.05, delta=3.0, nv=NV1, agg=AGG1, sap_block=(2, 2, 2, 2), cycle_prec=F32,
            levels=3, nv2=NV2, agg2=AGG2, sap_block1=(2, 1, 1, 1), coarse_mma=3, max_rhs=4)
    prm = ThreeLevelParams(m0=-0.3, c_sw=1.4, mu=0.05, delta=3.0, nv=NV1, agg=AGG1, sap_block=(2, 2, 2, 2),
                           nv2=NV2, agg2=AGG2, sap_block1=(2, 1, 1, 1))
    tl = ThreeLevel(U, prm)
    Lc1 = tuple(L[d] // AGG1[d] for d in range(4))
    v0 = inputs.random_test_vectors(L, NV1, 2007)
    w0 = inputs.random_coarse_vectors(Lc1, 2 * NV1, NV2, 2008)
    tm.tm_setup_from_vectors(g.h, np.concatenate([v0.ravel(), w0.ravel()]))
    tl.build_level1(v0)
    tl.build_level2(w0)
    Lc2 = tuple(Lc1[d] // AGG2[d] for d in range(4))
    got, expect = _schur_case(g, tl.oe2, Lc2, 2 * NV2, 4, 77)
    for r in range(4):
        assert rel(got[r], expect[r]) <= TOL[3]


@pytest.mark.parametrize("mma", [1, 2, 3])
def test_solves_with_tensor_core_coarse_solve(mma):
    g, U, op, tv, oe, seed = _two_level("16x8x8x8_nv12", mma, setup_iters=2)
    tm.tm_setup(g.h, tv)
    b = inputs.gaussian_spinor(g.L, seed + inputs.RHS_SEED_OFFSET, nrhs=3)
    x = np.zeros_like(b)
    st, info = tm.tm_solve(g.h, b, x, 3, 1e-10)
    assert st == tm.TM_OK and info.converged and info.true_relres <= 1e-10
    for r in range(3):
        assert np.linalg.norm(b[r] - op.apply(x[r])) / np.linalg.norm(b[r]) <= 1e-10
    # same solve with the CUDA-core coarse solve: comparable outer iteration counts
    g0, *_ = _two_level("16x8x8x8_nv12", 0, setup_iters=2)
    tm.tm_setup(g0.h, tv)
    x0 = np.zeros_like(b)
    st0, info0 = tm.tm_solve(g0.h, b, x0, 3, 1e-10)
    assert st0 == tm.TM_OK
    assert info.iters <= 1.5 * info0.iters + 3


def test_bounded_waits_time_out_cleanly():
    """A tensor-core Schur application whose pipeline waits may poll only once
    gives up: the call returns TM_ERR_TIMEOUT (the kernel drained its copies and
    MMAs and freed its tensor memory), the handle keeps working, and a fresh
    handle on the same GPU still matches the oracle on the tensor cores."""
    g, U, op, tv, oe, seed = _two_level("8x8x8x8_nv24", 1, tc_spin_limit=1)
    n = 2 * g.nv
    with pytest.raises(tm.TMError) as e:
        _schur_case(g, oe, g.Lc, n, 12, seed + 700)
    assert e.value.status == tm.TM_ERR_TIMEOUT
    # the handle keeps working: the coarse operator on the CUDA cores
    v = inputs.random_coarse_vectors(g.Lc, n, 1, seed + 701).reshape(g.Lc + (n,))
    fo = g.field(1, F32)
    tm.tm_apply(g.h, 1, F32, g.pack(1, F32, v), fo, 1)
    assert rel(g.unpack(1, F32, fo, v.shape), oe.Dc.apply(v)) <= 1e-5
    g2, *_ = _two_level("8x8x8x8_nv24", 1)
    got, expect = _schur_case(g2, oe, g2.Lc, n, 12, seed + 702)
    assert max(rel(got[r], expect[r]) for r in range(12)) <= TOL[1]
