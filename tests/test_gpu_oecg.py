"""GPU oeCG (the comparison solver of Fig. 1, Sec. 1; the odd-even reduced
operator of Sec. 3) against oracle.oecg and dense / oracle operators.

The GPU iterates in FP32 inside FP64 defect correction and the oracle in
FP64, so iterates differ; what is unique is the solution.  Checks: the
oracle's true residual |b - D x| of the GPU solution is at most 1.05 tol |b|
(FP64 on both sides, the 5 % covers the different summation order of the
two residual evaluations); the GPU solution matches a dense LU solve (4^4)
or the oracle's oeCG solution (8^4) to cond * tol; an odd twisted-mass shift
rho and a start vector are honoured; maxit too small reports
TM_ERR_NOT_CONVERGED with the best iterate.
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator, dense_matrix
from oracle import oecg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1611_01034_gb300 as tm  # noqa: E402
from tests.gpu_helpers import GPU, rel  # noqa: E402

CASES = {
    # name: (L, eps, seed, m0, c_sw, mu, rho)
    "4x4x4x4": ((4, 4, 4, 4), 0.3, 1, -0.15, 1.0, 0.01, 0.07),
    "8x8x8x8": ((8, 8, 8, 8), 0.5, 5, -0.4, 1.5, 0.005, 0.0),
    "8x4x4x8": ((8, 4, 4, 8), 0.4, 9, -0.3, 1.2, -0.02, 0.03),
}


def _setup(name):
    L, eps, seed, m0, csw, mu, rho = CASES[name]
    U = inputs.gauge_field(L, eps, seed)
    g = GPU(U, m0=m0, c_sw=csw, mu=mu, nv=4, agg=(2, 2, 2, 2), sap_block=(2, 2, 2, 2))
    tm.tm_set_mu_eo(g.h, mu, mu + rho, 1.0)
    return U, g, Operator(U, m0, csw, mu, rho=rho), seed


@pytest.mark.parametrize("name", list(CASES))
def test_oecg_solution_has_the_oracle_residual(name):
    U, g, op, seed = _setup(name)
    tol = 1e-10
    b = inputs.gaussian_spinor(g.L, seed + 100, nrhs=2)
    x = np.zeros_like(b)
    st, info = tm.tm_solve_oecg(g.h, b, x, 2, tol)
    assert st == tm.TM_OK and info.converged
    assert info.iters > 0 and info.restarts >= 1 and info.true_relres <= tol
    for r in range(2):
        res = np.linalg.norm(b[r] - op.apply(x[r])) / np.linalg.norm(b[r])
        assert res <= 1.05 * tol, (r, res)


def test_oecg_matches_a_dense_solve():
    U, g, op, seed = _setup("4x4x4x4")
    b = inputs.gaussian_spinor(g.L, seed + 7)
    x = np.zeros_like(b)
    st, info = tm.tm_solve_oecg(g.h, b, x, 1, 1e-12)
    assert st == tm.TM_OK
    D = dense_matrix(op.apply, g.L)
    xd = np.linalg.solve(D, b.ravel())
    cond = np.linalg.cond(D)
    assert rel(x, xd) <= 1e-12 * cond * 2


def test_oecg_matches_the_oracle_oecg():
    U, g, op, seed = _setup("8x8x8x8")
    b = inputs.gaussian_spinor(g.L, seed + 8)
    x = np.zeros_like(b)
    st, info = tm.tm_solve_oecg(g.h, b, x, 1, 1e-11)
    assert st == tm.TM_OK
    xo, res = oecg.solve(op, b, tol=1e-11)
    assert res.converged
    # both solutions have residual <= 1e-11 |b|; their difference is bounded by |D^-1| 2e-11 |b|
    assert rel(x, xo) <= 1e-7


def test_oecg_start_vector_and_maxit():
    U, g, op, seed = _setup("8x4x4x8")
    b = inputs.gaussian_spinor(g.L, seed + 9)
    x = np.zeros_like(b)
    st, info = tm.tm_solve_oecg(g.h, b, x, 1, 1e-10)
    assert st == tm.TM_OK
    # starting from the solution needs no CG iteration
    x2 = x.copy()
    st, info2 = tm.tm_solve_oecg(g.h, b, x2, 1, 1e-9)
    assert st == tm.TM_OK and info2.iters == 0
    assert rel(x2, x) <= 1e-9
    # too few iterations: not converged, the residual went down
    x3 = np.zeros_like(b)
    st, info3 = tm.tm_solve_oecg(g.h, b, x3, 1, 1e-10, maxit=3)
    assert st == tm.TM_ERR_NOT_CONVERGED and not info3.converged and info3.iters <= 3
    assert np.linalg.norm(b - op.apply(x3)) < np.linalg.norm(b)
