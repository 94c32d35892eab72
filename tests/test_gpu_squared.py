"""GPU: one setup serves D(+mu) and D(-mu), and the squared-operator solve
(Sec. 1 and Sec. 3 of the paper) through the C ABI, checked by the oracle.

The oracle recomputes D(mu)^dagger D(mu) x with D(mu)^dagger applied as
Gamma5 D(-mu) Gamma5 (pinned against the dense adjoint on CPU) and requires
it to reproduce b; the +mu and -mu solves with the same setup must need a
comparable number of outer iterations (the Fig. 2 statement on stability).
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator, gamma5_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1611_01034_gb300 as tm  # noqa: E402
from tests.gpu_helpers import GPU  # noqa: E402


@pytest.mark.parametrize("prec", [tm.TM_F64, tm.TM_F32])
def test_squared_solve_and_sign_of_mu(prec):
    L = (8, 8, 8, 8)
    U = inputs.gauge_field(L, 0.5, 5)
    m0, csw, mu = -0.4, 1.5, 0.005
    g = GPU(U, m0=m0, c_sw=csw, mu=mu, delta=5.0, nv=8, agg=(4, 4, 4, 4), sap_block=(4, 4, 4, 4),
            setup_iters=2, cycle_prec=prec, max_rhs=2)
    tm.tm_setup(g.h, inputs.random_test_vectors(L, 8, 2005))
    op = Operator(U, m0, csw, mu)
    opm = op.with_mu(-mu)
    b = inputs.gaussian_spinor(L, 1005, nrhs=2)
    iters = {}
    for sgn in (+1, -1):
        tm.tm_set_mu(g.h, sgn * mu, 5.0)
        x = np.zeros_like(b)
        st, info = tm.tm_solve(g.h, b, x, 2, 1e-10)
        assert st == tm.TM_OK
        o = op if sgn > 0 else opm
        for r in range(2):
            assert np.linalg.norm(b[r] - o.apply(x[r])) / np.linalg.norm(b[r]) <= 1e-10
        iters[sgn] = info.iters
    assert abs(iters[+1] - iters[-1]) <= max(2, 0.2 * iters[+1])
    tm.tm_set_mu(g.h, mu, 5.0)
    x = np.zeros_like(b)
    # the D^dagger D residual is the solves' residual amplified by ~ ||D|| / mu
    st, info = tm.tm_solve_squared(g.h, b, x, 2, 1e-12)
    assert st == tm.TM_OK and info.converged
    for r in range(2):
        ddx = gamma5_field(opm.apply(gamma5_field(op.apply(x[r]))))
        assert np.linalg.norm(ddx - b[r]) / np.linalg.norm(b[r]) <= 1e-8
    # the handle is back at +mu
    x1 = np.zeros_like(b[0])
    st, _ = tm.tm_solve(g.h, b[0], x1, 1, 1e-10)
    assert np.linalg.norm(b[0] - op.apply(x1)) / np.linalg.norm(b[0]) <= 1e-10
