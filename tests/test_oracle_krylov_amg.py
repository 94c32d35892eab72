"""Pins of the oracle's GMRES/FGMRES, K-cycle (eq. 1) and solve (CPU only).

Checks: GMRES equals a dense solve and its Arnoldi relation holds; FGMRES
with an exact preconditioner converges in one step; Givens rotations are
unitary and annihilate; with exact block solves and an exact coarse solve
the K-cycle's error propagator I - B D equals eq. (1) assembled from dense
matrices; the full FGMRES + AMG solve at 4^4 matches a dense LU solve.
"""
import numpy as np

import inputs
from oracle.dirac import Operator, dense_matrix
from oracle.krylov import gmres, givens
from oracle.sap import SAP
from oracle.amg import TwoLevel, AMGParams


def _rand_system(n, seed, shift=4.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = A / np.sqrt(n) + shift * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b


def test_givens_rotation():
    for a, b in [(1 + 2j, 0.5), (-3j, 2.0), (0.0, 1.0), (2.0, 0.0)]:
        c, s, rho = givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        assert np.allclose(G @ G.conj().T, np.eye(2))
        out = G @ np.array([a, b])
        assert abs(out[1]) < 1e-14 and abs(out[0] - rho) < 1e-14


def test_gmres_matches_dense_solve():
    A, b = _rand_system(60, 1)
    res = gmres(lambda v: A @ v, b, tol=1e-13, restart=15, maxit=500)
    assert res.converged
    assert np.allclose(res.x, np.linalg.solve(A, b), atol=1e-11)


def test_fgmres_exact_preconditioner_one_step():
    A, b = _rand_system(40, 2, shift=1.0)
    Ainv = np.linalg.inv(A)
    res = gmres(lambda v: A @ v, b, tol=1e-12, restart=10, maxit=10, M=lambda v: Ainv @ v)
    assert res.iters == 1 and res.relres < 1e-12


def _dense_setup():
    L = (4, 4, 2, 2)
    prm = AMGParams(m0=-0.3, c_sw=1.3, mu=0.05, delta=1.0, nv=3, agg=(2, 2, 1, 1),
                    sap_block=(2, 2, 1, 1), mr_iters=2, pre_smooth=1, post_smooth=2)
    tl = TwoLevel(inputs.gauge_field(L, 0.6, 41), prm)
    tl.build_coarse(inputs.random_test_vectors(L, prm.nv, 42))
    return L, prm, tl


def test_kcycle_error_propagation_is_eq1():
    """Exact solves make B linear; I - B D must equal (I-MD)^k (I-P Dc^-1 P^+ D) (I-MD)^j."""
    L, prm, tl = _dense_setup()
    D = dense_matrix(tl.op.apply, L)
    n = D.shape[0]
    sap = tl.sap
    colour = np.repeat(sap.colour.ravel(), 12)
    from tests.test_oracle_sap import _block_index
    bid = _block_index(L, prm.sap_block)

    def exact(r, mask):
        out = np.zeros(r.size, dtype=complex)
        m = np.repeat(mask.ravel(), 12)
        for blk in np.unique(bid[m]):
            s = bid == blk
            out[s] = np.linalg.solve(D[np.ix_(s, s)], r.ravel()[s])
        return out.reshape(r.shape)

    Dc_dense = None
    nc = int(np.prod(tl.P.Lc)) * 2 * prm.nv
    E = np.eye(nc, dtype=complex).reshape((nc,) + tl.P.Lc + (2 * prm.nv,))
    Dc_dense = tl.Dc.apply(E).reshape(nc, nc).T

    sap_exact = SAP(tl.op, prm.sap_block)
    tl.sap = type("S", (), {})()
    tl.sap.smooth = lambda b, x, k: _smooth(sap_exact, exact, b, x, k)
    tl.coarse_solve = lambda rc, *a: np.linalg.solve(Dc_dense, rc.ravel()).reshape(rc.shape)

    # dense error propagators
    I = np.eye(n)
    def prop(c):
        s = colour == c
        M = np.zeros((n, n), dtype=complex)
        for blk in np.unique(bid[s]):
            t = bid == blk
            M[np.ix_(t, t)] = np.linalg.inv(D[np.ix_(t, t)])
        return I - M @ D
    E_sweep = prop(1) @ prop(0)
    Pd = np.stack([tl.P.prolong(e).ravel() for e in E]).T
    E_cgc = I - Pd @ np.linalg.inv(Dc_dense) @ Pd.conj().T @ D
    E_eq1 = np.linalg.matrix_power(E_sweep, prm.post_smooth) @ E_cgc \
        @ np.linalg.matrix_power(E_sweep, prm.pre_smooth)

    eps = inputs.gaussian_spinor(L, 43)
    got = eps - tl.kcycle(tl.op.apply(eps))
    assert np.allclose(got.ravel(), E_eq1 @ eps.ravel(), atol=1e-11)


def _smooth(sap, exact, b, x, k):
    for _ in range(k):
        x = sap.sweep(b, x, block_solve=exact)
    return x


def test_two_level_solve_matches_dense_lu():
    L = (4, 4, 4, 4)
    prm = AMGParams(m0=1 / (2 * 0.13) - 4, c_sw=1.0, mu=0.01, delta=1.0, nv=8,
                    agg=(2, 2, 2, 2), sap_block=(2, 2, 2, 2), setup_iters=2)
    tl = TwoLevel(inputs.gauge_field(L, 0.3, 1), prm)
    tl.setup(inputs.random_test_vectors(L, prm.nv, 1 + 2000))
    b = inputs.gaussian_spinor(L, 1 + 1000)
    res = tl.solve(b, tol=1e-10)
    assert res.converged and res.relres <= 1e-10
    D = dense_matrix(tl.op.apply, L)
    x_ref = np.linalg.solve(D, b.ravel())
    rel = np.linalg.norm(res.x.ravel() - x_ref) / np.linalg.norm(x_ref)
    cond = np.linalg.cond(D)
    assert rel <= 1e-10 * cond
    assert rel < 1e-8
    # the preconditioner is doing its job: far fewer steps than unpreconditioned GMRES
    plain = gmres(tl.op.apply, b, tol=1e-10, restart=25, maxit=res.iters * 3)
    assert not plain.converged


def test_squared_operator_solve_with_one_setup():
    """Sec. 1 and 3: one setup serves D(+mu) and D(-mu); (D^dagger D)^-1 b
    from two non-squared solves satisfies D(mu)^dagger D(mu) x = b, with
    D(mu)^dagger applied as Gamma5 D(-mu) Gamma5 and checked densely."""
    from oracle.dirac import gamma5_field
    L = (4, 4, 4, 4)
    prm = AMGParams(m0=1 / (2 * 0.13) - 4, c_sw=1.0, mu=0.01, delta=2.0, nv=8,
                    agg=(2, 2, 2, 2), sap_block=(2, 2, 2, 2), setup_iters=1)
    tl = TwoLevel(inputs.gauge_field(L, 0.3, 1), prm)
    tl.setup(inputs.random_test_vectors(L, prm.nv, 2001))
    b = inputs.gaussian_spinor(L, 1001)
    x, (r1, r2) = tl.solve_squared(b, tol=1e-11)
    assert r1.converged and r2.converged and tl.prm.mu == 0.01
    D = dense_matrix(tl.op.apply, L)
    ddx = D.conj().T @ (D @ x.ravel())
    assert np.linalg.norm(ddx - b.ravel()) / np.linalg.norm(b) < 1e-8
    # D(mu)^dagger = Gamma5 D(-mu) Gamma5 on a vector
    Dm = tl.op.with_mu(-tl.op.mu)
    y = inputs.gaussian_spinor(L, 5)
    assert np.allclose(gamma5_field(Dm.apply(gamma5_field(y))).ravel(), D.conj().T @ y.ravel(), atol=1e-12)
