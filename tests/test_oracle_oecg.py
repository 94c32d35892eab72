"""Pins of the odd-even CG baseline (oracle.oecg; Sec. 1, Fig. 1 and Sec. 3), CPU only.

CGLS against numpy.linalg.solve on dense systems and against brute-force
least squares over its Krylov spaces (a wrong alpha, beta or adjoint moves
the iterates off the minimiser); the reduced right-hand side, the
reconstruction of the even sites and the reduced adjoint against the dense
Schur complement of D(mu, mu + rho) on a small lattice; the full oeCG
solution against a dense LU solve.  Planted mistakes (the adjoint without
the sign flip of the odd shift, the reconstruction without the hop term)
fail.
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator, dense_matrix, site_parity
from oracle import evenodd, oecg

L = (4, 4, 2, 2)
MU, RHO = 0.05, 0.13


def _op(mu=MU, rho=RHO):
    return Operator(inputs.gauge_field(L, 0.6, 7), -0.3, 1.3, mu, rho=rho)


def _idx():
    par = np.repeat(site_parity(L).ravel(), 12)
    return np.flatnonzero(par == 0), np.flatnonzero(par == 1)


def _dense_system(n=14, seed=2):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 4 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b


def test_cgls_solves_dense_systems():
    A, b = _dense_system()
    res = oecg.cgls(lambda v: A @ v, lambda v: A.conj().T @ v, b, 1e-13, 500)
    assert res.converged
    assert np.allclose(res.x, np.linalg.solve(A, b), atol=1e-11)
    assert np.linalg.norm(b - A @ res.x) <= 1e-13 * np.linalg.norm(b) * 1.0001


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_cgls_iterates_minimise_the_residual_over_krylov_spaces(k):
    A, b = _dense_system(seed=k)
    res = oecg.cgls(lambda v: A @ v, lambda v: A.conj().T @ v, b, 0.0, k)
    assert res.iters == k
    N = A.conj().T @ A
    K = [A.conj().T @ b]
    for _ in range(k - 1):
        K.append(N @ K[-1])
    K = np.stack(K, axis=1)
    c = np.linalg.lstsq(A @ K, b, rcond=None)[0]
    assert np.allclose(res.x, K @ c, atol=1e-9 * np.linalg.norm(K @ c))


def test_wrong_adjoint_moves_the_iterates():
    A, b = _dense_system(seed=3)
    good = oecg.cgls(lambda v: A @ v, lambda v: A.conj().T @ v, b, 0.0, 3)
    bad = oecg.cgls(lambda v: A @ v, lambda v: A.T @ v, b, 0.0, 3)  # planted: transpose without conjugation
    assert not np.allclose(good.x, bad.x, atol=1e-6)


def test_reduced_rhs_reconstruction_and_adjoint_against_dense_schur():
    op = _op()
    D = dense_matrix(op.apply, L)
    e, o = _idx()
    Dee, Deo, Doe, Doo = D[np.ix_(e, e)], D[np.ix_(e, o)], D[np.ix_(o, e)], D[np.ix_(o, o)]
    S = Doo - Doe @ np.linalg.solve(Dee, Deo)
    b = inputs.gaussian_spinor(L, 11)
    bv = b.ravel()
    bh = oecg.reduced_rhs(op, b).ravel()
    assert np.allclose(bh[o], bv[o] - Doe @ np.linalg.solve(Dee, bv[e]), atol=1e-12)
    assert np.allclose(bh[e], 0)
    xo = inputs.gaussian_spinor(L, 12)
    x = oecg.reconstruct(op, b, xo).ravel()
    assert np.allclose(x[e], np.linalg.solve(Dee, bv[e] - Deo @ xo.ravel()[o]), atol=1e-12)
    assert np.allclose(x[o], xo.ravel()[o])
    v = inputs.gaussian_spinor(L, 13)
    assert np.allclose(oecg.reduced_adjoint(op, v).ravel()[o], S.conj().T @ v.ravel()[o], atol=1e-12)
    # planted: the adjoint with -mu but the odd shift kept fails
    op_m = op.with_mu_eo(-op.mu, -op.mu + op.rho)
    wrong = evenodd.gamma5(evenodd.reduced_apply(op_m, evenodd.gamma5(v))).ravel()[o]
    assert not np.allclose(wrong, S.conj().T @ v.ravel()[o], atol=1e-6)
    # planted: a reconstruction without the hop term fails
    od = evenodd.odd_mask(op)
    naive = (evenodd.diag_solve(op, b * ~od) * ~od).ravel()
    assert not np.allclose(naive[e], x[e], atol=1e-6)


def test_oecg_solves_the_full_system():
    op = _op()
    D = dense_matrix(op.apply, L)
    b = inputs.gaussian_spinor(L, 21)
    x, res = oecg.solve(op, b, tol=1e-12)
    assert res.converged and res.iters > 5
    xd = np.linalg.solve(D, b.ravel())
    assert np.linalg.norm(x.ravel() - xd) <= 1e-9 * np.linalg.norm(xd)
    # the recurrence residual is the full residual: even sites solved exactly
    r = b - op.apply(x)
    assert np.linalg.norm(r) <= 1.01e-12 * np.linalg.norm(b) + 1e-14
