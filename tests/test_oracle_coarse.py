"""Pins of the oracle's aggregation P and coarse operator D_c (CPU only).

Checks: P^dagger P = 1; Gamma5 P = P Gamma5_c (Sec. 1); the QR factor equals
modified Gram-Schmidt (a different algorithm) on every aggregate; the local
9-point D_c equals the dense P^dagger D_W P, including lattices with only two
aggregates in a direction; D_c + i mu Gamma5_c = P^dagger D(mu) P (Sec. 1);
Gamma5_c-hermiticity (Sec. 1); the odd-even Schur solve equals the dense
solve; the exact coarse-grid correction is a projector.
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator, dense_matrix, gamma5_field
from oracle.coarse import Interpolation, CoarseOperator, OddEvenCoarse, to_agg, from_agg


def _setup(L, agg, nv, seed=31, mu=0.03):
    op = Operator(inputs.gauge_field(L, 0.6, seed), -0.35, 1.2, mu)
    tv = inputs.random_test_vectors(L, nv, seed + 2000)
    return op, Interpolation(tv, agg), tv


def _dense_P(P):
    return P.columns().reshape(2 * P.nv, -1).T       # fine x (k) for one coarse site each


def _dense_P_full(P):
    Lc, nv = P.Lc, P.nv
    nc = int(np.prod(Lc)) * 2 * nv
    E = np.eye(nc, dtype=complex).reshape((nc,) + Lc + (2 * nv,))
    return P.prolong(E).reshape(nc, -1).T


def _dense_coarse(apply, Lc, nv):
    nc = int(np.prod(Lc)) * 2 * nv
    E = np.eye(nc, dtype=complex).reshape((nc,) + Lc + (2 * nv,))
    return apply(E).reshape(nc, nc).T


def test_agg_view_roundtrip():
    L = (4, 6, 2, 4)
    psi = inputs.gaussian_spinor(L, 1)
    assert np.array_equal(from_agg(to_agg(psi, (2, 3, 1, 2)), (2, 3, 1, 2)), psi)


@pytest.mark.parametrize("L,agg", [((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 4, 2, 4), (2, 2, 1, 2))])
def test_P_orthonormal_and_gamma5_compatible(L, agg):
    op, P, _ = _setup(L, agg, 4)
    Pd = _dense_P_full(P)
    assert np.allclose(Pd.conj().T @ Pd, np.eye(Pd.shape[1]), atol=1e-13)
    G5 = dense_matrix(gamma5_field, L)
    g5c = np.tile(np.concatenate([-np.ones(P.nv), np.ones(P.nv)]), int(np.prod(P.Lc)))
    assert np.allclose(G5 @ Pd, Pd * g5c[None, :], atol=1e-14)


def test_P_equals_modified_gram_schmidt():
    L, agg, nv = (4, 4, 2, 2), (2, 2, 1, 1), 5
    _, P, tv = _setup(L, agg, nv)
    W = np.moveaxis(to_agg(tv, agg), 0, -1)             # [Lc, 2, rows, Nv]
    Wf = W.reshape(-1, W.shape[-2], nv)
    Qf = P.Q.reshape(-1, W.shape[-2], nv)
    for w, q in zip(Wf, Qf):
        Q = np.zeros_like(w)
        for j in range(nv):
            v = w[:, j].copy()
            for i in range(j):
                v -= np.vdot(Q[:, i], v) * Q[:, i]
            Q[:, j] = v / np.linalg.norm(v)
        assert np.allclose(Q, q, atol=1e-12)


@pytest.mark.parametrize("L,agg", [((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 4, 4, 2), (2, 2, 2, 1))])
def test_local_coarse_operator_equals_dense_galerkin(L, agg):
    op, P, _ = _setup(L, agg, 3)
    Dc = CoarseOperator.build(op, P, mu_c=0.0)
    Pd = _dense_P_full(P)
    W = dense_matrix(op.apply_W, L)
    galerkin = Pd.conj().T @ W @ Pd
    local = _dense_coarse(Dc.apply, P.Lc, P.nv)
    assert np.allclose(local, galerkin, atol=1e-12)
    # twisted mass stays diagonal: D_c + i mu Gamma5_c = P^dagger D(mu) P
    Dmu = dense_matrix(op.apply, L)
    local_mu = _dense_coarse(Dc.with_mu(op.mu).apply, P.Lc, P.nv)
    assert np.allclose(local_mu, Pd.conj().T @ Dmu @ Pd, atol=1e-12)
    # Gamma5_c-hermiticity of D_c
    g5c = np.tile(Dc.g5c, int(np.prod(P.Lc)))
    assert np.allclose(local.conj().T, g5c[:, None] * local * g5c[None, :], atol=1e-12)


def test_odd_even_schur_solve_equals_dense():
    L, agg = (4, 4, 4, 4), (2, 2, 2, 2)
    op, P, _ = _setup(L, agg, 3)
    Dc = CoarseOperator.build(op, P, mu_c=0.1)
    oe = OddEvenCoarse(Dc)
    rng = np.random.default_rng(2)
    b = rng.standard_normal(P.Lc + (2 * P.nv,)) + 1j * rng.standard_normal(P.Lc + (2 * P.nv,))
    dense = _dense_coarse(Dc.apply, P.Lc, P.nv)
    x_ref = np.linalg.solve(dense, b.ravel()).reshape(b.shape)
    even = oe.even.ravel()
    S = _dense_coarse(oe.schur, P.Lc, P.nv)
    ev = np.repeat(even, 2 * P.nv)
    xe = np.zeros(b.size, dtype=complex)
    xe[ev] = np.linalg.solve(S[np.ix_(ev, ev)], oe.reduced_rhs(b).ravel()[ev])
    x = oe.reconstruct(b, xe.reshape(b.shape))
    assert np.allclose(x, x_ref, atol=1e-11)


def test_exact_coarse_correction_is_projector():
    """P^dagger D (I - P D_c^-1 P^dagger D) eps = 0 with the exact D_c = P^dagger D P."""
    L, agg = (4, 4, 4, 4), (2, 2, 2, 2)
    op, P, _ = _setup(L, agg, 4)
    Dc = CoarseOperator.build(op, P, mu_c=op.mu)
    dense = _dense_coarse(Dc.apply, P.Lc, P.nv)
    eps = inputs.gaussian_spinor(L, 8)
    rc = P.restrict(op.apply(eps))
    ec = np.linalg.solve(dense, rc.ravel()).reshape(rc.shape)
    eps2 = eps - P.prolong(ec)
    assert np.linalg.norm(P.restrict(op.apply(eps2))) < 1e-11 * np.linalg.norm(rc)
