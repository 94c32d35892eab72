"""Pins of the oracle's gamma matrices, clover term and D(mu) (CPU only).

Each check fixes the oracle against something other than itself: the gamma5
printed in the paper (Sec. 2, eq. 2), the Clifford algebra, the free-field
plane-wave closed form, Gamma5-hermiticity and D^dagger D = D_W^dagger D_W +
mu^2 (Sec. 1), gauge covariance, a hand-evaluated clover term for a uniform
abelian field, and a site-by-site evaluation of the stencil.
"""
import os

import numpy as np
import pytest

import inputs
from oracle.dirac import (GAMMA, GAMMA5, Operator, dense_matrix, gamma5_field,
                          clover_matrix, clover_blocks)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gamma5_matches_eq2():
    g5 = np.loadtxt(os.path.join(GOLDEN, "gamma5_eq2.txt"))
    assert np.array_equal(GAMMA5.real, g5) and not GAMMA5.imag.any()


def test_clifford_algebra_and_gamma5_product():
    for a in range(4):
        assert np.allclose(GAMMA[a], GAMMA[a].conj().T)
        for b in range(4):
            ac = GAMMA[a] @ GAMMA[b] + GAMMA[b] @ GAMMA[a]
            assert np.allclose(ac, 2.0 * (a == b) * np.eye(4))
    # directions T, Z, Y, X carry gamma_4, gamma_3, gamma_2, gamma_1
    g1, g2, g3, g4 = GAMMA[3], GAMMA[2], GAMMA[1], GAMMA[0]
    assert np.allclose(g1 @ g2 @ g3 @ g4, GAMMA5)
    for a in range(4):  # gamma5 anticommutes with every gamma_mu
        assert np.allclose(GAMMA5 @ GAMMA[a], -GAMMA[a] @ GAMMA5)
        for b in range(4):  # sigma_mu_nu is block diagonal in chirality
            G = GAMMA[a] @ GAMMA[b]
            assert np.allclose(G[0:2, 2:4], 0) and np.allclose(G[2:4, 0:2], 0)


@pytest.mark.parametrize("L", [(6, 4, 2, 4), (4, 6, 4, 2)])
@pytest.mark.parametrize("bc", [-1.0, 1.0])
def test_free_field_plane_wave(L, bc):
    """U = 1: D psi = [m0 + sum(1 - cos p) + i sum gamma_mu sin p + i mu g5] psi."""
    m0, mu = -0.3, 0.07
    op = Operator(inputs.unit_gauge(L), m0, 1.7, mu, bc_t=bc)
    rng = np.random.default_rng(3)
    coords = np.meshgrid(*[np.arange(n) for n in L], indexing="ij")
    for trial in range(4):
        n = [int(rng.integers(0, L[d])) for d in range(4)]
        p = [2 * np.pi * n[d] / L[d] for d in range(4)]
        if bc < 0:
            p[0] = (2 * n[0] + 1) * np.pi / L[0]
        phase = np.exp(1j * sum(p[d] * coords[d] for d in range(4)))
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = phase[..., None, None] * u
        M = (m0 + sum(1 - np.cos(p[d]) for d in range(4))) * np.eye(4) \
            + 1j * sum(np.sin(p[d]) * GAMMA[d] for d in range(4)) + 1j * mu * GAMMA5
        expect = phase[..., None, None] * (M @ u)
        assert np.allclose(op.apply(psi), expect, atol=1e-13)


def _small_op(L=(4, 2, 2, 4), mu=0.15, seed=11, c_sw=1.3):
    U = inputs.gauge_field(L, 0.7, seed)
    return Operator(U, -0.2, c_sw, mu)


def test_gamma5_hermiticity_dense():
    """D(mu)^dagger = Gamma5 D(-mu) Gamma5 (Sec. 1)."""
    op = _small_op()
    Dp = dense_matrix(op.apply, op.L)
    Dm = dense_matrix(op.with_mu(-op.mu).apply, op.L)
    G5 = dense_matrix(gamma5_field, op.L)
    assert np.allclose(Dp.conj().T, G5 @ Dm @ G5, atol=1e-13)


def test_normal_operator_identity():
    """D(mu)^dagger D(mu) = D_W^dagger D_W + mu^2 (Sec. 1)."""
    op = _small_op()
    D = dense_matrix(op.apply, op.L)
    W = dense_matrix(op.apply_W, op.L)
    n = D.shape[0]
    assert np.allclose(D.conj().T @ D, W.conj().T @ W + op.mu ** 2 * np.eye(n), atol=1e-12)
    # and the lower bound mu on the singular values
    assert np.linalg.svd(D, compute_uv=False).min() >= op.mu * (1 - 1e-12)


def test_gauge_covariance():
    """D[U^g](g psi) = g D[U] psi, U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dagger."""
    L = (4, 4, 2, 6)
    U = inputs.gauge_field(L, 0.8, 5)
    g = inputs.random_gauge_transform(L, 6)
    Ug = np.empty_like(U)
    for d in range(4):
        gf = np.roll(g, -1, axis=d)
        Ug[..., d, :, :] = g @ U[..., d, :, :] @ np.conj(np.swapaxes(gf, -1, -2))
    psi = inputs.gaussian_spinor(L, 7)
    gpsi = np.einsum("...ab,...sb->...sa", g, psi)
    op = Operator(U, -0.4, 1.9, 0.05)
    opg = Operator(Ug, -0.4, 1.9, 0.05)
    lhs = opg.apply(gpsi)
    rhs = np.einsum("...ab,...sb->...sa", g, op.apply(psi))
    assert np.allclose(lhs, rhs, atol=1e-12)


def test_clover_uniform_abelian_field():
    """U_X(x) = exp(i phi y), phi = 2 pi n / L_Y, all other links 1.

    Every leaf in the (X, Y) plane is exp(-i phi), so evaluating the clover
    formula by hand gives A = (m0 + 4) - (c_sw sin(phi) / 2) diag(1,-1,1,-1) (x) 1_3
    (gamma_1 gamma_2 = i diag(1,-1,1,-1) in this basis).
    """
    L = (2, 2, 6, 4)
    m0, c_sw = -0.25, 1.6
    phi = 2 * np.pi * 1 / L[2]
    U = inputs.unit_gauge(L)
    y = np.arange(L[2])
    U[..., 3, :, :] = np.exp(1j * phi * y)[None, None, :, None, None, None] * np.eye(3)
    A = clover_matrix(U, m0, c_sw)
    spin = np.array([1, -1, 1, -1])
    expect = np.diag(np.repeat(m0 + 4 - c_sw * np.sin(phi) / 2 * spin, 3))
    assert np.allclose(A, expect, atol=1e-13)


def test_clover_hermitian_and_chiral():
    op = _small_op(L=(4, 4, 4, 2))
    A = op.A
    assert np.allclose(A, np.conj(np.swapaxes(A, -1, -2)), atol=1e-14)
    assert np.allclose(A[..., 0:6, 6:12], 0, atol=1e-14)
    assert np.allclose(A[..., 6:12, 0:6], 0, atol=1e-14)
    assert clover_blocks(A).shape == op.L + (2, 6, 6)


def test_stencil_against_site_by_site_definition():
    L = (4, 6, 2, 4)
    op = Operator(inputs.gauge_field(L, 0.5, 9), -0.6, 1.5, 0.02)
    psi = inputs.gaussian_spinor(L, 10)
    y = op.apply(psi)
    rng = np.random.default_rng(0)
    sites = [tuple(int(rng.integers(0, n)) for n in L) for _ in range(12)]
    sites += [(0, 0, 0, 0), (L[0] - 1, L[1] - 1, L[2] - 1, L[3] - 1)]
    ys = op.apply_at_sites(psi, sites)
    for k, s in enumerate(sites):
        assert np.allclose(y[s], ys[k], atol=1e-13)


def test_dense_lu_solve_matches_operator():
    """x = D^-1 b from a dense LU satisfies the stencil equation D x = b."""
    op = _small_op(L=(4, 4, 2, 2))
    D = dense_matrix(op.apply, op.L)
    b = inputs.gaussian_spinor(op.L, 12)
    x = np.linalg.solve(D, b.ravel()).reshape(b.shape)
    assert np.linalg.norm(op.apply(x) - b) / np.linalg.norm(b) < 1e-12
