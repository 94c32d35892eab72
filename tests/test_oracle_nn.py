"""Pins of the learned-layer oracle (``oracle.nn``), CPU only.

* Free field: a plane wave exp(i p.x) u is an eigenvector of every transport
  T_d with eigenvalue exp(+-i p_mu) (times bc_t's twist for antiperiodic T),
  so one layer acts on it as the closed-form spin matrix sum_d W_d phase_d.
* Gauge covariance: N[U^g](g r) = g N[U](r).
* One layer with the Wilson weights equals D_W at c_sw = 0 and mu = 0 from
  ``oracle.dirac`` (written independently).
* Adjoint: <y, L x> = <L^dagger y, x> for random fields and weights.
* Gradients: central finite differences of the loss in the real and imaginary
  part of single weights of both layers.
"""
import numpy as np
import pytest

import inputs
from oracle import nn
from oracle.dirac import Operator

L = (4, 4, 4, 4)


def _rand_w(shape, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def _rand_field(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("bc_t", [1.0, -1.0])
def test_free_field_plane_wave(bc_t):
    U = inputs.unit_gauge(L)
    twist = 0.0 if bc_t == 1.0 else np.pi        # antiperiodic in T: p_T = (2 pi k + pi) / L_T
    p = np.array([(2 * np.pi * 1 + twist) / L[0], 2 * np.pi * 2 / L[1], 2 * np.pi * 1 / L[2], 2 * np.pi * 3 / L[3]])
    x = np.stack(np.meshgrid(*[np.arange(n) for n in L], indexing="ij"), axis=-1)
    phase = np.exp(1j * (x @ p))
    u = _rand_field((4, 3), 3)
    psi = phase[..., None, None] * u
    W = _rand_w((2, 1, nn.NDIR, 4, 4), 4)
    y = nn.layer(U, psi[None], W, bc_t)
    for o in range(2):
        M = W[o, 0, 0].copy()
        for mu in range(4):
            M = M + W[o, 0, 1 + 2 * mu] * np.exp(1j * p[mu]) + W[o, 0, 2 + 2 * mu] * np.exp(-1j * p[mu])
        expect = phase[..., None, None] * (M @ u)
        assert np.allclose(y[o], expect, atol=1e-12)


def test_gauge_covariance():
    U = inputs.gauge_field(L, 0.5, 11)
    g = inputs.random_gauge_transform(L, 12)
    # U^g_mu(x) = g(x) U_mu(x) g(x + mu)^dagger
    Ug = np.empty_like(U)
    for mu in range(4):
        gn = np.roll(g, -1, axis=mu)
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gn, -1, -2))
    r = _rand_field(L + (4, 3), 13)
    W1 = _rand_w((nn.HIDDEN, 1, nn.NDIR, 4, 4), 14)
    W2 = _rand_w((1, nn.HIDDEN, nn.NDIR, 4, 4), 15)
    gr = np.einsum("...ab,...sb->...sa", g, r)
    lhs = nn.network(Ug, gr, W1, W2)
    rhs = np.einsum("...ab,...sb->...sa", g, nn.network(U, r, W1, W2))
    assert np.allclose(lhs, rhs, atol=1e-11)


@pytest.mark.parametrize("bc_t", [1.0, -1.0])
def test_wilson_weights_give_dirac_operator(bc_t):
    U = inputs.gauge_field(L, 0.5, 21)
    m0 = -0.37
    op = Operator(U, m0, 0.0, 0.0, bc_t)
    psi = _rand_field(L + (4, 3), 22)
    y = nn.layer(U, psi[None], nn.wilson_weights(m0), bc_t)[0]
    assert np.allclose(y, op.apply(psi), atol=1e-12)


def test_adjoint_layer():
    U = inputs.gauge_field(L, 0.5, 31)
    W = _rand_w((3, 2, nn.NDIR, 4, 4), 32)
    x = _rand_field((2,) + L + (4, 3), 33)
    y = _rand_field((3,) + L + (4, 3), 34)
    assert np.isclose(np.vdot(y, nn.layer(U, x, W)), np.vdot(nn.layer_adjoint(U, y, W), x), rtol=1e-12)


def test_gradients_match_finite_differences():
    U = inputs.gauge_field((4, 4, 2, 2), 0.5, 41)
    Lx = U.shape[:4]
    R = _rand_field((2,) + Lx + (4, 3), 42)
    E = _rand_field((2,) + Lx + (4, 3), 43)
    W1 = _rand_w((nn.HIDDEN, 1, nn.NDIR, 4, 4), 44)
    W2 = _rand_w((1, nn.HIDDEN, nn.NDIR, 4, 4), 45)
    loss, G1, G2 = nn.loss_and_grad(U, R, E, W1, W2)
    eps = 1e-6
    picks = [(1, (3, 0, 2, 1, 3)), (1, (0, 0, 0, 0, 0)), (2, (0, 5, 7, 2, 2)), (2, (0, 1, 0, 3, 0))]
    for which, idx in picks:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            Wp1, Wp2, Wm1, Wm2 = W1.copy(), W2.copy(), W1.copy(), W2.copy()
            if which == 1:
                Wp1[idx] += eps * unit
                Wm1[idx] -= eps * unit
                G = G1
            else:
                Wp2[idx] += eps * unit
                Wm2[idx] -= eps * unit
                G = G2
            lp = nn.loss_and_grad(U, R, E, Wp1, Wp2)[0]
            lm = nn.loss_and_grad(U, R, E, Wm1, Wm2)[0]
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - 2 * part(G[idx])) <= 1e-6 * max(1.0, abs(fd)), (which, idx, fd, G[idx])


def test_pack_roundtrip():
    W1 = _rand_w((nn.HIDDEN, 1, nn.NDIR, 4, 4), 51)
    W2 = _rand_w((1, nn.HIDDEN, nn.NDIR, 4, 4), 52)
    a, b = nn.unpack_weights(nn.pack_weights(W1, W2))
    assert np.array_equal(a, W1) and np.array_equal(b, W2)
    assert nn.pack_weights(W1, W2).size == 2304
