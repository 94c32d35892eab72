"""Learned gauge-covariant preconditioner layer (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

This component is NOT in the paper (arXiv:1611.01034 has no learned parts).
It is an added preconditioner stage whose definition is fixed here once and
implemented independently by the CUDA library:

* Directions d = 0 (self), 1 + 2 mu (forward), 2 + 2 mu (backward) for
  mu = 0..3 = T, Z, Y, X, the order of the coarse 9-point stencil.
* Parallel transport: (T_0 psi)(x) = psi(x),
  (T_{+mu} psi)(x) = U_mu(x) psi(x + mu_hat),
  (T_{-mu} psi)(x) = U_mu(x - mu_hat)^dagger psi(x - mu_hat), with the fermion
  boundary factor bc_t on hops across the T boundary (the same factor as in
  D(mu), so the layer sees the operator's boundary).
* One layer: y_o(x) = sum_i sum_d W[o, i, d] (T_d psi_i)(x), W[o, i, d] a
  complex 4 x 4 spin matrix acting trivially on colour.  It commutes with
  gauge transformations (gauge covariance).
* Network N = L2 o L1 with L1: 1 -> 8 channels and L2: 8 -> 1, no
  nonlinearity (reading: the layer description lists none; a linear N keeps
  the preconditioner a fixed linear map per weight set).
* Preconditioner: z = B(v) + N(v - D B(v)) with B the K-cycle of eq. (1).
* Training pairs: e = (1 - B D) e0 for random e0 (the error left by one
  K-cycle), r = D e.  Loss L = sum_p ||N(r_p) - e_p||^2 / sum_p ||e_p||^2;
  gradients are the Wirtinger derivatives dL/d conj(W) (the steepest-descent
  direction of a real loss in complex weights is minus twice this).

Pins (tests/test_oracle_nn.py): plane waves in the free field are
eigenvectors of every T_d with the closed-form phase; gauge covariance under
a random SU(3) transformation; one layer with the Wilson weights reproduces
D_W at c_sw = 0 from ``oracle.dirac`` (independent code); the adjoint layer
satisfies <y, L x> = <L^dagger y, x>; gradients match central finite
differences of the loss.
"""
from __future__ import annotations

import numpy as np

NDIR = 9
HIDDEN = 8


def _transport(U: np.ndarray, psi: np.ndarray, d: int, bc_t: float) -> np.ndarray:
    """(T_d psi)(x) for psi [..., T, Z, Y, X, 4, 3] (leading axes allowed)."""
    if d == 0:
        return psi.copy()
    mu, back = (d - 1) // 2, (d - 1) % 2 == 1
    ax = psi.ndim - 6 + mu  # lattice axis of direction mu
    Lmu = psi.shape[ax]
    if not back:
        nb = np.roll(psi, -1, axis=ax)            # psi(x + mu)
        if mu == 0 and bc_t != 1.0:
            sl = [slice(None)] * psi.ndim
            sl[ax] = Lmu - 1
            nb[tuple(sl)] *= bc_t
        link = U[..., mu, :, :]                  # U_mu(x)
        return np.einsum("...ab,...sb->...sa", link, nb)
    link = np.roll(U[..., mu, :, :], 1, axis=mu)  # U_mu(x - mu)
    nb = np.roll(psi, 1, axis=ax)                 # psi(x - mu)
    if mu == 0 and bc_t != 1.0:
        sl = [slice(None)] * psi.ndim
        sl[ax] = 0
        nb[tuple(sl)] *= bc_t
    return np.einsum("...ba,...sb->...sa", link.conj(), nb)


def opposite(d: int) -> int:
    return 0 if d == 0 else (d + 1 if (d - 1) % 2 == 0 else d - 1)


def layer(U: np.ndarray, psi: np.ndarray, W: np.ndarray, bc_t: float = -1.0) -> np.ndarray:
    """y [Cout, L, 4, 3] = sum_i sum_d W[o, i, d] T_d psi_i, psi [Cin, L, 4, 3]."""
    cout, cin = W.shape[:2]
    y = np.zeros((cout,) + psi.shape[1:], dtype=np.complex128)
    for d in range(NDIR):
        t = _transport(U, psi, d, bc_t)          # [Cin, L, 4, 3]
        y += np.einsum("oist,i...tc->o...sc", W[:, :, d], t)
    return y


def layer_adjoint(U: np.ndarray, g: np.ndarray, W: np.ndarray, bc_t: float = -1.0) -> np.ndarray:
    """L^dagger g [Cin, ...] = sum_o sum_d T_d^dagger (W[o, i, d]^H g_o); T_d^dagger = T_{-d}."""
    cout, cin = W.shape[:2]
    x = np.zeros((cin,) + g.shape[1:], dtype=np.complex128)
    for d in range(NDIR):
        m = np.einsum("oits,o...tc->i...sc", W[:, :, d].conj(), g)   # W^H acting on spin
        x += _transport(U, m, opposite(d), bc_t)
    return x


def network(U: np.ndarray, r: np.ndarray, W1: np.ndarray, W2: np.ndarray, bc_t: float = -1.0) -> np.ndarray:
    """N(r) for one field r [L, 4, 3]."""
    h = layer(U, r[None], W1, bc_t)
    return layer(U, h, W2, bc_t)[0]


def weight_grad(U: np.ndarray, psi: np.ndarray, g: np.ndarray, cout: int, bc_t: float = -1.0) -> np.ndarray:
    """G[o, i, d, s, s'] = sum_x sum_c g_o(x)[s, c] conj((T_d psi_i)(x)[s', c])."""
    cin = psi.shape[0]
    G = np.zeros((cout, cin, NDIR, 4, 4), dtype=np.complex128)
    for d in range(NDIR):
        t = _transport(U, psi, d, bc_t).reshape(cin, -1, 4, 3)
        G[:, :, d] = np.einsum("oxsc,ixtc->oist", g.reshape(cout, -1, 4, 3), t.conj())
    return G


def loss_and_grad(U: np.ndarray, R: np.ndarray, E: np.ndarray, W1: np.ndarray, W2: np.ndarray,
                  bc_t: float = -1.0):
    """Loss and Wirtinger gradients (G1, G2) over pairs R[p], E[p] of fields [L, 4, 3]."""
    S = float(sum(np.vdot(e, e).real for e in E))
    loss = 0.0
    G1 = np.zeros_like(W1)
    G2 = np.zeros_like(W2)
    for r, e in zip(R, E):
        h = layer(U, r[None], W1, bc_t)
        y = layer(U, h, W2, bc_t)[0]
        g = y - e
        loss += float(np.vdot(g, g).real)
        G2 += weight_grad(U, h, g[None], W2.shape[0], bc_t)
        gh = layer_adjoint(U, g[None], W2, bc_t)
        G1 += weight_grad(U, r[None], gh, W1.shape[0], bc_t)
    return loss / S, G1 / S, G2 / S


def wilson_weights(m0: float) -> np.ndarray:
    """W[1, 1, 9] with one layer equal to D_W(m0) at c_sw = 0 (Sec. 1 normalisation)."""
    from .dirac import GAMMA
    W = np.zeros((1, 1, NDIR, 4, 4), dtype=np.complex128)
    W[0, 0, 0] = (m0 + 4) * np.eye(4)
    for mu in range(4):
        W[0, 0, 1 + 2 * mu] = -0.5 * (np.eye(4) - GAMMA[mu])
        W[0, 0, 2 + 2 * mu] = -0.5 * (np.eye(4) + GAMMA[mu])
    return W


def pack_weights(W1: np.ndarray, W2: np.ndarray) -> np.ndarray:
    """Flat complex weights: W1 [8, 1, 9, 4, 4] then W2 [1, 8, 9, 4, 4]."""
    return np.concatenate([W1.ravel(), W2.ravel()])


def unpack_weights(w: np.ndarray):
    n1 = HIDDEN * 1 * NDIR * 16
    return w[:n1].reshape(HIDDEN, 1, NDIR, 4, 4), w[n1:].reshape(1, HIDDEN, NDIR, 4, 4)
