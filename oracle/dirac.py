"""Wilson-clover twisted-mass operator D(mu) = D_W + i*mu*Gamma5 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed
-----------------------
* Sec. 1: D_W is the Wilson clover operator; D(+-mu) = D_W +- i*Gamma5*mu.
* Sec. 2, eq. (2): gamma_5 = diag(-1, -1, +1, +1); the other gamma matrices
  may be chosen freely; lexicographic site order TZYX.

Readings where the paper is silent
----------------------------------------------------------------
* Gamma matrices: chiral basis gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]
  (k = 1, 2, 3), gamma_4 = [[0, -1], [-1, 0]]; lattice directions
  X, Y, Z, T carry gamma_1, gamma_2, gamma_3, gamma_4.  Direction index
  mu = 0..3 means T, Z, Y, X (the order of the array axes).
* Normalisation: diagonal (m0 + 4), hopping -1/2 [(1 - gamma_mu) U_mu(x)
  psi(x + mu) + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu)].
* Clover: A(x) = (m0 + 4) 1 - (c_sw / 32) sum_{mu,nu} (gamma_mu gamma_nu)
  (x) (Q_mu_nu(x) - Q_nu_mu(x)), Q the sum of the four plaquette leaves in
  the mu-nu plane that start and end at x.
* Boundary conditions: periodic in X, Y, Z; hops across the T boundary get
  the factor ``bc_t`` (-1 = antiperiodic, the default).

Pins (tests/test_oracle_dirac.py): gamma algebra and eq. (2); free-field
plane-wave closed form; Gamma5-hermiticity; D^dagger D = D_W^dagger D_W + mu^2;
gauge covariance; a uniform abelian field whose clover term has a closed form;
agreement of the dense assembly with the stencil.
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------
# gamma matrices (Sec. 2, eq. 2)
# ----------------------------------------------------------------------------

_S1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_S3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def _chiral(A: np.ndarray) -> np.ndarray:
    g = np.zeros((4, 4), dtype=np.complex128)
    g[0:2, 2:4] = A
    g[2:4, 0:2] = A.conj().T
    return g


def gamma_matrices() -> tuple[np.ndarray, np.ndarray]:
    """(gammas[4, 4, 4] indexed by lattice direction T, Z, Y, X; gamma5)."""
    g1 = _chiral(-1j * _S1)
    g2 = _chiral(-1j * _S2)
    g3 = _chiral(-1j * _S3)
    g4 = _chiral(-_I2)
    g5 = np.diag([-1, -1, 1, 1]).astype(np.complex128)
    return np.stack([g4, g3, g2, g1]), g5


GAMMA, GAMMA5 = gamma_matrices()
ONE4 = np.eye(4, dtype=np.complex128)

# spinor arrays: [..., T, Z, Y, X, 4, 3]; lattice axis of direction mu:
_SPIN_AXIS = (-6, -5, -4, -3)


def lattice_shape(psi: np.ndarray) -> tuple[int, int, int, int]:
    return tuple(psi.shape[-6:-2])


# ----------------------------------------------------------------------------
# shifts and hops
# ----------------------------------------------------------------------------

def shift_gauge(F: np.ndarray, mu: int, sign: int) -> np.ndarray:
    """F(x + sign*mu_hat) at x for a site field [T,Z,Y,X,...] (periodic)."""
    return np.roll(F, -sign, axis=mu)


def shift_spinor(psi: np.ndarray, mu: int, sign: int, bc_t: float) -> np.ndarray:
    """psi(x + sign*mu_hat) at x, with the factor bc_t on hops across T."""
    out = np.roll(psi, -sign, axis=_SPIN_AXIS[mu])
    if mu == 0 and bc_t != 1:
        edge = -1 if sign > 0 else 0
        idx = [slice(None)] * out.ndim
        idx[_SPIN_AXIS[0]] = edge
        out[tuple(idx)] *= bc_t
    return out


def color_mul(U: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(U psi)(x) on colour, U [T,Z,Y,X,3,3], psi [...,T,Z,Y,X,4,3]."""
    return np.einsum("...ab,...sb->...sa", U, psi)


def color_mul_dag(U: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(U^dagger psi)(x) on colour."""
    return np.einsum("...ba,...sb->...sa", U.conj(), psi)


def spin_mul(G: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(G psi)(x) on spin, G [4, 4]."""
    return np.einsum("st,...tc->...sc", G, psi)


def hop_forward(U: np.ndarray, psi: np.ndarray, mu: int, bc_t: float) -> np.ndarray:
    """U_mu(x) psi(x + mu_hat)."""
    return color_mul(U[..., mu, :, :], shift_spinor(psi, mu, +1, bc_t))


def hop_backward(U: np.ndarray, psi: np.ndarray, mu: int, bc_t: float) -> np.ndarray:
    """U_mu(x - mu_hat)^dagger psi(x - mu_hat)."""
    return shift_spinor(color_mul_dag(U[..., mu, :, :], psi), mu, -1, bc_t)


# ----------------------------------------------------------------------------
# clover term
# ----------------------------------------------------------------------------

def _dag(M: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(M, -1, -2))


def clover_leaves(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Q_mu_nu(x): the four plaquettes in the mu-nu plane at x, same orientation."""
    Um = U[..., mu, :, :]
    Un = U[..., nu, :, :]
    sh = shift_gauge
    l1 = Um @ sh(Un, mu, +1) @ _dag(sh(Um, nu, +1)) @ _dag(Un)
    l2 = Un @ _dag(sh(sh(Um, nu, +1), mu, -1)) @ _dag(sh(Un, mu, -1)) @ sh(Um, mu, -1)
    l3 = (_dag(sh(Um, mu, -1)) @ _dag(sh(sh(Un, mu, -1), nu, -1))
          @ sh(sh(Um, mu, -1), nu, -1) @ sh(Un, nu, -1))
    l4 = _dag(sh(Un, nu, -1)) @ sh(Um, nu, -1) @ sh(sh(Un, nu, -1), mu, +1) @ _dag(Um)
    return l1 + l2 + l3 + l4


def clover_matrix(U: np.ndarray, m0: float, c_sw: float) -> np.ndarray:
    """A(x) = (m0+4) 1 - (c_sw/32) sum_{mu,nu} gamma_mu gamma_nu (x) (Q_mu_nu - Q_nu_mu).

    Returns [T,Z,Y,X,12,12] with row index 3*spin + colour.  mu-free: the
    twisted-mass term is added by :func:`apply_D`.
    """
    L = U.shape[:4]
    A = np.zeros(L + (12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            F = clover_leaves(U, mu, nu) - clover_leaves(U, nu, mu)
            G = GAMMA[mu] @ GAMMA[nu]
            A += np.einsum("st,...ab->...satb", G, F).reshape(L + (12, 12))
    A *= -c_sw / 32.0
    A += (m0 + 4.0) * np.eye(12)
    return A


def clover_blocks(A: np.ndarray) -> np.ndarray:
    """The two 6x6 chiral blocks of A (spins {0,1} and {2,3}), [T,Z,Y,X,2,6,6]."""
    return np.stack([A[..., 0:6, 0:6], A[..., 6:12, 6:12]], axis=-3)


# ----------------------------------------------------------------------------
# the operator
# ----------------------------------------------------------------------------

def site_parity(L) -> np.ndarray:
    """(t + z + y + x) mod 2 per site, [T, Z, Y, X]: the even (0) and odd (1)
    sites of the odd-even decomposition."""
    c = np.indices(tuple(L))
    return c.sum(axis=0) % 2


class Operator:
    """D(mu) on a fixed gauge field: diagonal A(x) + i mu gamma5, Wilson hops.

    ``rho`` (Sec. 2: a different twisted mass on the even and the odd sites)
    adds i rho gamma5 on the odd sites only: the twisted mass is mu on even
    and mu + rho on odd sites."""

    def __init__(self, U: np.ndarray, m0: float, c_sw: float, mu: float,
                 bc_t: float = -1.0, rho: float = 0.0):
        self.U = U
        self.L = tuple(U.shape[:4])
        self.m0, self.c_sw, self.mu, self.bc_t = m0, c_sw, mu, bc_t
        self.rho = rho
        self.odd = site_parity(self.L) == 1
        self.A = clover_matrix(U, m0, c_sw)

    def with_mu(self, mu: float) -> "Operator":
        """The same operator with twisted mass mu on even sites (and mu + rho on odd)."""
        other = object.__new__(Operator)
        other.__dict__.update(self.__dict__)
        other.mu = mu
        return other

    def with_mu_eo(self, mu_even: float, mu_odd: float) -> "Operator":
        """Twisted mass mu_even on the even and mu_odd on the odd sites."""
        other = self.with_mu(mu_even)
        other.rho = mu_odd - mu_even
        return other

    def mu_field(self, mu: float | None = None) -> np.ndarray:
        """The twisted mass per site, [T, Z, Y, X] (mu of the even sites
        overridden by ``mu`` if given; the odd shift rho is kept)."""
        mu = self.mu if mu is None else mu
        return mu + self.rho * self.odd

    # -- pieces --------------------------------------------------------------
    def diag(self, psi: np.ndarray, mu: float | None = None) -> np.ndarray:
        """A(x) psi(x) + i mu(x) gamma5 psi(x), mu(x) = mu (+ rho on odd sites)."""
        sh = psi.shape
        y = np.einsum("...ij,...j->...i", self.A, psi.reshape(sh[:-2] + (12,)))
        y = y.reshape(sh)
        return y + 1j * self.mu_field(mu)[..., None, None] * spin_mul(GAMMA5, psi)

    def hop_term(self, psi: np.ndarray, mu: int, direction: int) -> np.ndarray:
        """-1/2 (1 - gamma_mu) U psi(x+mu) (direction +1) or
        -1/2 (1 + gamma_mu) U^dagger psi(x-mu) (direction -1)."""
        if direction > 0:
            return -0.5 * spin_mul(ONE4 - GAMMA[mu], hop_forward(self.U, psi, mu, self.bc_t))
        return -0.5 * spin_mul(ONE4 + GAMMA[mu], hop_backward(self.U, psi, mu, self.bc_t))

    def apply(self, psi: np.ndarray, mu: float | None = None) -> np.ndarray:
        """(D(mu) psi)(x); psi [..., T, Z, Y, X, 4, 3]."""
        y = self.diag(psi, mu)
        for d in range(4):
            y = y + self.hop_term(psi, d, +1) + self.hop_term(psi, d, -1)
        return y

    __call__ = apply

    def apply_W(self, psi: np.ndarray) -> np.ndarray:
        """D_W psi (mu = 0)."""
        return self.apply(psi, mu=0.0)

    def apply_at_sites(self, psi: np.ndarray, sites) -> np.ndarray:
        """(D psi)(x) for a list of sites x = (t, z, y, x); returns [n, 4, 3].

        Computed one site at a time from the definition, for sampled checks
        of full-size outputs.
        """
        L = self.L
        out = []
        for s in sites:
            s = tuple(int(v) for v in s)
            y = (self.A[s] @ psi[s].reshape(12)).reshape(4, 3)
            y = y + 1j * (self.mu + self.rho * (sum(s) % 2)) * (GAMMA5 @ psi[s])
            for d in range(4):
                f = list(s)
                f[d] = (s[d] + 1) % L[d]
                b = list(s)
                b[d] = (s[d] - 1) % L[d]
                pf = psi[tuple(f)] * (self.bc_t if (d == 0 and s[0] == L[0] - 1) else 1)
                pb = psi[tuple(b)] * (self.bc_t if (d == 0 and s[0] == 0) else 1)
                uf = self.U[s + (d,)]
                ub = self.U[tuple(b) + (d,)]
                y = y - 0.5 * (ONE4 - GAMMA[d]) @ (pf @ uf.T)
                y = y - 0.5 * (ONE4 + GAMMA[d]) @ (pb @ ub.conj())
            out.append(y)
        return np.array(out)


def dense_matrix(apply, L) -> np.ndarray:
    """The dense matrix of a linear map on spinor fields of lattice L (tiny L)."""
    n = 12 * int(np.prod(L))
    E = np.eye(n, dtype=np.complex128).reshape((n,) + tuple(L) + (4, 3))
    cols = apply(E).reshape(n, n)
    return cols.T.copy()


def gamma5_field(psi: np.ndarray) -> np.ndarray:
    """Gamma5 psi (site-diagonal gamma5)."""
    return spin_mul(GAMMA5, psi)


def vdot(a: np.ndarray, b: np.ndarray) -> complex:
    """<a, b> = sum conj(a) b."""
    return complex(np.vdot(a.ravel(), b.ravel()))


def norm(a: np.ndarray) -> float:
    return float(np.linalg.norm(a.ravel()))
