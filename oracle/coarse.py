"""Aggregation, interpolation P and the coarse operator D_c (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed
-----------------------
* Sec. 1: P spans approximately the low modes; it is built by aggregating a
  small set of N_v test vectors over blocks of the lattice ("local
  coherence").  D_c = P^dagger D_W P.
* Sec. 1: P is Gamma5-compatible, Gamma5 P = P Gamma5_c, so that D_c keeps
  Gamma5-hermiticity, D_c^dagger = Gamma5_c D_c Gamma5_c.
* Sec. 1: the twisted-mass term stays diagonal on the coarse grid,
  D_c(mu) = D_c + i mu Gamma5_c; on the coarsest grid mu is replaced by
  delta*mu with delta >= 1.
* Sec. 3: odd-even preconditioning is used on the coarsest level.

Readings (choices where the paper is silent)
------------------------------
* Aggregate = block of ``agg`` dims; each aggregate is split by chirality
  (spins {0,1} have gamma5 = -1, spins {2,3} have +1), giving 2 N_v coarse
  degrees of freedom per coarse site, ordered (chirality, i).
* For aggregate a and chirality chi the 6|a| x N_v matrix of test-vector
  pieces is orthonormalised by thin QR with a real positive R diagonal
  (unique), P_{a,chi} = Q.
* D_c is a 9-point stencil: a self block and, per direction mu, a forward
  block (hops from x in a across a's upper mu-face, coupling to a + mu) and a
  backward block (across the lower face, coupling to a - mu).  With two
  aggregates in a direction the forward and backward neighbour coincide; the
  two blocks are still kept apart.
* The stored blocks are mu-free; i*mu_c*Gamma5_c is added at apply time.
* Coarse site parity = (sum of coarse coordinates) mod 2.

Canonical layouts (used to compare with the CUDA path's exports)
----------------------------------------------------------------
* P columns as fine fields: [2 N_v, T, Z, Y, X, 4, 3]; column k = chi*N_v + i
  is, on every aggregate, P_{a,chi} e_i (zero on the other chirality).
* Coarse vector: [Tc, Zc, Yc, Xc, 2 N_v].
* D_c blocks: [Tc, Zc, Yc, Xc, 9, 2N_v, 2N_v]; block 0 = self, 1 + 2*mu =
  forward mu, 2 + 2*mu = backward mu; matrices [row, col].

Pins (tests/test_oracle_coarse.py): P^dagger P = 1; Gamma5 P = P Gamma5_c;
QR agrees with numpy's Householder QR after phase fixing; the local D_c
equals the dense P^dagger D_W P; D_c v = P^dagger D P v; Gamma5_c-hermiticity;
the odd-even Schur solve equals the dense solve.
"""
from __future__ import annotations

import numpy as np

from .dirac import Operator, ONE4, GAMMA, spin_mul, hop_forward, hop_backward


# ----------------------------------------------------------------------------
# aggregate views
# ----------------------------------------------------------------------------

def coarse_dims(L, agg):
    for d in range(4):
        if L[d] % agg[d]:
            raise ValueError("lattice not divisible by aggregate")
    return tuple(L[d] // agg[d] for d in range(4))


def to_agg(psi: np.ndarray, agg) -> np.ndarray:
    """[..., T,Z,Y,X,4,3] -> [..., Tc,Zc,Yc,Xc, 2(chi), 6|a|] (rows: site, spin, colour)."""
    L = psi.shape[-6:-2]
    Lc = coarse_dims(L, agg)
    lead = psi.shape[:-6]
    n = len(lead)
    p = psi.reshape(lead + (Lc[0], agg[0], Lc[1], agg[1], Lc[2], agg[2], Lc[3], agg[3], 2, 2, 3))
    # axes: lead..., Tc aT Zc aZ Yc aY Xc aX chi s c
    perm = list(range(n)) + [n + 0, n + 2, n + 4, n + 6, n + 8,
                             n + 1, n + 3, n + 5, n + 7, n + 9, n + 10]
    p = p.transpose(perm)
    asz = int(np.prod(agg))
    return p.reshape(lead + Lc + (2, 6 * asz))


def from_agg(a: np.ndarray, agg) -> np.ndarray:
    """Inverse of :func:`to_agg`."""
    lead = a.shape[:-6]
    Lc = a.shape[-6:-2]
    n = len(lead)
    p = a.reshape(lead + Lc + (2,) + tuple(agg) + (2, 3))
    # axes: lead..., Tc Zc Yc Xc chi aT aZ aY aX s c
    perm = list(range(n)) + [n + 0, n + 5, n + 1, n + 6, n + 2, n + 7, n + 3, n + 8,
                             n + 4, n + 9, n + 10]
    p = p.transpose(perm)
    L = tuple(Lc[d] * agg[d] for d in range(4))
    return p.reshape(lead + L + (4, 3))


# ----------------------------------------------------------------------------
# interpolation
# ----------------------------------------------------------------------------

class Interpolation:
    """P for one coarsening step: Q factors per (aggregate, chirality)."""

    def __init__(self, test_vectors: np.ndarray, agg):
        """test_vectors [Nv, T,Z,Y,X,4,3]."""
        self.agg = tuple(int(a) for a in agg)
        self.nv = test_vectors.shape[0]
        self.L = tuple(test_vectors.shape[-6:-2])
        self.Lc = coarse_dims(self.L, self.agg)
        W = to_agg(test_vectors, self.agg)              # [Nv, Tc..Xc, 2, 6|a|]
        W = np.moveaxis(W, 0, -1)                       # [Tc..Xc, 2, 6|a|, Nv]
        Q, R = np.linalg.qr(W)
        d = np.diagonal(R, axis1=-2, axis2=-1)
        if np.any(np.abs(d) < 1e-12 * np.linalg.norm(W, axis=(-2, -1))[..., None]):
            raise ValueError("test vectors rank deficient on an aggregate")
        ph = d / np.abs(d)
        self.Q = Q * np.conj(ph)[..., None, :]           # R diagonal now real > 0
        self.R = R * np.conj(ph)[..., :, None]

    def restrict(self, psi: np.ndarray) -> np.ndarray:
        """P^dagger psi: [..., T,Z,Y,X,4,3] -> [..., Tc,Zc,Yc,Xc, 2 Nv]."""
        a = to_agg(psi, self.agg)                        # [..., Lc, 2, 6|a|]
        c = np.einsum("...xk,...x->...k", self.Q.conj(), a)   # [..., Lc, 2, Nv]
        return c.reshape(c.shape[:-2] + (2 * self.nv,))

    def prolong(self, v: np.ndarray) -> np.ndarray:
        """P v: [..., Tc,Zc,Yc,Xc, 2 Nv] -> [..., T,Z,Y,X,4,3]."""
        c = v.reshape(v.shape[:-1] + (2, self.nv))
        a = np.einsum("...xk,...k->...x", self.Q, c)
        return from_agg(a, self.agg)

    def columns(self) -> np.ndarray:
        """P in the canonical column layout [2Nv, T,Z,Y,X,4,3]."""
        E = np.zeros((2 * self.nv,) + self.Lc + (2 * self.nv,), dtype=np.complex128)
        for k in range(2 * self.nv):
            E[k, ..., k] = 1.0
        return self.prolong(E)


# ----------------------------------------------------------------------------
# coarse operator
# ----------------------------------------------------------------------------

def _face_masks(L, agg):
    c = np.meshgrid(*[np.arange(n) for n in L], indexing="ij")
    up = [c[d] % agg[d] == agg[d] - 1 for d in range(4)]
    lo = [c[d] % agg[d] == 0 for d in range(4)]
    return up, lo


class CoarseOperator:
    """D_c(mu_c) = P^dagger D_W P + i mu_c Gamma5_c as a 9-point stencil."""

    def __init__(self, blocks: np.ndarray, nv: int, mu_c: float):
        self.blocks = blocks                      # [Tc,Zc,Yc,Xc,9,2Nv,2Nv], mu-free
        self.nv = nv
        self.Lc = tuple(blocks.shape[:4])
        self.mu_c = mu_c
        self.g5c = np.concatenate([-np.ones(nv), np.ones(nv)])

    @staticmethod
    def build(op: Operator, P: Interpolation, mu_c: float) -> "CoarseOperator":
        """Local formula: project each piece of D_W between aggregates."""
        L, agg, nv = op.L, P.agg, P.nv
        up, lo = _face_masks(L, agg)
        cols = P.columns()                                     # [2Nv, fine]
        blocks = np.zeros(P.Lc + (9, 2 * nv, 2 * nv), dtype=np.complex128)
        # self block: site-diagonal part + hops that stay inside the aggregate
        y = op.diag(cols, mu=0.0)
        for d in range(4):
            y = y + (~up[d])[..., None, None] * op.hop_term(cols, d, +1)
            y = y + (~lo[d])[..., None, None] * op.hop_term(cols, d, -1)
        blocks[..., 0, :, :] = np.moveaxis(P.restrict(y), 0, -1)
        for d in range(4):
            yf = up[d][..., None, None] * op.hop_term(cols, d, +1)
            yb = lo[d][..., None, None] * op.hop_term(cols, d, -1)
            blocks[..., 1 + 2 * d, :, :] = np.moveaxis(P.restrict(yf), 0, -1)
            blocks[..., 2 + 2 * d, :, :] = np.moveaxis(P.restrict(yb), 0, -1)
        return CoarseOperator(blocks, nv, mu_c)

    def with_mu(self, mu_c: float) -> "CoarseOperator":
        return CoarseOperator(self.blocks, self.nv, mu_c)

    def apply(self, v: np.ndarray, mu_c: float | None = None) -> np.ndarray:
        """y(a) = S(a) v(a) + sum_mu [F_mu(a) v(a+mu) + B_mu(a) v(a-mu)] + i mu_c G5c v(a)."""
        mu_c = self.mu_c if mu_c is None else mu_c
        B = self.blocks
        y = np.einsum("...ij,...j->...i", B[..., 0, :, :], v)
        for d in range(4):
            ax = v.ndim - 5 + d
            vf = np.roll(v, -1, axis=ax)
            vb = np.roll(v, +1, axis=ax)
            y = y + np.einsum("...ij,...j->...i", B[..., 1 + 2 * d, :, :], vf)
            y = y + np.einsum("...ij,...j->...i", B[..., 2 + 2 * d, :, :], vb)
        return y + 1j * mu_c * self.g5c * v

    __call__ = apply

    # -- odd-even ----------------------------------------------------------------
    def parity(self) -> np.ndarray:
        c = np.meshgrid(*[np.arange(n) for n in self.Lc], indexing="ij")
        return (c[0] + c[1] + c[2] + c[3]) % 2

    def self_inverse(self) -> np.ndarray:
        """(S(a) + i mu_c Gamma5_c)^-1 per coarse site."""
        M = self.blocks[..., 0, :, :] + 1j * self.mu_c * np.diag(self.g5c)
        return np.linalg.inv(M)

    def hop(self, v: np.ndarray) -> np.ndarray:
        """Off-diagonal (hopping) part of D_c."""
        return self.apply(v, mu_c=0.0) - np.einsum(
            "...ij,...j->...i", self.blocks[..., 0, :, :], v)

    def diag_apply(self, v: np.ndarray) -> np.ndarray:
        return np.einsum("...ij,...j->...i", self.blocks[..., 0, :, :], v) \
            + 1j * self.mu_c * self.g5c * v


class OddEvenCoarse:
    """Schur complement S = D_ee - D_eo D_oo^-1 D_oe of D_c(mu_c) (Sec. 3)."""

    def __init__(self, Dc: CoarseOperator):
        for n in Dc.Lc:
            if n % 2:
                raise ValueError("odd-even needs even coarse extents")
        self.Dc = Dc
        par = Dc.parity()
        self.even = (par == 0)[..., None]
        self.odd = (par == 1)[..., None]
        self.inv = Dc.self_inverse()

    def _oo_inv(self, v):
        return np.einsum("...ij,...j->...i", self.inv, v) * self.odd

    def schur(self, ve: np.ndarray) -> np.ndarray:
        """S v_e for v_e supported on even sites."""
        Dc = self.Dc
        t = self._oo_inv(Dc.hop(ve * self.even))
        return (Dc.diag_apply(ve) - Dc.hop(t)) * self.even

    def reduced_rhs(self, b: np.ndarray) -> np.ndarray:
        """b_e - D_eo D_oo^-1 b_o."""
        return (b - self.Dc.hop(self._oo_inv(b))) * self.even

    def reconstruct(self, b: np.ndarray, xe: np.ndarray) -> np.ndarray:
        """x = x_e + D_oo^-1 (b_o - D_oe x_e)."""
        xe = xe * self.even
        return xe + self._oo_inv(b - self.Dc.hop(xe))
