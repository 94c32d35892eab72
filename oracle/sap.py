"""The SAP smoother M of eq. (1) (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed
-----------------------
* Sec. 1: the smoother M in eq. (1) is the Schwarz Alternating Procedure, a
  domain-decomposition method that damps the UV part of the error.
* Sec. 3: odd-even preconditioning is used in the smoother (and on the
  coarsest level) but not on the full fine operator.

Readings where the paper is silent
--------------------------------------------------------
* Domains are the blocks of ``block`` dims.  A block's colour is the parity
  of the sum of its block coordinates; colour 0 ("red") goes first.
* The block operator D_B is D restricted to the block with Dirichlet
  boundaries: hops whose target lies in another block are dropped.
* One sweep: for each colour in (red, black): r = b - D x on the whole
  lattice; on every block B of that colour, independently, e_B is n_MR
  minimal-residual steps on D_B e = r_B from e = 0; then x_B += e_B.
* MR step: q = D_B r; alpha = <q, r>/<q, q>; e += alpha r; r -= alpha q.
* Odd-even option (``block_oe``): the MR steps run on the block Schur
  complement D_ee - D_eo D_oo^-1 D_oe over the block's even sites (site
  parity = (t+z+y+x) mod 2), with the odd sites recovered afterwards.

Pins (tests/test_oracle_sap.py): one block covering the lattice is textbook
global MR; D_B is the sub-matrix of the dense D; with exact block solves a
sweep equals dense block Gauss-Seidel (red then black); the MR residual norm
never increases; the odd-even variant solves the same block system.
"""
from __future__ import annotations

import numpy as np

from .dirac import Operator, ONE4, GAMMA, GAMMA5, spin_mul, hop_forward, hop_backward


def _site_coords(L):
    return np.meshgrid(*[np.arange(n) for n in L], indexing="ij")


def block_ids(L, block) -> np.ndarray:
    """Per-site block coordinates, [4, T, Z, Y, X]."""
    c = _site_coords(L)
    return np.stack([c[d] // block[d] for d in range(4)])


def block_colour(L, block) -> np.ndarray:
    """Per-site block colour (sum of block coordinates mod 2), [T,Z,Y,X]."""
    return block_ids(L, block).sum(axis=0) % 2


def same_block_masks(L, block):
    """masks[d][s]: True where the hop from x in direction s*d_hat stays in x's block."""
    c = _site_coords(L)
    out = []
    for d in range(4):
        n = L[d]
        fw = ((c[d] + 1) % n) // block[d] == c[d] // block[d]
        bw = ((c[d] - 1) % n) // block[d] == c[d] // block[d]
        out.append((fw, bw))
    return out


class SAP:
    """Red/black multiplicative Schwarz with block-local MR (or exact) solves."""

    def __init__(self, op: Operator, block, n_mr: int = 4, block_oe: bool = False):
        self.op = op
        self.L = op.L
        self.block = tuple(int(b) for b in block)
        for d in range(4):
            if self.L[d] % self.block[d]:
                raise ValueError("lattice not divisible by SAP block")
        self.n_mr = n_mr
        self.block_oe = block_oe
        self.colour = block_colour(self.L, self.block)
        self.masks = same_block_masks(self.L, self.block)
        c = _site_coords(self.L)
        self.site_parity = (c[0] + c[1] + c[2] + c[3]) % 2

    # -- block operator ------------------------------------------------------
    def apply_block(self, psi: np.ndarray, mu: float | None = None) -> np.ndarray:
        """D_B psi for every block at once (Dirichlet: cross-block hops dropped)."""
        op = self.op
        y = op.diag(psi, mu)
        for d in range(4):
            fw, bw = self.masks[d]
            y = y - 0.5 * fw[..., None, None] * spin_mul(
                ONE4 - GAMMA[d], hop_forward(op.U, psi, d, op.bc_t))
            y = y - 0.5 * bw[..., None, None] * spin_mul(
                ONE4 + GAMMA[d], hop_backward(op.U, psi, d, op.bc_t))
        return y

    def block_sum(self, f: np.ndarray) -> np.ndarray:
        """Sum a per-site array [..., T,Z,Y,X] over each block -> [..., nT,nZ,nY,nX]."""
        L, b = self.L, self.block
        sh = f.shape[:-4] + (L[0] // b[0], b[0], L[1] // b[1], b[1],
                             L[2] // b[2], b[2], L[3] // b[3], b[3])
        return f.reshape(sh).sum(axis=(-7, -5, -3, -1))

    def block_expand(self, g: np.ndarray) -> np.ndarray:
        """Broadcast a per-block array [..., nT,nZ,nY,nX] back to sites."""
        for d in range(4):
            g = np.repeat(g, self.block[d], axis=g.ndim - 4 + d)
        return g

    def _block_dot(self, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        return self.block_sum((np.conj(a) * b).sum(axis=(-2, -1)))

    # -- block solvers ----------------------------------------------------------
    def mr(self, r: np.ndarray, mask: np.ndarray) -> np.ndarray:
        """n_MR minimal-residual steps on D_B e = r for all blocks in ``mask``."""
        m = mask[..., None, None]
        r = r * m
        e = np.zeros_like(r)
        for _ in range(self.n_mr):
            q = self.apply_block(r) * m
            qr = self._block_dot(q, r)
            qq = self._block_dot(q, q).real
            alpha = np.where(qq > 0, qr / np.where(qq > 0, qq, 1.0), 0.0)
            a = self.block_expand(alpha)[..., None, None]
            e = e + a * r
            r = r - a * q
        return e

    def mr_history(self, r: np.ndarray, mask: np.ndarray) -> list[np.ndarray]:
        """Per-block residual norms after each MR step (for the monotonicity pin)."""
        m = mask[..., None, None]
        r = r * m
        hist = [np.sqrt(self.block_sum((np.abs(r) ** 2).sum(axis=(-2, -1))))]
        for _ in range(self.n_mr):
            q = self.apply_block(r) * m
            qr = self._block_dot(q, r)
            qq = self._block_dot(q, q).real
            alpha = np.where(qq > 0, qr / np.where(qq > 0, qq, 1.0), 0.0)
            a = self.block_expand(alpha)[..., None, None]
            r = r - a * q
            hist.append(np.sqrt(self.block_sum((np.abs(r) ** 2).sum(axis=(-2, -1)))))
        return hist

    # odd-even block solve ------------------------------------------------------
    def _diag_inverse(self):
        """Per-site inverse of A(x) + i mu(x) gamma5 (12x12), computed once per mu."""
        key = (self.op.mu, self.op.rho)
        if getattr(self, "_dinv_mu", None) != key:
            D = self.op.A + 1j * self.op.mu_field()[..., None, None] * np.kron(GAMMA5, np.eye(3))
            self._dinv = np.linalg.inv(D)
            self._dinv_mu = key
        return self._dinv

    def _diag_solve(self, psi):
        sh = psi.shape
        y = np.einsum("...ij,...j->...i", self._diag_inverse(), psi.reshape(sh[:-2] + (12,)))
        return y.reshape(sh)

    def _hop_block(self, psi):
        """D_B psi - diag psi: the intra-block hopping part."""
        return self.apply_block(psi) - self.op.diag(psi)

    def mr_oe(self, r: np.ndarray, mask: np.ndarray) -> np.ndarray:
        """n_MR MR steps on the block Schur complement, then odd back-substitution.

        D_B = [[D_ee, D_eo], [D_oe, D_oo]] on each block (site parity); the
        hopping part only couples even and odd sites, D_ee and D_oo are the
        site-diagonal terms.  S = D_ee - D_eo D_oo^-1 D_oe acts on even sites;
        rhs r_e - D_eo D_oo^-1 r_o; e_o = D_oo^-1 (r_o - D_oe e_e).
        """
        m = mask[..., None, None]
        ev = (self.site_parity == 0)[..., None, None]
        od = ~ev
        r = r * m

        def S(v):  # v supported on even sites of masked blocks
            t = self._diag_solve(self._hop_block(v) * od)
            return (self.op.diag(v) - self._hop_block(t)) * ev * m

        rhs = (r * ev - self._hop_block(self._diag_solve(r * od)) * ev) * m
        e = np.zeros_like(r)
        res = rhs
        for _ in range(self.n_mr):
            q = S(res)
            qr = self._block_dot(q, res)
            qq = self._block_dot(q, q).real
            alpha = np.where(qq > 0, qr / np.where(qq > 0, qq, 1.0), 0.0)
            a = self.block_expand(alpha)[..., None, None]
            e = e + a * res
            res = res - a * q
        e_o = self._diag_solve((r * od - self._hop_block(e) * od)) * m * od
        return e * ev + e_o

    # -- sweeps ------------------------------------------------------------------
    def sweep(self, b: np.ndarray, x: np.ndarray, block_solve=None) -> np.ndarray:
        """One SAP sweep on D x = b: red blocks, then black blocks."""
        solve = block_solve or (self.mr_oe if self.block_oe else self.mr)
        x = x.copy()
        for colour in (0, 1):
            mask = self.colour == colour
            if not mask.any():
                continue
            r = b - self.op.apply(x)
            x = x + solve(r, mask) * mask[..., None, None]
        return x

    def smooth(self, b: np.ndarray, x: np.ndarray, sweeps: int) -> np.ndarray:
        for _ in range(sweeps):
            x = self.sweep(b, x)
        return x
