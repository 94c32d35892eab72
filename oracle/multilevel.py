"""Three-level DD-alphaAMG (oracle): coarse-grid SAP, a second aggregation and
the level-1 K-cycle inside the fine K-cycle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed
-----------------------
* Sec. 2: the standard DD-alphaAMG setup is a three-level multigrid with
  aggregates of 4^4 fine sites, then 2^4 sites of the first coarse grid.
* Sec. 1: mu_coarse = delta * mu is used on the coarsest grid only.
* Sec. 1, eq. (1): each level's preconditioner is the K-cycle error
  propagation (I - M D)^k (I - P D_c^-1 P^dagger D) (I - M D)^j.
* Sec. 3 (Listing 1): MGSetupIter fine setup iterations and
  MGCoarseSetupIter setup iterations on the first coarse grid.
* Sec. 3: odd-even preconditioning on the coarsest level and in the smoother.

Readings (choices where the paper is silent)
------------------------------
* Level 1 carries D_c1(mu) = P1^dagger D_W P1 + i mu Gamma5_c (mu itself);
  level 2 D_c2(delta mu) = P2^dagger D_c1(0) P2 + i delta mu Gamma5_c2.
* The coarse solve of the fine K-cycle is FGMRES(coarse_restart) on
  D_c1(mu) from zero to ``coarse_tol``, preconditioned by the level-1 K-cycle:
  x = 0; j1 coarse SAP sweeps; r = v - D_c1 x; e_2 = odd-even GMRES on
  D_c2(delta mu) to ``coarsest_tol``; x += P2 e_2; k1 coarse SAP sweeps.
* Coarse SAP: blocks of ``sap_block1`` coarse sites, colour = parity of the
  block coordinates, Dirichlet block operator of the 9-point stencil, n_MR
  MR steps, red then black.
* Level-1 aggregation: aggregates of ``agg2`` coarse sites, split by level-1
  chirality (first N_v1 components chirality -1); P2 per (aggregate,
  chirality) is the thin QR with real positive R diagonal of the
  N_v2 level-1 test vectors.
* Setup: fine initial phase (random v_i, init SAP sweeps, P1, D_c1); level-1
  initial phase (random level-1 vectors w_j, init coarse SAP sweeps on
  D_c1 w = 0, P2, D_c2); then ``setup_iters`` times every v_i <- B(v_i) with the
  three-level cycle, P1, D_c1 rebuilt and P2, D_c2 rebuilt from the current
  w_j; finally ``coarse_setup_iters`` times every w_j <- B1(w_j) with the
  level-1 cycle and P2, D_c2 rebuilt.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .dirac import Operator
from .sap import SAP
from .coarse import Interpolation, CoarseOperator, OddEvenCoarse, coarse_dims
from .krylov import gmres
from .amg import AMGParams, normalise


# ----------------------------------------------------------------------------
# coarse-lattice helpers
# ----------------------------------------------------------------------------

def _coords(Lc):
    return np.meshgrid(*[np.arange(n) for n in Lc], indexing="ij")


class CoarseSAP:
    """Red/black SAP with block MR on a 9-point coarse stencil."""

    def __init__(self, Dc: CoarseOperator, block, n_mr: int):
        self.Dc = Dc
        self.Lc = Dc.Lc
        self.block = tuple(int(b) for b in block)
        for d in range(4):
            if self.Lc[d] % self.block[d]:
                raise ValueError("coarse lattice not divisible by the coarse SAP block")
        self.n_mr = n_mr
        c = _coords(self.Lc)
        bid = [c[d] // self.block[d] for d in range(4)]
        self.colour = (bid[0] + bid[1] + bid[2] + bid[3]) % 2
        # hop (forward / backward in d) stays inside the block?
        self.fw, self.bw = [], []
        for d in range(4):
            n = self.Lc[d]
            self.fw.append(((c[d] + 1) % n) // self.block[d] == bid[d])
            self.bw.append(((c[d] - 1) % n) // self.block[d] == bid[d])

    def apply_block(self, v: np.ndarray) -> np.ndarray:
        """D_B v for every block (hops to other blocks dropped)."""
        B = self.Dc.blocks
        y = np.einsum("...ij,...j->...i", B[..., 0, :, :], v)
        for d in range(4):
            ax = v.ndim - 5 + d
            vf = np.roll(v, -1, axis=ax)
            vb = np.roll(v, +1, axis=ax)
            y = y + self.fw[d][..., None] * np.einsum("...ij,...j->...i", B[..., 1 + 2 * d, :, :], vf)
            y = y + self.bw[d][..., None] * np.einsum("...ij,...j->...i", B[..., 2 + 2 * d, :, :], vb)
        return y + 1j * self.Dc.mu_c * self.Dc.g5c * v

    def block_sum(self, f: np.ndarray) -> np.ndarray:
        L, b = self.Lc, self.block
        sh = f.shape[:-4] + (L[0] // b[0], b[0], L[1] // b[1], b[1], L[2] // b[2], b[2], L[3] // b[3], b[3])
        return f.reshape(sh).sum(axis=(-7, -5, -3, -1))

    def block_expand(self, g: np.ndarray) -> np.ndarray:
        for d in range(4):
            g = np.repeat(g, self.block[d], axis=g.ndim - 4 + d)
        return g

    def mr(self, r: np.ndarray, mask: np.ndarray) -> np.ndarray:
        m = mask[..., None]
        r = r * m
        e = np.zeros_like(r)
        for _ in range(self.n_mr):
            q = self.apply_block(r) * m
            qr = self.block_sum((np.conj(q) * r).sum(axis=-1))
            qq = self.block_sum((np.abs(q) ** 2).sum(axis=-1))
            alpha = np.where(qq > 0, qr / np.where(qq > 0, qq, 1.0), 0.0)
            a = self.block_expand(alpha)[..., None]
            e = e + a * r
            r = r - a * q
        return e

    def sweep(self, b: np.ndarray, x: np.ndarray, block_solve=None) -> np.ndarray:
        solve = block_solve or self.mr
        x = x.copy()
        for colour in (0, 1):
            mask = self.colour == colour
            if not mask.any():
                continue
            r = b - self.Dc.apply(x)
            x = x + solve(r, mask) * mask[..., None]
        return x

    def smooth(self, b, x, sweeps):
        for _ in range(sweeps):
            x = self.sweep(b, x)
        return x


def to_cagg(v: np.ndarray, agg, nv1: int) -> np.ndarray:
    """[..., Lc1(4), 2 Nv1] -> [..., Lc2(4), 2(chi), |a| * Nv1] (rows: site, i)."""
    Lc1 = v.shape[-5:-1]
    Lc2 = coarse_dims(Lc1, agg)
    lead = v.shape[:-5]
    n = len(lead)
    p = v.reshape(lead + (Lc2[0], agg[0], Lc2[1], agg[1], Lc2[2], agg[2], Lc2[3], agg[3], 2, nv1))
    perm = list(range(n)) + [n + 0, n + 2, n + 4, n + 6, n + 8, n + 1, n + 3, n + 5, n + 7, n + 9]
    p = p.transpose(perm)
    return p.reshape(lead + Lc2 + (2, int(np.prod(agg)) * nv1))


def from_cagg(a: np.ndarray, agg, nv1: int) -> np.ndarray:
    lead = a.shape[:-6]
    Lc2 = a.shape[-6:-2]
    n = len(lead)
    p = a.reshape(lead + Lc2 + (2,) + tuple(agg) + (nv1,))
    perm = list(range(n)) + [n + 0, n + 5, n + 1, n + 6, n + 2, n + 7, n + 3, n + 8, n + 4, n + 9]
    p = p.transpose(perm)
    Lc1 = tuple(Lc2[d] * agg[d] for d in range(4))
    return p.reshape(lead + Lc1 + (2 * nv1,))


class CoarseInterpolation:
    """P2 between level 1 (n1 = 2 Nv1 per site) and level 2 (2 Nv2 per site)."""

    def __init__(self, w: np.ndarray, agg, nv1: int):
        """w: level-1 test vectors [Nv2, Lc1(4), 2 Nv1]."""
        self.agg = tuple(int(a) for a in agg)
        self.nv1 = nv1
        self.nv = w.shape[0]
        self.Lc1 = tuple(w.shape[1:5])
        self.Lc = coarse_dims(self.Lc1, self.agg)
        W = np.moveaxis(to_cagg(w, self.agg, nv1), 0, -1)     # [Lc2, 2, rows, Nv2]
        Q, R = np.linalg.qr(W)
        d = np.diagonal(R, axis1=-2, axis2=-1)
        if np.any(np.abs(d) < 1e-12 * np.linalg.norm(W, axis=(-2, -1))[..., None]):
            raise ValueError("level-1 test vectors rank deficient on an aggregate")
        ph = d / np.abs(d)
        self.Q = Q * np.conj(ph)[..., None, :]

    def restrict(self, v: np.ndarray) -> np.ndarray:
        a = to_cagg(v, self.agg, self.nv1)
        c = np.einsum("...xk,...x->...k", self.Q.conj(), a)
        return c.reshape(c.shape[:-2] + (2 * self.nv,))

    def prolong(self, v: np.ndarray) -> np.ndarray:
        c = v.reshape(v.shape[:-1] + (2, self.nv))
        a = np.einsum("...xk,...k->...x", self.Q, c)
        return from_cagg(a, self.agg, self.nv1)

    def columns(self) -> np.ndarray:
        """P2 as level-1 fields, [2 Nv2, Lc1(4), 2 Nv1] (column chi*Nv2 + j)."""
        E = np.zeros((2 * self.nv,) + self.Lc + (2 * self.nv,), dtype=np.complex128)
        for k in range(2 * self.nv):
            E[k, ..., k] = 1.0
        return self.prolong(E)


def galerkin_coarse(Dc1: CoarseOperator, P2: CoarseInterpolation, mu_c: float) -> CoarseOperator:
    """D_c2 = P2^dagger D_c1(0) P2 as a 9-point stencil (blocks by crossed face)."""
    Lc1, agg = Dc1.Lc, P2.agg
    c = _coords(Lc1)
    up = [c[d] % agg[d] == agg[d] - 1 for d in range(4)]
    lo = [c[d] % agg[d] == 0 for d in range(4)]
    B = Dc1.blocks
    cols = P2.columns()                                   # [K, Lc1, n1]
    nv2 = P2.nv
    blocks = np.zeros(P2.Lc + (9, 2 * nv2, 2 * nv2), dtype=np.complex128)

    def hop(d, fwd):
        ax = cols.ndim - 5 + d
        src = np.roll(cols, -1 if fwd else +1, axis=ax)
        return np.einsum("...ij,...j->...i", B[..., (1 if fwd else 2) + 2 * d, :, :], src)

    y = np.einsum("...ij,...j->...i", B[..., 0, :, :], cols)
    for d in range(4):
        y = y + (~up[d])[..., None] * hop(d, True) + (~lo[d])[..., None] * hop(d, False)
    blocks[..., 0, :, :] = np.moveaxis(P2.restrict(y), 0, -1)
    for d in range(4):
        blocks[..., 1 + 2 * d, :, :] = np.moveaxis(P2.restrict(up[d][..., None] * hop(d, True)), 0, -1)
        blocks[..., 2 + 2 * d, :, :] = np.moveaxis(P2.restrict(lo[d][..., None] * hop(d, False)), 0, -1)
    return CoarseOperator(blocks, nv2, mu_c)


# ----------------------------------------------------------------------------
# three levels
# ----------------------------------------------------------------------------

@dataclass
class ThreeLevelParams(AMGParams):
    nv2: int = 4
    agg2: tuple = (2, 2, 2, 2)
    sap_block1: tuple = (2, 2, 2, 2)
    mr_iters1: int = 4
    pre_smooth1: int = 0
    post_smooth1: int = 2
    init_sweeps1: int = 3
    coarse_setup_iters: int = 3
    coarsest_tol: float = 5e-2
    coarsest_maxit: int = 200


class ThreeLevel:
    """Fine level, first coarse level (FGMRES + K-cycle), coarsest level (odd-even GMRES)."""

    def __init__(self, U: np.ndarray, prm: ThreeLevelParams):
        self.prm = prm
        self.op = Operator(U, prm.m0, prm.c_sw, prm.mu, prm.bc_t, rho=prm.rho)
        self.sap = SAP(self.op, prm.sap_block, prm.mr_iters, prm.block_oe)
        self.coarse_iters = []
        self.coarsest_iters = []

    # -- hierarchy ---------------------------------------------------------------
    def build_level1(self, v: np.ndarray) -> None:
        prm = self.prm
        self.P1 = Interpolation(v, prm.agg)
        self.Dc1 = CoarseOperator.build(self.op, self.P1, prm.mu)       # level 1 keeps mu
        self.csap = CoarseSAP(self.Dc1, prm.sap_block1, prm.mr_iters1)

    def build_level2(self, w: np.ndarray) -> None:
        prm = self.prm
        self.P2 = CoarseInterpolation(w, prm.agg2, prm.nv)
        self.Dc2 = galerkin_coarse(self.Dc1, self.P2, prm.delta * prm.mu)  # coarsest: delta mu
        self.oe2 = OddEvenCoarse(self.Dc2)

    # -- cycles ------------------------------------------------------------------
    def coarsest_solve(self, r2: np.ndarray, tol=None, maxit=None) -> np.ndarray:
        prm = self.prm
        tol = prm.coarsest_tol if tol is None else tol
        maxit = prm.coarsest_maxit if maxit is None else maxit
        res = gmres(self.oe2.schur, self.oe2.reduced_rhs(r2), tol=tol, restart=prm.coarse_restart,
                    maxit=maxit)
        self.coarsest_iters.append(res.iters)
        return self.oe2.reconstruct(r2, res.x)

    def kcycle1(self, v1: np.ndarray, coarsest_tol=None, coarsest_maxit=None) -> np.ndarray:
        """B1(v1): the level-1 K-cycle of eq. (1)."""
        prm = self.prm
        x = np.zeros_like(v1)
        x = self.csap.smooth(v1, x, prm.pre_smooth1)
        r = v1 - self.Dc1.apply(x) if prm.pre_smooth1 else v1
        e2 = self.coarsest_solve(self.P2.restrict(r), coarsest_tol, coarsest_maxit)
        x = x + self.P2.prolong(e2)
        return self.csap.smooth(v1, x, prm.post_smooth1)

    def level1_solve(self, r1: np.ndarray, tol=None, maxit=None) -> np.ndarray:
        prm = self.prm
        tol = prm.coarse_tol if tol is None else tol
        maxit = prm.coarse_maxit if maxit is None else maxit
        res = gmres(self.Dc1.apply, r1, tol=tol, restart=prm.coarse_restart, maxit=maxit, M=self.kcycle1)
        self.coarse_iters.append(res.iters)
        return res.x

    def kcycle(self, v: np.ndarray) -> np.ndarray:
        """B(v): the fine K-cycle with the level-1 FGMRES as coarse solve."""
        prm = self.prm
        x = np.zeros_like(v)
        x = self.sap.smooth(v, x, prm.pre_smooth)
        r = v - self.op.apply(x) if prm.pre_smooth else v
        x = x + self.P1.prolong(self.level1_solve(self.P1.restrict(r)))
        return self.sap.smooth(v, x, prm.post_smooth)

    # -- setup and solve -------------------------------------------------------------
    def setup(self, v0: np.ndarray, w0: np.ndarray):
        prm = self.prm
        v = v0.copy()
        zero = np.zeros_like(v)
        for _ in range(prm.init_sweeps):
            v = self.sap.sweep(zero, v)
        v = normalise(v)
        self.build_level1(v)
        w = w0.copy()
        zw = np.zeros_like(w)
        for _ in range(prm.init_sweeps1):
            w = self.csap.sweep(zw, w)
        w = normalise(w)
        self.build_level2(w)
        for _ in range(prm.setup_iters):
            v = normalise(np.stack([self.kcycle(v[i]) for i in range(v.shape[0])]))
            self.build_level1(v)
            self.build_level2(w)
        for _ in range(prm.coarse_setup_iters):
            w = normalise(np.stack([self.kcycle1(w[j]) for j in range(w.shape[0])]))
            self.build_level2(w)
        self.test_vectors, self.test_vectors1 = v, w
        return v, w

    def update(self, fine_iters: int, coarse_iters: int, v=None, w=None):
        """Setup update (Sec. 3: one fine and three first-coarse-grid iterations
        after the gauge field changes): P1, D_c1 and P2, D_c2 from the current
        test vectors, then the fine and the level-1 iterations of setup."""
        v = (self.test_vectors if v is None else v).copy()
        w = (self.test_vectors1 if w is None else w).copy()
        self.build_level1(v)
        self.build_level2(w)
        for _ in range(fine_iters):
            v = normalise(np.stack([self.kcycle(v[i]) for i in range(v.shape[0])]))
            self.build_level1(v)
            self.build_level2(w)
        for _ in range(coarse_iters):
            w = normalise(np.stack([self.kcycle1(w[j]) for j in range(w.shape[0])]))
            self.build_level2(w)
        self.test_vectors, self.test_vectors1 = v, w
        return v, w

    def solve(self, b: np.ndarray, tol: float = 1e-10, x0=None):
        prm = self.prm
        return gmres(self.op.apply, b, x0=x0, tol=tol, restart=prm.restart, maxit=prm.maxit, M=self.kcycle)
