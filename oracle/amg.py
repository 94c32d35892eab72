"""Two-level DD-alphaAMG: K-cycle of eq. (1), adaptive setup, FGMRES solve (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed
-----------------------
* Sec. 1, eq. (1): the preconditioner's error propagation is
  (I - M D)^k (I - P D_c^-1 P^dagger D) (I - M D)^j: j pre-smoothing SAP
  sweeps, a coarse-grid correction, k post-smoothing sweeps.
* Sec. 1: the test vectors come from an adaptive setup phase; Fig. 1 uses
  three setup iterations for few right-hand sides and five for many.
* Sec. 1: mu_coarse = delta * mu on the coarsest grid, delta >= 1.
* Sec. 3: odd-even preconditioning on the coarsest level; the full fine
  operator is used by the outer solver.
* Sec. 1: one setup serves D(+mu) and D(-mu) (D_c(mu) = D_c + i mu Gamma5_c,
  so only the coarse diagonal shift changes); Sec. 3: the squared operator is
  inverted by two solves of the non-squared operator,
  (D(mu)^dagger D(mu))^-1 = D(mu)^-1 Gamma5 D(-mu)^-1 Gamma5, using
  D(mu)^dagger = Gamma5 D(-mu) Gamma5.

Readings (choices where the paper is silent)
------------------------------
* B(v): x = 0; j sweeps of SAP on D x = v; r = v - D x; e_c = coarse solve of
  D_c(delta*mu) e_c = P^dagger r; x += P e_c; k sweeps of SAP on D x = v.
* Coarse solve: GMRES(coarse_restart) on the odd-even Schur complement of
  D_c(delta*mu) from zero, to a residual ``coarse_tol`` relative to the
  reduced right-hand side, at most ``coarse_maxit`` steps.
* Odd-site twisted-mass shift rho (Sec. 2): the fine operator carries mu on
  even and mu + rho on odd sites; the coarse operator is the Galerkin
  projection P^dagger (D_W + i rho Pi_odd Gamma5) P with i delta mu Gamma5_c
  added, i.e. delta raises the common twisted mass only.
* Setup: each random v_i gets ``init_sweeps`` SAP sweeps on D v = 0 (i.e.
  v_i <- (I - M D) v_i) and is normalised; P and D_c are built; then
  ``setup_iters`` times: every v_i <- B(v_i) with the current P, D_c,
  normalised; P and D_c are rebuilt after each full pass over i.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .dirac import Operator
from .sap import SAP
from .coarse import Interpolation, CoarseOperator, OddEvenCoarse
from .krylov import gmres


@dataclass
class AMGParams:
    m0: float
    c_sw: float
    mu: float
    delta: float = 1.0
    bc_t: float = -1.0
    nv: int = 8
    agg: tuple = (2, 2, 2, 2)
    sap_block: tuple = (2, 2, 2, 2)
    mr_iters: int = 4
    pre_smooth: int = 0
    post_smooth: int = 4
    block_oe: bool = False
    init_sweeps: int = 3
    setup_iters: int = 3
    coarse_tol: float = 5e-2
    coarse_restart: int = 30
    coarse_maxit: int = 200
    restart: int = 25
    maxit: int = 1000
    rho: float = 0.0          # odd-site twisted-mass shift (Sec. 2): mu + rho on odd sites
    extra: dict = field(default_factory=dict)


def normalise(v: np.ndarray) -> np.ndarray:
    """v_i / ||v_i|| for a stack of vectors [n, ...]."""
    n = np.sqrt((np.abs(v) ** 2).reshape(v.shape[0], -1).sum(axis=1))
    return v / n.reshape((-1,) + (1,) * (v.ndim - 1))


class TwoLevel:
    """Operators of a two-level hierarchy for a fixed gauge field."""

    def __init__(self, U: np.ndarray, prm: AMGParams):
        self.prm = prm
        self.op = Operator(U, prm.m0, prm.c_sw, prm.mu, prm.bc_t, rho=prm.rho)
        self.sap = SAP(self.op, prm.sap_block, prm.mr_iters, prm.block_oe)
        self.P = None
        self.Dc = None
        self.oe = None
        self.coarse_iters = []

    # -- hierarchy -----------------------------------------------------------------
    def build_coarse(self, test_vectors: np.ndarray) -> None:
        """P from the test vectors, D_c(delta*mu), odd-even Schur data."""
        self.P = Interpolation(test_vectors, self.prm.agg)
        self.Dc = CoarseOperator.build(self.op, self.P, self.prm.delta * self.prm.mu)
        self.oe = OddEvenCoarse(self.Dc)

    def coarse_solve(self, rc: np.ndarray, tol=None, maxit=None) -> np.ndarray:
        """Odd-even GMRES on D_c(delta*mu) e = rc (one coarse vector)."""
        prm = self.prm
        tol = prm.coarse_tol if tol is None else tol
        maxit = prm.coarse_maxit if maxit is None else maxit
        bh = self.oe.reduced_rhs(rc)
        res = gmres(self.oe.schur, bh, tol=tol, restart=prm.coarse_restart, maxit=maxit)
        self.coarse_iters.append(res.iters)
        return self.oe.reconstruct(rc, res.x)

    def kcycle(self, v: np.ndarray, coarse_tol=None, coarse_maxit=None) -> np.ndarray:
        """z = B(v), eq. (1)."""
        prm = self.prm
        x = np.zeros_like(v)
        x = self.sap.smooth(v, x, prm.pre_smooth)
        r = v - self.op.apply(x) if prm.pre_smooth else v
        rc = self.P.restrict(r)
        ec = self.coarse_solve(rc, coarse_tol, coarse_maxit)
        x = x + self.P.prolong(ec)
        x = self.sap.smooth(v, x, prm.post_smooth)
        return x

    # -- setup -------------------------------------------------------------------------
    def setup(self, v0: np.ndarray, setup_iters=None) -> np.ndarray:
        """Adaptive setup from random vectors v0 [Nv, T,Z,Y,X,4,3]; returns the v_i."""
        prm = self.prm
        iters = prm.setup_iters if setup_iters is None else setup_iters
        v = v0.copy()
        zero = np.zeros_like(v)
        for _ in range(prm.init_sweeps):
            v = self.sap.sweep(zero, v)
        v = normalise(v)
        self.build_coarse(v)
        for _ in range(iters):
            v = np.stack([self.kcycle(v[i]) for i in range(v.shape[0])])
            v = normalise(v)
            self.build_coarse(v)
        self.test_vectors = v
        return v

    def update(self, iters: int, v: np.ndarray | None = None) -> np.ndarray:
        """Setup update (Sec. 3: after the gauge field changes the setup is updated
        by a few iterations instead of rebuilt): P and D_c from the current test
        vectors on this operator, then `iters` iterations v_i <- B(v_i) as in setup."""
        v = (self.test_vectors if v is None else v).copy()
        self.build_coarse(v)
        for _ in range(iters):
            v = np.stack([self.kcycle(v[i]) for i in range(v.shape[0])])
            v = normalise(v)
            self.build_coarse(v)
        self.test_vectors = v
        return v

    # -- solve -----------------------------------------------------------------------
    def solve(self, b: np.ndarray, tol: float = 1e-10, x0=None):
        prm = self.prm
        return gmres(self.op.apply, b, x0=x0, tol=tol, restart=prm.restart,
                     maxit=prm.maxit, M=self.kcycle)

    def set_mu(self, mu: float) -> None:
        """Switch to D(mu) keeping P and the mu-free D_c (only shifts change)."""
        self.prm.mu = mu
        self.op = self.op.with_mu(mu)
        self.sap = SAP(self.op, self.prm.sap_block, self.prm.mr_iters, self.prm.block_oe)
        if self.Dc is not None:
            self.Dc = self.Dc.with_mu(self.prm.delta * mu)
            self.oe = OddEvenCoarse(self.Dc)

    def set_mu_eo(self, mu_even: float, mu_odd: float) -> None:
        """Twisted mass mu_even on the even and mu_odd on the odd sites (Sec. 2)
        with the same P; the odd shift enters D_c through the Galerkin
        projection, so D_c is projected again from the kept P."""
        self.prm.mu, self.prm.rho = mu_even, mu_odd - mu_even
        self.op = self.op.with_mu_eo(mu_even, mu_odd)
        self.sap = SAP(self.op, self.prm.sap_block, self.prm.mr_iters, self.prm.block_oe)
        if self.P is not None:
            self.Dc = CoarseOperator.build(self.op, self.P, self.prm.delta * mu_even)
            self.oe = OddEvenCoarse(self.Dc)

    def solve_squared(self, b: np.ndarray, tol: float = 1e-10):
        """x = (D(mu)^dagger D(mu))^-1 b as D(mu)^-1 Gamma5 D(-mu)^-1 Gamma5 b."""
        from .dirac import gamma5_field
        mu = self.prm.mu
        self.set_mu(-mu)
        r1 = self.solve(gamma5_field(b), tol=tol)
        self.set_mu(mu)
        r2 = self.solve(gamma5_field(r1.x), tol=tol)
        return r2.x, (r1, r2)
