"""Odd-even conjugate gradient on the normal equations: the comparison solver of Fig. 1 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed
-----------------------
* Sec. 1, Fig. 1: DD-alphaAMG is compared with oeCG, the conjugate gradient
  method on the odd-even preconditioned twisted-mass clover operator, the
  standard solver before multigrid; the speed-up includes the setup time and
  grows with the number of right-hand sides.
* Sec. 3: the odd-even reduced operator lives on the odd sites,
  D^ = D_oo - D_oe D_ee^-1 D_eo (``oracle.evenodd.reduced_apply``), and
  D^(mu)^dagger = G^5 D^(-mu) G^5 (Gamma5-hermiticity; a shift rho on the odd
  sites flips sign with mu).

Readings (choices where the paper is silent)
------------------------------
* oeCG is CG on D^dagger D^ x_o = D^dagger b^, written in the CGLS form that
  carries the residual r = b^ - D^ x_o of the non-squared system:
    x = 0, r = b^, s = D^dagger r, p = s, gamma = |s|^2;
    per step: q = D^ p, alpha = gamma / |q|^2, x += alpha p, r -= alpha q,
    s = D^dagger r, beta = |s|^2 / gamma, gamma = |s|^2, p = s + beta p.
* Right-hand side and solution of the full system D x = b:
    b^ = b_o - D_oe D_ee^-1 b_e,   x_e = D_ee^-1 (b_e - D_eo x_o).
  With x_e so reconstructed the full residual is (0 on even sites, b^ - D^ x_o
  on odd sites), so the solve stops once |b^ - D^ x_o| <= tol |b| -- the same
  criterion as the DD-alphaAMG solves of the full operator.

Pins (tests/test_oracle_oecg.py): CGLS on small dense systems equals
``numpy.linalg.solve``; its k-th iterate is the least-squares solution over
the Krylov space K_k(A^H A, A^H b) (brute force); the reduced right-hand
side, the reconstruction and D^dagger against the dense Schur complement at
4^4; the full solution against a dense LU solve of D.
"""
from __future__ import annotations

import numpy as np

from .dirac import Operator
from . import evenodd


class CGResult:
    def __init__(self, x, iters, relres, history, converged):
        self.x, self.iters, self.relres = x, iters, relres
        self.history, self.converged = history, converged


def cgls(A, A_dag, b: np.ndarray, tol: float, maxit: int, bnorm: float | None = None) -> CGResult:
    """CG on A^H A x = A^H b in the CGLS form; stops when |b - A x| <= tol * bnorm
    (the recurrence residual), bnorm = |b| unless given."""
    bnorm = float(np.linalg.norm(b)) if bnorm is None else bnorm
    x = np.zeros_like(b)
    r = b.copy()
    s = A_dag(r)
    p = s.copy()
    gamma = float(np.vdot(s, s).real)
    hist = [float(np.linalg.norm(r))]
    it = 0
    while hist[-1] > tol * bnorm and it < maxit and gamma > 0:
        q = A(p)
        alpha = gamma / float(np.vdot(q, q).real)
        x = x + alpha * p
        r = r - alpha * q
        s = A_dag(r)
        gamma_new = float(np.vdot(s, s).real)
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        it += 1
        hist.append(float(np.linalg.norm(r)))
    return CGResult(x, it, hist[-1] / bnorm if bnorm > 0 else 0.0, hist, hist[-1] <= tol * bnorm)


def reduced_adjoint(op: Operator, v: np.ndarray) -> np.ndarray:
    """D^(mu)^dagger v = G^5 D^(-mu) G^5 v on the odd sites (mu and the odd
    shift rho both change sign)."""
    op_m = op.with_mu_eo(-op.mu, -op.mu - op.rho)
    return evenodd.gamma5(evenodd.reduced_apply(op_m, evenodd.gamma5(v)))


def reduced_rhs(op: Operator, b: np.ndarray) -> np.ndarray:
    """b^ = b_o - D_oe D_ee^-1 b_e (zero on the even sites)."""
    od = evenodd.odd_mask(op)
    t = evenodd.diag_solve(op, b * ~od) * ~od  # D_ee^-1 b_e
    return (b - op.apply(t)) * od


def reconstruct(op: Operator, b: np.ndarray, xo: np.ndarray) -> np.ndarray:
    """x = (D_ee^-1 (b_e - D_eo x_o) on even, x_o on odd sites)."""
    od = evenodd.odd_mask(op)
    xo = xo * od
    xe = evenodd.diag_solve(op, (b - op.apply(xo)) * ~od) * ~od
    return xe + xo


def solve(op: Operator, b: np.ndarray, tol: float = 1e-10, maxit: int = 100000) -> tuple[np.ndarray, CGResult]:
    """Full-system solution of D x = b by oeCG; returns (x, CGLS result)."""
    bh = reduced_rhs(op, b)
    res = cgls(lambda v: evenodd.reduced_apply(op, v), lambda v: reduced_adjoint(op, v), bh, tol, maxit,
               bnorm=float(np.linalg.norm(b)))
    return reconstruct(op, b, res.x), res
