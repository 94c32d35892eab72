"""Restarted (flexible) GMRES with CGS2 Arnoldi and Givens rotations (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed
-----------------------
* Sec. 1: DD-alphaAMG preconditions a flexible Krylov solver at every
  iteration by the multigrid error propagation of eq. (1); Fig. 3 names it
  FGMRES.  Flexible GMRES keeps the preconditioned vectors z_k because the
  preconditioner changes from step to step.
* Sec. 3: the coarsest level is solved with odd-even preconditioning (here:
  GMRES on the Schur complement, :mod:`oracle.coarse`).

Readings (choices where the paper is silent)
------------------------------
* Right preconditioning, x = x0 + Z y.  Arnoldi by classical Gram-Schmidt
  applied twice (CGS2).  The least-squares problem is reduced by complex
  Givens rotations G = [[c, s], [-conj(s), c]] with real c.
* A restart cycle ends when the estimated residual |g_{k+1}| <= tol*||b||,
  when the cycle has ``restart`` steps or when ``maxit`` steps were done in
  total; the true residual b - A x is then recomputed, and the solve stops
  once it is <= tol*||b|| or maxit is reached.

Pins (tests/test_oracle_krylov.py): GMRES on small dense systems equals
``numpy.linalg.solve``; the Arnoldi relation A V_k = V_{k+1} H holds; with
an exact preconditioner FGMRES converges in one step; the residual estimate
equals the true residual in exact arithmetic.
"""
from __future__ import annotations

import numpy as np


def _dot(a, b):
    return complex(np.vdot(a.ravel(), b.ravel()))


def _norm(a):
    return float(np.linalg.norm(a.ravel()))


def givens(a: complex, b: float):
    """(c, s, rho) with [[c, s], [-conj(s), c]] [a, b]^T = [rho, 0]^T, c real."""
    if b == 0:
        return 1.0, 0.0 + 0.0j, a
    if a == 0:
        return 0.0, 1.0 + 0.0j, complex(b)
    nu = np.hypot(abs(a), abs(b))
    c = abs(a) / nu
    ph = a / abs(a)
    s = ph * np.conj(b) / nu
    return c, s, ph * nu


class GMRESResult:
    def __init__(self, x, iters, relres, history, converged):
        self.x, self.iters, self.relres = x, iters, relres
        self.history, self.converged = history, converged


def gmres(A, b: np.ndarray, x0: np.ndarray | None = None, tol: float = 1e-10,
          restart: int = 25, maxit: int = 1000, M=None) -> GMRESResult:
    """Solve A x = b.  With ``M`` it is flexible GMRES (z_k = M(v_k) kept)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = _norm(b)
    if bnorm == 0:
        return GMRESResult(np.zeros_like(b), 0, 0.0, [], True)
    r = b - A(x)
    beta = _norm(r)
    iters = 0
    history = [beta / bnorm]
    while beta > tol * bnorm and iters < maxit:
        m = restart
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        while k < m:
            z = M(V[k]) if M is not None else V[k]
            w = A(z)
            h = np.array([_dot(v, w) for v in V])
            for hi, v in zip(h, V):
                w = w - hi * v
            h2 = np.array([_dot(v, w) for v in V])
            for hi, v in zip(h2, V):
                w = w - hi * v
            h = h + h2
            hn = _norm(w)
            col = np.zeros(m + 1, dtype=np.complex128)
            col[: k + 1] = h
            col[k + 1] = hn
            for j in range(k):
                t = cs[j] * col[j] + sn[j] * col[j + 1]
                col[j + 1] = -np.conj(sn[j]) * col[j] + cs[j] * col[j + 1]
                col[j] = t
            c, s, rho = givens(col[k], hn)
            cs[k], sn[k] = c, s
            col[k], col[k + 1] = rho, 0.0
            H[:, k] = col
            g[k + 1] = -np.conj(s) * g[k]
            g[k] = c * g[k]
            if M is not None:
                Z.append(z)
            iters += 1
            k += 1
            history.append(abs(g[k]) / bnorm)
            if hn == 0 or abs(g[k]) <= tol * bnorm or iters >= maxit:
                break
            V.append(w / hn)
        # back substitution R y = g
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        basis = Z if M is not None else V
        for i in range(k):
            x = x + y[i] * basis[i]
        r = b - A(x)
        beta = _norm(r)
        history.append(beta / bnorm)
    return GMRESResult(x, iters, beta / bnorm, history, beta <= tol * bnorm)
