"""Odd-site reduced operator and the Hasenbusch two-solve sequence (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed
-----------------------
* Sec. 2: the library applies a different twisted mass on the even and the
  odd sites, as Hasenbusch mass preconditioning with odd-even preconditioning
  needs.
* Sec. 3: the HMC inverts D^(mu) + i rho G^5 and then G^5 D^(-mu) G^5 - i rho
  G^5, D^ the odd-even reduced operator on the odd sites and G^5 = Gamma5
  restricted to them; DD-alphaAMG inverts the full operator even when the
  reduced one is wanted.

Readings
--------
* Site parity (t + z + y + x) mod 2; the reduced operator lives on the odd
  sites: D^ = D_oo - D_oe D_ee^-1 D_eo, D_ee and D_oo the site-diagonal parts
  A(x) + i mu(x) gamma5.
* A twisted mass mu on the even and mu + rho on the odd sites changes D_oo
  only, so the odd Schur complement of D(mu, mu + rho) is exactly
  D^(mu) + i rho G^5: the reduced system D^ x_o = b_o is solved with the full
  operator on b = (0 on even, b_o on odd), x_o the odd part of the solution.
* The two solves are applied in the order Sec. 3 lists them: y = (D^(mu) +
  i rho G^5)^-1 b, then x = (G^5 D^(-mu) G^5 - i rho G^5)^-1 y; the second
  operator is the adjoint of the first (Gamma5-hermiticity of D^), so x =
  (A A^dagger)^-1 b with A = D^(mu) + i rho G^5.  Its inverse is
  G^5 (D^(-mu) - i rho G^5)^-1 G^5, the odd Schur complement of
  D(-mu, -mu - rho) between two G^5.

Pins (tests/test_oracle_evenodd.py): dense Schur complements at 4^4, the
shift identity, Gamma5-hermiticity of D^, the full-operator route to the
reduced solution, A A^dagger x = b for the sequence, and the Galerkin coarse
operator of D(mu, mu + rho) against dense projection.
"""
from __future__ import annotations

import numpy as np

from .dirac import Operator, GAMMA5, spin_mul


def odd_mask(op: Operator) -> np.ndarray:
    return op.odd[..., None, None]


def restrict_odd(op: Operator, psi: np.ndarray) -> np.ndarray:
    """psi on the odd sites, zero on the even ones."""
    return psi * odd_mask(op)


def diag_solve(op: Operator, psi: np.ndarray) -> np.ndarray:
    """(A(x) + i mu(x) gamma5)^-1 psi(x) at every site."""
    D = op.A + 1j * op.mu_field()[..., None, None] * np.kron(GAMMA5, np.eye(3))
    sh = psi.shape
    y = np.linalg.solve(D, psi.reshape(sh[:-2] + (12,))[..., None])[..., 0]
    return y.reshape(sh)


def reduced_apply(op: Operator, x: np.ndarray) -> np.ndarray:
    """D^ x_o = D_oo x_o - D_oe D_ee^-1 D_eo x_o on the odd sites (x's even
    sites are ignored; the result is zero on even sites)."""
    od = odd_mask(op)
    xo = x * od
    t = op.apply(xo)                      # odd part D_oo x_o, even part D_eo x_o
    u = diag_solve(op, t * ~od)           # D_ee^-1 D_eo x_o on even sites
    return (t - op.apply(u)) * od         # minus D_oe u on odd sites


def reduced_solve_by_full(solve, op: Operator, b: np.ndarray) -> np.ndarray:
    """x_o with D^ x_o = b_o from a solver of the full operator D (``solve``
    maps a right-hand side to the solution of D x = rhs)."""
    return restrict_odd(op, solve(restrict_odd(op, b)))


def gamma5(psi: np.ndarray) -> np.ndarray:
    return spin_mul(GAMMA5, psi)


def hasenbusch(solve_eo, mu: float, rho: float, b: np.ndarray, op: Operator) -> np.ndarray:
    """x = (G^5 D^(-mu) G^5 - i rho G^5)^-1 (D^(mu) + i rho G^5)^-1 b_o.

    ``solve_eo(mu_even, mu_odd, rhs)`` solves the full D(mu_even, mu_odd) x = rhs."""
    y = reduced_solve_by_full(lambda r: solve_eo(mu, mu + rho, r), op, b)
    z = reduced_solve_by_full(lambda r: solve_eo(-mu, -mu - rho, r), op, gamma5(y))
    return gamma5(z)
