"""True residual ||b - D(mu) x|| of a large lattice, T-slab by T-slab (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The oracle's ``Operator`` holds the clover term of every site as a 12x12
complex matrix (2.3 KB per site, 24 GB at 48^3 x 96), so the residual of a
solution at that size is taken slab by slab: rows t0..t1-1 of D(mu) x need
x, the links and the clover term of those rows only, and the clover term of a
row only needs links within one row of it (the plaquette leaves of Sec. 2's
clover term reach one site in each direction).  So each slab is evaluated
with the unchanged ``Operator`` on a sub-lattice of rows t0-1 .. t1 (one halo
row each side), periodic in T, and only its interior rows are kept.  The
fermion boundary factor bc_t of the hops across the T boundary is carried by
the links U_T of row T-1 instead (multiplied by bc_t), which changes no
plaquette (each one holding U_T(row T-1) also holds its adjoint).

Pins (tests/test_oracle_slabs.py): on small lattices the slab-wise residual
equals the full-lattice ``Operator`` residual for both boundary conditions,
for slabs that contain the T boundary and for one-row slabs.
"""
from __future__ import annotations

import numpy as np

from .dirac import Operator


def _sub_lattice(U: np.ndarray, rows: np.ndarray, bc_t: float) -> np.ndarray:
    """Links of the given full-lattice rows, U_T of row T-1 times bc_t."""
    T = U.shape[0]
    Us = U[rows].copy()
    last = np.flatnonzero(rows == T - 1)
    if last.size and bc_t != 1.0:
        Us[last, ..., 0, :, :] *= bc_t
    return Us


def slab_residual_norms(U, x, b, m0, c_sw, mu, bc_t, t0, t1):
    """(||b - D x||^2, ||b||^2) summed over rows t0 <= t < t1 (t1 - t0 >= 1,
    T >= t1 - t0 + 2).  x and b may carry leading right-hand-side axes."""
    T = U.shape[0]
    rows = np.arange(t0 - 1, t1 + 1) % T
    op = Operator(_sub_lattice(U, rows, bc_t), m0, c_sw, mu, bc_t=1.0)
    lead = x.ndim - 6
    xs = np.take(x, rows, axis=lead)
    y = op.apply(xs)
    inner = slice(1, 1 + (t1 - t0))
    idx = (slice(None),) * lead + (inner,)
    r = np.take(b, np.arange(t0, t1), axis=lead) - y[idx]
    bb = np.take(b, np.arange(t0, t1), axis=lead)
    return float(np.vdot(r, r).real), float(np.vdot(bb, bb).real)


def residual_by_slabs(U, x, b, m0, c_sw, mu, bc_t=-1.0, slab=4):
    """||b - D(mu) x|| / ||b|| over the whole lattice, one slab at a time."""
    T = U.shape[0]
    rr = bb = 0.0
    for t0 in range(0, T, slab):
        r2, b2 = slab_residual_norms(U, x, b, m0, c_sw, mu, bc_t, t0, min(T, t0 + slab))
        rr += r2
        bb += b2
    return float(np.sqrt(rr / bb))
