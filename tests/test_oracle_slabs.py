"""Pins of the slab-wise true residual (oracle/slabs.py) against the full-lattice
oracle operator (CPU only): equal residual norms for antiperiodic and periodic
T, for slabs that contain the T boundary, one-row slabs and several
right-hand sides; a planted mistake (the boundary factor left off) fails."""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator
from oracle import slabs


def _system(L, bc_t, seed=3, nrhs=None):
    U = inputs.gauge_field(L, 0.6, seed)
    op = Operator(U, -0.4, 1.3, 0.02, bc_t=bc_t)
    x = inputs.gaussian_spinor(L, seed + 1, nrhs=nrhs)
    b = inputs.gaussian_spinor(L, seed + 2, nrhs=nrhs)
    # a near-solution, so that the residual is small and cancellation matters
    b = op.apply(x) + 1e-6 * b
    return U, op, x, b


@pytest.mark.parametrize("bc_t", [-1.0, 1.0])
@pytest.mark.parametrize("slab", [1, 2, 3, 6])
def test_slab_residual_equals_full(bc_t, slab):
    L = (8, 4, 4, 6)
    U, op, x, b = _system(L, bc_t)
    full = np.linalg.norm(b - op.apply(x)) / np.linalg.norm(b)
    got = slabs.residual_by_slabs(U, x, b, op.m0, op.c_sw, op.mu, bc_t, slab=slab)
    assert abs(got - full) <= 1e-9 * full


def test_slab_rows_equal_full_rows_with_rhs_axis():
    L = (6, 4, 4, 4)
    U, op, x, b = _system(L, -1.0, nrhs=2)
    r = b - op.apply(x)
    for t0, t1 in [(0, 1), (5, 6), (2, 5)]:
        r2, b2 = slabs.slab_residual_norms(U, x, b, op.m0, op.c_sw, op.mu, -1.0, t0, t1)
        assert abs(r2 - np.vdot(r[:, t0:t1], r[:, t0:t1]).real) <= 1e-10 * r2
        assert abs(b2 - np.vdot(b[:, t0:t1], b[:, t0:t1]).real) <= 1e-12 * b2


def test_boundary_factor_left_off_is_caught():
    L = (6, 4, 4, 4)
    U, op, x, b = _system(L, -1.0)
    r = b - op.apply(x)
    want = np.vdot(r[5:6], r[5:6]).real
    orig = slabs._sub_lattice
    try:
        slabs._sub_lattice = lambda U_, rows, bc: U_[rows].copy()
        r2, _ = slabs.slab_residual_norms(U, x, b, op.m0, op.c_sw, op.mu, -1.0, 5, 6)
    finally:
        slabs._sub_lattice = orig
    assert abs(r2 - want) > 1e-3 * want
