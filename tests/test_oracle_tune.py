"""Pins of the oracle's m0 tuner (CPU only).

The sparse D_W equals the stencil operator on random fields (both boundary
conditions); the ARPACK leftmost eigenvalues agree with a dense eigenvalue
solve at 4^4; the tuned m0 puts the left edge of D_W(m0)'s spectrum at the
target, as the dense spectrum confirms.
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator, dense_matrix
from oracle.tune_m0 import sparse_dirac, leftmost_eigenvalues, tune_m0


@pytest.mark.parametrize("bc", [-1.0, 1.0])
def test_sparse_matrix_equals_stencil(bc):
    L = (4, 6, 2, 4)
    U = inputs.gauge_field(L, 0.7, 3)
    D = sparse_dirac(U, -0.2, 1.3, bc)
    op = Operator(U, -0.2, 1.3, 0.0, bc_t=bc)
    psi = inputs.gaussian_spinor(L, 4)
    assert np.allclose(D @ psi.ravel(), op.apply(psi).ravel(), atol=1e-13)


def test_leftmost_eigenvalues_and_tuned_edge():
    L = (4, 4, 4, 4)
    U = inputs.gauge_field(L, 0.5, 1)
    dense = dense_matrix(Operator(U, 0.0, 1.5, 0.0).apply, L)
    ev = np.linalg.eigvals(dense)
    ev = ev[np.argsort(ev.real)]
    got = leftmost_eigenvalues(sparse_dirac(U, 0.0, 1.5), k=6, ncv=60, tol=1e-10)
    assert abs(got[0].real - ev[0].real) < 1e-8
    res = tune_m0(U, 1.5, target=1e-3, k=6, ncv=60, tol=1e-10)
    shifted = np.linalg.eigvals(dense + res["m0"] * np.eye(len(dense)))
    assert abs(shifted.real.min() - 1e-3) < 1e-8
    assert res["sigma_min_bound"] >= np.linalg.svd(dense + res["m0"] * np.eye(len(dense)),
                                                   compute_uv=False).min() - 1e-9
