"""Pins of the oracle's SAP smoother (CPU only).

Checks: one block covering the lattice is textbook global MR; the Dirichlet
block operator is the block-diagonal sub-matrix of the dense D; with exact
block solves a sweep equals dense block Gauss-Seidel written in splitting
form; MR never increases a block's residual; the odd-even block solve
converges to the exact block solve.
"""
import numpy as np

import inputs
from oracle.dirac import Operator, dense_matrix
from oracle.sap import SAP, block_ids


def _op(L, seed=21, mu=0.05):
    return Operator(inputs.gauge_field(L, 0.6, seed), -0.3, 1.4, mu)


def test_single_block_is_global_mr():
    L = (4, 2, 2, 2)
    op = _op(L)
    sap = SAP(op, L, n_mr=5)
    b = inputs.gaussian_spinor(L, 1)
    x0 = inputs.gaussian_spinor(L, 2) * 0.1
    D = dense_matrix(op.apply, L)
    xv, bv = x0.ravel().copy(), b.ravel()
    r = bv - D @ xv
    e = np.zeros_like(r)
    for _ in range(5):
        q = D @ r
        a = np.vdot(q, r) / np.vdot(q, q)
        e += a * r
        r -= a * q
    expect = xv + e
    got = sap.sweep(b, x0)
    assert np.allclose(got.ravel(), expect, atol=1e-12)


def _block_index(L, block):
    ids = block_ids(L, block)
    nb = [L[d] // block[d] for d in range(4)]
    flat = ((ids[0] * nb[1] + ids[1]) * nb[2] + ids[2]) * nb[3] + ids[3]
    return np.repeat(flat.ravel(), 12)


def test_block_operator_is_dense_submatrix():
    L, block = (4, 4, 2, 2), (2, 2, 1, 1)
    op = _op(L)
    sap = SAP(op, block)
    D = dense_matrix(op.apply, L)
    DB = dense_matrix(sap.apply_block, L)
    bid = _block_index(L, block)
    same = bid[:, None] == bid[None, :]
    assert np.allclose(DB[same], D[same], atol=1e-14)
    assert np.allclose(DB[~same], 0, atol=1e-14)


def test_exact_block_solves_equal_block_gauss_seidel():
    L, block = (4, 4, 2, 2), (2, 2, 1, 1)
    op = _op(L)
    sap = SAP(op, block)
    D = dense_matrix(op.apply, L)
    bid = _block_index(L, block)
    colour = np.repeat(sap.colour.ravel(), 12)

    def exact(r, mask):
        out = np.zeros(r.size, dtype=complex)
        rv = r.ravel()
        m = np.repeat(mask.ravel(), 12)
        for blk in np.unique(bid[m]):
            s = bid == blk
            out[s] = np.linalg.solve(D[np.ix_(s, s)], rv[s])
        return out.reshape(r.shape)

    b = inputs.gaussian_spinor(L, 3)
    x0 = inputs.gaussian_spinor(L, 4)
    got = sap.sweep(b, x0, block_solve=exact)
    # splitting form: x_R = D_RR^-1 (b_R - D_RB x_B); x_B = D_BB^-1 (b_B - D_BR x_R)
    R, B = colour == 0, colour == 1
    x = x0.ravel().copy()
    bv = b.ravel()
    x[R] = np.linalg.solve(D[np.ix_(R, R)], bv[R] - D[np.ix_(R, B)] @ x[B])
    x[B] = np.linalg.solve(D[np.ix_(B, B)], bv[B] - D[np.ix_(B, R)] @ x[R])
    assert np.allclose(got.ravel(), x, atol=1e-12)


def test_mr_residual_monotone():
    L, block = (4, 4, 4, 4), (2, 2, 2, 2)
    sap = SAP(_op(L, mu=0.01), block, n_mr=8)
    r = inputs.gaussian_spinor(L, 5)
    hist = sap.mr_history(r, sap.colour == 0)
    for a, b in zip(hist[:-1], hist[1:]):
        assert np.all(b <= a * (1 + 1e-14))
    assert np.all(hist[-1][hist[0] > 0] < hist[0][hist[0] > 0])


def test_odd_even_block_solve_converges_to_exact():
    L, block = (4, 4, 2, 2), (2, 2, 2, 2)
    op = _op(L, mu=0.2)
    D = dense_matrix(op.apply, L)
    sap = SAP(op, block, n_mr=150, block_oe=True)
    r = inputs.gaussian_spinor(L, 6)
    mask = sap.colour == 0
    got = sap.mr_oe(r, mask)
    bid = _block_index(L, block)
    m = np.repeat(mask.ravel(), 12)
    expect = np.zeros(r.size, dtype=complex)
    for blk in np.unique(bid[m]):
        s = bid == blk
        expect[s] = np.linalg.solve(D[np.ix_(s, s)], r.ravel()[s])
    assert np.linalg.norm(got.ravel() - expect) / np.linalg.norm(expect) < 1e-10
