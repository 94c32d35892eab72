"""Pins of the oracle's three-level pieces (CPU only).

Coarse SAP on the 9-point stencil: one block is global MR; exact block
solves give dense block Gauss-Seidel.  Level-1 aggregation P2: orthonormal,
Gamma5_c-compatible, equal to modified Gram-Schmidt.  D_c2 equals the dense
P2^dagger D_c1 P2, and the twisted mass stays diagonal.  The level-1 K-cycle
with exact solves is eq. (1) assembled from dense matrices.  The three-level
FGMRES solve reaches 1e-10 and matches a dense LU solve.
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator, dense_matrix
from oracle.coarse import Interpolation, CoarseOperator
from oracle.multilevel import (CoarseSAP, CoarseInterpolation, ThreeLevel, ThreeLevelParams,
                               galerkin_coarse, to_cagg, from_cagg)

L = (8, 4, 4, 4)
AGG1, NV1 = (2, 2, 2, 2), 6
AGG2, NV2 = (2, 1, 1, 1), 4


def _level1(mu=0.05, seed=7):
    U = inputs.gauge_field(L, 0.5, seed)
    op = Operator(U, -0.3, 1.4, mu)
    P1 = Interpolation(inputs.random_test_vectors(L, NV1, seed + 1), AGG1)
    Dc1 = CoarseOperator.build(op, P1, mu)
    return op, P1, Dc1


def _coarse_random(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _dense_c(apply, Lc, n):
    N = int(np.prod(Lc)) * n
    E = np.eye(N, dtype=complex).reshape((N,) + tuple(Lc) + (n,))
    return apply(E).reshape(N, N).T


def test_cagg_roundtrip():
    v = _coarse_random((3, 4, 2, 2, 2, 2 * NV1), 1)
    assert np.array_equal(from_cagg(to_cagg(v, AGG2, NV1), AGG2, NV1), v)


def test_coarse_sap_single_block_is_global_mr():
    op, P1, Dc1 = _level1()
    sap = CoarseSAP(Dc1, Dc1.Lc, n_mr=5)
    D = _dense_c(Dc1.apply, Dc1.Lc, 2 * NV1)
    b = _coarse_random(Dc1.Lc + (2 * NV1,), 2)
    x0 = 0.1 * _coarse_random(Dc1.Lc + (2 * NV1,), 3)
    xv, r = x0.ravel().copy(), b.ravel() - D @ x0.ravel()
    e = np.zeros_like(r)
    for _ in range(5):
        q = D @ r
        a = np.vdot(q, r) / np.vdot(q, q)
        e += a * r
        r -= a * q
    assert np.allclose(sap.sweep(b, x0).ravel(), xv + e, atol=1e-12)


def test_coarse_sap_exact_block_solves_are_block_gauss_seidel():
    op, P1, Dc1 = _level1()
    blk = (2, 1, 1, 1)
    sap = CoarseSAP(Dc1, blk, n_mr=1)
    n = 2 * NV1
    D = _dense_c(Dc1.apply, Dc1.Lc, n)
    c = np.meshgrid(*[np.arange(k) for k in Dc1.Lc], indexing="ij")
    nb = [Dc1.Lc[d] // blk[d] for d in range(4)]
    bid = ((c[0] // blk[0] * nb[1] + c[1] // blk[1]) * nb[2] + c[2] // blk[2]) * nb[3] + c[3] // blk[3]
    bid = np.repeat(bid.ravel(), n)
    colour = np.repeat(sap.colour.ravel(), n)

    def exact(r, mask):
        out = np.zeros(r.size, dtype=complex)
        m = np.repeat(mask.ravel(), n)
        for k in np.unique(bid[m]):
            s = bid == k
            out[s] = np.linalg.solve(D[np.ix_(s, s)], r.ravel()[s])
        return out.reshape(r.shape)

    b = _coarse_random(Dc1.Lc + (n,), 4)
    x0 = _coarse_random(Dc1.Lc + (n,), 5)
    got = sap.sweep(b, x0, block_solve=exact)
    R, B = colour == 0, colour == 1
    x = x0.ravel().copy()
    bv = b.ravel()
    x[R] = np.linalg.solve(D[np.ix_(R, R)], bv[R] - D[np.ix_(R, B)] @ x[B])
    x[B] = np.linalg.solve(D[np.ix_(B, B)], bv[B] - D[np.ix_(B, R)] @ x[R])
    assert np.allclose(got.ravel(), x, atol=1e-11)


def _level2(mu=0.05, mu2=0.0):
    op, P1, Dc1 = _level1(mu)
    w = _coarse_random((NV2,) + Dc1.Lc + (2 * NV1,), 9)
    P2 = CoarseInterpolation(w, AGG2, NV1)
    return op, P1, Dc1, w, P2, galerkin_coarse(Dc1, P2, mu2)


def test_level1_interpolation_orthonormal_gamma5_and_mgs():
    op, P1, Dc1, w, P2, Dc2 = _level2()
    cols = P2.columns().reshape(2 * NV2, -1)
    N = int(np.prod(P2.Lc)) * 2 * NV2
    E = np.eye(N, dtype=complex).reshape((N,) + P2.Lc + (2 * NV2,))
    Pd = P2.prolong(E).reshape(N, -1).T
    assert np.allclose(Pd.conj().T @ Pd, np.eye(N), atol=1e-13)
    g1 = np.tile(Dc1.g5c, int(np.prod(Dc1.Lc)))
    g2 = np.tile(np.concatenate([-np.ones(NV2), np.ones(NV2)]), int(np.prod(P2.Lc)))
    assert np.allclose(g1[:, None] * Pd, Pd * g2[None, :], atol=1e-14)
    W = np.moveaxis(to_cagg(w, AGG2, NV1), 0, -1).reshape(-1, int(np.prod(AGG2)) * NV1, NV2)
    for wk, qk in zip(W, P2.Q.reshape(W.shape)):
        Q = np.zeros_like(wk)
        for j in range(NV2):
            v = wk[:, j].copy()
            for i in range(j):
                v -= np.vdot(Q[:, i], v) * Q[:, i]
            Q[:, j] = v / np.linalg.norm(v)
        assert np.allclose(Q, qk, atol=1e-12)
    assert cols.shape[0] == 2 * NV2


def test_level2_galerkin_equals_dense():
    op, P1, Dc1, w, P2, Dc2 = _level2(mu=0.05, mu2=0.0)
    n1, n2 = 2 * NV1, 2 * NV2
    D1 = _dense_c(Dc1.with_mu(0.0).apply, Dc1.Lc, n1)
    N = int(np.prod(P2.Lc)) * n2
    E = np.eye(N, dtype=complex).reshape((N,) + P2.Lc + (n2,))
    Pd = P2.prolong(E).reshape(N, -1).T
    assert np.allclose(_dense_c(Dc2.apply, P2.Lc, n2), Pd.conj().T @ D1 @ Pd, atol=1e-12)
    # the twisted mass stays diagonal: P2^dagger D_c1(mu) P2 = D_c2 + i mu Gamma5_c2
    D1mu = _dense_c(Dc1.apply, Dc1.Lc, n1)
    assert np.allclose(_dense_c(Dc2.with_mu(0.05).apply, P2.Lc, n2), Pd.conj().T @ D1mu @ Pd, atol=1e-12)


def test_level1_kcycle_is_eq1_with_exact_solves():
    prm = ThreeLevelParams(m0=-0.3, c_sw=1.4, mu=0.05, delta=3.0, nv=NV1, agg=AGG1, sap_block=(2, 2, 2, 2),
                           nv2=NV2, agg2=AGG2, sap_block1=(2, 1, 1, 1), pre_smooth1=1, post_smooth1=2)
    tl = ThreeLevel(inputs.gauge_field(L, 0.5, 7), prm)
    tl.build_level1(inputs.random_test_vectors(L, NV1, 8))
    tl.build_level2(_coarse_random((NV2,) + tl.Dc1.Lc + (2 * NV1,), 9))
    n1, n2 = 2 * NV1, 2 * NV2
    D1 = _dense_c(tl.Dc1.apply, tl.Dc1.Lc, n1)
    D2 = _dense_c(tl.Dc2.apply, tl.P2.Lc, n2)
    tl.coarsest_solve = lambda r2, *a: np.linalg.solve(D2, r2.ravel()).reshape(r2.shape)
    blk = tl.csap.block
    c = np.meshgrid(*[np.arange(k) for k in tl.Dc1.Lc], indexing="ij")
    nbk = [tl.Dc1.Lc[d] // blk[d] for d in range(4)]
    bid = ((c[0] // blk[0] * nbk[1] + c[1] // blk[1]) * nbk[2] + c[2] // blk[2]) * nbk[3] + c[3] // blk[3]
    bid = np.repeat(bid.ravel(), n1)
    colour = np.repeat(tl.csap.colour.ravel(), n1)

    def exact(r, mask):
        out = np.zeros(r.size, dtype=complex)
        m = np.repeat(mask.ravel(), n1)
        for k in np.unique(bid[m]):
            s = bid == k
            out[s] = np.linalg.solve(D1[np.ix_(s, s)], r.ravel()[s])
        return out.reshape(r.shape)

    csap = tl.csap
    tl.csap = type("S", (), {})()
    tl.csap.smooth = lambda b, x, k: _smooth(csap, exact, b, x, k)
    I = np.eye(D1.shape[0])

    def prop(col):
        s = colour == col
        M = np.zeros_like(D1)
        for k in np.unique(bid[s]):
            t = bid == k
            M[np.ix_(t, t)] = np.linalg.inv(D1[np.ix_(t, t)])
        return I - M @ D1
    Es = prop(1) @ prop(0)
    N = int(np.prod(tl.P2.Lc)) * n2
    E = np.eye(N, dtype=complex).reshape((N,) + tl.P2.Lc + (n2,))
    Pd = tl.P2.prolong(E).reshape(N, -1).T
    Ecgc = I - Pd @ np.linalg.inv(D2) @ Pd.conj().T @ D1
    Eeq1 = np.linalg.matrix_power(Es, 2) @ Ecgc @ Es
    eps = _coarse_random(tl.Dc1.Lc + (n1,), 11)
    got = eps - tl.kcycle1(tl.Dc1.apply(eps))
    assert np.allclose(got.ravel(), Eeq1 @ eps.ravel(), atol=1e-10)


def _smooth(sap, exact, b, x, k):
    for _ in range(k):
        x = sap.sweep(b, x, block_solve=exact)
    return x


def test_three_level_solve_matches_dense_lu():
    prm = ThreeLevelParams(m0=-0.3, c_sw=1.4, mu=0.02, delta=3.0, nv=NV1, agg=AGG1, sap_block=(2, 2, 2, 2),
                           nv2=NV2, agg2=AGG2, sap_block1=(2, 1, 1, 1), setup_iters=1, coarse_setup_iters=1)
    U = inputs.gauge_field(L, 0.5, 7)
    tl = ThreeLevel(U, prm)
    w0 = _coarse_random((NV2,) + tuple(L[d] // AGG1[d] for d in range(4)) + (2 * NV1,), 12)
    tl.setup(inputs.random_test_vectors(L, NV1, 2007), w0)
    b = inputs.gaussian_spinor(L, 1007)
    res = tl.solve(b, tol=1e-10)
    assert res.converged and res.relres <= 1e-10
    D = dense_matrix(tl.op.apply, L)
    x_ref = np.linalg.solve(D, b.ravel())
    assert np.linalg.norm(res.x.ravel() - x_ref) / np.linalg.norm(x_ref) < 1e-8
    assert tl.coarse_iters and tl.coarsest_iters
