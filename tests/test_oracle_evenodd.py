"""Pins of the even/odd twisted mass and the Hasenbusch sequence (oracle.evenodd,
the odd shift rho of oracle.dirac.Operator; Sec. 2 and Sec. 3), CPU only.

Against dense linear algebra on small lattices: D(mu, mu + rho) is D_W plus
the site-diagonal i mu(x) Gamma5; its odd Schur complement is the dense
D_oo - D_oe D_ee^-1 D_eo and equals D^(mu) + i rho G^5; D^ is
Gamma5-hermitian; the full-operator route (b = (0, b_o)) solves the reduced
system; the two-solve sequence gives x with A A^dagger x = b; the coarse
operator with the shift is the dense Galerkin projection; the two-level solve
with the shift matches a dense solve.  A planted mistake (the shift on even
sites) fails.
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import Operator, dense_matrix, site_parity, GAMMA5
from oracle.coarse import Interpolation, CoarseOperator
from oracle.amg import TwoLevel, AMGParams
from oracle import evenodd

L = (4, 4, 2, 2)
MU, RHO = 0.07, 0.31


def _op(mu=MU, rho=0.0, Lat=L, seed=3):
    return Operator(inputs.gauge_field(Lat, 0.6, seed), -0.35, 1.4, mu, rho=rho)


def _idx(Lat):
    par = np.repeat(site_parity(Lat).ravel(), 12)
    return np.flatnonzero(par == 0), np.flatnonzero(par == 1)


def _schur(D, Lat):
    e, o = _idx(Lat)
    return D[np.ix_(o, o)] - D[np.ix_(o, e)] @ np.linalg.solve(D[np.ix_(e, e)], D[np.ix_(e, o)])


def _g5(Lat):
    return np.kron(np.ones(int(np.prod(Lat))), np.repeat(np.diag(GAMMA5).real, 3))


def test_operator_is_dw_plus_sitewise_twisted_mass():
    op = _op(rho=RHO)
    D = dense_matrix(op.apply, L)
    DW = dense_matrix(op.with_mu_eo(0.0, 0.0).apply, L)
    mu_x = np.repeat(MU + RHO * site_parity(L).ravel(), 12)
    assert np.allclose(D, DW + 1j * np.diag(mu_x * _g5(L)), atol=1e-13)
    # the per-site evaluation agrees
    psi = inputs.gaussian_spinor(L, 4)
    sites = [(0, 0, 0, 0), (1, 0, 0, 0), (3, 2, 1, 1)]
    y = op.apply(psi)
    assert np.allclose(op.apply_at_sites(psi, sites), np.array([y[s] for s in sites]), atol=1e-13)


def test_reduced_operator_is_the_dense_schur_complement_and_the_hasenbusch_shift():
    op = _op(rho=RHO)
    D = dense_matrix(op.apply, L)
    S = _schur(D, L)
    e, o = _idx(L)
    x = inputs.gaussian_spinor(L, 5)
    got = evenodd.reduced_apply(op, x).ravel()
    assert np.allclose(got[o], S @ x.ravel()[o], atol=1e-12)
    assert np.allclose(got[e], 0)
    # odd shift rho = the shift i rho G5 of the reduced operator
    S0 = _schur(dense_matrix(_op().apply, L), L)
    assert np.allclose(S, S0 + 1j * RHO * np.diag(_g5(L)[o]), atol=1e-12)


def test_reduced_operator_gamma5_hermiticity():
    e, o = _idx(L)
    g5o = np.diag(_g5(L)[o])
    Sp = _schur(dense_matrix(_op(MU, 0.0).apply, L), L)
    Sm = _schur(dense_matrix(_op(-MU, 0.0).apply, L), L)
    assert np.allclose(Sp.conj().T, g5o @ Sm @ g5o, atol=1e-12)
    A = Sp + 1j * RHO * g5o
    assert np.allclose(A.conj().T, g5o @ Sm @ g5o - 1j * RHO * g5o, atol=1e-12)


def test_full_operator_route_solves_the_reduced_system():
    op = _op(rho=RHO)
    D = dense_matrix(op.apply, L)
    S = _schur(D, L)
    e, o = _idx(L)
    b = inputs.gaussian_spinor(L, 6)
    x = evenodd.reduced_solve_by_full(lambda r: np.linalg.solve(D, r.ravel()).reshape(r.shape), op, b)
    assert np.allclose(x.ravel()[e], 0)
    assert np.allclose(S @ x.ravel()[o], b.ravel()[o], atol=1e-11)


def test_hasenbusch_sequence_inverts_A_A_dagger():
    op = _op()
    e, o = _idx(L)
    g5o = np.diag(_g5(L)[o])

    def solve_eo(mu_e, mu_o, r):
        D = dense_matrix(op.with_mu_eo(mu_e, mu_o).apply, L)
        return np.linalg.solve(D, r.ravel()).reshape(r.shape)

    b = inputs.gaussian_spinor(L, 7)
    x = evenodd.hasenbusch(solve_eo, MU, RHO, b, op).ravel()
    A = _schur(dense_matrix(op.apply, L), L) + 1j * RHO * g5o
    bo = b.ravel()[o]
    assert np.allclose(x[e], 0)
    assert np.linalg.norm(A @ (A.conj().T @ x[o]) - bo) <= 1e-11 * np.linalg.norm(bo)
    # the order matters: this is not (A^dagger A)^-1 b
    assert np.linalg.norm(A.conj().T @ (A @ x[o]) - bo) > 1e-6 * np.linalg.norm(bo)


def test_coarse_operator_with_the_shift_is_the_dense_galerkin_projection():
    Lat, agg, nv = (4, 4, 4, 4), (2, 2, 2, 2), 3
    op = _op(rho=RHO, Lat=Lat)
    P = Interpolation(inputs.random_test_vectors(Lat, nv, 8), agg)
    delta = 3.0
    Dc = CoarseOperator.build(op, P, mu_c=delta * MU)
    n = 2 * nv
    N = int(np.prod(P.Lc)) * n
    E = np.eye(N, dtype=complex).reshape((N,) + P.Lc + (n,))
    Pd = np.stack([P.prolong(v).ravel() for v in E]).T
    Dc_dense = Dc.apply(E).reshape(N, N).T
    DW_rho = dense_matrix(op.with_mu(0.0).apply, Lat)   # D_W + i rho Pi_odd Gamma5
    g5c = np.tile(np.concatenate([-np.ones(nv), np.ones(nv)]), N // n)
    assert np.allclose(Dc_dense, Pd.conj().T @ DW_rho @ Pd + 1j * delta * MU * np.diag(g5c), atol=1e-12)


def test_two_level_solve_with_the_shift_matches_dense():
    Lat = (4, 4, 4, 4)
    prm = AMGParams(m0=-0.3, c_sw=1.2, mu=0.02, delta=2.0, nv=6, agg=(2, 2, 2, 2), sap_block=(2, 2, 2, 2),
                    setup_iters=1, rho=0.05, block_oe=True)
    tl = TwoLevel(inputs.gauge_field(Lat, 0.4, 9), prm)
    tl.setup(inputs.random_test_vectors(Lat, 6, 10))
    b = inputs.gaussian_spinor(Lat, 11)
    res = tl.solve(b, tol=1e-10)
    assert res.converged
    D = dense_matrix(tl.op.apply, Lat)
    assert np.linalg.norm(D @ res.x.ravel() - b.ravel()) <= 1e-10 * np.linalg.norm(b)
    # switching the shift sign with the same P still solves
    tl.set_mu_eo(-0.02, -0.07)
    res2 = tl.solve(b, tol=1e-10)
    D2 = dense_matrix(tl.op.apply, Lat)
    assert res2.converged and np.linalg.norm(D2 @ res2.x.ravel() - b.ravel()) <= 1e-10 * np.linalg.norm(b)


def test_shift_on_even_sites_is_caught(monkeypatch):
    op = _op(rho=RHO)
    S = _schur(dense_matrix(op.apply, L), L)
    wrong = op.with_mu(MU)
    wrong.odd = ~wrong.odd  # planted: the shift lands on the even sites
    S_wrong = _schur(dense_matrix(wrong.apply, L), L)
    S0 = _schur(dense_matrix(_op().apply, L), L)
    e, o = _idx(L)
    assert not np.allclose(S_wrong, S0 + 1j * RHO * np.diag(_g5(L)[o]), atol=1e-6)
    assert np.allclose(S, S0 + 1j * RHO * np.diag(_g5(L)[o]), atol=1e-12)
