"""Pins of the oracle's adaptive setup (Sec. 1; Sec. 3's MGSetupIter and
MGCoarseSetupIter) against dense linear algebra (CPU only).

With exact block solves in SAP and an exact coarse solve the smoother and the
K-cycle are linear maps, so every phase of the setup has a closed form that is
assembled here from dense matrices, independently of the oracle's sequencing:

* initial phase: v_i = normalise(E_sweep^s v0_i), E_sweep = (I - M_black D)
  (I - M_red D) the dense propagator of one red/black sweep on D v = 0;
* one setup pass: v_i <- normalise(B v_i) with B = (I - E_eq1) D^-1 built
  from the P of the previous pass (eq. (1) with exact solves), the same B for
  every i, and P, D_c rebuilt from the new vectors only after the pass;
* three levels: the fine pass with an exact level-1 solve (then D_c2 is the
  Galerkin product of the new D_c1 with the P2 of the unchanged w_j), and the
  level-1 pass w_j <- normalise(B1 w_j), B1 = (I - E1_eq1) D_c1^-1.

Three plausible sequencing mistakes are planted in copies of the oracle's
setup (on the CPU) and each must fail at least one of these pins: P rebuilt
after every vector instead of after the pass, the normalisation dropped, and
the initial sweeps run on D v = v instead of D v = 0.
"""
import numpy as np
import pytest

import inputs
from oracle.dirac import dense_matrix
from oracle.coarse import Interpolation
from oracle.amg import TwoLevel, AMGParams, normalise
from oracle.multilevel import (ThreeLevel, ThreeLevelParams, CoarseInterpolation, galerkin_coarse)

L = (4, 4, 2, 2)
NV = 3
AGG = (2, 2, 1, 1)
BLK = (2, 2, 1, 1)


# ----------------------------------------------------------------------------
# dense building blocks
# ----------------------------------------------------------------------------

def _block_ids(Ls, blk):
    c = np.meshgrid(*[np.arange(n) for n in Ls], indexing="ij")
    nb = [Ls[d] // blk[d] for d in range(4)]
    bid = ((c[0] // blk[0] * nb[1] + c[1] // blk[1]) * nb[2] + c[2] // blk[2]) * nb[3] + c[3] // blk[3]
    col = sum(c[d] // blk[d] for d in range(4)) % 2
    return bid.ravel(), col.ravel()


class ExactSmoother:
    """Red/black multiplicative Schwarz with exact block solves on a dense matrix;
    vectors of shape [..., *site_shape] with any leading stack dimensions."""

    def __init__(self, D, bid, col, site_shape):
        self.D = D
        self.shape = tuple(site_shape)
        self.sets = []
        for c in (0, 1):
            blocks = [np.flatnonzero(bid == k) for k in np.unique(bid[col == c])]
            self.sets.append([(s, np.linalg.inv(D[np.ix_(s, s)])) for s in blocks])

    def _sweep1(self, b, x):
        x = x.copy()
        for blocks in self.sets:
            r = b - self.D @ x
            for s, inv in blocks:
                x[s] += inv @ r[s]
        return x

    def sweep(self, b, x):
        lead = x.shape[:x.ndim - len(self.shape)]
        n = int(np.prod(self.shape))
        xs = x.reshape((-1, n))
        bs = np.broadcast_to(b, x.shape).reshape((-1, n))
        out = np.stack([self._sweep1(bs[i], xs[i]) for i in range(xs.shape[0])])
        return out.reshape(lead + self.shape)

    def smooth(self, b, x, k):
        for _ in range(k):
            x = self.sweep(b, x)
        return x

    def propagator(self):
        """E_sweep = (I - M_1 D)(I - M_0 D)."""
        n = self.D.shape[0]
        E = np.eye(n, dtype=complex)
        for blocks in self.sets:
            M = np.zeros((n, n), dtype=complex)
            for s, inv in blocks:
                M[np.ix_(s, s)] = inv
            E = (np.eye(n) - M @ self.D) @ E
        return E


def _dense_coarse(apply, Lc, n):
    N = int(np.prod(Lc)) * n
    E = np.eye(N, dtype=complex).reshape((N,) + tuple(Lc) + (n,))
    return apply(E).reshape(N, N).T


def _prolong_matrix(P, Lc, n):
    N = int(np.prod(Lc)) * n
    E = np.eye(N, dtype=complex).reshape((N,) + tuple(Lc) + (n,))
    return np.stack([P.prolong(e).ravel() for e in E]).T


def _B_dense(D, E_sweep, Pd, Dc, pre, post):
    """B = (I - E_eq1) D^-1 with E_eq1 = E^post (I - P Dc^-1 P^+ D) E^pre."""
    n = D.shape[0]
    E_cgc = np.eye(n) - Pd @ np.linalg.solve(Dc, Pd.conj().T @ D)
    E_eq1 = np.linalg.matrix_power(E_sweep, post) @ E_cgc @ np.linalg.matrix_power(E_sweep, pre)
    return (np.eye(n) - E_eq1) @ np.linalg.inv(D)


def _norm_rows(V):
    return V / np.linalg.norm(V, axis=1, keepdims=True)


# ----------------------------------------------------------------------------
# two levels
# ----------------------------------------------------------------------------

def _two_level(cls=TwoLevel, init_sweeps=2, setup_iters=1):
    prm = AMGParams(m0=-0.3, c_sw=1.3, mu=0.05, delta=2.0, nv=NV, agg=AGG, sap_block=BLK, mr_iters=2,
                    pre_smooth=1, post_smooth=2, init_sweeps=init_sweeps, setup_iters=setup_iters)
    tl = cls(inputs.gauge_field(L, 0.6, 41), prm)
    D = dense_matrix(tl.op.apply, L)
    bid, col = _block_ids(L, BLK)
    sm = ExactSmoother(D, np.repeat(bid, 12), np.repeat(col, 12), L + (4, 3))
    tl.sap = sm
    cache = {}

    def exact_coarse(rc, *a):
        key = id(tl.Dc)
        if key not in cache:
            cache.clear()
            cache[key] = _dense_coarse(tl.Dc.apply, tl.P.Lc, 2 * NV)
        return np.linalg.solve(cache[key], rc.ravel()).reshape(rc.shape)

    tl.coarse_solve = exact_coarse
    return tl, D, sm


def _pin_initial_phase(cls):
    tl, D, sm = _two_level(cls, init_sweeps=2, setup_iters=0)
    v0 = inputs.random_test_vectors(L, NV, 42)
    v = tl.setup(v0)
    Es = sm.propagator()
    want = _norm_rows((np.linalg.matrix_power(Es, 2) @ v0.reshape(NV, -1).T).T)
    return np.max(np.abs(v.reshape(NV, -1) - want))


def _pin_setup_pass(cls):
    tl, D, sm = _two_level(cls, init_sweeps=1, setup_iters=1)
    v0 = inputs.random_test_vectors(L, NV, 42)
    v = tl.setup(v0)
    Es = sm.propagator()
    v1 = _norm_rows((Es @ v0.reshape(NV, -1).T).T)
    P1 = Interpolation(v1.reshape(v0.shape), AGG)
    Pd = _prolong_matrix(P1, P1.Lc, 2 * NV)
    Dc = Pd.conj().T @ D @ Pd      # the Galerkin operator with the fine twisted mass ...
    n_c = Dc.shape[0]
    g5c = np.tile(np.concatenate([-np.ones(NV), np.ones(NV)]), n_c // (2 * NV))
    Dc = Dc + 1j * (tl.prm.delta - 1.0) * tl.prm.mu * np.diag(g5c)   # ... raised to delta mu
    B = _B_dense(D, Es, Pd, Dc, tl.prm.pre_smooth, tl.prm.post_smooth)
    v2 = _norm_rows((B @ v1.T).T)
    dev_v = np.max(np.abs(v.reshape(NV, -1) - v2))
    # P and D_c are rebuilt from the new vectors after the pass
    P2 = Interpolation(v2.reshape(v0.shape), AGG)
    dev_p = np.max(np.abs(tl.P.Q - P2.Q))
    return max(dev_v, dev_p)


def test_initial_phase_is_normalised_sweep_propagator():
    assert _pin_initial_phase(TwoLevel) < 1e-12


def test_setup_pass_is_dense_B_with_the_previous_P():
    assert _pin_setup_pass(TwoLevel) < 1e-10


# planted mistakes ------------------------------------------------------------------

class RebuildPerVector(TwoLevel):
    """Mistake: P and D_c rebuilt after every vector of a pass."""

    def setup(self, v0, setup_iters=None):
        prm = self.prm
        v = v0.copy()
        zero = np.zeros_like(v)
        for _ in range(prm.init_sweeps):
            v = self.sap.sweep(zero, v)
        v = normalise(v)
        self.build_coarse(v)
        for _ in range(prm.setup_iters if setup_iters is None else setup_iters):
            for i in range(v.shape[0]):
                v[i] = self.kcycle(v[i])
                v = normalise(v)
                self.build_coarse(v)
        self.test_vectors = v
        return v


class NoNormalisation(TwoLevel):
    """Mistake: the vectors are never normalised."""

    def setup(self, v0, setup_iters=None):
        prm = self.prm
        v = v0.copy()
        zero = np.zeros_like(v)
        for _ in range(prm.init_sweeps):
            v = self.sap.sweep(zero, v)
        self.build_coarse(v)
        for _ in range(prm.setup_iters if setup_iters is None else setup_iters):
            v = np.stack([self.kcycle(v[i]) for i in range(v.shape[0])])
            self.build_coarse(v)
        self.test_vectors = v
        return v


class SweepsOnDvEqualsV(TwoLevel):
    """Mistake: the initial sweeps smooth D v = v0 instead of D v = 0."""

    def setup(self, v0, setup_iters=None):
        prm = self.prm
        v = v0.copy()
        for _ in range(prm.init_sweeps):
            v = self.sap.sweep(v0, v)
        v = normalise(v)
        self.build_coarse(v)
        for _ in range(prm.setup_iters if setup_iters is None else setup_iters):
            v = normalise(np.stack([self.kcycle(v[i]) for i in range(v.shape[0])]))
            self.build_coarse(v)
        self.test_vectors = v
        return v


@pytest.mark.parametrize("mutant", [RebuildPerVector, NoNormalisation, SweepsOnDvEqualsV])
def test_planted_setup_mistakes_fail_a_pin(mutant):
    devs = [_pin_initial_phase(mutant), _pin_setup_pass(mutant)]
    assert max(devs) > 1e-6, devs


# ----------------------------------------------------------------------------
# three levels
# ----------------------------------------------------------------------------

L3 = (4, 4, 4, 4)
AGG1, NV1 = (2, 2, 2, 2), 4
AGG2, NV2 = (1, 1, 1, 1), 3


def _w0(Lc, seed):
    rng = np.random.default_rng(seed)
    s = (NV2,) + tuple(Lc) + (2 * NV1,)
    return rng.standard_normal(s) + 1j * rng.standard_normal(s)


def _three_level(fine_iters, coarse_iters):
    prm = ThreeLevelParams(m0=-0.3, c_sw=1.4, mu=0.05, delta=3.0, nv=NV1, agg=AGG1, sap_block=(2, 2, 2, 2),
                           mr_iters=2, pre_smooth=1, post_smooth=1, init_sweeps=1, setup_iters=fine_iters,
                           nv2=NV2, agg2=AGG2, sap_block1=(1, 1, 1, 1), pre_smooth1=1, post_smooth1=2,
                           init_sweeps1=1, coarse_setup_iters=coarse_iters)
    tl = ThreeLevel(inputs.gauge_field(L3, 0.5, 7), prm)
    D = dense_matrix(tl.op.apply, L3)
    bid, col = _block_ids(L3, prm.sap_block)
    fine_sm = ExactSmoother(D, np.repeat(bid, 12), np.repeat(col, 12), L3 + (4, 3))
    tl.sap = fine_sm
    Lc1 = tuple(L3[d] // AGG1[d] for d in range(4))
    n1, n2 = 2 * NV1, 2 * NV2
    cbid, ccol = _block_ids(Lc1, prm.sap_block1)
    state = {}
    build1 = tl.build_level1

    def build_level1_exact(v):
        build1(v)
        D1 = _dense_coarse(tl.Dc1.apply, Lc1, n1)
        state["D1"] = D1
        tl.csap = ExactSmoother(D1, np.repeat(cbid, n1), np.repeat(ccol, n1), Lc1 + (n1,))

    tl.build_level1 = build_level1_exact

    def coarsest_exact(r2, *a):
        D2 = _dense_coarse(tl.Dc2.apply, tl.P2.Lc, n2)
        return np.linalg.solve(D2, r2.ravel()).reshape(r2.shape)

    def level1_exact(r1, *a):
        return np.linalg.solve(state["D1"], r1.ravel()).reshape(r1.shape)

    tl.coarsest_solve = coarsest_exact
    tl.level1_solve = level1_exact
    return tl, D, fine_sm, Lc1, state


def test_three_level_fine_pass_is_dense_B_and_rebuilds_level2_from_w():
    tl, D, fsm, Lc1, state = _three_level(fine_iters=1, coarse_iters=0)
    v0 = inputs.random_test_vectors(L3, NV1, 8)
    w0 = _w0(Lc1, 9)
    v, w = tl.setup(v0, w0)
    Es = fsm.propagator()
    v1 = _norm_rows((Es @ v0.reshape(NV1, -1).T).T)
    P1 = Interpolation(v1.reshape(v0.shape), AGG1)
    Pd = _prolong_matrix(P1, P1.Lc, 2 * NV1)
    Dc1 = Pd.conj().T @ D @ Pd              # level 1 keeps the fine twisted mass
    B = _B_dense(D, Es, Pd, Dc1, tl.prm.pre_smooth, tl.prm.post_smooth)
    v2 = _norm_rows((B @ v1.T).T)
    assert np.max(np.abs(v.reshape(NV1, -1) - v2)) < 1e-10
    # level 2 after the fine pass: the unchanged w_j on the new D_c1
    assert np.max(np.abs(tl.P1.Q - Interpolation(v2.reshape(v0.shape), AGG1).Q)) < 1e-10
    P2 = CoarseInterpolation(w, AGG2, NV1)
    D2 = galerkin_coarse(tl.Dc1, P2, tl.prm.delta * tl.prm.mu)
    assert np.max(np.abs(tl.Dc2.blocks - D2.blocks)) < 1e-12


def test_three_level_coarse_pass_is_dense_B1():
    tl, D, fsm, Lc1, state = _three_level(fine_iters=0, coarse_iters=1)
    v0 = inputs.random_test_vectors(L3, NV1, 8)
    w0 = _w0(Lc1, 9)
    v, w = tl.setup(v0, w0)
    D1 = state["D1"]
    E1 = tl.csap.propagator()
    w1 = _norm_rows((E1 @ w0.reshape(NV2, -1).T).T)
    P2 = CoarseInterpolation(w1.reshape(w0.shape), AGG2, NV1)
    n2 = 2 * NV2
    N2 = int(np.prod(P2.Lc)) * n2
    Ec = np.eye(N2, dtype=complex).reshape((N2,) + P2.Lc + (n2,))
    P2d = P2.prolong(Ec).reshape(N2, -1).T
    # coarsest operator: the Galerkin product of D_c1(0) plus i delta mu Gamma5_c2
    D1_0 = D1 - 1j * tl.prm.mu * np.diag(np.tile(np.concatenate([-np.ones(NV1), np.ones(NV1)]),
                                                 D1.shape[0] // (2 * NV1)))
    g5c2 = np.tile(np.concatenate([-np.ones(NV2), np.ones(NV2)]), N2 // n2)
    D2 = P2d.conj().T @ D1_0 @ P2d + 1j * tl.prm.delta * tl.prm.mu * np.diag(g5c2)
    B1 = _B_dense(D1, E1, P2d, D2, tl.prm.pre_smooth1, tl.prm.post_smooth1)
    w2 = _norm_rows((B1 @ w1.T).T)
    assert np.max(np.abs(w.reshape(NV2, -1) - w2)) < 1e-10
    assert np.max(np.abs(tl.P2.Q - CoarseInterpolation(w2.reshape(w0.shape), AGG2, NV1).Q)) < 1e-10


class CoarseRebuildPerVector(ThreeLevel):
    """Mistake: P2 and D_c2 rebuilt after every level-1 vector of a pass."""

    def setup(self, v0, w0):
        prm = self.prm
        v = v0.copy()
        zero = np.zeros_like(v)
        for _ in range(prm.init_sweeps):
            v = self.sap.sweep(zero, v)
        v = normalise(v)
        self.build_level1(v)
        w = w0.copy()
        zw = np.zeros_like(w)
        for _ in range(prm.init_sweeps1):
            w = self.csap.sweep(zw, w)
        w = normalise(w)
        self.build_level2(w)
        for _ in range(prm.coarse_setup_iters):
            for j in range(w.shape[0]):
                w[j] = self.kcycle1(w[j])
                w = normalise(w)
                self.build_level2(w)
        self.test_vectors, self.test_vectors1 = v, w
        return v, w


def test_planted_level1_rebuild_per_vector_fails_the_level1_pin():
    ThreeLevel_ = ThreeLevel
    import oracle.multilevel as ml
    try:
        globals()["ThreeLevel"] = CoarseRebuildPerVector
        with pytest.raises(AssertionError):
            test_three_level_coarse_pass_is_dense_B1()
    finally:
        globals()["ThreeLevel"] = ThreeLevel_
    assert ml.ThreeLevel is ThreeLevel_
