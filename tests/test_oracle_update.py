"""Pins of the oracle's setup update (Sec. 3): on an unchanged gauge field, a
setup with k iterations followed by an update with one fine iteration equals
a setup with k + 1 iterations (two levels; three levels with the level-1
iterations after the fine ones); an update on a new field builds D_c from
that field (equal to a build from the same vectors on it)."""
import numpy as np

import inputs
from oracle.amg import TwoLevel, AMGParams
from oracle.multilevel import ThreeLevel, ThreeLevelParams


def _two(U, iters):
    prm = AMGParams(m0=-0.3, c_sw=1.4, mu=0.02, delta=2.0, nv=6, agg=(2, 2, 2, 2), sap_block=(2, 2, 2, 2),
                    setup_iters=iters)
    return TwoLevel(U, prm)


def test_two_level_setup_plus_update_is_longer_setup():
    L = (4, 4, 4, 4)
    U = inputs.gauge_field(L, 0.5, 3)
    v0 = inputs.random_test_vectors(L, 6, 2003)
    a = _two(U, 1)
    a.setup(v0)
    a.update(1)
    b = _two(U, 2)
    b.setup(v0)
    assert np.allclose(a.test_vectors, b.test_vectors, atol=1e-13)
    assert np.allclose(a.Dc.blocks, b.Dc.blocks, atol=1e-12)


def test_two_level_update_on_new_field_builds_from_it():
    L = (4, 4, 4, 4)
    U = inputs.gauge_field(L, 0.5, 3)
    U2 = inputs.evolve_gauge(U, 0.05, 77)
    v0 = inputs.random_test_vectors(L, 6, 2003)
    a = _two(U, 1)
    a.setup(v0)
    c = _two(U2, 1)
    c.update(0, a.test_vectors)
    d = _two(U2, 1)
    d.build_coarse(a.test_vectors)
    assert np.allclose(c.Dc.blocks, d.Dc.blocks, atol=1e-14)
    assert not np.allclose(c.Dc.blocks, a.Dc.blocks, atol=1e-6)


def test_evolved_field_is_su3():
    U = inputs.gauge_field((2, 2, 2, 2), 0.5, 5)
    U2 = inputs.evolve_gauge(U, 0.1, 6)
    I = np.eye(3)
    assert np.allclose(np.einsum("...ij,...kj->...ik", U2, U2.conj()), I, atol=1e-13)
    assert np.allclose(np.linalg.det(U2), 1, atol=1e-13)


def test_three_level_setup_plus_update_is_longer_setup():
    L, agg1, nv1, agg2, nv2 = (8, 4, 4, 4), (2, 2, 2, 2), 6, (2, 1, 1, 1), 4

    def make(fi, ci):
        prm = ThreeLevelParams(m0=-0.3, c_sw=1.4, mu=0.02, delta=3.0, nv=nv1, agg=agg1, sap_block=(2, 2, 2, 2),
                               nv2=nv2, agg2=agg2, sap_block1=(2, 1, 1, 1), setup_iters=fi, coarse_setup_iters=ci)
        return ThreeLevel(U, prm)
    U = inputs.gauge_field(L, 0.5, 7)
    v0 = inputs.random_test_vectors(L, nv1, 2007)
    Lc1 = tuple(L[d] // agg1[d] for d in range(4))
    w0 = inputs.random_coarse_vectors(Lc1, 2 * nv1, nv2, 2008)
    a = make(1, 0)
    a.setup(v0, w0)
    a.update(1, 1)
    b = make(2, 1)
    b.setup(v0, w0)
    assert np.allclose(a.test_vectors, b.test_vectors, atol=1e-12)
    assert np.allclose(a.test_vectors1, b.test_vectors1, atol=1e-12)
    assert np.allclose(a.Dc2.blocks, b.Dc2.blocks, atol=1e-11)
