"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds input generation only: random gauge links, sources and the
random starting test vectors that the adaptive setup draws.  It contains none
of the method's arithmetic (no Dirac operator, smoother, aggregation or
solver), so both sides may import it without sharing code.

The paper measures on real ensembles (cA2.09.48, 48^3x96, Sec. 1; cA2.09.64,
64^3x128, Sec. 3) that are not available here.  The stand-ins are random
near-unit gauge fields U = exp(i*eps*H) with H a Gaussian traceless Hermitian
3x3 matrix per link, on lattices of the same shapes.

Conventions
-----------
* Lattice extents are (T, Z, Y, X) with X fastest; the lexicographic order
  TZYX is the one the paper fixes for its library interface (Sec. 2).
* Gauge field: complex128 array [T, Z, Y, X, 4, 3, 3]; direction index
  0..3 = T, Z, Y, X; colour matrices row-major.
* Spinor field: complex128 array [T, Z, Y, X, 4, 3] (spin, colour).
* Random generator: numpy PCG64.  Gauge seed s, right-hand sides s + 1000,
  test vectors s + 2000.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann",
    "random_hermitian_traceless",
    "gauge_field",
    "unit_gauge",
    "gaussian_spinor",
    "point_sources",
    "random_test_vectors",
    "random_gauge_transform",
    "RHS_SEED_OFFSET",
    "TV_SEED_OFFSET",
]

RHS_SEED_OFFSET = 1000
TV_SEED_OFFSET = 2000


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape [8, 3, 3], complex128."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def random_hermitian_traceless(rng: np.random.Generator, shape) -> np.ndarray:
    """H = sum_a h_a lambda_a / 2 with h_a ~ N(0, 1) i.i.d.; shape + (3, 3)."""
    h = rng.standard_normal(tuple(shape) + (8,))
    return np.einsum("...a,aij->...ij", h, gell_mann() / 2)


def _expi_hermitian(H: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*H) for Hermitian H via the eigendecomposition H = W e W^H."""
    e, W = np.linalg.eigh(H)
    ph = np.exp(1j * eps * e)
    return np.einsum("...ik,...k,...jk->...ij", W, ph, W.conj())


def _gauge_chunk(args):
    """Worker of gauge_field: links lo..hi from the shared normals."""
    from multiprocessing import shared_memory
    name_h, name_u, n, lo, hi, eps = args
    sh = shared_memory.SharedMemory(name=name_h)
    su = shared_memory.SharedMemory(name=name_u)
    try:
        h = np.ndarray((n, 8), dtype=np.float64, buffer=sh.buf)
        u = np.ndarray((n, 3, 3), dtype=np.complex128, buffer=su.buf)
        H = np.einsum("...a,aij->...ij", h[lo:hi], gell_mann() / 2)
        u[lo:hi] = _expi_hermitian(H, eps)
        del h, u
    finally:
        sh.close()
        su.close()


def gauge_field(L, eps: float, seed: int, workers: int = 1) -> np.ndarray:
    """Random SU(3) links U_mu(x) = exp(i*eps*H_mu(x)), shape [T,Z,Y,X,4,3,3].

    ``workers`` > 1 evaluates the exponentials in that many spawned processes
    (same random numbers, same per-link arithmetic); for large lattices."""
    T, Z, Y, X = (int(v) for v in L)
    rng = np.random.Generator(np.random.PCG64(seed))
    if workers <= 1:
        H = random_hermitian_traceless(rng, (T, Z, Y, X, 4))
        return _expi_hermitian(H, eps)
    import multiprocessing as mp
    from multiprocessing import shared_memory
    n = T * Z * Y * X * 4
    sh = shared_memory.SharedMemory(create=True, size=n * 8 * 8)
    su = shared_memory.SharedMemory(create=True, size=n * 9 * 16)
    try:
        h = np.ndarray((n, 8), dtype=np.float64, buffer=sh.buf)
        h[...] = rng.standard_normal((n, 8))
        step = -(-n // (4 * workers))
        jobs = [(sh.name, su.name, n, lo, min(n, lo + step), eps) for lo in range(0, n, step)]
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_gauge_chunk, jobs)
        U = np.ndarray((n, 3, 3), dtype=np.complex128, buffer=su.buf).copy()
        del h
    finally:
        sh.close()
        sh.unlink()
        su.close()
        su.unlink()
    return U.reshape(T, Z, Y, X, 4, 3, 3)


def evolve_gauge(U: np.ndarray, eta: float, seed: int) -> np.ndarray:
    """A nearby gauge field exp(i*eta*H'(x)) U_mu(x) with a fresh random H'
    (a stand-in for one molecular-dynamics step of an HMC trajectory)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = _expi_hermitian(random_hermitian_traceless(rng, U.shape[:-2]), eta)
    return np.einsum("...ij,...jk->...ik", R, U)


def unit_gauge(L) -> np.ndarray:
    """The free field U_mu(x) = 1."""
    T, Z, Y, X = (int(v) for v in L)
    U = np.zeros((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def gaussian_spinor(L, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Spinor(s) with re, im ~ N(0, 1) i.i.d.; shape [nrhs?, T,Z,Y,X,4,3]."""
    T, Z, Y, X = (int(v) for v in L)
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (T, Z, Y, X, 4, 3) if nrhs is None else (nrhs, T, Z, Y, X, 4, 3)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def point_source_site(L, seed: int) -> tuple:
    """The site x0 of the twelve point sources (drawn uniformly, seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return tuple(int(rng.integers(0, int(n))) for n in L)


def point_sources(L, seed: int) -> tuple[np.ndarray, tuple]:
    """Twelve spin-colour point sources at one random site x0.

    Returns (sources [12, T,Z,Y,X,4,3], x0) with source k = 3*s0 + c0 equal
    to delta_{x,x0} delta_{s,s0} delta_{c,c0}.
    """
    T, Z, Y, X = (int(v) for v in L)
    x0 = point_source_site(L, seed)
    b = np.zeros((12, T, Z, Y, X, 4, 3), dtype=np.complex128)
    for s in range(4):
        for c in range(3):
            b[(3 * s + c,) + x0 + (s, c)] = 1.0
    return b, x0


def random_test_vectors(L, nv: int, seed: int) -> np.ndarray:
    """The random starting vectors v_1..v_Nv of the adaptive setup.

    Shape [Nv, T,Z,Y,X,4,3]; re, im ~ N(0, 1) i.i.d.
    """
    return gaussian_spinor(L, seed, nrhs=nv)


def random_coarse_vectors(Lc, n: int, count: int, seed: int) -> np.ndarray:
    """Random vectors on a coarse lattice with n complex components per site
    (the level-1 starting vectors w_j of a three-level setup, or coarse
    right-hand sides).  Shape [count, Tc,Zc,Yc,Xc, n]; re, im ~ N(0, 1) i.i.d."""
    rng = np.random.default_rng(seed)
    shape = (count,) + tuple(int(x) for x in Lc) + (n,)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_gauge_transform(L, seed: int, eps: float = 1.0) -> np.ndarray:
    """A random SU(3) matrix g(x) per site, shape [T,Z,Y,X,3,3]."""
    T, Z, Y, X = (int(v) for v in L)
    rng = np.random.Generator(np.random.PCG64(seed))
    H = random_hermitian_traceless(rng, (T, Z, Y, X))
    return _expi_hermitian(H, eps)
