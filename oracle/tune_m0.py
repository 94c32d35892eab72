"""Near-critical bare mass m0 for a synthetic gauge field (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``); run as a script it
writes ``inputs/m0_tuned.json``, the m0 values the synthetic workloads use.

The workloads ask for "m0 fixed per seed so that the smallest singular value
of D_W is about 1e-3" (the paper's ensembles are tuned to the physical point,
Sec. 1; the synthetic stand-ins are not).  D_W(m0) = D_W(0) + m0, so its
eigenvalues move rigidly with m0.  Reading used here: find the eigenvalues
of D_W(0) with the smallest real part and set m0 = target - Re(lambda_left),
so that the spectrum of D_W(m0) just touches Re = target from the right (the
onset of eigenvalues with negative real part, i.e. the critical edge).  With
v the eigenvector of lambda_left, sigma_min(D_W) <= |lambda_left(m0)|; when the
field has a real eigenvalue at its left edge this bound equals the target,
otherwise it is the edge pair's modulus, which the output records.

D_W(0) is assembled as a sparse matrix (the same conventions as
:class:`oracle.dirac.Operator`, checked against it by
tests/test_oracle_tune.py) and ARPACK finds the eigenvalues of smallest real
part.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .dirac import GAMMA, ONE4, clover_matrix


def sparse_dirac(U: np.ndarray, m0: float, c_sw: float, bc_t: float = -1.0) -> sp.csr_matrix:
    """D_W(m0) as a CSR matrix, row/column index 12*site + 3*spin + colour."""
    L = U.shape[:4]
    V = int(np.prod(L))
    site = np.arange(V).reshape(L)
    rows, cols, vals = [], [], []
    A = clover_matrix(U, m0, c_sw).reshape(V, 12, 12)
    ii, jj = np.nonzero(np.abs(A).max(axis=0) > 0)
    for i, j in zip(ii, jj):
        rows.append(site.ravel() * 12 + i)
        cols.append(site.ravel() * 12 + j)
        vals.append(A[:, i, j])
    for mu in range(4):
        for sign in (+1, -1):
            nb = np.roll(site, -sign, axis=mu).ravel()
            phase = np.ones(L)
            if mu == 0 and bc_t != 1:
                idx = [slice(None)] * 4
                idx[0] = -1 if sign > 0 else 0
                phase[tuple(idx)] = bc_t
            phase = phase.ravel()
            if sign > 0:
                S = ONE4 - GAMMA[mu]
                Um = U[..., mu, :, :].reshape(V, 3, 3)              # U_mu(x)
            else:
                S = ONE4 + GAMMA[mu]
                Ub = np.roll(U[..., mu, :, :], 1, axis=mu)         # U_mu(x - mu)
                Um = np.conj(np.swapaxes(Ub, -1, -2)).reshape(V, 3, 3)
            for s in range(4):
                for t in range(4):
                    if S[s, t] == 0:
                        continue
                    for a in range(3):
                        for b in range(3):
                            rows.append(site.ravel() * 12 + 3 * s + a)
                            cols.append(nb * 12 + 3 * t + b)
                            vals.append(-0.5 * S[s, t] * Um[:, a, b] * phase)
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    return sp.csr_matrix((v, (r, c)), shape=(12 * V, 12 * V))


def leftmost_eigenvalues(D: sp.spmatrix, k: int = 16, ncv: int = 120, tol: float = 1e-7,
                         seed: int = 0) -> np.ndarray:
    """The k eigenvalues of smallest real part (ARPACK), sorted by real part."""
    rng = np.random.default_rng(seed)
    v0 = rng.standard_normal(D.shape[0]) + 1j * rng.standard_normal(D.shape[0])
    ev = spla.eigs(D, k=k, which="SR", ncv=ncv, tol=tol, v0=v0, return_eigenvectors=False,
                   maxiter=100000)
    return ev[np.argsort(ev.real)]


def tune_m0(U: np.ndarray, c_sw: float, target: float = 1e-3, bc_t: float = -1.0, **kw) -> dict:
    D0 = sparse_dirac(U, 0.0, c_sw, bc_t)
    t0 = time.time()
    ev = leftmost_eigenvalues(D0, **kw)
    lam = ev[0]
    real = ev[np.abs(ev.imag) < 1e-6]
    m0 = target - float(lam.real)
    return {"m0": m0, "lambda_left": [float(lam.real), float(lam.imag)],
            "sigma_min_bound": float(abs(complex(target, lam.imag))),
            "real_eigenvalue_at_edge": bool(real.size and abs(real[0].real - lam.real) < 1e-6),
            "target": target, "leftmost": [[float(e.real), float(e.imag)] for e in ev],
            "seconds": time.time() - t0}


WORKLOADS = {
    # name: (L = T,Z,Y,X, eps, seed, c_sw)
    "16x16x16x32_eps0.5_seed1": ((32, 16, 16, 16), 0.5, 1, 1.5),
    "24x24x24x48_eps0.5_seed1": ((48, 24, 24, 24), 0.5, 1, 1.5),
    # the 48^3x96 field strength and clover coefficient, tuned on a 16^3x32 volume
    "16x16x16x32_eps0.6_seed1_csw1.57551": ((32, 16, 16, 16), 0.6, 1, 1.57551),
}


def main(argv):
    import inputs
    out_path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "inputs", "m0_tuned.json")
    table = json.load(open(out_path)) if os.path.exists(out_path) else {}
    names = argv or list(WORKLOADS)
    for name in names:
        L, eps, seed, c_sw = WORKLOADS[name]
        U = inputs.gauge_field(L, eps, seed)
        res = tune_m0(U, c_sw)
        res.update({"L": list(L), "eps": eps, "seed": seed, "c_sw": c_sw})
        table[name] = res
        print(name, json.dumps(res))
        json.dump(table, open(out_path, "w"), indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
