"""FP64 CPU oracle for DD-alphaAMG with twisted-mass fermions (arXiv:1611.01034).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The CUDA library never calls it, links it or falls back to it, and it shares
no code with the CUDA path: the only common module is ``inputs`` (seeded
random inputs, none of the method's arithmetic).

Everything is plain numpy in complex128, vectorised over lattice sites (and
over independent blocks or right-hand sides where the method treats them
independently), with no blocking, fusion or reordering beyond what the
definitions state.

Modules
-------
* ``dirac``  -- gamma matrices (eq. 2), clover term, D(mu) = D_W + i*mu*Gamma5
  (Sec. 1), dense assembly for tiny lattices.
* ``sap``    -- the SAP smoother M with block-local minimal residual (Sec. 1,
  eq. 1; odd-even option of Sec. 3).
* ``coarse`` -- Gamma5-compatible aggregation P, the coarse operator
  D_c = P^dagger D_W P + i*mu_c*Gamma5_c (Sec. 1), its odd-even Schur
  complement (Sec. 3).
* ``krylov`` -- restarted (flexible) GMRES with CGS2 Arnoldi and Givens
  rotations (Sec. 1, Fig. 3).
* ``amg``    -- the K-cycle of eq. (1), the adaptive setup (Sec. 1, Sec. 3)
  and the FGMRES + AMG solve.
* ``multilevel`` -- the three-level hierarchy of Sec. 2 (coarse-grid SAP,
  level-1 aggregation, the level-1 K-cycle).
* ``evenodd`` -- the odd-site reduced operator with even/odd twisted masses
  and the Hasenbusch two-solve sequence (Sec. 2, Sec. 3).
* ``oecg``   -- odd-even CG on the normal equations, the comparison solver of
  Fig. 1 (Sec. 1).
* ``slabs``  -- the true residual of a large lattice evaluated T-slab by
  T-slab with the unchanged operator (for solutions too large for one
  full-lattice oracle apply).
* ``nn``     -- the learned gauge-covariant layer (not in the paper).
* ``tune_m0`` -- the m0 reading of the synthetic workloads.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, algebraic identities, dense brute force or library
routines; see the module docstrings for which pin covers which function.
"""
