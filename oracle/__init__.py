"""FP64 CPU oracle for the MRHS Wilson-clover multigrid solver (arXiv:2211.13719).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library; the only module both sides use is ``synth``
(seeded random inputs, no solver arithmetic).

Everything here is plain numpy in complex128, written for a reader checking it
against the paper by eye: whole-lattice shifts with ``np.roll``, ``einsum`` for
the small matrix products, ``numpy.linalg`` for QR and least squares.

Modules
-------
conventions  gamma matrices (chiral basis), sigma_{mu nu}
wilson       fine Wilson-clover operator D (Sec. 4): clover-leaf field strength,
             clover term, hopping term, per-site evaluation, dense matrix
coarse       aggregation, chirally split prolongator (Sec. 5), restriction and
             prolongation, Galerkin coarse operator R D P as a 9-point stencil
             (Sec. 6), coarse apply
krylov       per-RHS GMRES / flexible GMRES with batched inner products (Sec. 7, 8)
mg           null-vector setup, V-cycle, MG-preconditioned FGMRES solve (Sec. 8)
evenodd      checkerboard decomposition, Schur complement D_hat (Sec. 4, M_eooe)
sap          Schwarz alternating procedure smoother (Sec. 9 outlook)
gcrodr       GCRO-DR coarsest-level solver with subspace recycling (Sec. 9 outlook)

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against a closed form, an invariant or a brute-force
dense computation.  The null-vector relaxation (``mg.setup_nullvecs``) has no
closed form; it is pinned only through properties (it lowers ||D v|| / ||v||
and feeds a preconditioner that converges), which the tests check.
"""
