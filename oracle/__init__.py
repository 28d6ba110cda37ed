"""CPU FP64 oracle for the hybridised Crouzeix-Raviart Stokes / Navier-Stokes solve.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of what the paper computes, used to prove the CUDA library right.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import it; the library never does, and it imports nothing from the
library.  It shares with the library only the seeded inputs of ``synth``.

Modules (each function cites the passage it follows):

* ``topology``   faces, interior/exterior, owners and C_K signs, K_0, the
                 maximal independent set M_1 used when mu = 0.
* ``elements``   geometry, the CR basis, S_K, A_K, D_K, R_K (Sections 2, 3.1).
* ``convection`` the co-volume convection form b_h (Eq. 9) and its Newton /
                 Oseen linearisations.
* ``coupled``    assembly of the coupled system (Eq. 10) and its direct solve:
                 the plain definition of the result the method reaches.
* ``hybrid``     E_K, C_K, B_K, G_K, S (Section 3.2, item 4) and the recovery
                 of U and P (item 2), step by step.
* ``krylov``     textbook Jacobi-PCG, restarted GMRES and iterative refinement.

No function here is left unpinned: each is checked in ``tests/test_oracle_*.py``
against closed forms, invariants, brute force or a library routine, and
``tests/test_oracle_mutations.py`` plants mistakes that those pins catch.
"""

from . import topology, elements, convection, coupled, hybrid, krylov  # noqa: F401
