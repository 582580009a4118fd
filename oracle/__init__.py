"""CPU oracle for the hierarchical solver (test infrastructure only).

A plain, slow, float64 restatement of the paper's method, written for
checking the CUDA library and nothing else.  Only ``tests/``, the smoke check
in ``__graft_entry__`` and the CPU-baseline / reference legs of ``bench.py``
may import it; the library never calls into it and it shares no code with the
CUDA path (the only common module is the input generator
``paper_1712_07297_gb300.inputs``, which holds none of the method's
arithmetic).

Modules
-------
hsolver      Sec. 2: clustering (Alg. 1 partition step), block pattern A_B
             (Eq. quotient), distance-2 colouring (Sec. 3.2 independence rule),
             LowRank_Elimination (Eqs. lra, scaling, elim, perm), the level
             recursion of Alg. 1 and the substitution sweeps of Alg. 2.
krylov       Sec. 5: preconditioned CG and right-preconditioned FGMRES, used
             with the factorization as preconditioner.
matrix_form  Eqs. scaling/elim/perm built as full N x N operators for tiny
             problems, used to pin the block oracle's structure.

Parity status: every function is pinned by a ``-m "not gpu"`` test against
closed forms, library routines or invariants; see ``tests/test_oracle_*``.
"""
