"""Plain FP64 CPU oracle for the spin-restricted CCSDT (RCCSDT) residual path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library, its
Python binding) may import, call or link anything in this package; only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` do.
It shares no code with the CUDA path.

Modules
-------
``rccsdt``     RCCSD / RCCSDT on full storage, written term by term from the
               working equations of the paper's appendix A.5 (T1-dressed
               integrals of A.4, spin summation of Eq. triples-spin-sum, the
               permutation operator of Eq. rcc-perm-op), the energy, the Jacobi
               update of A.1 and the DIIS of Sec. III.A.5.
``compact``    The same residual on compact ``i <= j <= k`` storage, following
               Sec. II.C (direct traversal, unpacking, the representative
               contractions of the operation-count table) and the post-processing
               of Sec. II.D (symmetrisation, purification, orthogonalisation).
``detcc``      Brute-force FCI and determinant-space spin-orbital CC at any
               truncation, straight from the projective definition of A.1, and
               the spin-orbital CCSDT(Q) energy from its determinant definition.
``q_correction`` The RCCSDT(Q) energy correction on full storage, from the (Q)
               appendix (Eqs. ener-pt-q, resi-pt-q, q_t3_terms, q_w_vvv_voo,
               q_w_vvo_ooo, q_w_alter) and Eq. quadruples-spin-sum.
``nullspace``  The spin-free overlap metric of appendix B.
``opcount``    Leading operation counts (Sec. II.C.3 and its table).

Every function is FP64 and cites the passage it follows.
"""
