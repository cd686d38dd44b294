"""Plain FP64 CPU oracle for the randomized restarted Krylov method for f(A)b.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code, table or constant generator
with the CUDA path; the two meet only through the seeded inputs of the
``workloads`` package.

Every routine is written for a reader who checks it against the paper by eye:
loops in the paper's order and notation, FP64 throughout, library primitives
(matrix products, linear solves) only as single steps.

Modules
-------
philox    Philox4x32-10 counter-based generator (Salmon et al., SC'11).
sketch    sparse sign embedding S of Eq. (3), generated column by column.
dense     small dense kernels: Householder QR with positive diagonal, the
          matrix exponential (scaling and squaring with the degree-13 Pade
          approximant, Higham 2005), the inverse square root (Denman-Beavers),
          the inverse.
krylov    the restarted methods: classical restarted Arnoldi, the paper's
          randomized restart (Algorithms 1 and 2), and the truncated +
          whitened restart (Appendix A, Eq. A.1) used by the GPU path.
truth     closed-form references: Kronecker-sum exponentials of the grid
          operators, dense eigendecomposition on tiny matrices.
"""
