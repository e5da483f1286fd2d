"""CPU FP64 oracle for arrowhead LPs -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct implementations of what the GPU path computes,
written from the paper (arXiv 2412.07731) and from the textbook primal-dual
interior-point method it builds on.  Only the test-suite, the smoke check and
the CPU-baseline leg of the benchmark may import this package; the library
itself never does, and it shares no code with the CUDA path (only the seeded
input generators in ``instances`` serve both).

Modules
  lp       monolithic assembly of the constraint matrix (Sec. 3.2/3.3) and
           LP residual / gap measures (Sec. 2.2)
  newton   the Newton system of Sec. 2.3 solved monolithically (dense LU or
           sparse LU of the augmented system)
  ipm      Mehrotra predictor-corrector IPM on the monolithic system
  schur    Alg. 1 / Alg. 2 / Alg. 3 on the paper's augmented block form, the
           App. A Schur block structure and the Observation-1 nnz bound
  vertex   brute-force vertex enumeration for tiny LPs
  adjoint  transposed Newton solve for implicit differentiation
  general  the full LP statement of Sec. 3.2 (inequality rows, bounds of every
           kind) reduced to the standard form by textbook transformations,
           solved by ipm and mapped back

Every function is pinned by a test in tests/test_oracle_*.py against something
other than itself (brute force, planted optima, library routines, closed forms).
"""
