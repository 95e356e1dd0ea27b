"""CPU oracle for the adaptive s-step conjugate gradient method (Carson 2019).

TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 numpy/scipy restatements of the
paper's algorithms, written to be checked against the paper by eye.  Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA library never calls it and
shares no code, table or constant generator with it.

Modules
  operators  stencil -> sparse matrix assembly (the operator's definition)
  basis      eq. (rho) basis polynomials, eq. (B), Newton/Leja (eq. newtbasis)
             and Chebyshev (eq. chebbasis) parameters
  ritz       eq. (T), eq. (lit) and Algorithms 3-4 (Meurant-Tichy estimates)
  cg         Algorithm 1 (HSCG) and Algorithm 5 (improved adaptive s-step CG)
  adjoint    dense adjoint of the differentiable solve (tiny systems)

Parity status: every function is pinned by a ``-m "not gpu"`` test except the
adaptive-s decision sequence of Algorithm 5 against the paper's own tables,
which needs the SuiteSparse matrices of Table 1 ("parity unpinned" there: the
decisions are pinned only oracle-vs-GPU, through decision logs).
"""
