"""CPU oracle for the parallel-in-time preconditioned Biot solver (arxiv 2310.10430).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, FP64 restatement of the
method, written from the paper, against which the CUDA path is checked. Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline may import
it. The product path (the C-ABI library and its Python binding) never imports,
calls or links anything here, and this package never imports the product path.

Modules
-------
mesh      structured right-triangle mesh (Sec. 4: uniform grid, h = 1/2^k)
fem       P1 element matrices and assembly of A, B, C (Sec. 2.2) into the
          saddle-point matrix of Eq. (fullysystem) and the previous-step matrix A'
problems  boundary data, loads and exact solutions for the Terzaghi column and the
          trigonometric manufactured solution (Sec. 4.1)
system    Dirichlet elimination and the per-step right-hand sides f^n
solvers   Algorithm 1 with an exact solve (seq_solve), the block preconditioners
          P1/P2 (Eqs. p1, p2), the inner Krylov solver K (right-preconditioned
          FGMRES), Algorithm 3 literally, and the windowed sweep schedule
analytic  Terzaghi series solution, L2 error quadrature

Parity status: every function is pinned by a test under tests/ (test_oracle_*.py).
"""
