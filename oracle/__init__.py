"""Plain FP64 CPU oracle of block PLHR (Vecharynski & Knyazev, arXiv 1408.0042).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
executes this directory; only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path:
operators are built as scipy sparse matrices from their textbook definitions,
the multigrid preconditioner follows Algorithm 4 step by step, and the
eigensolver follows Algorithm 3 (real arithmetic) / Algorithm 2 (complex
arithmetic) with explicit blockwise B-orthonormalisation.  Library primitives
(sparse and dense products, Cholesky, LAPACK eig/eigh) serve as single steps.

Modules:
  operators  - finite-difference and finite-element model operators
  avmg       - the absolute-value multigrid preconditioner (Appendix A, Alg. 4)
  plhr       - block PLHR (Section 4, Alg. 2 and Alg. 3)
  spectral   - the Teter-Payne-Allan preconditioner of Section 5.3 on a grid
  grad       - potential gradients of eigenvalues and eigenvector losses
                 of H(V) = -1/2 Lap + diag(V) (dense perturbation formulas)
"""
