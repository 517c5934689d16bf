"""Oracle: a plain, slow, FP64 CPU statement of what the embedding method computes.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) may import, call or link anything in this package.  It is used by
``tests/``, by ``__graft_entry__.smoke()`` (to check one small GPU result) and by the
CPU-baseline leg of ``bench.py``.  It shares no code with the CUDA path; the only
module both sides use is the seeded input generator ``manifold_graphs``.

Layout
  graph_ops  the sparse pair (A, B) of Sec. 4: two-hop sets T_i, Laplacian L, the
             disconnected two-hop difference matrix Q (Eq. 5), epsilon = lambda_2(Q),
             mu (Eq. 7-9), the Gershgorin radii r_i and b_i (Sec. 4.3).
  eigen      the first K generalized eigenpairs of (A, B) (Eq. 10-11): by dense
             symmetric eigendecomposition of B^{-1/2} A B^{-1/2} (small N) and by a
             textbook FP64 LOBPCG (the solver the paper names) for larger N; the
             residual / backward-error definitions used as convergence criteria.

Every floating point computation here is FP64.  Library primitives (sparse products,
dense symmetric eigendecomposition, connected components) serve as single steps; no
blocking, fusion or reordering beyond the definitions is done.

Pinned by the ``-m "not gpu"`` tests in tests/test_oracle_*.py against brute force on
tiny graphs, closed forms (odd rings, paths, rings with mu = epsilon = 0), structural
invariants and independent library routines.  Parity unpinned: nothing in this package
(the clustering experiments of Sec. 5, which need the paper's datasets, are not here).
"""
from . import graph_ops, eigen  # noqa: F401
