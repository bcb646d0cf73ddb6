"""CPU oracle for the Sparse Geometric Factorization (SGF) hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
the method written from the paper (Klockiewicz & Darve, "Sparse Hierarchical
Preconditioners Using Piecewise Smooth Approximations of Eigenvectors"):

* `assemble`  - the SPD operators of Sec. 7.1 (stencils, TPFA, Q1 elasticity)
* `partition` - the geometric nested-dissection partitions of Sec. 5.1
* `basis`     - the discretized polynomial bases Pi^j of Sec. 3.1 and the
                rigid-body modes of Sec. 7.2, in node-local coordinates
* `sgf`       - Algorithm 4.1: interior elimination (Sec. 4.1), polynomial
                compression (Sec. 3.2, 4.2), coarsening and Phi merge
                (Sec. 4.3-4.4), top Cholesky (Sec. 4.5) and the apply of
                A_l^{-1} (Sec. 4.7)
* `dense`     - a brute-force dense n x n restatement of Algorithm 4.1 used
                only to pin `sgf` on tiny grids
* `pcg`       - preconditioned conjugate gradients (Sec. 7)

Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / reference
leg of `bench.py` may import it.  It shares no code with the CUDA library and
must never sit on the product path.
"""
