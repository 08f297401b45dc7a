"""CPU oracle for recursive skeletonization (Ho & Greengard, arXiv 1110.3105).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 (complex128
for Helmholtz) restatement of the method, written from the paper, used to
check the GPU library.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the GPU library: it reads inputs only from the seeded generators in
``rs_inputs`` and never from the library.

Modules
  tree     quadtree / octree with contiguous index blocks (Sec. 2.1, Ex. 1;
           Sec. 6 opening paragraph)
  kernels  Green's functions (eqs. 2d-laplace, 3d-laplace, 2d-helmholtz,
           3d-helmholtz) and
           the system matrix A = I + w K with K_ii = 0
  interp   interpolative decomposition by column-pivoted Householder QR with
           adaptive rank (Sec. 2.2, Def. 2.3)
  rskel    proxy compression (Sec. 3.1-3.2), telescoping forward operator
           (eq. multilevel-compression, Sec. 3.3), compressed inverse
           (eqs. compressed-inverse, multilevel-inverse, Sec. 3.4) and solve
  dense    dense matrices and dense solves for small N (brute-force checks)

Parity status per function is listed in each module header.
"""
from . import tree, kernels, interp, rskel, dense  # noqa: F401
