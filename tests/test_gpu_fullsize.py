"""Full-size workloads (the configurations of the benchmark family).

At these sizes the oracle cannot factor the matrix in test time, so the
checks use what it can compute one by one or what holds at any size:
  * the tree (permutation, box ranges, parents, colleagues) equals the
    oracle's tree bit for bit;
  * rows of the true A = I + w K, sampled and evaluated by the oracle's
    kernel function, applied to the GPU solution give back b to within
    10 eps (root-mean-square over the sampled rows, relative to b);
  * the refined mixed-precision solve meets its residual target and agrees
    with the FP64 solve.
"""
import numpy as np
import pytest

import rs_inputs as ri
from oracle.kernels import green
from oracle.tree import Tree

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NAMES = ["laplace2d_starfish_131072", "helmholtz2d_starfish_65536", "laplace3d_sphere_32768"]


@pytest.mark.parametrize("name", NAMES)
def test_full_size(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    wl = ri.WORKLOADS[name]
    pts, w = ri.geometry(wl["geom"], wl["n"])
    n, kw = wl["n"], wl.get("kwave", 0.0)
    cplx = wl["kernel"] == "helmholtz2d"
    H = rs.rs_build(pts, wl["kernel"], w, wl["eps"], wl["leaf"], wl["nproxy"], k_wave=kw)
    try:
        T = Tree(pts, wl["leaf"])
        assert np.array_equal(rs.rs_tree_perm(H), T.perm)
        for l in (T.L, T.L // 2, 1):
            g = rs.rs_tree_level(H, l)
            assert np.array_equal(g["begin"], T.levels[l].begin)
            assert np.array_equal(g["parent"], T.levels[l].parent)
        B = ri.rhs(n, 2, seed=5, complex_=cplx)
        X = np.zeros_like(B)
        rs.rs_solve(H, B, X)
        rows = np.random.default_rng(0).choice(n, 32, replace=False)
        G = green(wl["kernel"], pts[:, rows], pts, kw)
        G[np.arange(len(rows)), rows] = 0.0
        Ax = X[rows] + w * (G @ X)
        res = np.sqrt(np.mean(np.abs(Ax - B[rows]) ** 2, axis=0)) / np.sqrt(np.mean(np.abs(B) ** 2, axis=0))
        assert np.all(res <= 10 * wl["eps"]), res
        tol = 1e-9 if cplx else 1e-10
        Xr = np.zeros_like(B)
        its, rel = rs.rs_solve_refined(H, B, Xr, tol=tol, max_it=8)
        assert np.all(rel <= tol)
        assert np.linalg.norm(Xr - X) / np.linalg.norm(X) <= 10 * tol
    finally:
        H.free()
