"""The randomized-ID build (Sec. 2.2) on the GPU against the oracle's
randomized build with the same sample (Omega from the same normal stream):
tree bit-exact, leaf ranks within +-2, solutions within 10 eps of the
oracle's, the compressed operator within 10 eps of the dense matrix."""
import numpy as np
import pytest

import rs_inputs as ri
from oracle import dense, rskel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    ("laplace2d", "starfish", 4096, 1e-10, 64, 64),
    ("helmholtz2d", "starfish", 4096, 1e-9, 64, 64),
    ("laplace3d", "sphere", 4096, 1e-6, 128, 216),
]
P_OVER, SEED = 8, 3


@pytest.mark.parametrize("kind,geom,n,eps,leaf,nproxy", CASES, ids=lambda v: str(v))
def test_randomized_build_matches_oracle(kind, geom, n, eps, leaf, nproxy):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    pts, w = ri.geometry(geom, n)
    kw = 10.0 if kind.startswith("helmholtz") else 0.0
    cplx = kind.startswith("helmholtz")
    F = rskel.build(pts, rskel.Params(kind=kind, w=w, eps=eps, leaf=leaf, nproxy=nproxy, kwave=kw,
                                      id_oversample=P_OVER, id_seed=SEED))
    H = rs.rs_build(pts, kind, w, eps, leaf, nproxy, k_wave=kw, id_oversample=P_OVER, id_seed=SEED)
    try:
        assert np.array_equal(rs.rs_tree_perm(H), F.tree.perm)
        L = F.tree.L
        _, k = rs.rs_box_ranks(H, L, F.tree.levels[L].nbox)
        assert np.max(np.abs(k - np.array([f.k for f in F.boxes[L]]))) <= 2
        B = ri.rhs(n, 3, seed=81, complex_=cplx)
        X = np.zeros_like(B)
        rs.rs_solve(H, B, X)
        Xo = F.solve(B)
        err = np.linalg.norm(X - Xo, axis=0) / np.linalg.norm(Xo, axis=0)
        assert np.all(err <= 10 * eps), err
        Y = np.zeros_like(B)
        rs.rs_matvec(H, B, Y)
        A = dense.dense_matrix(kind, pts, w, kw)
        ya = A @ B
        assert np.all(np.linalg.norm(Y - ya, axis=0) / np.linalg.norm(ya, axis=0) <= 10 * eps)
    finally:
        H.free()


def test_randomized_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    pts, h = ri.circle(512)
    with pytest.raises(rs.RSError):
        rs.rs_build(pts, "laplace2d", h, 1e-9, 64, 64, id_oversample=-1)
    with pytest.raises(rs.RSError):
        rs.rs_build(pts, "laplace2d", h, 1e-9, 64, 64, id_oversample=8, id_arith="dfloat")
