"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Tolerances: tree and box indexing bit-exact; solutions within 10 eps of the
oracle's (relative 2-norm, Sec. 5 error bound for second-kind operators);
skeleton counts per leaf box within +-2 of the oracle's (pivot near-ties may
resolve differently under different rounding orders).
"""
import math

import numpy as np
import pytest

import rs_inputs as ri
from oracle import dense, rskel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    rs.load()


def rs_mod():
    import paper_1110_3105_gb300 as rs
    return rs


def _oracle(kind, pts, w, eps, leaf, nproxy, kwave=0.0):
    return rskel.build(pts, rskel.Params(kind=kind, w=w, eps=eps, leaf=leaf, nproxy=nproxy, kwave=kwave))


def _compare_tree(H, T):
    rs = rs_mod()
    assert np.array_equal(rs.rs_tree_perm(H), T.perm)
    stats = H.stats()
    assert stats["depth"] == T.L
    for l, lv in enumerate(T.levels):
        g = rs.rs_tree_level(H, l)
        assert np.array_equal(g["begin"], lv.begin), l
        if l > 0:
            assert np.array_equal(g["parent"], lv.parent), l
        assert len(g["colleagues"]) == lv.nbox
        for b in range(lv.nbox):
            assert np.array_equal(g["colleagues"][b], lv.colleagues[b]), (l, b)


def _tree_clouds():
    rng = np.random.default_rng(7)
    yield "circle4096", ri.circle(4096)[0], 64
    yield "starfish20000", ri.starfish(20000)[0], 64
    yield "sphere6000", ri.fibonacci_sphere(6000)[0], 128
    yield "uniform2d_ragged", rng.random((2, 4097)), 16
    yield "clustered3d", np.hstack([0.5 + rng.random((3, 500)) * 1e-4, rng.random((3, 1500))]), 40
    yield "tiny", ri.circle(7)[0], 64


@pytest.mark.parametrize("name,pts,leaf", list(_tree_clouds()), ids=lambda v: v if isinstance(v, str) else "")
def test_tree_bit_exact(name, pts, leaf):
    from oracle.tree import Tree
    rs = rs_mod()
    dim = pts.shape[0]
    kind = "laplace3d" if dim == 3 else "laplace2d"
    T = Tree(pts, leaf)
    H = rs.rs_build(pts, kind, 1.0 / pts.shape[1], 1e-6, leaf, 216 if dim == 3 else 64)
    try:
        _compare_tree(H, T)
    finally:
        H.free()


SOLVE_CASES = [
    ("laplace2d", "circle", 4096, 1e-9, 64, 64),
    ("laplace2d", "starfish", 8192, 1e-10, 64, 64),
    ("helmholtz2d", "starfish", 4096, 1e-9, 64, 64),
    ("laplace3d", "sphere", 4096, 1e-6, 128, 216),
    ("helmholtz3d", "sphere", 2048, 1e-6, 128, 216),
]


@pytest.fixture(scope="module", params=SOLVE_CASES, ids=lambda c: f"{c[0]}-{c[1]}-{c[2]}")
def built(request):
    rs = rs_mod()
    kind, geom, n, eps, leaf, nproxy = request.param
    pts, w = ri.geometry(geom, n)
    kw = 10.0 if kind.startswith("helmholtz") else 0.0   # 3D: k = 10 is omega = 3.18 on the unit sphere (Sec. 6.2)
    F = _oracle(kind, pts, w, eps, leaf, nproxy, kw)
    H = rs.rs_build(pts, kind, w, eps, leaf, nproxy, k_wave=kw)
    yield dict(kind=kind, n=n, eps=eps, F=F, H=H, pts=pts, w=w, kw=kw, cplx=kind.startswith("helmholtz"))
    H.free()


def test_build_tree_matches(built):
    _compare_tree(built["H"], built["F"].tree)


def test_leaf_ranks_match(built):
    rs = rs_mod()
    F, H = built["F"], built["H"]
    L = F.tree.L
    n, k = rs.rs_box_ranks(H, L, F.tree.levels[L].nbox)
    on = np.array([f.n for f in F.boxes[L]])
    ok = np.array([f.k for f in F.boxes[L]])
    assert np.array_equal(n, on)
    assert np.max(np.abs(k - ok)) <= 2


def test_solve_fp64_matches_oracle(built):
    rs = rs_mod()
    n, eps = built["n"], built["eps"]
    B = ri.rhs(n, 3, seed=21, complex_=built["cplx"])
    X = np.zeros_like(B)
    rs.rs_solve(built["H"], B, X)
    Xo = built["F"].solve(B)
    err = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
    assert err <= 10 * eps, err


def test_matvec_matches_dense_and_inverts(built):
    rs = rs_mod()
    n, eps = built["n"], built["eps"]
    x = ri.rhs(n, 2, seed=3, complex_=built["cplx"])
    y = np.zeros_like(x)
    rs.rs_matvec(built["H"], x, y)
    A = dense.dense_matrix(built["kind"], built["pts"], built["w"], built["kw"])
    ya = A @ x
    assert np.linalg.norm(y - ya) / np.linalg.norm(ya) <= 10 * eps
    z = np.zeros_like(x)
    rs.rs_solve(built["H"], y, z)
    assert np.linalg.norm(z - x) / np.linalg.norm(x) < 1e-11


def test_fp32_solve_and_refinement(built):
    rs = rs_mod()
    n = built["n"]
    B = ri.rhs(n, 4, seed=8, complex_=built["cplx"])
    X64 = np.zeros_like(B)
    rs.rs_solve(built["H"], B, X64)
    X32 = np.zeros_like(B)
    rs.rs_solve(built["H"], B, X32, precision=rs.RS_PREC_FP32)
    assert np.linalg.norm(X32 - X64) / np.linalg.norm(X64) < 1e-4
    Xr = np.zeros_like(B)
    its, rel = rs.rs_solve_refined(built["H"], B, Xr, tol=1e-10, max_it=8)
    assert np.all(rel <= 1e-10), rel
    assert its >= 1
    assert np.linalg.norm(Xr - X64) / np.linalg.norm(X64) < 1e-9
    # the reported residual is what an independent FP64 apply of A_RS measures
    Y = np.zeros_like(Xr)
    rs.rs_matvec(built["H"], Xr, Y)
    true_rel = np.linalg.norm(Y - B, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(true_rel <= 1e-10), true_rel
    assert np.all(np.abs(true_rel - rel) <= 1e-12 + 1e-3 * true_rel), (true_rel, rel)


def test_matvec_matches_oracle_apply(built):
    """rs_matvec (FP64 forward operator, Sec. 3.3) against the oracle's own
    compressed operator A_RS, column by column: the two compress A with their
    own skeletons, each within eps of A (Def. 2.3), so they agree to 10 eps."""
    rs = rs_mod()
    n, eps = built["n"], built["eps"]
    x = ri.rhs(n, 3, seed=31, complex_=built["cplx"])
    y = np.zeros_like(x)
    rs.rs_matvec(built["H"], x, y)
    yo = built["F"].apply(x)
    err = np.linalg.norm(y - yo, axis=0) / np.linalg.norm(yo, axis=0)
    assert np.all(err <= 10 * eps), err


def _check_refined_against_oracle(built, B, Xr, rel, tol):
    """The refined solution against the oracle's FP64 solve (10 eps per
    column); the residual of the GPU's X under the oracle's A_RS and under
    the dense A (both within 10 eps: the GPU's operator differs from each by
    at most that); and the library's reported residual against the oracle's
    measurement of it (they may differ by the two operators' difference)."""
    eps = built["eps"]
    Xo = built["F"].solve(B)
    err = np.linalg.norm(Xr - Xo, axis=0) / np.linalg.norm(Xo, axis=0)
    assert np.all(err <= 10 * eps), err.max()
    nb = np.linalg.norm(B, axis=0)
    r_oracle = np.linalg.norm(built["F"].apply(Xr) - B, axis=0) / nb
    assert np.all(r_oracle <= 10 * eps), r_oracle.max()
    assert np.all(rel <= tol), rel.max()
    assert np.all(np.abs(r_oracle - rel) <= 10 * eps), np.abs(r_oracle - rel).max()
    if built["n"] <= 8192:
        A = dense.dense_matrix(built["kind"], built["pts"], built["w"], built["kw"])
        r_true = np.linalg.norm(A @ Xr - B, axis=0) / nb
        assert np.all(r_true <= 10 * eps), r_true.max()


def test_refined_matches_oracle(built):
    rs = rs_mod()
    n = built["n"]
    B = ri.rhs(n, 5, seed=33, complex_=built["cplx"])
    Xr = np.zeros_like(B)
    its, rel = rs.rs_solve_refined(built["H"], B, Xr, tol=1e-10, max_it=8)
    assert its >= 1
    _check_refined_against_oracle(built, B, Xr, rel, 1e-10)


@pytest.mark.parametrize("nrhs", [40, 70, 130])
def test_many_rhs_tiles(built, nrhs):
    """Block-tiled multi-column solve (column blocks of 32/64/128 with a ragged
    last block) against the oracle, in FP64, FP32 and refined form."""
    rs = rs_mod()
    n, eps = built["n"], built["eps"]
    B = ri.rhs(n, nrhs, seed=40 + nrhs, complex_=built["cplx"])
    X = np.zeros_like(B)
    rs.rs_solve(built["H"], B, X)
    Xo = built["F"].solve(B)
    err = np.linalg.norm(X - Xo, axis=0) / np.linalg.norm(Xo, axis=0)
    assert np.all(err <= 10 * eps), err.max()
    X32 = np.zeros_like(B)
    rs.rs_solve(built["H"], B, X32, precision=rs.RS_PREC_FP32)
    assert np.all(np.linalg.norm(X32 - X, axis=0) / np.linalg.norm(X, axis=0) < 1e-4)
    # the first call of a column count tuned the tile shape; later calls use
    # the chosen one and agree bit for bit
    X2 = np.zeros_like(B)
    rs.rs_solve(built["H"], B, X2)
    assert np.array_equal(X2, X)
    X32b = np.zeros_like(B)
    rs.rs_solve(built["H"], B, X32b, precision=rs.RS_PREC_FP32)
    assert np.array_equal(X32b, X32)
    Xr = np.zeros_like(B)
    its, rel = rs.rs_solve_refined(built["H"], B, Xr, tol=1e-10, max_it=8)
    Y = np.zeros_like(Xr)
    rs.rs_matvec(built["H"], Xr, Y)
    true_rel = np.linalg.norm(Y - B, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(true_rel <= 1e-10), true_rel.max()
    assert np.all(np.abs(true_rel - rel) <= 1e-12 + 1e-3 * true_rel)
    _check_refined_against_oracle(built, B, Xr, rel, 1e-10)


def test_device_pointers_same_as_host(built):
    rs = rs_mod()
    n = built["n"]
    B = ri.rhs(n, 2, seed=2, complex_=built["cplx"])
    Xh = np.zeros_like(B)
    rs.rs_solve(built["H"], B, Xh)
    Bd = torch.from_numpy(B).cuda().t().contiguous().t()
    Xd = torch.zeros_like(Bd)
    rs.rs_solve(built["H"], Bd, Xd)
    torch.cuda.synchronize()
    assert np.array_equal(Xd.cpu().numpy(), Xh)


def test_dfloat_id_matches_oracle(built):
    """The double-float QR of the ID (rs_id_arith) against the same oracle:
    ranks within +-2 per leaf, solutions within 10 eps (real kernels)."""
    if built["cplx"]:
        pytest.skip("complex kernels always run the FP64 QR")
    rs = rs_mod()
    F, n, eps = built["F"], built["n"], built["eps"]
    leaf, nproxy = (128, 216) if built["kind"] == "laplace3d" else (64, 64)
    H = rs.rs_build(built["pts"], built["kind"], built["w"], eps, leaf, nproxy, id_arith="dfloat")
    try:
        _compare_tree(H, F.tree)
        L = F.tree.L
        nb, kb = rs.rs_box_ranks(H, L, F.tree.levels[L].nbox)
        assert np.max(np.abs(kb - np.array([f.k for f in F.boxes[L]]))) <= 2
        B = ri.rhs(n, 3, seed=23)
        X = np.zeros_like(B)
        rs.rs_solve(H, B, X)
        Xo = F.solve(B)
        assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 10 * eps
    finally:
        H.free()


def _circle_eig(n, m):
    s = math.fsum(math.log(2 * math.sin(math.pi * j / n)) * math.cos(2 * math.pi * m * j / n)
                  for j in range(1, n))
    return 1.0 - s / n


def test_circle_closed_form_gpu():
    rs = rs_mod()
    n, eps = 4096, 1e-9
    pts, h = ri.circle(n)
    H = rs.rs_build(pts, "laplace2d", h, eps, 64, 64)
    th = 2 * np.pi * np.arange(n) / n
    ms = (0, 1, 5, 17)
    B = np.asfortranarray(np.stack([np.cos(m * th) for m in ms], axis=1))
    X = np.zeros_like(B)
    rs.rs_solve(H, B, X)
    H.free()
    for i, m in enumerate(ms):
        ref = B[:, i] / _circle_eig(n, m)
        assert np.linalg.norm(X[:, i] - ref) / np.linalg.norm(ref) <= 10 * eps


def test_edge_cases():
    rs = rs_mod()
    # single point, a tree with one box, one more point than a leaf
    for n in (1, 5, 64, 65):
        pts, h = ri.circle(n)
        H = rs.rs_build(pts, "laplace2d", h, 1e-9, 64, 64)
        B = ri.rhs(n, 1, seed=1)
        X = np.zeros_like(B)
        rs.rs_solve(H, B, X)
        A = dense.dense_matrix("laplace2d", pts, h)
        assert np.linalg.norm(A @ X - B) / np.linalg.norm(B) < 1e-8, n
        H.free()
    # too many coincident points
    pts = np.zeros((2, 100))
    with pytest.raises(rs.RSError) as e:
        rs.rs_build(pts, "laplace2d", 0.01, 1e-9, 64, 64)
    assert e.value.code == -1
    # non-finite coordinate
    pts, h = ri.circle(100)
    pts[0, 3] = np.nan
    with pytest.raises(rs.RSError) as e:
        rs.rs_build(pts, "laplace2d", h, 1e-9, 64, 64)
    assert e.value.code == -6
    # bad arguments
    pts, h = ri.circle(100)
    for kw in (dict(eps=0.0), dict(eps=2.0), dict(leaf=0), dict(proxy_n=0)):
        args = dict(eps=1e-9, leaf=64, proxy_n=64)
        args.update(kw)
        with pytest.raises(rs.RSError):
            rs.rs_build(pts, "laplace2d", h, args["eps"], args["leaf"], args["proxy_n"])
