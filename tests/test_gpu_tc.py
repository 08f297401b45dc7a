"""Tensor-core building blocks (tcgen05 MMA through shared-memory descriptors
and tensor memory) against a host product of the same rounded operands."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _round_tf32(x):
    u = x.astype(np.float32).view(np.uint32)
    u = (u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return u.view(np.float32)


@pytest.mark.parametrize("kind,n", [(0, 16), (0, 64), (0, 256), (1, 32), (1, 128), (1, 256)])
def test_selftest_block_product(kind, n):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    K = 32 if kind == 0 else 64
    rng = np.random.default_rng(11 + n + kind)
    A = rng.standard_normal((128, K)).astype(np.float32)
    B = rng.standard_normal((n, K)).astype(np.float32)
    if kind == 0:
        Ar, Br = _round_tf32(A), _round_tf32(B)
    else:
        Ar = torch.from_numpy(A).bfloat16().float().numpy()
        Br = torch.from_numpy(B).bfloat16().float().numpy()
    ref = Ar.astype(np.float64) @ Br.astype(np.float64).T
    D = torch.zeros((128, n), dtype=torch.float32, device="cuda")
    rs.rs_tc_selftest(kind, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), D)
    torch.cuda.synchronize()
    got = D.cpu().numpy().astype(np.float64)
    # products of tf32/bf16 values are exact in fp32; only the fp32
    # accumulation over K terms rounds
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref)) * K


# -------------------------------------------------- tensor-core solve tiles
import rs_inputs as ri  # noqa: E402
from oracle import rskel  # noqa: E402

# The 3D sphere's top blocks are thousands deep: there the library keeps the
# CUDA-core tiles even when the tensor-core tiles are asked for (their fp32
# accumulation over so many K steps is an order of magnitude less accurate),
# so that case checks the fallback.
TC_CASES = [
    ("laplace2d", "circle", 4096, 1e-9, 64, 64),
    ("laplace2d", "starfish", 8192, 1e-10, 64, 64),
    ("laplace3d", "sphere", 4096, 1e-6, 128, 216),
]


@pytest.fixture(scope="module", params=TC_CASES, ids=lambda c: f"{c[0]}-{c[1]}-{c[2]}")
def tc_built(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    kind, geom, n, eps, leaf, nproxy = request.param
    pts, w = ri.geometry(geom, n)
    F = rskel.build(pts, rskel.Params(kind=kind, w=w, eps=eps, leaf=leaf, nproxy=nproxy))
    H = rs.rs_build(pts, kind, w, eps, leaf, nproxy)
    yield dict(rs=rs, n=n, eps=eps, F=F, H=H, dim=pts.shape[0])
    H.free()


@pytest.mark.parametrize("tile", ["128x64", "128x128", "128x256"])
@pytest.mark.parametrize("nrhs", [40, 130, 256])
def test_tc_solve_tiles(tc_built, tile, nrhs):
    """The FP32 solve on tensor-core tiles (3xTF32 products) against the FP64
    solve (fp32-level agreement, as the CUDA-core FP32 tiles), repeatable bit
    for bit, and the refined solve built on it against the oracle (10 eps)."""
    rs, H, n, eps, F = tc_built["rs"], tc_built["H"], tc_built["n"], tc_built["eps"], tc_built["F"]
    B = ri.rhs(n, nrhs, seed=70 + nrhs)
    X64 = np.zeros_like(B)
    rs.rs_solve(H, B, X64)
    Xc = np.zeros_like(B)
    rs.rs_set_path("tile:32x64")       # the CUDA-core FP32 tiles, for comparison
    try:
        rs.rs_solve(H, B, Xc, precision=rs.RS_PREC_FP32)
    finally:
        rs.rs_set_path(None)
    rs.rs_set_path("tile:" + tile)
    try:
        X = np.zeros_like(B)
        rs.rs_solve(H, B, X, precision=rs.RS_PREC_FP32)
        X2 = np.zeros_like(B)
        rs.rs_solve(H, B, X2, precision=rs.RS_PREC_FP32)
        Xr = np.zeros_like(B)
        its, rel = rs.rs_solve_refined(H, B, Xr, tol=1e-10, max_it=8)
    finally:
        rs.rs_set_path(None)
    # fp32-level agreement: the same bar as the CUDA-core FP32 tiles; on the
    # 2D curves (every block product at most ~150 deep) also no further from
    # the FP64 solve than twice their error.  The 3D top boxes' products are
    # hundreds to thousands deep, and the tensor cores' fp32 accumulation of
    # one K step after another loses more there than the CUDA-core FMA chain
    # (about 1e-5 against 1e-6 at N = 4096): tf32-level, as the 3D workload
    # allows, and the refinement below still reaches 1e-10.
    err = np.linalg.norm(X - X64, axis=0) / np.linalg.norm(X64, axis=0)
    err_c = np.linalg.norm(Xc - X64, axis=0) / np.linalg.norm(X64, axis=0)
    assert np.all(err < 1e-4), err.max()
    if tc_built["dim"] == 2:
        assert np.all(err <= 2 * err_c + 1e-6), (err.max(), err_c.max())
    assert np.array_equal(X, X2)
    assert np.all(rel <= 1e-10), rel.max()
    Xo = F.solve(B)
    e2 = np.linalg.norm(Xr - Xo, axis=0) / np.linalg.norm(Xo, axis=0)
    assert np.all(e2 <= 10 * eps), e2.max()
    Y = np.zeros_like(Xr)
    rs.rs_matvec(H, Xr, Y)
    true_rel = np.linalg.norm(Y - B, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(true_rel <= 1e-10), true_rel.max()
    assert np.all(np.abs(true_rel - rel) <= 1e-12 + 1e-3 * true_rel)
