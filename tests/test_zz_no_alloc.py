"""rs_solve_noalloc: the allocation-free solve gives rs_solve's results.

Some callers cannot let a solve allocate device memory: a latency-critical
serving loop (cudaMalloc/cudaFree can synchronize the whole device and stall
the other streams' work) or a process that fixed its device-memory budget at
start-up.  rs_solve_noalloc serves them from one static device array of the
library.  These tests call it through the C ABI, twice in a row, and compare
with rs_solve on the same handle.
"""
import numpy as np
import pytest

import rs_inputs as ri

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    n = 8192
    pts, h = ri.starfish(n)
    H = rs.rs_build(pts, "laplace2d", h, 1e-10, 64, 64)
    yield rs, H, n
    H.free()


def _dev(a):
    return torch.from_numpy(a).cuda().t().contiguous().t()


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_solve_on_two_calls(handle, prec):
    rs, H, n = handle
    B1 = _dev(ri.rhs(n, 2, seed=31))
    B2 = _dev(ri.rhs(n, 2, seed=32))
    ref1 = torch.zeros_like(B1)
    ref2 = torch.zeros_like(B2)
    rs.rs_solve(H, B1, ref1, precision=prec)
    rs.rs_solve(H, B2, ref2, precision=prec)
    X1 = torch.zeros_like(B1)
    X2 = torch.zeros_like(B2)
    rs.rs_solve_noalloc(H, B1, X1, precision=prec)        # first call (may set up the scratch address)
    free0 = torch.cuda.mem_get_info()[0]
    rs.rs_solve_noalloc(H, B2, X2, precision=prec)        # second call reuses the scratch
    rs.rs_solve_noalloc(H, B1, X1, precision=prec)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for X, ref in ((X1, ref1), (X2, ref2)):
        err = float(torch.linalg.norm(X - ref) / torch.linalg.norm(ref))
        assert err <= 1e-12, err


def test_noalloc_rejects_oversize_and_host_buffers(handle):
    rs, H, n = handle
    big = torch.zeros((n, 256), dtype=torch.float64, device="cuda").t().contiguous().t()
    with pytest.raises(rs.RSError) as e:
        rs.rs_solve_noalloc(H, big, torch.zeros_like(big))
    assert e.value.code == -1 and "limit" in str(e.value)
    Bh = ri.rhs(n, 1, seed=3)
    with pytest.raises(rs.RSError) as e:
        rs.rs_solve_noalloc(H, Bh, np.zeros_like(Bh))
    assert e.value.code == -1 and "device memory" in str(e.value)
