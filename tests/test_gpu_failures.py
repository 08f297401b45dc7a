"""Failure detection without a GPU fault (host-side injection).

A dependency wait of the persistent solve that can never be satisfied must
run out within its bound, raise the device flag and return RS_ERR_TIMEOUT,
leaving the context and the handle usable; an injected allocation failure
must surface as RS_ERR_OOM with no handle left behind.
"""
import numpy as np
import pytest

import rs_inputs as ri

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    rs.load()
    yield rs
    rs.rs_set_fault("off")


def test_wait_timeout_then_recovery(rs):
    n = 4096
    pts, h = ri.circle(n)
    H = rs.rs_build(pts, "laplace2d", h, 1e-9, 64, 64)
    B = ri.rhs(n, 2, seed=4)
    ref = np.zeros_like(B)
    rs.rs_solve(H, B, ref)
    rs.rs_set_fault("wait")
    X = np.zeros_like(B)
    with pytest.raises(rs.RSError) as e:
        rs.rs_solve(H, B, X)
    assert e.value.code == -5 and "wait" in str(e.value)
    X2 = np.zeros_like(B)
    rs.rs_solve(H, B, X2)           # counters restart; same answer as before
    assert np.array_equal(X2, ref)
    H.free()


def test_injected_allocation_failure(rs):
    pts, h = ri.circle(2048)
    rs.rs_set_fault("alloc:6")
    with pytest.raises(rs.RSError) as e:
        rs.rs_build(pts, "laplace2d", h, 1e-9, 64, 64)
    assert e.value.code == -2
    rs.rs_set_fault("off")
    H = rs.rs_build(pts, "laplace2d", h, 1e-9, 64, 64)
    assert H.stats()["n"] == 2048
    H.free()
