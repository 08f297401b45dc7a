"""Serving: continuous batching, admission, and alone-versus-mix results.

The server coalesces requests that arrive while a batch is on the GPU into
one multi-column refined solve.  Each request's result must be the same when
it is served alone and when it is served inside a mixed batch (every column
is computed independently; the refinement target is a relative residual of
1e-10, so the two must agree to about that level), and every result must
meet the residual target against the compressed operator.
"""
import numpy as np
import pytest

import rs_inputs as ri

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    n = 8192
    pts, h = ri.starfish(n)
    H = rs.rs_build(pts, "laplace2d", h, 1e-10, 64, 64)
    yield rs, H, n
    H.free()


def _residual(rs, H, X, B):
    Y = np.zeros_like(X)
    rs.rs_matvec(H, X, Y)
    return np.linalg.norm(Y - B, axis=0) / np.linalg.norm(B, axis=0)


def test_same_alone_and_in_mix(setup):
    rs, H, n = setup
    S = rs.Server(max_cols=128)
    hid = S.add(H)
    B0 = ri.rhs(n, 5, seed=77)
    X_alone = np.zeros_like(B0)
    r = S.wait(S.submit(hid, B0, X_alone))
    assert r["status"] == 0 and r["relres"] <= 1e-10
    # the same request inside a burst of others (coalesced into shared batches)
    rng = np.random.default_rng(5)
    tickets, outs = [], []
    for i in range(24):
        if i == 11:
            B, X = B0, np.zeros_like(B0)
        else:
            B = ri.rhs(n, int(rng.integers(1, 9)), seed=100 + i)
            X = np.zeros_like(B)
        tickets.append(S.submit(hid, B, X))
        outs.append((B, X))
    res = [S.wait(t) for t in tickets]
    st = S.stats()
    S.destroy()
    assert all(q["status"] == 0 and q["relres"] <= 1e-10 for q in res)
    X_mix = outs[11][1]
    assert np.linalg.norm(X_mix - X_alone) / np.linalg.norm(X_alone) <= 1e-10
    for B, X in outs:
        assert np.all(_residual(rs, H, X, B) <= 1e-10)
    # requests were coalesced: fewer batches than requests
    assert st["batches"] < st["requests"]
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_build_admission_and_new_handle(setup):
    rs, H, n = setup
    pts, h = ri.starfish(4096, arms=3, amp=0.2)
    tiny = rs.Server(max_cols=16, hbm_budget_bytes=1 << 20)
    r = tiny.wait(tiny.submit_build(pts, "laplace2d", h, 1e-10, 64, 64))
    tiny.destroy()
    assert r["status"] == -2                       # not admitted under a 1 MiB budget
    S = rs.Server(max_cols=16)
    r = S.wait(S.submit_build(pts, "laplace2d", h, 1e-10, 64, 64))
    assert r["status"] == 0
    hid = r["result"]
    B = ri.rhs(4096, 3, seed=9)
    X = np.zeros_like(B)
    q = S.wait(S.submit(hid, B, X))
    S.destroy()
    assert q["status"] == 0 and q["relres"] <= 1e-10
    Href = rs.rs_build(pts, "laplace2d", h, 1e-10, 64, 64)
    Xr = np.zeros_like(B)
    rs.rs_solve(Href, B, Xr)
    Href.free()
    assert np.linalg.norm(X - Xr) / np.linalg.norm(Xr) <= 1e-9


def test_two_handles_interleaved(setup):
    rs, H, n = setup
    pts2, h2 = ri.circle(4096)
    H2 = rs.rs_build(pts2, "laplace2d", h2, 1e-9, 64, 64)
    S = rs.Server(max_cols=64)
    a, b = S.add(H), S.add(H2)
    jobs = []
    for i in range(10):
        hid, nn, HH = (a, n, H) if i % 2 == 0 else (b, 4096, H2)
        B = ri.rhs(nn, 4, seed=300 + i)
        X = np.zeros_like(B)
        jobs.append((S.submit(hid, B, X), B, X, HH))
    for t, B, X, HH in jobs:
        assert S.wait(t)["status"] == 0
        assert np.all(_residual(rs, HH, X, B) <= 1e-10)
    S.destroy()
    H2.free()
