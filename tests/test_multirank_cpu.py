"""The multi-GPU form is replicas (every rank builds and solves its own
problem, no collective on the data path); the only cross-rank step is the
timing reduction.  Checked here with two gloo ranks on the CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
        q.put((rank, ms, bench.replica_throughput(ws, 256, 5, ms)))
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 20.0                      # the slower rank's time on every rank
        assert value == pytest.approx(2 * 256 * 5 / 0.020)


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.replica_throughput(1, 256, 5, 500.0) == pytest.approx(2560.0)


def test_column_ranges_cover_each_column_once():
    sys.path.insert(0, ROOT)
    from paper_1110_3105_gb300.replicas import column_range
    for total in (0, 1, 7, 256, 1000):
        for world in (1, 2, 3, 8):
            seen = []
            prev = 0
            for r in range(world):
                c0, c1 = column_range(total, world, r)
                assert c0 == prev and c1 >= c0
                assert c1 - c0 in (total // world, total // world + 1)
                seen.extend(range(c0, c1))
                prev = c1
            assert seen == list(range(total))


def _mock_solve(B, c0):
    """Stand-in for a replica's solve: any column-wise map (here it depends
    on the column's global index, so a misplaced slice would show)."""
    import numpy as np
    return B * 2.0 + (c0 + np.arange(B.shape[1]))[None, :]


def _split_worker(rank, ws, port, q, n, total):
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import rs_inputs as ri
    from paper_1110_3105_gb300.replicas import column_range, gather_columns
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        c0, c1 = column_range(total, ws, rank)
        B = ri.rhs_columns(n, c0, c1, seed=100)          # this rank's slice of one global batch
        X = gather_columns(_mock_solve(B, c0), total, dist, ws, rank)
        q.put((rank, None if X is None else X.copy()))
    finally:
        dist.destroy_process_group()


def test_two_rank_column_split_and_gather():
    """Two gloo ranks solve their column slices of one batch and X is
    reassembled on rank 0: identical to a one-rank run of the same map."""
    import multiprocessing as mp
    import socket
    import numpy as np
    sys.path.insert(0, ROOT)
    import rs_inputs as ri
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    n, total = 97, 11
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_split_worker, args=(r, 2, port, q, n, total)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[1] is None
    ref = _mock_solve(ri.rhs(n, total, seed=100), 0)
    assert np.array_equal(out[0], ref)
