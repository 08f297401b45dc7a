"""Oracle tree pinned by brute force (Sec. 2.1, Ex. 1, Sec. 6 opening)."""
import itertools

import numpy as np
import pytest

import rs_inputs as ri
from oracle.tree import Tree


def _clouds():
    rng = np.random.default_rng(3)
    yield "circle", ri.circle(1000)[0], 32
    yield "starfish", ri.starfish(3000)[0], 64
    yield "sphere", ri.fibonacci_sphere(3000)[0], 128
    yield "uniform2d", rng.random((2, 777)), 16
    yield "clustered3d", np.hstack([rng.random((3, 300)) * 1e-3, rng.random((3, 300))]), 40


@pytest.mark.parametrize("name,pts,leaf", list(_clouds()), ids=lambda v: v if isinstance(v, str) else "")
def test_tree_invariants(name, pts, leaf):
    T = Tree(pts, leaf)
    dim, N = pts.shape
    assert sorted(T.perm.tolist()) == list(range(N))
    assert np.array_equal(T.points, pts[:, T.perm])
    for l, lv in enumerate(T.levels):
        # boxes partition [0, N) into contiguous ranges in order
        assert lv.begin[0] == 0 and lv.end[-1] == N
        assert np.array_equal(lv.begin[1:], lv.end[:-1]) and np.all(lv.end > lv.begin)
        side = T.width / 2 ** l
        for b in range(lv.nbox):
            lo = T.lower + lv.coords[:, b] * side
            x = T.points[:, lv.begin[b]:lv.end[b]]
            assert np.all(x >= lo[:, None] - 1e-12) and np.all(x <= lo[:, None] + side + 1e-12)
        if l > 0:
            # parent contains child
            assert np.array_equal(T.levels[l - 1].coords[:, lv.parent], lv.coords >> 1)
        # colleagues equal a brute-force search over all pairs
        for b in range(lv.nbox):
            brute = [c for c in range(lv.nbox) if c != b and
                     np.all(np.abs(lv.coords[:, c] - lv.coords[:, b]) <= 1)]
            assert list(lv.colleagues[b]) == brute
    assert max(lv.end[-1] for lv in T.levels) == N
    leaves = T.levels[-1]
    assert np.max(leaves.end - leaves.begin) <= leaf
    if T.L > 0:
        up = T.levels[-2]
        assert np.max(up.end - up.begin) > leaf            # depth L is minimal
    # within a leaf, points keep their original relative order
    for b in range(leaves.nbox):
        seg = T.perm[leaves.begin[b]:leaves.end[b]]
        assert np.all(np.diff(seg) > 0)


def test_morton_child_order():
    # four points, one per quadrant: Morton order is (x bit, y bit) = 00, 10, 01, 11
    pts = np.array([[0.9, 0.1, 0.9, 0.1], [0.9, 0.9, 0.1, 0.1]])
    T = Tree(pts, 1)
    assert T.L == 1
    assert T.perm.tolist() == [3, 2, 1, 0]


def test_single_box():
    pts = ri.circle(10)[0]
    T = Tree(pts, 64)
    assert T.L == 0 and T.levels[0].nbox == 1 and T.perm.tolist() == list(range(10))
