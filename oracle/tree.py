"""Oracle: uniform quadtree / octree with contiguous index blocks.

Test infrastructure (see the package header).  Follows Sec. 2.1 (index tree
whose nodes are contiguous index ranges, Fig. tree-struct), Example 1
(recursive subdivision of the root box into 2^d equal children with the
points reordered so every box holds a contiguous range) and the opening of
Sec. 6 (uniform subdivision until every block is O(1), empty boxes dropped).

Readings taken where the paper is silent (recorded with the others in the
design notes):
  * root box: centre = midpoint of the bounding box, half-width
    a = 0.5 * (largest extent) * (1 + 2^-20);
  * integer cell of a point per axis: q = min(2^D - 1,
    floor((x - (c - a)) / (2a) * 2^D)), D = 30 in 2D and 20 in 3D; the box
    of a point at depth l is q >> (D - l);
  * depth L = the smallest l at which no box holds more than `leaf` points;
  * points ordered by (Morton key of their depth-L box, original index);
    boxes of each depth numbered in Morton order with empty boxes dropped;
  * colleagues = the other boxes of the same depth whose integer
    coordinates differ by at most one on every axis, ascending box index.

Pins (tests/test_oracle_tree.py): brute-force invariants -- every point in
exactly one box per depth, boxes contain their points geometrically, leaves
hold at most `leaf` points, depth L is minimal, colleague lists equal a
brute-force search over all box pairs.
"""
from __future__ import annotations

import numpy as np


def key_bits(dim: int) -> int:
    return 30 if dim == 2 else 20


def root_box(points: np.ndarray):
    """Centre (dim,) and half-width of the root box."""
    lo = points.min(axis=1)
    hi = points.max(axis=1)
    center = (lo + hi) * 0.5
    ext = float((hi - lo).max())
    a = (ext * 0.5) * (1.0 + 2.0 ** -20) if ext > 0.0 else 1.0
    return center, a


def integer_cells(points: np.ndarray, center: np.ndarray, a: float, nbits: int):
    """Finest integer cell of every point, shape (dim, N), int64."""
    lower = center - a
    width = a * 2.0
    q = np.floor((points - lower[:, None]) / width * (2.0 ** nbits))
    return np.minimum(q, 2 ** nbits - 1).astype(np.int64)


def morton(coords: np.ndarray, bits: int) -> np.ndarray:
    """Interleave `bits` low bits of each axis: axis d goes to bit dim*b + d."""
    dim = coords.shape[0]
    key = np.zeros(coords.shape[1], dtype=np.int64)
    for b in range(bits):
        for d in range(dim):
            key |= ((coords[d] >> b) & 1) << (dim * b + d)
    return key


class Level:
    """Boxes of one depth l (root is l = 0)."""

    def __init__(self, depth, keys, coords, begin, end):
        self.depth = depth
        self.keys = keys          # Morton key of each box at this depth
        self.coords = coords      # (dim, nbox) integer box coordinates
        self.begin = begin        # first point (tree order) of each box
        self.end = end            # one past the last point
        self.parent = None        # index of the parent box at depth l-1
        self.child_begin = None   # children occupy [child_begin, child_end)
        self.child_end = None
        self.colleagues = None    # list of int64 arrays, ascending

    @property
    def nbox(self):
        return len(self.keys)


class Tree:
    def __init__(self, points: np.ndarray, leaf: int):
        points = np.asarray(points, dtype=np.float64)
        self.dim, self.N = points.shape
        self.leaf = leaf
        self.nbits = key_bits(self.dim)
        self.center, self.a = root_box(points)
        self.lower = self.center - self.a
        self.width = self.a * 2.0
        q = integer_cells(points, self.center, self.a, self.nbits)

        # depth L: smallest depth with every box holding <= leaf points
        L = None
        for l in range(self.nbits + 1):
            _, counts = np.unique(morton(q >> (self.nbits - l), l), return_counts=True)
            if counts.max() <= leaf:
                L = l
                break
        if L is None:
            raise ValueError("more than `leaf` coincident points")
        self.L = L

        # order points by (depth-L Morton key, original index): stable sort
        keyL = morton(q >> (self.nbits - L), L)
        self.perm = np.argsort(keyL, kind="stable").astype(np.int64)
        self.points = points[:, self.perm]          # tree order
        keyL_sorted = keyL[self.perm]
        q_sorted = q[:, self.perm]

        self.levels = []
        for l in range(L + 1):
            kl = keyL_sorted >> (self.dim * (L - l))
            start = np.concatenate([[True], kl[1:] != kl[:-1]])
            begin = np.nonzero(start)[0].astype(np.int64)
            end = np.append(begin[1:], self.N).astype(np.int64)
            coords = q_sorted[:, begin] >> (self.nbits - l)
            self.levels.append(Level(l, kl[begin], coords, begin, end))

        for l in range(1, L + 1):
            lv, up = self.levels[l], self.levels[l - 1]
            lv.parent = np.searchsorted(up.keys, lv.keys >> self.dim).astype(np.int64)
        for l in range(L + 1):
            lv = self.levels[l]
            if l < L:
                par = self.levels[l + 1].parent
                lv.child_begin = np.searchsorted(par, np.arange(lv.nbox), side="left")
                lv.child_end = np.searchsorted(par, np.arange(lv.nbox), side="right")
            else:
                lv.child_begin = np.zeros(lv.nbox, dtype=np.int64)
                lv.child_end = np.zeros(lv.nbox, dtype=np.int64)
            lv.colleagues = self._colleagues(lv)

    def _colleagues(self, lv: Level):
        offs = np.array(np.meshgrid(*([[-1, 0, 1]] * self.dim), indexing="ij")).reshape(self.dim, -1)
        offs = offs[:, np.any(offs != 0, axis=0)]
        out = []
        lim = 2 ** lv.depth
        for b in range(lv.nbox):
            nb = lv.coords[:, b:b + 1] + offs
            ok = np.all((nb >= 0) & (nb < lim), axis=0)
            keys = morton(nb[:, ok], lv.depth)
            pos = np.searchsorted(lv.keys, keys)
            found = np.array([p for p, kk in zip(pos, keys)
                              if p < lv.nbox and lv.keys[p] == kk], dtype=np.int64)
            out.append(np.sort(found).astype(np.int64))
        return out

    def box_center(self, depth: int, b: int) -> np.ndarray:
        side = self.width / (2 ** depth)
        return self.lower + (self.levels[depth].coords[:, b] + 0.5) * side

    def box_side(self, depth: int) -> float:
        return self.width / (2 ** depth)
