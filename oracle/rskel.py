"""Oracle: recursive skeletonization -- compression, inverse, solve, apply.

Test infrastructure (see the package header).  Symmetric kernels (the four
Green's functions give A = A^T) need a single ID per box whose projection P
serves as both R_i = P and L_i = P^T (Sec. 3.1 with identical row and column
skeletons; complex symmetric Helmholtz uses the transpose, not the conjugate
transpose).  The double-layer kernel is not symmetric: each box gets a
column ID of its off-diagonal block column (R_i = P_i, column skeletons) and
a row ID of its off-diagonal block row (L_i = Q_i^T, row skeletons), as the
one-level scheme of Sec. 3.1 states it; the two are taken at the same rank
k_i = max(row rank, column rank) (the pivoted QR of the side with the lower
rank runs on to k_i steps), the equal-dimension case in which Sec. 3.4
writes the block elimination.  A box then carries a row active set
(targets) and a column active set (sources) of equal size: its points at the
leaves, above them the children's row and column skeletons.

Build, level by level from the leaves (Sec. 3.1, the two-step multilevel
procedure; depth L of the tree is compression level 1, depth 1 is level
lambda, depth 0 the root):
  active set of a box: its points at the leaves, otherwise the skeletons of
  its children in child order (regrouping, Fig. multi-comp);
  proxy compression (Sec. 3.2): rows = all active points of the colleague
  boxes (the near neighbours) plus the proxy surface, each scaled by w;
  2D Laplace adds one constant row when |log rho| < 0.1 (the single layer on
  a circle of radius 1 cannot make constants);
  double layer, column ID: the colleagues' row active points and the proxy
  points as targets of the box's sources (the field the box sends out);
  row ID: the transpose of the box's targets against the colleagues' column
  active points and against single-layer charges on the proxy circle plus a
  constant (the fields the box receives from far away: harmonic inside the
  circle, so single-layer charges on it and a constant represent them);
  ID of that matrix (interp.interp_decomp) -> skeletons, P;
  diagonal block D_i: at the leaves A(I_i, I_i); above, the children's
  Lambda on the diagonal and w G between skeletons of different children
  (S^(l-1) regrouped, with Lambda^(l-1) added: the system S z = y of eq.
  sparse-embedding expanded again, eq. multilevel-embedding);
  block elimination (eq. compressed-inverse):
    Lambda = (R D^-1 L)^-1,  calD = D^-1 - D^-1 L Lambda R D^-1,
    calL = D^-1 L Lambda,    calR = Lambda R D^-1;
root: calS = the root's diagonal block built the same way; solved by dense
LU with partial pivoting (numpy.linalg.solve, a library primitive).

Solve (eq. multilevel-inverse applied right to left, Sec. 4.3):
  upward   u_i = calD_i b_i, c_i = calR_i b_i -> parent's active slots
  root     x = calS^-1 c
  downward x_i = u_i + calL_i x_parent[slots of i]
Forward apply of the compressed matrix (eq. multilevel-compression, Sec. 3.3):
  upward   z -> P z (column projections), D^(l) z kept per box, where D^(l)
           is A(I_i, I_i) at the leaves and the sibling blocks (zero blocks
           on the children) above
  top      S z on the root's active set (sibling blocks of the depth-1 boxes)
  downward y_i = D^(l)_i z_i + Q_i^T y_parent[slots of i]   (Q_i = P_i if symmetric)

Pins (tests/test_oracle_solver.py): ||A - A_RS|| / ||A|| <= 10 eps against the
dense matrix; the solve equals dense Gaussian elimination on A_RS to rounding
and on A within 10 eps; closed-form circulant spectrum on the unit circle
(Laplace and Helmholtz); sphere harmonics eigenvalues (3D, loose).
(tests/test_oracle_pins.py): every box's proxy ID compresses the TRUE
off-diagonal block row A(other boxes' active points, I) to eps, and its rank
is at least that of the ID of that block itself (Sec. 3.2).

build() takes an optional box_map to run the independent boxes of a level
elsewhere; process_box_map spreads them over forked processes (the CPU
baseline of the benchmark); the arithmetic is unchanged.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .interp import interp_decomp, interp_decomp_randomized, projection
from .kernels import (green, green_dl, is_complex, is_symmetric, offdiag_block, proxy_points, proxy_radius_2d,
                      system_block)
from .tree import Tree


@dataclasses.dataclass
class Params:
    kind: str = "laplace2d"
    w: float = 1.0            # quadrature weight in A = I + w K
    eps: float = 1e-9
    leaf: int = 64
    nproxy: int = 64
    ratio: float = 1.5
    kwave: float = 0.0
    id_oversample: int = 0    # > 0: randomized ID with n + id_oversample sample rows (Sec. 2.2)
    id_seed: int = 0
    normals: np.ndarray | None = None     # (2, N) outward unit normals (double layer), input order
    curvature: np.ndarray | None = None   # (N,) curvature (double layer), input order


@dataclasses.dataclass
class BoxFactor:
    I: np.ndarray            # column active point ids (tree order positions)
    sk_loc: np.ndarray       # column skeleton positions within I (pivot order)
    rd_loc: np.ndarray       # redundant positions within I
    T: np.ndarray            # k x (n - k) interpolation matrix
    P: np.ndarray            # k x n column projection (R_i = P)
    D: np.ndarray            # n x n diagonal block of the inverse recursion
    Lam: np.ndarray          # k x k
    calD: np.ndarray         # n x n
    calL: np.ndarray         # n x k
    calR: np.ndarray         # k x n
    m: int = 0               # rows of the compressed matrix
    # row side (L_i = Q^T); the same objects as the column side for symmetric kernels
    Ir: np.ndarray = None    # row active point ids
    skr_loc: np.ndarray = None
    rdr_loc: np.ndarray = None
    Tr: np.ndarray = None
    Q: np.ndarray = None     # k x n row projection

    @property
    def sk(self):
        return self.I[self.sk_loc]

    @property
    def skr(self):
        return self.Ir[self.skr_loc]

    @property
    def n(self):
        return len(self.I)

    @property
    def k(self):
        return len(self.sk_loc)


class Factorization:
    def __init__(self, tree: Tree, params: Params):
        self.tree = tree
        self.params = params
        self.geom = None      # (normals, curvature) in tree order (double layer)
        if params.normals is not None:
            self.geom = (np.asarray(params.normals)[:, tree.perm], np.asarray(params.curvature)[tree.perm])
        self.boxes = {}       # depth -> list[BoxFactor] for depths L..1
        self.root_I = None    # active set of the root
        self.calS = None      # root diagonal block (dense)
        self.fwd_blocks = {}  # depth -> list of forward D^(l) blocks (0..L), root at 0

    # ------------------------------------------------------------------ helpers
    def _dtype(self):
        return np.complex128 if is_complex(self.params.kind) else np.float64

    def _blocks_from_children(self, depth, b, with_lambda: bool):
        """Diagonal block of box b (depth < L) from its children at depth+1."""
        tr, pr = self.tree, self.params
        lv = tr.levels[depth]
        kids = range(lv.child_begin[b], lv.child_end[b])
        cf = [self.boxes[depth + 1][c] for c in kids]
        sizes = [f.k for f in cf]
        offs = np.concatenate([[0], np.cumsum(sizes)])
        n = int(offs[-1])
        D = np.zeros((n, n), dtype=self._dtype())
        for a, fa in enumerate(cf):
            for c, fc in enumerate(cf):
                ra = slice(offs[a], offs[a + 1])
                rc = slice(offs[c], offs[c + 1])
                if a == c:
                    if with_lambda:
                        D[ra, rc] = fa.Lam
                else:   # rows: row skeletons of child a; columns: column skeletons of child c
                    D[ra, rc] = offdiag_block(pr.kind, tr.points, fa.skr, fc.sk, pr.w, pr.kwave, self.geom)
        return D

    def _active(self, depth, b):
        """(row active set, column active set) of box b."""
        tr = self.tree
        lv = tr.levels[depth]
        if depth == tr.L:
            I = np.arange(lv.begin[b], lv.end[b])
            return I, I
        kids = range(lv.child_begin[b], lv.child_end[b])
        fs = [self.boxes[depth + 1][c] for c in kids]
        I = np.concatenate([f.sk for f in fs])
        return (I if is_symmetric(self.params.kind) else np.concatenate([f.skr for f in fs])), I

    def _proxy(self, depth, b):
        tr, pr = self.tree, self.params
        side = tr.box_side(depth)
        return proxy_points(tr.dim, tr.box_center(depth, b), side, pr.nproxy, pr.ratio), side

    def _compress_matrix(self, depth, b, I, active_of):
        """Column compression of box b: rows = near-neighbour (row) active
        points and proxy points as targets of the box's sources I (Sec. 3.2)."""
        tr, pr = self.tree, self.params
        lv = tr.levels[depth]
        near = [active_of[c][0] for c in lv.colleagues[b]]
        near = np.concatenate(near) if near else np.zeros(0, dtype=np.int64)
        prox, side = self._proxy(depth, b)
        rows = [offdiag_block(pr.kind, tr.points, near, I, pr.w, pr.kwave, self.geom)]
        if pr.kind == "laplace2d_dl":
            rows.append(pr.w * green_dl(prox, tr.points[:, I], self.geom[0][:, I]))
        else:
            rows.append(pr.w * green(pr.kind, prox, tr.points[:, I], pr.kwave))
        if pr.kind == "laplace2d" and abs(np.log(proxy_radius_2d(side, pr.ratio))) < 0.1:
            rows.append(pr.w * np.ones((1, len(I))))
        return np.vstack(rows)

    def _compress_matrix_rows(self, depth, b, Ir, active_of):
        """Row compression of box b (non-symmetric kernels), transposed:
        rows = the colleagues' column active points and single-layer charges
        on the proxy circle plus a constant, as sources acting on the box's
        targets Ir (Sec. 3.2)."""
        tr, pr = self.tree, self.params
        lv = tr.levels[depth]
        near = [active_of[c][1] for c in lv.colleagues[b]]
        near = np.concatenate(near) if near else np.zeros(0, dtype=np.int64)
        prox, _ = self._proxy(depth, b)
        rows = [offdiag_block(pr.kind, tr.points, Ir, near, pr.w, pr.kwave, self.geom).T,
                pr.w * green("laplace2d", tr.points[:, Ir], prox).T,
                pr.w * np.ones((1, len(Ir)))]
        return np.vstack(rows)

    def _id(self, M, kmin=0):
        pr = self.params
        if pr.id_oversample > 0:
            return interp_decomp_randomized(M, pr.eps, pr.id_oversample, pr.id_seed, kmin)
        return interp_decomp(M, pr.eps, kmin)

    # -------------------------------------------------------------------- build
    def _factor_box(self, depth, b, active_of):
        """Compression and block elimination of box b at `depth` (its children,
        if any, are done)."""
        tr, pr = self.tree, self.params
        Ir, I = active_of[b]
        M = self._compress_matrix(depth, b, I, active_of)
        sk_loc, rd_loc, T = self._id(M)
        if is_symmetric(pr.kind):
            skr_loc, rdr_loc, Tr = sk_loc, rd_loc, T
        else:   # row ID at the column rank, then the column ID again if the row rank is higher
            Mr = self._compress_matrix_rows(depth, b, Ir, active_of)
            skr_loc, rdr_loc, Tr = self._id(Mr, kmin=len(sk_loc))
            if len(skr_loc) > len(sk_loc):
                sk_loc, rd_loc, T = self._id(M, kmin=len(skr_loc))
            if len(skr_loc) != len(sk_loc):
                raise ValueError("row and column ranks differ: a block of rank below the other side's")
        P = projection(sk_loc, rd_loc, T, len(I)).astype(self._dtype())
        Q = P if is_symmetric(pr.kind) else projection(skr_loc, rdr_loc, Tr, len(Ir)).astype(self._dtype())
        if depth == tr.L:
            D = system_block(pr.kind, tr.points, Ir, I, pr.w, pr.kwave, self.geom)
            Dfwd = D
        else:
            D = self._blocks_from_children(depth, b, with_lambda=True)
            Dfwd = self._blocks_from_children(depth, b, with_lambda=False)
        # block elimination, eq. compressed-inverse (L = Q^T, R = P)
        DinvL = np.linalg.solve(D, Q.T)              # D^-1 L
        RDinv = np.linalg.solve(D.T, P.T).T          # R D^-1
        Lam = np.linalg.inv(P @ DinvL)               # (R D^-1 L)^-1
        Dinv = np.linalg.inv(D)
        calD = Dinv - DinvL @ Lam @ RDinv
        calL = DinvL @ Lam
        calR = Lam @ RDinv
        return BoxFactor(I, sk_loc, rd_loc, T, P, D, Lam, calD, calL, calR, m=M.shape[0],
                         Ir=Ir, skr_loc=skr_loc, rdr_loc=rdr_loc, Tr=Tr, Q=Q), Dfwd

    def build(self, box_map=None):
        """Level by level from the leaves.  box_map(f, items) -> list may run the
        independent boxes of one level elsewhere (e.g. a process pool); the
        default runs them in order.  The arithmetic is the same either way."""
        tr = self.tree
        for depth in range(tr.L, 0, -1):
            lv = tr.levels[depth]
            active_of = [self._active(depth, b) for b in range(lv.nbox)]
            if box_map is None:
                res = [self._factor_box(depth, b, active_of) for b in range(lv.nbox)]
            else:
                res = box_map(self, depth, active_of, range(lv.nbox))
            self.boxes[depth] = [r[0] for r in res]
            self.fwd_blocks[depth] = [r[1] for r in res]
        # root (depth 0)
        pr = self.params
        self.root_Ir, self.root_I = self._active(0, 0)
        if tr.L == 0:
            self.calS = system_block(pr.kind, tr.points, self.root_Ir, self.root_I, pr.w, pr.kwave, self.geom)
            self.fwd_blocks[0] = [self.calS]
        else:
            self.calS = self._blocks_from_children(0, 0, with_lambda=True)
            self.fwd_blocks[0] = [self._blocks_from_children(0, 0, with_lambda=False)]
        return self

    # ------------------------------------------------------------ structure info
    def ranks(self):
        """Per depth (L..1): list of (n_i, k_i)."""
        return {d: [(f.n, f.k) for f in fs] for d, fs in self.boxes.items()}

    def skeleton_count(self):
        return len(self.root_I)

    def storage_scalars(self):
        tot = len(self.root_I) ** 2
        for fs in self.boxes.values():
            for f in fs:
                tot += f.n * f.n + 2 * f.n * f.k
        return tot

    def _child_slots(self, depth, b):
        """Slots of box b (depth) within its parent's active vector."""
        tr = self.tree
        p = tr.levels[depth].parent[b]
        up = tr.levels[depth - 1]
        off = 0
        for c in range(up.child_begin[p], b):
            off += self.boxes[depth][c].k
        return p, slice(off, off + self.boxes[depth][b].k)

    # -------------------------------------------------------------------- solve
    def solve(self, B: np.ndarray) -> np.ndarray:
        """x = A_RS^{-1} b for each column of B (original point order)."""
        tr = self.tree
        B2 = np.asarray(B).reshape(tr.N, -1)
        dt = np.result_type(B2.dtype, self._dtype())
        bt = B2[tr.perm].astype(dt)
        if tr.L == 0:
            xt = np.linalg.solve(self.calS, bt)
        else:
            lvL = tr.levels[tr.L]
            vec = [bt[lvL.begin[b]:lvL.end[b]] for b in range(lvL.nbox)]
            u = {}
            for depth in range(tr.L, 0, -1):
                fs = self.boxes[depth]
                u[depth] = [f.calD @ v for f, v in zip(fs, vec)]
                c = [f.calR @ v for f, v in zip(fs, vec)]
                up = tr.levels[depth - 1]
                vec = [np.concatenate([c[i] for i in range(up.child_begin[p], up.child_end[p])])
                       for p in range(up.nbox)]
            xs = [np.linalg.solve(self.calS, vec[0])]
            for depth in range(1, tr.L + 1):
                fs = self.boxes[depth]
                nxt = []
                for b, f in enumerate(fs):
                    p, sl = self._child_slots(depth, b)
                    nxt.append(u[depth][b] + f.calL @ xs[p][sl])
                xs = nxt
            xt = np.concatenate(xs)
        X = np.empty_like(xt)
        X[tr.perm] = xt
        return X.reshape(np.shape(B)) if np.ndim(B) == 1 else X

    # ------------------------------------------------------------ forward apply
    def apply(self, X: np.ndarray) -> np.ndarray:
        """y = A_RS x (telescoping forward operator, Sec. 3.3)."""
        tr = self.tree
        X2 = np.asarray(X).reshape(tr.N, -1)
        dt = np.result_type(X2.dtype, self._dtype())
        xt = X2[tr.perm].astype(dt)
        if tr.L == 0:
            yt = self.fwd_blocks[0][0] @ xt
        else:
            lvL = tr.levels[tr.L]
            z = [xt[lvL.begin[b]:lvL.end[b]] for b in range(lvL.nbox)]
            yD = {}
            for depth in range(tr.L, 0, -1):
                fs = self.boxes[depth]
                yD[depth] = [Df @ v for Df, v in zip(self.fwd_blocks[depth], z)]
                c = [f.P @ v for f, v in zip(fs, z)]
                up = tr.levels[depth - 1]
                z = [np.concatenate([c[i] for i in range(up.child_begin[p], up.child_end[p])])
                     for p in range(up.nbox)]
            ys = [self.fwd_blocks[0][0] @ z[0]]
            for depth in range(1, tr.L + 1):
                fs = self.boxes[depth]
                nxt = []
                for b, f in enumerate(fs):
                    p, sl = self._child_slots(depth, b)
                    nxt.append(yD[depth][b] + f.Q.T @ ys[p][sl])
                ys = nxt
            yt = np.concatenate(ys)
        Y = np.empty_like(yt)
        Y[tr.perm] = yt
        return Y.reshape(np.shape(X)) if np.ndim(X) == 1 else Y


def build(points: np.ndarray, params: Params, box_map=None) -> Factorization:
    """Tree + compression + factorization of A = I + w K on `points` (dim x N)."""
    tree = Tree(points, params.leaf)
    return Factorization(tree, params).build(box_map)


# ------------------------------------------------------- parallel box driver
# The boxes of one level are independent once the level below is done (Sec.
# 3.1: each box's ID and elimination read only its own and its colleagues'
# active sets and its children's Lambda).  `process_box_map` runs them on a
# pool of forked worker processes, one pool per level so that the workers see
# the finished lower levels.  Only for processes that never initialise CUDA
# (a fork after CUDA initialisation is unsafe).
_POOL_STATE = None


def _pool_worker(b):
    fac, depth, active_of = _POOL_STATE
    return fac._factor_box(depth, b, active_of)


def process_box_map(workers: int):
    import multiprocessing as mp

    def box_map(fac, depth, active_of, boxes):
        global _POOL_STATE
        boxes = list(boxes)
        if workers <= 1 or len(boxes) < 2:
            return [fac._factor_box(depth, b, active_of) for b in boxes]
        _POOL_STATE = (fac, depth, active_of)
        try:
            with mp.get_context("fork").Pool(min(workers, len(boxes))) as pool:
                return pool.map(_pool_worker, boxes, chunksize=max(1, len(boxes) // (4 * workers)))
        finally:
            _POOL_STATE = None
    return box_map
