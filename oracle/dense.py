"""Oracle: dense reference matrices for small N (brute force).

Test infrastructure (see the package header).  A = I + w K in the original
point order, K_ij = G(x_i, x_j), K_ii = 0 (Sec. 2 problem statement
sum_j A_ij x_j = b_i; kernels from oracle.kernels).  Dense solves use
numpy.linalg.solve (LU with partial pivoting, a library primitive): the
brute-force Gaussian elimination the compressed inverse is compared with
(Sec. 4.3 states the hand-rolled elimination is one ordering of it).

coupled_matrix (several patches, Sec. 6.4) is pinned by its special cases:
one patch is dense_matrix, equal weights give a (complex) symmetric matrix,
a common translation of all patches leaves it unchanged.

Pins (tests/test_oracle_pins.py): norm2_est against the 2-norm from the
singular value decomposition (LAPACK through numpy.linalg.norm(E, 2)) on
random real and complex matrices and on A - A_RS, and against closed forms
(a diagonal matrix, rank-one products u v^H).
"""
from __future__ import annotations

import numpy as np

from .kernels import system_block


def dense_matrix(kind: str, points: np.ndarray, w: float, kwave: float = 0.0, geom=None) -> np.ndarray:
    """geom = (normals, curvature) in the same order as points (double layer)."""
    idx = np.arange(points.shape[1])
    return system_block(kind, points, idx, idx, w, kwave, geom)


def coupled_matrix(kind: str, pts_list, w_list, kwave: float = 0.0) -> np.ndarray:
    """The matrix coupling several patches (Sec. 6.4): block (i, j) is
    delta_ij I + w_j K(X_i, X_j) with K_ii = 0 on the diagonal, i.e. every
    column carries its own patch's weight."""
    pts = np.hstack(pts_list)
    n = pts.shape[1]
    w = np.concatenate([np.full(p.shape[1], wj) for p, wj in zip(pts_list, w_list)])
    idx = np.arange(n)
    return system_block(kind, pts, idx, idx, 1.0, kwave) * w[None, :] + np.diag(1.0 - w)


def dense_solve(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    return np.linalg.solve(A, B)


def operator_matrix(apply, n: int, dtype=np.float64) -> np.ndarray:
    """Dense matrix of a linear operator given by its action on columns."""
    return apply(np.eye(n, dtype=dtype))


def norm2_est(E: np.ndarray, iters: int = 60, seed: int = 1) -> float:
    """2-norm of a dense matrix by power iteration on E^H E."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(E.shape[1]).astype(E.dtype)
    v /= np.linalg.norm(v)
    s = 0.0
    for _ in range(iters):
        w = E.conj().T @ (E @ v)
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        s = np.sqrt(nw)
        v = w / nw
    return float(s)
