"""Oracle: interpolative decomposition by column-pivoted QR.

Test infrastructure (see the package header).

Definition 2.3 (Sec. 2.2): a rank-k ID of M (m x n) is M ~ B P with B = k
columns of M (the skeletons) and P (k x n) containing the k x k identity on
those columns.  The rank is chosen on the fly to a relative precision eps
(Sec. 2.2, the paragraph after Def. 2.4).  The paper's own code uses random
sampling; the deterministic column-pivoted QR route is used here.

Steps (Householder QR with column pivoting, Golub & Van Loan Sec. 5.4.1):
  for j = 0, 1, ...:
    norms of the trailing columns over rows j..m-1 (recomputed each step)
    pivot p = the largest norm (lowest index on ties); |R_jj| = that norm
    stop when |R_jj| <= eps * |R_00|   (rank k = j)
    swap columns j and p, reflect column j onto e_1, update the rest
  R11 = R[:k, :k] (upper triangular), R12 = R[:k, k:]
  T = R11^{-1} R12,   skeletons = first k pivots,  redundant = the rest
so that M[:, rd] ~ M[:, sk] T and P[:, sk] = I, P[:, rd] = T.

Pins (tests/test_oracle_interp.py): skeleton columns reproduced exactly; an
exactly rank-r matrix gives k = r with a residual at rounding level; the pivot
order equals LAPACK's dgeqp3 (scipy.linalg.qr with pivoting) on matrices with
well separated column norms; the ID error sits within a modest factor of
sigma_{k+1} (Def. 2.3).  The randomized ID (interp_decomp_randomized): an
exactly rank-r matrix again gives k = r and a rounding-level residual (the
sample of a rank-r matrix has rank r with probability one), the sample is
the product with the stated normal stream, and on kernel matrices its error
stays within a modest factor of eps.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular


def cpqr(M: np.ndarray, eps: float, kmin: int = 0):
    """Column-pivoted Householder QR stopped at relative precision eps, but
    not before kmin steps (kmin > 0: the two-sided ID of a non-symmetric
    kernel asks both sides for the same rank).

    Returns (R, piv, k): R holds the triangular factor in its first k rows,
    piv the column permutation, k the numerical rank.
    """
    R = np.array(M, dtype=np.complex128 if np.iscomplexobj(M) else np.float64, copy=True)
    m, n = R.shape
    piv = np.arange(n)
    k = 0
    r00 = 0.0
    for j in range(min(m, n)):
        norms = np.sqrt(np.sum(np.abs(R[j:, j:]) ** 2, axis=0))
        p = j + int(np.argmax(norms))          # argmax returns the lowest index on ties
        rjj = norms[p - j]
        if j == 0:
            r00 = rjj
            if r00 == 0.0:
                break
        elif rjj <= eps * r00 and (j >= kmin or rjj == 0.0):
            break
        R[:, [j, p]] = R[:, [p, j]]
        piv[[j, p]] = piv[[p, j]]
        x = R[j:, j].copy()
        alpha = x[0]
        phase = alpha / abs(alpha) if alpha != 0 else 1.0
        beta = -phase * rjj
        u = x
        u[0] = alpha - beta
        uu = np.vdot(u, u).real
        if uu > 0.0:
            R[j:, j:] -= (2.0 / uu) * np.outer(u, np.conj(u) @ R[j:, j:])
        R[j + 1:, j] = 0.0
        R[j, j] = beta
        k = j + 1
    return R, piv, k


def interp_decomp(M: np.ndarray, eps: float, kmin: int = 0):
    """ID of M to relative precision eps (rank at least kmin where M allows
    it): returns (sk, rd, T) with local indices."""
    R, piv, k = cpqr(M, eps, kmin)
    sk = piv[:k].copy()
    rd = piv[k:].copy()
    if k == 0:
        return sk, rd, np.zeros((0, M.shape[1]), dtype=R.dtype)
    T = solve_triangular(np.triu(R[:k, :k]), R[:k, k:], lower=False)
    return sk, rd, T


# Randomized ID (the paper's own ID, Sec. 2.2: compression of a random
# sample of the matrix's row space instead of the matrix itself).  The
# sample is Y = Omega M with Omega an l x m matrix of independent N(0,1)
# entries, l = n + p (p oversampling rows); the ID of Y (the same pivoted QR,
# same rank rule) is taken as the ID of M: with probability close to one the
# column relations of Y are those of M up to the precision asked for.  Used
# only when it shrinks the matrix (m > l).  The paper samples with a
# structured random transform; a Gaussian Omega is the plain form of the same
# scheme.  Omega's entries are an input of the method: entry (i, r) is element
# r * SKETCH_STRIDE + i of the counter-based normal stream `SKETCH_STREAM` of
# the seed (rs_inputs), the same entries the GPU build draws.
SKETCH_STRIDE = 1024
SKETCH_STREAM = 77


def sketch_matrix(seed: int, l: int, m: int) -> np.ndarray:
    """Omega (l x m): entry (i, r) = normal stream element r * SKETCH_STRIDE + i."""
    import rs_inputs
    Z = rs_inputs.normal(seed, (m, SKETCH_STRIDE), stream=SKETCH_STREAM)
    return Z[:, :l].T.copy()


def interp_decomp_randomized(M: np.ndarray, eps: float, p: int, seed: int, kmin: int = 0):
    """Randomized ID of M: the ID of the sample Omega M (l = n + p rows)."""
    m, n = M.shape
    l = n + p
    if m <= l:
        return interp_decomp(M, eps, kmin)
    Y = sketch_matrix(seed, l, m) @ M
    return interp_decomp(Y, eps, kmin)


def projection(sk, rd, T, n):
    """P (k x n) with P[:, sk] = I and P[:, rd] = T, so M ~ M[:, sk] P."""
    k = len(sk)
    P = np.zeros((k, n), dtype=T.dtype if T.size else np.float64)
    P[np.arange(k), sk] = 1.0
    if len(rd):
        P[:, rd] = T
    return P
