"""Oracle ID pinned against Def. 2.3 and LAPACK's pivoted QR (Sec. 2.2)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.interp import cpqr, interp_decomp, projection


def _lowrank(m, n, r, seed, complex_=False):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((m, r))
    V = rng.standard_normal((r, n))
    if complex_:
        U = U + 1j * rng.standard_normal((m, r))
        V = V + 1j * rng.standard_normal((r, n))
    return U @ V


@pytest.mark.parametrize("complex_", [False, True])
def test_exact_rank(complex_):
    M = _lowrank(80, 50, 13, 1, complex_)
    sk, rd, T = interp_decomp(M, 1e-12)
    assert len(sk) == 13
    P = projection(sk, rd, T, 50)
    assert np.linalg.norm(M - M[:, sk] @ P) < 1e-12 * np.linalg.norm(M)


def test_skeleton_columns_exact():
    M = _lowrank(60, 40, 25, 2) + 1e-6 * np.random.default_rng(0).standard_normal((60, 40))
    sk, rd, T = interp_decomp(M, 1e-3)
    P = projection(sk, rd, T, 40)
    # P restricted to the skeleton columns is the identity, exactly
    assert np.array_equal(P[:, sk], np.eye(len(sk)))
    assert np.array_equal((M[:, sk] @ P)[:, sk], M[:, sk] @ np.eye(len(sk)))


def test_pivots_match_lapack():
    rng = np.random.default_rng(5)
    m, n = 70, 30
    scales = 2.0 ** -np.arange(n)
    M = rng.standard_normal((m, n)) * rng.permutation(scales)[None, :]
    R, piv, k = cpqr(M, 0.0)
    _, Rl, pl = sla.qr(M, pivoting=True)
    assert k == n
    assert np.array_equal(piv, pl)
    assert np.allclose(np.abs(np.diag(R[:n, :n])), np.abs(np.diag(Rl)), rtol=1e-10)


def test_error_near_sigma_k1():
    rng = np.random.default_rng(9)
    m, n = 90, 60
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = 10.0 ** (-np.arange(n) / 4.0)
    M = U @ np.diag(sig) @ V.T
    for eps in (1e-3, 1e-6, 1e-9):
        sk, rd, T = interp_decomp(M, eps)
        k = len(sk)
        err = np.linalg.norm(M - M[:, sk] @ projection(sk, rd, T, n), 2)
        assert err <= 10 * np.sqrt(1 + k * (n - k)) * sig[k]
        # adaptive rank lands where sigma crosses eps (within a small band)
        assert sig[k] <= 100 * eps * sig[0] and sig[max(k - 4, 0)] >= 1e-2 * eps * sig[0]


def test_rank_zero_and_full():
    sk, rd, T = interp_decomp(np.zeros((5, 4)), 1e-9)
    assert len(sk) == 0 and len(rd) == 4
    M = np.eye(6)[:, :4]
    sk, rd, T = interp_decomp(M, 1e-9)
    assert len(sk) == 4 and T.shape == (4, 0)
