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


# ------------------------------------------------------------ randomized ID
def test_randomized_id_exact_rank():
    """A rank-r matrix: the sample has rank r with probability one, so the
    randomized ID finds k = r and reproduces M to rounding."""
    from oracle import interp
    rng = np.random.default_rng(3)
    for m, n, r in ((300, 40, 7), (500, 90, 33)):
        M = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
        sk, rd, T = interp.interp_decomp_randomized(M, 1e-12, 8, seed=5)
        assert len(sk) == r
        P = interp.projection(sk, rd, T, n)
        assert np.linalg.norm(M - M[:, sk] @ P) <= 1e-12 * np.linalg.norm(M)


def test_sketch_is_the_stated_normal_stream():
    """Omega's entry (i, r) is element r * SKETCH_STRIDE + i of the normal
    stream (Box-Muller pairs of splitmix64 uniforms), independent of l, m."""
    from oracle import interp
    import rs_inputs as ri
    O = interp.sketch_matrix(9, 12, 30)
    O2 = interp.sketch_matrix(9, 5, 7)
    assert np.array_equal(O[:5, :7], O2)
    z = ri.normal_range(9, 17 * interp.SKETCH_STRIDE + 3, 1, stream=interp.SKETCH_STREAM)[0]
    assert O[3, 17] == z


def test_randomized_id_on_kernel_matrix():
    """On a proxy-compression matrix of a box: the randomized ID compresses
    it to a modest factor of eps (Def. 2.3), with a rank near the
    deterministic one."""
    import rs_inputs as ri
    from oracle import interp, rskel
    pts, h = ri.starfish(2048)
    F = rskel.build(pts, rskel.Params(kind="laplace2d", w=h, eps=1e-10, leaf=64, nproxy=64))
    L = F.tree.L
    lv = F.tree.levels[L]
    active = [F._active(L, b) for b in range(lv.nbox)]
    for b in (0, lv.nbox // 2, lv.nbox - 1):
        M = F._compress_matrix(L, b, active[b][1], active)
        sk, rd, T = interp.interp_decomp_randomized(M, 1e-10, 8, seed=1)
        P = interp.projection(sk, rd, T, M.shape[1])
        assert np.linalg.norm(M - M[:, sk] @ P, 2) <= 100 * 1e-10 * np.linalg.norm(M, 2)
        sk0, _, _ = interp.interp_decomp(M, 1e-10)
        assert abs(len(sk) - len(sk0)) <= 4
