"""Two more pins of the oracle against mathematics it does not compute itself.

1. dense.norm2_est (power iteration on E^H E) against the 2-norm from the
   singular value decomposition (numpy.linalg.norm(E, 2), LAPACK gesdd) and
   against closed forms: a diagonal matrix (its largest |entry|) and a rank-one
   matrix u v^H (|u| |v|).  The compression pin ||A - A_RS|| / ||A|| <= 10 eps
   divides two of its results, so a scale error in it would partly cancel
   there; here it cannot.
2. The proxy compression (Sec. 3.2): the ID computed from near rows plus the
   proxy surface must also compress the TRUE off-diagonal block row, i.e. the
   interactions of the box's active set I with the active points of every
   other box of its level:  ||A(out, I) - A(out, sk) P||_2 <= eps ||A(out, I)||_2
   (Def. 2.3 to relative precision eps), and its rank must not be below the
   rank of the ID of A(out, I) itself at the same eps (the proxy surface
   stands in for all far sources, so it can only ask for more skeletons).
"""
import numpy as np
import pytest

import rs_inputs as ri
from oracle import dense, interp, rskel
from oracle.kernels import offdiag_block


def test_norm2_est_closed_forms_and_svd():
    rng = np.random.default_rng(5)
    D = np.diag([0.5, -3.0, 2.0, 1e-3])
    assert abs(dense.norm2_est(D) - 3.0) < 1e-12
    u, v = rng.standard_normal(30), rng.standard_normal(17)
    assert abs(dense.norm2_est(np.outer(u, v)) - np.linalg.norm(u) * np.linalg.norm(v)) < 1e-10
    uc = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    vc = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    assert abs(dense.norm2_est(np.outer(uc, vc.conj())) - np.linalg.norm(uc) * np.linalg.norm(vc)) < 1e-10
    for shape, cplx in (((40, 40), False), ((60, 25), False), ((33, 47), True)):
        E = rng.standard_normal(shape) + (1j * rng.standard_normal(shape) if cplx else 0)
        s = np.linalg.norm(E, 2)
        # 60 steps of power iteration on a random Gaussian matrix: relative
        # accuracy set by (sigma_2 / sigma_1)^120, well below 1e-3 here
        assert abs(dense.norm2_est(E) - s) <= 1e-3 * s


def test_norm2_est_on_compression_error():
    n, eps = 1024, 1e-9
    pts, h = ri.circle(n)
    F = rskel.build(pts, rskel.Params(kind="laplace2d", w=h, eps=eps, leaf=64, nproxy=64))
    A = dense.dense_matrix("laplace2d", pts, h)
    E = A - F.apply(np.eye(n))
    for M in (A, E):
        s = np.linalg.norm(M, 2)
        assert abs(dense.norm2_est(M) - s) <= 1e-2 * s


PROXY_CASES = [
    ("laplace2d", "starfish", 2048, 1e-10, 64, 64),
    ("laplace2d", "circle", 2048, 1e-9, 64, 64),
    ("helmholtz2d", "starfish", 1024, 1e-9, 64, 64),
    ("laplace3d", "sphere", 1500, 1e-6, 128, 216),
]


@pytest.mark.parametrize("kind,geom,n,eps,leaf,nproxy", PROXY_CASES, ids=lambda v: str(v))
def test_proxy_id_compresses_true_far_field(kind, geom, n, eps, leaf, nproxy):
    pts, w = ri.geometry(geom, n)
    kw = 10.0 if kind.startswith("helmholtz") else 0.0
    F = rskel.build(pts, rskel.Params(kind=kind, w=w, eps=eps, leaf=leaf, nproxy=nproxy, kwave=kw))
    T = F.tree
    checked = 0
    for depth in range(T.L, 0, -1):
        fs = F.boxes[depth]
        for b, f in enumerate(fs):
            out = np.concatenate([fs[c].I for c in range(len(fs)) if c != b])
            if out.size == 0:
                continue
            Aout = offdiag_block(kind, T.points, out, f.I, w, kw)
            err = np.linalg.norm(Aout - Aout[:, f.sk_loc] @ f.P, 2)
            assert err <= eps * np.linalg.norm(Aout, 2), (depth, b, err)
            sk_true, _, _ = interp.interp_decomp(Aout, eps)
            assert f.k >= len(sk_true), (depth, b, f.k, len(sk_true))
            checked += 1
    assert checked >= 8


def _scatterer(n, center, scale=1.0 / 3.0, rotation=0.0):
    """r = (2 + cos 3 theta) / 6 (the paper's scatterer, Sec. 6.4) = the
    starfish with 3 arms, amplitude 1/2, scaled by 1/3; equal arc length."""
    pts, h = ri.starfish(n, arms=3, amp=0.5, rotation=rotation)
    return pts * scale + np.asarray(center, dtype=float)[:, None], h * scale


def test_coupled_matrix_special_cases():
    p1, w1 = _scatterer(96, (0.0, 0.0))
    p2, w2 = _scatterer(80, (1.3, 0.2), rotation=0.4)
    # one patch: the ordinary system matrix
    assert np.array_equal(dense.coupled_matrix("laplace2d", [p1], [w1]), dense.dense_matrix("laplace2d", p1, w1))
    for kind, kw in (("laplace2d", 0.0), ("helmholtz2d", 7.0)):
        # equal weights: (complex) symmetric, since G(x, y) = G(y, x)
        A = dense.coupled_matrix(kind, [p1, p2], [w1, w1], kw)
        assert np.allclose(A, A.T, rtol=0, atol=1e-15 * np.abs(A).max())
        # a common translation changes no distance
        At = dense.coupled_matrix(kind, [p1 + 5.0, p2 + 5.0], [w1, w2], kw)
        A2 = dense.coupled_matrix(kind, [p1, p2], [w1, w2], kw)
        assert np.allclose(At, A2, rtol=1e-12, atol=1e-13)
        # each column carries its own patch's weight
        n1 = p1.shape[1]
        A1 = dense.coupled_matrix(kind, [p1, p2], [1.0, 1.0], kw)
        assert np.allclose(A2[:n1, n1:], w2 * A1[:n1, n1:])
        assert np.allclose(A2[n1:, :n1], w1 * A1[n1:, :n1])
