"""Pins of the double-layer kernel and of the two-sided compression of the
oracle (Sec. 3.1 with row and column skeletons; Sec. 6.2's interior
Dirichlet problem on the ellipse of aspect ratio 2).

Closed forms and identities that the oracle does not compute itself:
  * on the unit circle the double-layer kernel is the constant -1/(4 pi)
    (x - y is a chord and (x - y) . nu_y = -|x - y|^2 / 2 there), and its
    diagonal limit -kappa/(4 pi) is the same constant;
  * Gauss's integral: the double layer of the unit density is -1 inside the
    curve, 0 outside and -1/2 on it, so h sum_j K_ij = -1/2 (trapezoid rule,
    spectrally accurate on a smooth closed curve) and A 1 = 2 with w = -2 h;
  * the interior Dirichlet problem with the field of an exterior point source
    as boundary data: the double-layer potential of the solved density
    reproduces that field inside the curve (the paper's error measure E);
  * ||A - A_RS||_2 <= 10 eps ||A||_2 with the norm from LAPACK's SVD;
  * the row ID of every box compresses its TRUE off-diagonal block row and the
    column ID its block column to eps (Def. 2.3), with equal ranks.
"""
import numpy as np
import pytest

import rs_inputs as ri
from oracle import dense, rskel
from oracle.kernels import green, green_dl, offdiag_block


def _dl_params(n, eps=1e-9, leaf=64, **kw):
    p, h, nr, cv = ri.ellipse(n, **kw)
    return p, h, (nr, cv), rskel.Params(kind="laplace2d_dl", w=-2.0 * h, eps=eps, leaf=leaf, nproxy=64,
                                        normals=nr, curvature=cv)


def test_circle_kernel_is_constant():
    n = 64
    th = 2 * np.pi * np.arange(n) / n
    p = np.vstack([np.cos(th), np.sin(th)])
    K = green_dl(p, p, p)                      # the outward normal of the unit circle is the point
    off = ~np.eye(n, dtype=bool)
    assert np.allclose(K[off], -1.0 / (4.0 * np.pi), rtol=0, atol=1e-14)
    A = dense.dense_matrix("laplace2d_dl", p, 0.3, geom=(p, np.ones(n)))
    assert np.allclose(A, np.eye(n) - 0.3 / (4.0 * np.pi) * np.ones((n, n)), rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [256, 1024])
def test_gauss_integral(n):
    p, h, nr, cv = ri.ellipse(n)
    A = dense.dense_matrix("laplace2d_dl", p, -2.0 * h, geom=(nr, cv))
    assert np.abs(A @ np.ones(n) - 2.0).max() < 1e-12
    inside = np.array([[0.3, -1.5, 1.6], [0.1, 0.2, 0.0]])
    outside = np.array([[2.5, 0.0, -3.0], [0.0, 1.3, 2.0]])
    assert np.allclose(h * green_dl(inside, p, nr).sum(1), -1.0, rtol=0, atol=1e-10)
    assert np.allclose(h * green_dl(outside, p, nr).sum(1), 0.0, rtol=0, atol=1e-10)


@pytest.mark.parametrize("n", [1024, 2048])
def test_interior_dirichlet_exact_solution(n):
    """Sec. 6.2: boundary data from a point source outside the ellipse; the
    double-layer potential of the RS solution matches the source's field
    inside (the paper reports E ~ 1e-10 at eps 1e-9)."""
    p, h, geom, prm = _dl_params(n)
    F = rskel.build(p, prm)
    src = np.array([3.0, 2.0])
    f = -np.log(np.hypot(*(p - src[:, None]))) / (2 * np.pi)
    sig = F.solve(-2.0 * f)
    for x in (np.array([0.5, 0.2]), np.array([-1.2, -0.3]), np.array([1.6, 0.1])):
        u = h * (green_dl(x[:, None], p, geom[0]) @ sig)[0]
        ex = -np.log(np.hypot(*(x - src))) / (2 * np.pi)
        assert abs(u - ex) <= 1e-10 * abs(ex), (x, u, ex)


def test_compression_and_dense_elimination():
    n, eps = 2048, 1e-9
    p, h, geom, prm = _dl_params(n, eps)
    F = rskel.build(p, prm)
    A = dense.dense_matrix("laplace2d_dl", p, prm.w, geom=geom)
    Ars = F.apply(np.eye(n))
    assert np.linalg.norm(A - Ars, 2) <= 10 * eps * np.linalg.norm(A, 2)
    assert not np.allclose(A, A.T)                 # the kernel is not symmetric
    b = ri.rhs(n, 3, seed=7)
    x = F.solve(b)
    assert np.linalg.norm(x - np.linalg.solve(Ars, b)) <= 1e-11 * np.linalg.norm(x)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 10 * eps * np.linalg.norm(x)


def test_two_sided_ids_compress_true_far_field():
    n, eps = 2048, 1e-9
    p, h, geom, prm = _dl_params(n, eps)
    F = rskel.build(p, prm)
    T = F.tree
    differ = 0
    for depth in range(T.L, 0, -1):
        fs = F.boxes[depth]
        for b, f in enumerate(fs):
            assert f.Q.shape == f.P.shape                  # equal row and column ranks
            out_r = np.concatenate([fs[c].Ir for c in range(len(fs)) if c != b])
            out_c = np.concatenate([fs[c].I for c in range(len(fs)) if c != b])
            col = offdiag_block("laplace2d_dl", T.points, out_r, f.I, prm.w, 0.0, F.geom)
            row = offdiag_block("laplace2d_dl", T.points, f.Ir, out_c, prm.w, 0.0, F.geom)
            assert np.linalg.norm(col - col[:, f.sk_loc] @ f.P, 2) <= eps * np.linalg.norm(col, 2)
            assert np.linalg.norm(row - f.Q.T @ row[f.skr_loc], 2) <= eps * np.linalg.norm(row, 2)
            differ += not np.array_equal(np.sort(f.sk), np.sort(f.skr))
    assert differ > 0                                      # row and column skeletons are distinct sets


def test_symmetric_kernel_keeps_one_id():
    p, h = ri.circle(1024)
    F = rskel.build(p, rskel.Params(kind="laplace2d", w=h, eps=1e-9, leaf=64, nproxy=64))
    for fs in F.boxes.values():
        for f in fs:
            assert f.Q is f.P and f.Ir is f.I
