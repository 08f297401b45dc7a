"""2D Helmholtz at the frequency of the paper's 2D solver experiments,
omega = k diam / (2 pi) = 10 (Sec. 6.2), on the unit circle (k = 10 pi,
about 31 wavelengths on the curve, N = 4096: 130 points per wavelength).

The oracle's compressed operator is held to 10 eps of the dense matrix
(Sec. 5), and the GPU's FP64 and refined solves to 10 eps of the oracle's
solve; the right-hand side cos(m theta) is an eigenfunction of the system on
the circle, so the solution is also checked against the closed form b /
lambda_m with lambda_m = 1 + h sum_j G(2 sin(pi j / N)) cos(2 pi m j / N) (the
discrete circulant eigenvalue, the punctured trapezoid rule).
"""
import numpy as np
import pytest
from scipy.special import hankel1

import rs_inputs as ri
from oracle import dense, rskel

torch = pytest.importorskip("torch")

N, EPS, K = 4096, 1e-9, 10 * np.pi


@pytest.fixture(scope="module")
def oracle():
    pts, h = ri.circle(N)
    return pts, h, rskel.build(pts, rskel.Params(kind="helmholtz2d", w=h, eps=EPS, leaf=64, nproxy=64, kwave=K))


def _closed_form(h, m):
    j = np.arange(1, N)
    row = h * 0.25j * hankel1(0, K * 2 * np.sin(np.pi * j / N))
    lam = 1 + np.sum(row * np.cos(2 * np.pi * m * j / N))
    th = 2 * np.pi * np.arange(N) / N
    b = np.cos(m * th).astype(np.complex128)
    return b, b / lam


def test_oracle_compression_at_omega10(oracle):
    pts, h, F = oracle
    A = dense.dense_matrix("helmholtz2d", pts, h, K)
    x = ri.rhs(N, 2, seed=61, complex_=True)
    assert np.linalg.norm(F.apply(x) - A @ x) <= 10 * EPS * np.linalg.norm(A @ x)
    for m in (0, 31, 200):
        b, xe = _closed_form(h, m)
        assert np.linalg.norm(F.solve(b) - xe) <= 10 * EPS * np.linalg.norm(xe)


@pytest.mark.gpu
def test_gpu_matches_oracle_at_omega10(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    pts, h, F = oracle
    H = rs.rs_build(pts, "helmholtz2d", h, EPS, 64, 64, k_wave=K)
    try:
        B = ri.rhs(N, 3, seed=62, complex_=True)
        X = np.zeros_like(B)
        rs.rs_solve(H, B, X)
        Xo = F.solve(B)
        assert np.all(np.linalg.norm(X - Xo, axis=0) <= 10 * EPS * np.linalg.norm(Xo, axis=0))
        Xr = np.zeros_like(B)
        its, rel = rs.rs_solve_refined(H, B, Xr, tol=1e-10, max_it=8)
        assert np.all(rel <= 1e-10)
        assert np.all(np.linalg.norm(Xr - Xo, axis=0) <= 10 * EPS * np.linalg.norm(Xo, axis=0))
        b, xe = _closed_form(h, 31)
        b = b[:, None].copy(order="F")
        x = np.zeros_like(b)
        rs.rs_solve(H, b, x)
        assert np.linalg.norm(x[:, 0] - xe) <= 10 * EPS * np.linalg.norm(xe)
    finally:
        H.free()
