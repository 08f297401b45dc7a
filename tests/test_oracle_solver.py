"""Oracle compression, inverse and solve pinned by closed forms and brute force.

Pins: Sec. 5 error bound (||A - A_RS|| / ||A|| within 10 eps for a
second-kind operator), Sec. 4.3 (the telescoping inverse is one ordering of
Gaussian elimination on the compressed matrix), and closed-form spectra of
A = I + h K on the unit circle (circulant) and the sphere; the 3D Helmholtz
kernel (eq. 3d-helmholtz) by the Helmholtz equation, the outgoing radiation
condition and its small-wavenumber expansion.
"""
import math

import numpy as np
import pytest
from scipy.special import hankel1, jv, spherical_jn, spherical_yn

import rs_inputs as ri
from oracle import dense, rskel
from oracle.kernels import green


def _build(kind, pts, w, eps, leaf, nproxy, kwave=0.0):
    return rskel.build(pts, rskel.Params(kind=kind, w=w, eps=eps, leaf=leaf, nproxy=nproxy, kwave=kwave))


CASES = [
    # kind, geometry, N, eps, leaf, nproxy
    ("laplace2d", "circle", 2048, 1e-9, 64, 64),
    ("laplace2d", "starfish", 2048, 1e-10, 64, 64),
    ("helmholtz2d", "starfish", 1024, 1e-9, 64, 64),
    ("laplace3d", "sphere", 1500, 1e-6, 128, 216),
    ("helmholtz3d", "sphere", 1500, 1e-6, 128, 216),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"{c[0]}-{c[1]}-{c[2]}")
def case(request):
    kind, geom, n, eps, leaf, nproxy = request.param
    pts, w = ri.geometry(geom, n)
    kw = 10.0 if kind.startswith("helmholtz") else 0.0
    F = _build(kind, pts, w, eps, leaf, nproxy, kw)
    A = dense.dense_matrix(kind, pts, w, kw)
    dt = np.complex128 if kind.startswith("helmholtz") else np.float64
    ARS = F.apply(np.eye(n, dtype=dt))
    return dict(kind=kind, n=n, eps=eps, F=F, A=A, ARS=ARS, dt=dt)


def test_compression_error_within_10eps(case):
    rel = dense.norm2_est(case["A"] - case["ARS"]) / dense.norm2_est(case["A"])
    assert rel <= 10 * case["eps"], rel


def test_solve_equals_dense_elimination(case):
    n = case["n"]
    B = ri.rhs(n, 3, seed=11, complex_=case["dt"] == np.complex128)
    X = case["F"].solve(B)
    Xd = np.linalg.solve(case["ARS"], B)
    assert np.linalg.norm(X - Xd) / np.linalg.norm(Xd) < 1e-12
    Xa = np.linalg.solve(case["A"], B)
    assert np.linalg.norm(X - Xa) / np.linalg.norm(Xa) <= 10 * case["eps"]


def test_forward_apply_consistent_with_solve(case):
    n = case["n"]
    x = ri.rhs(n, 1, seed=4, complex_=case["dt"] == np.complex128)[:, 0]
    y = case["F"].apply(x)
    assert np.linalg.norm(case["F"].solve(y) - x) / np.linalg.norm(x) < 1e-12


def test_tree_leaf_and_rank_structure(case):
    F = case["F"]
    for d, fs in F.boxes.items():
        for f in fs:
            assert 0 < f.k <= f.n
            assert f.calD.shape == (f.n, f.n) and f.calL.shape == (f.n, f.k) and f.calR.shape == (f.k, f.n)
    assert F.skeleton_count() == F.calS.shape[0]


def _circle_laplace_eig(n, m):
    """lambda_m = 1 - (1/N) sum_j ln(2 sin(pi j/N)) cos(2 pi m j / N), exact sum."""
    s = math.fsum(math.log(2 * math.sin(math.pi * j / n)) * math.cos(2 * math.pi * m * j / n)
                  for j in range(1, n))
    return 1.0 - s / n


def test_circle_laplace_closed_form():
    n, eps = 4096, 1e-9
    pts, h = ri.circle(n)
    F = _build("laplace2d", pts, h, eps, 64, 64)
    th = 2 * np.pi * np.arange(n) / n
    # constant mode: prod_j 2 sin(pi j / N) = N gives lambda_0 = 1 - ln(N)/N exactly
    assert abs(_circle_laplace_eig(n, 0) - (1 - math.log(n) / n)) < 1e-14
    for m in (0, 1, 5, 17):
        lam = _circle_laplace_eig(n, m)
        b = np.cos(m * th)
        x = F.solve(b)
        assert np.linalg.norm(x - b / lam) / np.linalg.norm(b / lam) <= 10 * eps
        if m > 0:
            # continuum single layer on the unit circle: S cos(m t) = cos(m t) / (2m)
            assert abs(lam - (1 + 1 / (2 * m))) < 5 * (2 * np.pi / n) * math.log(n)


def test_circle_helmholtz_closed_form():
    n, eps, k = 2048, 1e-9, 10.0
    pts, h = ri.circle(n)
    F = _build("helmholtz2d", pts, h, eps, 64, 64, k)
    th = 2 * np.pi * np.arange(n) / n
    j = np.arange(1, n)
    row = h * 0.25j * hankel1(0, k * 2 * np.sin(np.pi * j / n))
    for m in (0, 3, 11):
        lam = 1 + np.sum(row * np.cos(2 * np.pi * m * j / n))
        b = np.cos(m * th)
        x = F.solve(b)
        assert np.linalg.norm(x - b / lam) / np.linalg.norm(b / lam) <= 10 * eps
        # continuum: 1 + (i pi / 2) J_m(k) H_m^(1)(k)
        cont = 1 + 0.5j * np.pi * jv(m, k) * hankel1(m, k)
        assert abs(lam - cont) < 2e-2


def test_sphere_single_layer_eigenvalue():
    n = 3000
    pts, w = ri.fibonacci_sphere(n)
    F = _build("laplace3d", pts, w, 1e-6, 128, 216)
    for l, Y in ((0, np.ones(n)), (1, pts[2].copy())):
        x = F.solve(Y)
        lam = float(Y @ Y / (Y @ x))          # Rayleigh quotient of A^-1
        # S Y_l = Y_l / (2l + 1) on the unit sphere; the punctured rule drops
        # about 1/sqrt(N) of the self cell
        assert abs(lam - (1 + 1 / (2 * l + 1))) < 2.0 / np.sqrt(n)


def test_helmholtz3d_kernel_pins():
    """G = e^{ikr}/(4 pi r): (Laplacian + k^2) G = 0 off the source (second
    differences, O(h^2)); r (dG/dr - i k G) -> 0 (outgoing; the incoming
    e^{-ikr} leaves k/(2 pi)); G = 1/(4 pi r) + i k/(4 pi) - k^2 r/(8 pi) + O(k^3 r^2)."""
    k = 7.0
    y = np.zeros((3, 1))
    x0 = np.array([0.3, -0.2, 0.5])
    for hstep in (1e-2, 5e-3):
        g0 = green("helmholtz3d", x0[:, None], y, k)[0, 0]
        lap = 0.0
        for d in range(3):
            e = np.zeros(3)
            e[d] = hstep
            gp = green("helmholtz3d", (x0 + e)[:, None], y, k)[0, 0]
            gm = green("helmholtz3d", (x0 - e)[:, None], y, k)[0, 0]
            lap += (gp - 2 * g0 + gm) / hstep**2
        assert abs(lap + k * k * g0) < 2.0 * hstep**2 * abs(k**4 * g0) + 1e-9
    for r in (50.0, 500.0):
        dr = 1e-5   # k dr small: central-difference error (k dr)^2 / 6
        p = lambda t: np.array([[t], [0.0], [0.0]])
        g = green("helmholtz3d", p(r), y, k)[0, 0]
        dg = (green("helmholtz3d", p(r + dr), y, k)[0, 0] - green("helmholtz3d", p(r - dr), y, k)[0, 0]) / (2 * dr)
        assert abs(r * (dg - 1j * k * g)) < 2.0 / (4 * np.pi * r) + 1e-6
    kk, r = 1e-3, 0.5
    g = green("helmholtz3d", np.array([[r], [0.0], [0.0]]), y, kk)[0, 0]
    ser = 1 / (4 * np.pi * r) + 1j * kk / (4 * np.pi) - kk * kk * r / (8 * np.pi)
    assert abs(g - ser) < kk**3 * r * r / (4 * np.pi) + 1e-15


def test_helmholtz2d_kernel_pins():
    """G = (i/4) H0^(1)(k r) checked without the Bessel routines it is built
    from: (Laplacian + k^2) G = 0 off the source (second differences in x and
    y, O(h^2)); sqrt(r) (dG/dr - i k G) decays like 1/r (outgoing; the
    incoming wave would leave a term growing like sqrt(r)); and as k r -> 0,
    G + log(r) / (2 pi) -> i/4 - (log(k/2) + gamma) / (2 pi), the 2D Laplace
    kernel plus a constant (Euler's gamma)."""
    k = 7.0
    y = np.zeros((2, 1))
    x0 = np.array([0.45, -0.3])
    for hstep in (1e-2, 5e-3):
        g0 = green("helmholtz2d", x0[:, None], y, k)[0, 0]
        lap = 0.0
        for d in range(2):
            e = np.zeros(2)
            e[d] = hstep
            gp = green("helmholtz2d", (x0 + e)[:, None], y, k)[0, 0]
            gm = green("helmholtz2d", (x0 - e)[:, None], y, k)[0, 0]
            lap += (gp - 2 * g0 + gm) / hstep**2
        assert abs(lap + k * k * g0) < 2.0 * hstep**2 * abs(k**4 * g0) + 1e-9
    for r in (50.0, 500.0):
        dr = 1e-5
        p = lambda t: np.array([[t], [0.0]])
        g = green("helmholtz2d", p(r), y, k)[0, 0]
        dg = (green("helmholtz2d", p(r + dr), y, k)[0, 0] - green("helmholtz2d", p(r - dr), y, k)[0, 0]) / (2 * dr)
        bound = 2.0 * np.sqrt(2.0 / (np.pi * k)) / (8.0 * r)
        assert abs(np.sqrt(r) * (dg - 1j * k * g)) < bound
    gamma = 0.5772156649015329
    for r in (1e-5, 1e-6):
        kk = 10.0
        g = green("helmholtz2d", np.array([[r], [0.0]]), y, kk)[0, 0]
        lim = 0.25j - (np.log(kk / 2) + gamma) / (2 * np.pi)
        assert abs(g + np.log(r) / (2 * np.pi) - lim) < 1e-6


def test_sphere_helmholtz_single_layer_eigenvalue():
    """On the unit sphere the single layer of eq. 3d-helmholtz maps Y_l to
    i k j_l(k) h_l^(1)(k) Y_l; A = I + w K approximates I + S, to the same
    1/sqrt(N) self-cell error as the Laplace case."""
    n, k = 1500, 10.0
    pts, w = ri.fibonacci_sphere(n)
    F = _build("helmholtz3d", pts, w, 1e-6, 128, 216, k)
    for l, Y in ((0, np.ones(n)), (1, pts[2].copy())):
        x = F.solve(Y.astype(np.complex128))
        lam = (Y @ Y) / (Y @ x)
        cont = 1 + 1j * k * spherical_jn(l, k) * (spherical_jn(l, k) + 1j * spherical_yn(l, k))
        assert abs(lam - cont) < 2.0 / np.sqrt(n), (l, lam, cont)


@pytest.mark.parametrize("kind,geom,n,eps,leaf,nproxy", [
    ("laplace2d", "starfish", 2048, 1e-10, 64, 64),
    ("laplace3d", "sphere", 1500, 1e-6, 128, 216),
], ids=lambda v: str(v))
def test_randomized_build_compression_and_solve(kind, geom, n, eps, leaf, nproxy):
    """The randomized-ID build (Sec. 2.2) meets the same bars as the
    deterministic one: ||A - A_RS|| / ||A|| <= 10 eps and the solve equals
    dense elimination on A within 10 eps."""
    pts, w = ri.geometry(geom, n)
    F = rskel.build(pts, rskel.Params(kind=kind, w=w, eps=eps, leaf=leaf, nproxy=nproxy, id_oversample=8, id_seed=3))
    A = dense.dense_matrix(kind, pts, w)
    ARS = F.apply(np.eye(n))
    assert dense.norm2_est(A - ARS) / dense.norm2_est(A) <= 10 * eps
    B = ri.rhs(n, 2, seed=12)
    X = F.solve(B)
    Xa = np.linalg.solve(A, B)
    assert np.linalg.norm(X - Xa) / np.linalg.norm(Xa) <= 10 * eps
