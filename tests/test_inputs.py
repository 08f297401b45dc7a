"""Seeded input generators: determinism and geometric definitions."""
import numpy as np

import rs_inputs as ri


def test_rhs_deterministic_and_normal():
    a = ri.rhs(5000, 3, seed=7)
    b = ri.rhs(5000, 3, seed=7)
    assert a.flags["F_CONTIGUOUS"] and a.shape == (5000, 3)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, ri.rhs(5000, 3, seed=8))
    assert abs(a.mean()) < 0.05 and abs(a.std() - 1.0) < 0.05


def test_splitmix64_reference_value():
    # splitmix64 with state 0 after one increment: published first output
    assert int(ri.splitmix64(np.array([0], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF


def test_circle_and_sphere():
    p, h = ri.circle(64)
    assert np.allclose(np.hypot(p[0], p[1]), 1.0) and np.isclose(h, 2 * np.pi / 64)
    s, w = ri.fibonacci_sphere(500)
    assert np.allclose(np.sum(s * s, axis=0), 1.0) and np.isclose(w, 4 * np.pi / 500)


def test_starfish_equal_arclength():
    n = 2048
    p, h = ri.starfish(n)
    th = np.unwrap(np.arctan2(p[1], p[0]))
    r = np.hypot(p[0], p[1])
    assert np.allclose(r, 1.0 + 0.3 * np.cos(5 * th), atol=1e-12)
    assert np.isclose(p[0, 0], 1.3) and abs(p[1, 0]) < 1e-15
    # arc length of every step by 20-point Gauss-Legendre on the speed
    xg, wg = np.polynomial.legendre.leggauss(20)
    t0 = th
    t1 = np.append(th[1:], th[0] + 2 * np.pi)
    mid, half = (t0 + t1) / 2, (t1 - t0) / 2
    tt = mid[:, None] + half[:, None] * xg[None, :]
    rr = 1.0 + 0.3 * np.cos(5 * tt)
    dr = -1.5 * np.sin(5 * tt)
    arcs = half * (np.sqrt(rr * rr + dr * dr) @ wg)
    assert np.max(np.abs(arcs - h)) < 1e-12


def test_rhs_column_slices_match_the_batch():
    for n in (7, 8, 131):
        B = ri.rhs(n, 9, seed=4)
        for c0, c1 in ((0, 9), (2, 5), (3, 4), (8, 9)):
            assert np.array_equal(ri.rhs_columns(n, c0, c1, seed=4), B[:, c0:c1])
