"""Seeded synthetic inputs for the recursive-skeletonization solver.

This module only makes data: point clouds on the workload geometries, their
quadrature weights, and right-hand sides.  It holds none of the solver's
arithmetic (no kernel evaluation, no tree, no compression), so both the CPU
oracle and the GPU library can be fed the same bytes from it.

Geometries (Sec. 6 of Ho & Greengard uses a circle, ellipses and a sphere; the
workloads here use):
  * unit circle, theta_j = 2 pi j / N, weight h = 2 pi / N;
  * starfish r(theta) = 1 + amp*cos(arms*theta), N points equispaced in arc
    length starting at theta = 0, weight h = L / N with L the perimeter;
  * Fibonacci sphere z_i = 1 - (2i+1)/N, phi_i = i*pi*(3 - sqrt 5),
    weight w = 4 pi / N;
  * ellipse with semi-axes a = 2, b = 1 (aspect ratio 2, Sec. 6.2), N points
    equispaced in arc length, weight h = L / N, with outward unit normals and
    curvature (the double-layer kernel needs both).

Random numbers come from splitmix64 (Steele, Lea & Flood, OOPSLA 2014) as a
counter-based generator, mapped to N(0,1) with the Box-Muller transform, so
the streams are identical on every platform and numpy version.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """splitmix64 output for each 64-bit counter value (vectorised)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int, stream: int = 0, offset: int = 0) -> np.ndarray:
    """`count` doubles in (0, 1], counter-based from (seed, stream), starting
    at position `offset` of the stream."""
    base = (np.uint64(seed) * np.uint64(0x100000001B3)) ^ (np.uint64(stream) << np.uint64(40))
    ctr = np.arange(count, dtype=np.uint64) + base + np.uint64(offset)
    bits = splitmix64(ctr) >> np.uint64(11)
    return (bits.astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normal(seed: int, shape, stream: int = 0) -> np.ndarray:
    """Standard normal samples by Box-Muller on splitmix64 uniforms."""
    count = int(np.prod(shape))
    half = (count + 1) // 2
    u1 = uniform01(seed, half, 2 * stream)
    u2 = uniform01(seed, half, 2 * stream + 1)
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * half)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count].reshape(shape)


def normal_range(seed: int, start: int, count: int, stream: int = 0) -> np.ndarray:
    """Elements [start, start + count) of the stream normal(seed, ...) makes."""
    p0 = start // 2
    p1 = (start + count + 1) // 2
    u1 = uniform01(seed, p1 - p0, 2 * stream, offset=p0)
    u2 = uniform01(seed, p1 - p0, 2 * stream + 1, offset=p0)
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * (p1 - p0))
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[start - 2 * p0:start - 2 * p0 + count]


def rhs_columns(n: int, c0: int, c1: int, seed: int = 0) -> np.ndarray:
    """Columns [c0, c1) of rhs(n, nrhs, seed) for any nrhs >= c1 (real), so a
    rank can make its slice of one global batch without the rest."""
    z = normal_range(seed, c0 * n, (c1 - c0) * n, stream=0)
    return np.asfortranarray(z.reshape(c1 - c0, n).T)


def rhs(n: int, nrhs: int, seed: int = 0, complex_: bool = False) -> np.ndarray:
    """N x nrhs right-hand sides, i.i.d. N(0,1), Fortran (column-major) order."""
    if complex_:
        re = normal(seed, (nrhs, n), stream=0)
        im = normal(seed, (nrhs, n), stream=1)
        return np.asfortranarray((re + 1j * im).T)
    return np.asfortranarray(normal(seed, (nrhs, n), stream=0).T)


def circle(n: int):
    """Unit circle, theta_j = 2 pi j / n.  Returns (points 2 x n, weight)."""
    th = 2.0 * np.pi * np.arange(n) / n
    return np.vstack([np.cos(th), np.sin(th)]), 2.0 * np.pi / n


def _starfish_speed_coeffs(arms: int, amp: float, nodes: int = 4096):
    th = 2.0 * np.pi * np.arange(nodes) / nodes
    r = 1.0 + amp * np.cos(arms * th)
    dr = -amp * arms * np.sin(arms * th)
    c = np.fft.rfft(np.sqrt(r * r + dr * dr)) / nodes
    # truncate where the coefficients have decayed to the rounding floor
    small = np.abs(c) < 1e-15 * abs(c[0])
    keep = len(c)
    for m in range(len(c)):
        if small[m:].all():
            keep = m
            break
    return c[:keep]


def starfish(n: int, arms: int = 5, amp: float = 0.3, rotation: float = 0.0):
    """Starfish r = 1 + amp cos(arms theta), n points equispaced in arc length.

    The arc-length function s(theta) is the integral of the speed, whose
    Fourier series comes from a 4096-node periodic trapezoid rule; each node
    theta_j with s(theta_j) = j L / n is found by Newton's method from
    theta = 2 pi j / n.  Returns (points 2 x n, weight h = L / n).
    """
    c = _starfish_speed_coeffs(arms, amp)
    length = 2.0 * np.pi * c[0].real

    def s_of(t):
        # s(t) = c0 t + sum_m 2 Re(c_m (e^{imt} - 1) / (i m)), powers by recursion
        e1 = np.exp(1j * t)
        em = np.ones_like(e1)
        acc = np.zeros_like(t)
        for m in range(1, len(c)):
            em = em * e1
            acc += np.real(c[m] * (em - 1.0) / (1j * m))
        return c[0].real * t + 2.0 * acc

    def speed(t):
        r = 1.0 + amp * np.cos(arms * t)
        dr = -amp * arms * np.sin(arms * t)
        return np.sqrt(r * r + dr * dr)

    target = length * np.arange(n) / n
    t = 2.0 * np.pi * np.arange(n) / n
    for _ in range(12):
        step = (s_of(t) - target) / speed(t)
        t = t - step
        if np.max(np.abs(step)) < 1e-14:
            break
    r = 1.0 + amp * np.cos(arms * t)
    ang = t + rotation
    return np.vstack([r * np.cos(ang), r * np.sin(ang)]), length / n


def ellipse(n: int, a: float = 2.0, b: float = 1.0):
    """Ellipse x = a cos t, y = b sin t, n points equispaced in arc length.

    Returns (points 2 x n, weight h = L / n, outward unit normals 2 x n,
    curvature n).  Arc length from the Fourier series of the speed
    |x'(t)| = sqrt(a^2 sin^2 t + b^2 cos^2 t) (4096-node periodic trapezoid),
    nodes by Newton's method as for the starfish; the normal is
    (b cos t, a sin t) / |x'(t)| and the curvature a b / |x'(t)|^3.
    """
    nodes = 4096
    th = 2.0 * np.pi * np.arange(nodes) / nodes
    c = np.fft.rfft(np.sqrt((a * np.sin(th)) ** 2 + (b * np.cos(th)) ** 2)) / nodes
    keep = len(c)
    small = np.abs(c) < 1e-15 * abs(c[0])
    for m in range(len(c)):
        if small[m:].all():
            keep = m
            break
    c = c[:keep]
    length = 2.0 * np.pi * c[0].real

    def s_of(t):
        e1 = np.exp(1j * t)
        em = np.ones_like(e1)
        acc = np.zeros_like(t)
        for m in range(1, len(c)):
            em = em * e1
            acc += np.real(c[m] * (em - 1.0) / (1j * m))
        return c[0].real * t + 2.0 * acc

    def speed(t):
        return np.sqrt((a * np.sin(t)) ** 2 + (b * np.cos(t)) ** 2)

    target = length * np.arange(n) / n
    t = 2.0 * np.pi * np.arange(n) / n
    for _ in range(20):
        step = (s_of(t) - target) / speed(t)
        t = t - step
        if np.max(np.abs(step)) < 1e-14:
            break
    sp = speed(t)
    pts = np.vstack([a * np.cos(t), b * np.sin(t)])
    nrm = np.vstack([b * np.cos(t), a * np.sin(t)]) / sp
    curv = a * b / sp ** 3
    return pts, length / n, nrm, curv


def fibonacci_sphere(n: int):
    """Fibonacci points on the unit sphere.  Returns (points 3 x n, 4 pi / n)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    rr = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * np.pi * (3.0 - np.sqrt(5.0))
    return np.vstack([rr * np.cos(phi), rr * np.sin(phi), z]), 4.0 * np.pi / n


def serving_curve(seed: int, index: int):
    """Random starfish for the serving mix: (n, arms, amp, rotation)."""
    u = uniform01(seed, 4, stream=1000 + index)
    n = int([8192, 16384, 32768, 65536][min(3, int(u[0] * 4))])
    arms = 3 + min(4, int(u[1] * 5))
    amp = 0.1 + 0.2 * u[2]
    rot = 2.0 * np.pi * u[3]
    return n, arms, amp, rot


# Workload presets: (geometry, kernel, eps, leaf, proxy count) per workload.
WORKLOADS = {
    "laplace2d_circle_4096": dict(geom="circle", n=4096, kernel="laplace2d",
                                  eps=1e-9, leaf=64, nproxy=64),
    "laplace2d_starfish_131072": dict(geom="starfish", n=131072, kernel="laplace2d",
                                      eps=1e-10, leaf=64, nproxy=64),
    "helmholtz2d_starfish_65536": dict(geom="starfish", n=65536, kernel="helmholtz2d",
                                       eps=1e-9, leaf=64, nproxy=64, kwave=10.0),
    "laplace3d_sphere_32768": dict(geom="sphere", n=32768, kernel="laplace3d",
                                   eps=1e-6, leaf=128, nproxy=216),
    # 3D Helmholtz on the unit sphere, k = 10 (omega = k diam / 2 pi = 3.18)
    "helmholtz3d_sphere_8192": dict(geom="sphere", n=8192, kernel="helmholtz3d",
                                    eps=1e-6, leaf=128, nproxy=216, kwave=10.0),
    # the interior Dirichlet problem on the ellipse a = 2, b = 1 with the
    # double layer (Sec. 6.2), weight -2 h (A sigma = -2 f)
    "laplace2d_dl_ellipse_131072": dict(geom="ellipse", n=131072, kernel="laplace2d_dl",
                                        eps=1e-9, leaf=64, nproxy=64),
}


def geometry(name: str, n: int, **kw):
    if name == "circle":
        return circle(n)
    if name == "starfish":
        return starfish(n, **kw)
    if name == "sphere":
        return fibonacci_sphere(n)
    if name == "ellipse":
        return ellipse(n, **kw)[:2]
    raise ValueError(name)
