"""Oracle: Green's functions, the system matrix and proxy surfaces.

Test infrastructure (see the package header).

Green's functions (Sec. 2, Example 1 and 2; Sec. 6.1.2):
  laplace2d    G = -(1/2 pi) log|x - y|          (eq. 2d-laplace)
  laplace3d    G = 1 / (4 pi |x - y|)             (eq. 3d-laplace)
  helmholtz2d  G = (i/4) H0^(1)(k |x - y|)        (eq. 2d-helmholtz)
  helmholtz3d  G = exp(i k |x - y|) / (4 pi |x - y|) (eq. 3d-helmholtz)
  laplace2d_dl K = dG/dnu_y = (1/2 pi) (x - y) . nu_y / |x - y|^2, the kernel
               of the double-layer potential (eq. double-layer) with the 2D
               Laplace G, nu_y the outward unit normal at the source
System matrix: A = I + w K with K_ij = G(x_i, x_j) for i != j and K_ii = 0
(punctured trapezoid / one-point rule, the configuration the workloads
state; w = h for curves, 4 pi / N on the sphere).  The double-layer kernel
is smooth on a smooth curve: K_ii is its limit -kappa_i / (4 pi) (kappa the
curvature), and the trapezoid rule is used as it stands.  The second-kind
equation -sigma/2 + D sigma = f (eq. 2k-integral-eqn) times -2 is
A sigma = -2 f with w = -2 h.  The double-layer kernel is not symmetric
(K(x, y) != K(y, x)): the row and column skeletons of a box differ.

Proxy surfaces (Sec. 3.2, Fig. proxy-comp; count per Sec. 6 opening):
  2D  n_p points on a circle of radius ratio * (sqrt(2)/2) * s around the box
      centre (s = box side, so ratio times the box circumradius), angles
      2 pi j / n_p;
  3D  a g x g grid of cell centres on each of the 6 faces of a cube of
      half-width ratio * s / 2 (6 g^2 = n_p points), faces in the order
      -x, +x, -y, +y, -z, +z.
H0^(1) is taken from scipy.special.hankel1, a library primitive; the 3D
kernel is numpy's complex exponential.

Pins: tests/test_oracle_solver.py checks the Laplace 2D kernel through the
closed-form spectrum of A on the unit circle (eigenvalue 1 - ln(N)/N for the
constant mode, and its continuum limit 1 + 1/(2m)); the 2D Helmholtz kernel
through the Helmholtz equation (second differences), the outgoing radiation
condition and its small-argument limit (the Laplace kernel plus i/4 -
(log(k/2) + gamma)/(2 pi)), and the continuum limit 1 + (i pi / 2) J_m(k)
H_m^(1)(k) on the circle;
the 3D kernel through the single-layer eigenvalue 1 + 1/(2l+1) of the
spherical harmonics on the sphere; the 3D Helmholtz kernel through the
Helmholtz equation itself (a finite-difference Laplacian of G plus k^2 G
vanishes away from the source, for e^{+ikr} only with the outgoing
behaviour r (dG/dr - i k G) -> 0), its small-k expansion
1/(4 pi r) + i k/(4 pi) - k^2 r/(8 pi) + ..., and the single-layer
eigenvalue 1 + i k j_l(k) h_l^(1)(k) of the spherical harmonics on the unit
sphere.
"""
from __future__ import annotations

import numpy as np
from scipy.special import hankel1

KINDS = ("laplace2d", "helmholtz2d", "laplace3d", "helmholtz3d", "laplace2d_dl")


def is_complex(kind: str) -> bool:
    return kind in ("helmholtz2d", "helmholtz3d")


def is_symmetric(kind: str) -> bool:
    return kind != "laplace2d_dl"


def green_dl(X: np.ndarray, Y: np.ndarray, NY: np.ndarray) -> np.ndarray:
    """dG/dnu_y (x_i, y_j) for G = -(1/2 pi) log|x - y|: targets X (2, m),
    sources Y (2, n) with unit normals NY (2, n); x != y assumed."""
    diff = X[:, :, None] - Y[:, None, :]
    r2 = np.sum(diff * diff, axis=0)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.einsum("dij,dj->ij", diff, NY) / (2.0 * np.pi * r2)


def green(kind: str, X: np.ndarray, Y: np.ndarray, kwave: float = 0.0) -> np.ndarray:
    """G(x_i, y_j) for targets X (dim, m) and sources Y (dim, n); r > 0 assumed."""
    diff = X[:, :, None] - Y[:, None, :]
    r = np.sqrt(np.sum(diff * diff, axis=0))
    with np.errstate(divide="ignore", invalid="ignore"):
        if kind == "laplace2d":
            return -np.log(r) / (2.0 * np.pi)
        if kind == "laplace3d":
            return 1.0 / (4.0 * np.pi * r)
        if kind == "helmholtz2d":
            return 0.25j * hankel1(0, kwave * r)
        if kind == "helmholtz3d":
            return np.exp(1j * kwave * r) / (4.0 * np.pi * r)
    raise ValueError(kind)


def kernel_block(kind, pts, I, J, kwave=0.0, geom=None) -> np.ndarray:
    """K(x_i, y_j) for targets I and sources J (indices into pts); geom =
    (normals 2 x N, curvature N) for the double-layer kernel."""
    I = np.asarray(I)
    J = np.asarray(J)
    if kind == "laplace2d_dl":
        nrm, _ = geom
        return green_dl(pts[:, I], pts[:, J], nrm[:, J])
    return green(kind, pts[:, I], pts[:, J], kwave)


def system_block(kind, pts, I, J, w, kwave=0.0, geom=None) -> np.ndarray:
    """A(I, J) = delta_ij + w K(x_i, x_j); K_ii = 0, or for the double layer
    its limit -kappa_i / (4 pi)."""
    I = np.asarray(I)
    J = np.asarray(J)
    G = kernel_block(kind, pts, I, J, kwave, geom)
    same = I[:, None] == J[None, :]
    G[same] = 0.0
    A = w * G
    if kind == "laplace2d_dl":
        _, curv = geom
        ii, jj = np.nonzero(same)
        A[ii, jj] = 1.0 - w * curv[I[ii]] / (4.0 * np.pi)
    else:
        A[same] = 1.0
    return A


def offdiag_block(kind, pts, I, J, w, kwave=0.0, geom=None) -> np.ndarray:
    """w K(x_i, y_j) between two disjoint point sets (targets I, sources J)."""
    return w * kernel_block(kind, pts, I, J, kwave, geom)


def proxy_points(dim: int, center: np.ndarray, side: float, nproxy: int,
                 ratio: float = 1.5) -> np.ndarray:
    """Proxy surface points, shape (dim, nproxy)."""
    if dim == 2:
        rho = ratio * (np.sqrt(2.0) / 2.0) * side
        th = 2.0 * np.pi * np.arange(nproxy) / nproxy
        return center[:, None] + rho * np.vstack([np.cos(th), np.sin(th)])
    g = int(round(np.sqrt(nproxy / 6.0)))
    if 6 * g * g != nproxy:
        raise ValueError("3D proxy count must be 6 g^2")
    h = ratio * side / 2.0
    u = -h + (2.0 * np.arange(g) + 1.0) * h / g
    ua, ub = np.meshgrid(u, u, indexing="ij")
    ua = ua.ravel()
    ub = ub.ravel()
    faces = []
    for axis in range(3):
        others = [a for a in range(3) if a != axis]
        for sign in (-1.0, 1.0):
            f = np.zeros((3, g * g))
            f[axis] = sign * h
            f[others[0]] = ua
            f[others[1]] = ub
            faces.append(f)
    return center[:, None] + np.hstack(faces)


def proxy_radius_2d(side: float, ratio: float = 1.5) -> float:
    return ratio * (np.sqrt(2.0) / 2.0) * side
