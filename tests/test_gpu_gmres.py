"""Recursive skeletonization as a preconditioner (Sec. 6.4): GMRES on the
system coupling two scatterers, with and without the block-diagonal
preconditioner diag(A_ii^-1) (each block one RS handle), against the
oracle's dense solve of the coupled matrix."""
import numpy as np
import pytest

import rs_inputs as ri
from oracle import dense

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _scatterer(n, center, scale=1.0 / 3.0, rotation=0.0):
    """r = (2 + cos 3 theta) / 6 (Sec. 6.4): the starfish with 3 arms,
    amplitude 1/2, scaled by 1/3; equal arc length, weight h."""
    pts, h = ri.starfish(n, arms=3, amp=0.5, rotation=rotation)
    return pts * scale + np.asarray(center, dtype=float)[:, None], h * scale


# The configurations' A = I + h K is second kind and well conditioned: GMRES
# needs only a handful of iterations with or without a preconditioner.  With
# the single layer weighted 50 h the self-interactions dominate (condition
# numbers ~20-40 at N = 2 x 1024) and the unpreconditioned iteration count
# grows, as for the paper's scatterers; the block preconditioner removes the
# self-interactions and leaves the weak coupling.
@pytest.mark.parametrize("kind,kw,sep,ratio", [("helmholtz2d", 30.0, 1.2, 3), ("helmholtz2d", 30.0, 3.0, 3),
                                               ("laplace2d", 0.0, 1.2, 2)])
def test_preconditioned_gmres_two_scatterers(kind, kw, sep, ratio):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    n, eps = 1024, 1e-8
    cplx = kind.startswith("helmholtz")
    p1, w1 = _scatterer(n, (0.0, 0.0))
    p2, w2 = _scatterer(n, (sep, 0.0))
    w1, w2 = 50.0 * w1, 50.0 * w2
    H1 = rs.rs_build(p1, kind, w1, eps, 64, 64, k_wave=kw)
    H2 = rs.rs_build(p2, kind, w2, eps, 64, 64, k_wave=kw)
    try:
        pts = np.hstack([p1, p2])
        # incoming plane wave e^{i k x_2} (Laplace: a smooth field)
        f = np.exp(1j * kw * pts[1]) if cplx else np.cos(pts[0]) + pts[1]
        b = np.ascontiguousarray(f.astype(np.complex128 if cplx else np.float64))
        A = dense.coupled_matrix(kind, [p1, p2], [w1, w2], kw)
        x_ref = np.linalg.solve(A, b)
        x = np.zeros_like(b)
        its_p, rel_p = rs.rs_gmres_patches([H1, H2], pts, b, x, tol=1e-9, max_it=400, restart=60)
        assert rel_p <= 1e-9
        assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 2e-9
        assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-6
        x0 = np.zeros_like(b)
        its_0, rel_0 = rs.rs_gmres_patches([H1, H2], pts, b, x0, tol=1e-9, max_it=400, restart=60,
                                           precondition=False)
        # the preconditioner removes the scatterers' self-interaction: far
        # fewer iterations than plain GMRES on the same system
        assert its_p * ratio <= its_0, (its_p, its_0)
        assert its_p <= 30, its_p
    finally:
        H1.free()
        H2.free()


def test_gmres_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1110_3105_gb300 as rs
    p1, w1 = _scatterer(200, (0.0, 0.0))
    H1 = rs.rs_build(p1, "laplace2d", w1, 1e-8, 64, 64)
    H2 = rs.rs_build(p1, "helmholtz2d", w1, 1e-8, 64, 64, k_wave=5.0)
    try:
        b = np.ones(400)
        with pytest.raises(rs.RSError):   # mixed kernels
            rs.rs_gmres_patches([H1, H2], np.hstack([p1, p1]), b, np.zeros(400))
        with pytest.raises(rs.RSError):   # bad restart
            rs.rs_gmres_patches([H1], p1, b[:200], np.zeros(200), restart=0)
    finally:
        H1.free()
        H2.free()
