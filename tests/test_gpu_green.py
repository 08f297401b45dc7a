"""The device evaluation of the Green's functions (rs_green) against numpy /
scipy: the 2D Laplace kernel goes through the library's table-driven
logarithm (Tang 1990), checked here to a few units of 1e-16 over the whole
range of squared distances the solver meets."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _s2():
    rng = np.random.default_rng(5)
    s = np.concatenate([10.0 ** rng.uniform(-30, 6, 200000),
                        1.0 + rng.uniform(-1e-6, 1e-6, 20000),       # log near 0
                        np.array([1.0, 2.0, 0.5, 4.0, 1.0 + 2.0 ** -52, 2.0 ** -1022 * 3])])
    return s


def test_laplace2d_log_table():
    import paper_1110_3105_gb300 as rs
    s = _s2()
    g = rs.rs_green("laplace2d", s)
    ref = -np.log(s) / (4 * np.pi)
    err = np.abs(g - ref)
    # absolute error a few ulp of O(1) values, relative where |log s| is large
    assert np.all(err <= 4e-16 * np.maximum(1.0, np.abs(ref))), err.max()


def test_laplace3d_and_helmholtz():
    import paper_1110_3105_gb300 as rs
    from scipy.special import j0, y0
    rng = np.random.default_rng(6)
    s = 10.0 ** rng.uniform(-12, 2, 50000)
    g = rs.rs_green("laplace3d", s)
    ref = 1.0 / (4 * np.pi * np.sqrt(s))
    assert np.max(np.abs(g - ref) / ref) <= 8e-16   # rsqrt and the reference each round a few times
    k = 10.0
    h = rs.rs_green("helmholtz2d", s, k_wave=k)
    kr = k * np.sqrt(s)
    href = 0.25j * (j0(kr) + 1j * y0(kr))
    # CUDA j0 / y0 against scipy: a few units of 1e-13 absolute
    assert np.max(np.abs(h - href) / np.maximum(1.0, np.abs(href))) <= 1e-12


def test_helmholtz3d():
    import paper_1110_3105_gb300 as rs
    rng = np.random.default_rng(8)
    s = 10.0 ** rng.uniform(-10, 2, 50000)
    k = 10.0
    g = rs.rs_green("helmholtz3d", s, k_wave=k)
    r = np.sqrt(s)
    ref = np.exp(1j * k * r) / (4 * np.pi * r)
    # CUDA sincos and the reference each round a few times; kr up to 1e2
    assert np.max(np.abs(g - ref) / np.abs(ref)) <= 1e-14
