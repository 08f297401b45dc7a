"""The C-ABI library loads and exports every entry point include/rs.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1110_3105_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_exported(lib):
    names = _declared()
    assert "rs_build" in names and "rs_solve" in names and "rs_free" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_1110_3105_gb300 import _lib
    assert set(_declared()) <= set(_lib.EXPORTED)


def test_no_compute_without_gpu_errors_cleanly(lib):
    # argument validation happens before any device work
    from paper_1110_3105_gb300 import _lib
    _lib.load()
    out = ctypes.c_void_p()
    rc = _lib._lib.rs_build(None, 10, 2, None, 1e-9, 64, None, ctypes.byref(out))
    assert rc == -1 and out.value is None
    assert b"null" in _lib._lib.rs_last_error()
    assert _lib._lib.rs_free(None) == 0


def test_fault_spec_validation(lib):
    from paper_1110_3105_gb300 import _lib
    _lib.load()
    assert _lib._lib.rs_set_fault(b"bogus") == -1
    assert _lib._lib.rs_set_fault(b"alloc:0") == -1
    assert _lib._lib.rs_set_fault(b"off") == 0
    assert _lib._lib.rs_set_fault(None) == 0


def test_build_parameter_validation(lib):
    """Bad build parameters are rejected before any device work (no GPU needed)."""
    import numpy as np
    from paper_1110_3105_gb300 import _lib
    _lib.load()
    pts = np.asfortranarray(np.random.default_rng(0).random((2, 100)))
    out = ctypes.c_void_p()
    good = dict(kernel_id=0, k_wave=0.0, weight=0.01, proxy_n=64, proxy_ratio=1.5, id_arith=0)
    for field, bad in (("id_arith", 7), ("proxy_ratio", 1.0), ("proxy_n", 0), ("weight", -1.0), ("kernel_id", 9)):
        kw = dict(good)
        kw[field] = bad
        p = _lib.rs_params(**kw)
        rc = _lib._lib.rs_build(pts.ctypes.data, 100, 2, ctypes.byref(p), 1e-9, 64, None, ctypes.byref(out))
        assert rc == -1, field
        assert out.value is None
    # kernel / dimension mismatches and a Helmholtz kernel without a wavenumber
    for kid, dim, kwave in ((3, 2, 10.0), (2, 2, 0.0), (1, 3, 10.0), (3, 3, 0.0), (1, 2, 0.0)):
        kw = dict(good, kernel_id=kid, k_wave=kwave, proxy_n=216 if dim == 3 else 64)
        p = _lib.rs_params(**kw)
        q = np.asfortranarray(np.random.default_rng(1).random((dim, 100)))
        rc = _lib._lib.rs_build(q.ctypes.data, 100, dim, ctypes.byref(p), 1e-9, 64, None, ctypes.byref(out))
        assert rc == -1, (kid, dim, kwave)
        assert out.value is None
    # the double layer: normals and curvature required, 2D only, a nonzero
    # weight, the deterministic FP64 ID
    nrm = np.zeros(200)
    kap = np.zeros(100)
    for extra, dim in ((dict(), 2), (dict(normals=nrm.ctypes.data), 2),
                       (dict(normals=nrm.ctypes.data, curvature=kap.ctypes.data, weight=0.0), 2),
                       (dict(normals=nrm.ctypes.data, curvature=kap.ctypes.data, id_oversample=8), 2),
                       (dict(normals=nrm.ctypes.data, curvature=kap.ctypes.data, id_arith=1), 2),
                       (dict(normals=nrm.ctypes.data, curvature=kap.ctypes.data, proxy_n=216), 3)):
        p = _lib.rs_params(**dict(good, kernel_id=4, **extra))
        q = np.asfortranarray(np.random.default_rng(1).random((dim, 100)))
        rc = _lib._lib.rs_build(q.ctypes.data, 100, dim, ctypes.byref(p), 1e-9, 64, None, ctypes.byref(out))
        assert rc == -1, extra
        assert out.value is None


def test_handle_and_argument_errors(lib):
    """Null handles, bad sizes and bad kernel ids are rejected with RS_ERR_ARG
    and a message, before any device work."""
    import numpy as np
    from paper_1110_3105_gb300 import _lib
    _lib.load()
    L = _lib._lib
    x = np.zeros(4)
    assert L.rs_solve(None, 0, x.ctypes.data, 4, 1, x.ctypes.data, 4, None) == -1
    assert b"null handle" in L.rs_last_error()
    assert L.rs_solve_refined(None, x.ctypes.data, 4, 1, x.ctypes.data, 4, 1e-10, 8, None, None, None) == -1
    assert L.rs_matvec(None, x.ctypes.data, 4, 1, x.ctypes.data, 4, None) == -1
    assert L.rs_stats(None, None) == -1
    out = ctypes.c_void_p()
    assert L.rs_server_create(0, 0, ctypes.byref(out)) == -1 and out.value is None
    s2 = np.ones(3)
    g = np.zeros(6)
    assert L.rs_green(9, 0.0, s2.ctypes.data, 3, g.ctypes.data) == -1
    assert L.rs_green(4, 0.0, s2.ctypes.data, 3, g.ctypes.data) == -1   # the double layer needs normals
    assert L.rs_green(0, 0.0, s2.ctypes.data, -1, g.ctypes.data) == -1
    assert L.rs_version().startswith(b"rs-gb300")


def test_path_spec_validation(lib):
    from paper_1110_3105_gb300 import _lib
    _lib.load()
    assert _lib._lib.rs_set_path(b"id:bogus") == -1
    assert _lib._lib.rs_set_path(b"id:step,gj:coop") == 0
    assert _lib._lib.rs_set_path(b"off") == 0
    assert _lib._lib.rs_set_path(None) == 0
    counts = _lib.rs_path_counts(reset=True)
    assert len(counts) == 11 and all(v == 0 for v in counts.values())


def test_tile_spec_validation(lib):
    from paper_1110_3105_gb300 import _lib
    _lib.load()
    for good in (b"tile:128x128", b"tile:32x64", b"tile:warp", b"tile:128x256,id:big"):
        assert _lib._lib.rs_set_path(good) == 0, good
    for bad in (b"tile:128x32", b"tile:16x16", b"tile:"):
        assert _lib._lib.rs_set_path(bad) == -1, bad
    assert _lib._lib.rs_set_path(None) == 0
