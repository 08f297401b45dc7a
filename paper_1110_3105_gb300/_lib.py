"""ctypes binding of librs.so: argument marshalling only.

Every function maps one-to-one onto an entry point of include/rs.h.  Arrays
may be numpy arrays (host) or torch tensors (host or CUDA); the library
detects device pointers itself.  Nothing here computes any part of the
method: a missing or unloadable library raises immediately.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librs.so")

RS_LAPLACE2D, RS_HELMHOLTZ2D, RS_LAPLACE3D, RS_HELMHOLTZ3D, RS_LAPLACE2D_DL = 0, 1, 2, 3, 4
RS_PREC_FP64, RS_PREC_FP32 = 0, 1
KERNELS = {"laplace2d": RS_LAPLACE2D, "helmholtz2d": RS_HELMHOLTZ2D, "laplace3d": RS_LAPLACE3D,
           "helmholtz3d": RS_HELMHOLTZ3D, "laplace2d_dl": RS_LAPLACE2D_DL}
COMPLEX_KERNELS = ("helmholtz2d", "helmholtz3d")
STATUS = {0: "RS_OK", -1: "RS_ERR_ARG", -2: "RS_ERR_OOM", -3: "RS_ERR_CUDA", -4: "RS_ERR_SINGULAR",
          -5: "RS_ERR_TIMEOUT", -6: "RS_ERR_NAN", -7: "RS_ERR_STATE"}


class RSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class rs_params(ctypes.Structure):
    _fields_ = [("kernel_id", ctypes.c_int), ("k_wave", ctypes.c_double), ("weight", ctypes.c_double),
                ("proxy_n", ctypes.c_int), ("proxy_ratio", ctypes.c_double), ("id_arith", ctypes.c_int),
                ("id_oversample", ctypes.c_int), ("id_seed", ctypes.c_uint64),
                ("normals", ctypes.c_void_p), ("curvature", ctypes.c_void_p)]


def _dlayer(normals, curvature):
    """Point-major normals (2N doubles) and curvatures (N) for the double layer,
    or (None, None); returns the arrays to keep alive and their addresses."""
    if normals is None:
        return (), None, None
    nrm = np.ascontiguousarray(np.asarray(normals, dtype=np.float64).T)   # (N, 2): point-major
    kap = np.ascontiguousarray(np.asarray(curvature, dtype=np.float64))
    return (nrm, kap), nrm.ctypes.data, kap.ctypes.data


class rs_stats_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("dim", ctypes.c_int), ("depth", ctypes.c_int),
                ("top_skeletons", ctypes.c_int64), ("factor_bytes", ctypes.c_int64),
                ("factor_scalars", ctypes.c_int64), ("build_ms", ctypes.c_double),
                ("max_box_n", ctypes.c_int), ("max_box_m", ctypes.c_int), ("max_rank", ctypes.c_int)]


class rs_server_stats_t(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_int64), ("rhs", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("mean_batch_cols", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("elapsed_s", ctypes.c_double), ("handles", ctypes.c_int), ("resident_bytes", ctypes.c_int64)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_PROTOS = {
    "rs_build": (ctypes.c_int, [_P, _I64, ctypes.c_int, ctypes.POINTER(rs_params), ctypes.c_double,
                                ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "rs_solve": (ctypes.c_int, [_P, ctypes.c_int, _P, _I64, ctypes.c_int, _P, _I64, _P]),
    "rs_solve_noalloc": (ctypes.c_int, [_P, ctypes.c_int, _P, _I64, ctypes.c_int, _P, _I64, _P]),
    "rs_solve_refined": (ctypes.c_int, [_P, _P, _I64, ctypes.c_int, _P, _I64, ctypes.c_double, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), _P, _P]),
    "rs_matvec": (ctypes.c_int, [_P, _P, _I64, ctypes.c_int, _P, _I64, _P]),
    "rs_stats": (ctypes.c_int, [_P, ctypes.POINTER(rs_stats_t)]),
    "rs_tree_perm": (ctypes.c_int, [_P, _P]),
    "rs_tree_level": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _P, _P, _P, _P]),
    "rs_box_ranks": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "rs_free": (ctypes.c_int, [_P]),
    "rs_set_fault": (ctypes.c_int, [ctypes.c_char_p]),
    "rs_server_create": (ctypes.c_int, [ctypes.c_int, _I64, ctypes.POINTER(_P)]),
    "rs_server_add_handle": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int)]),
    "rs_server_submit_solve": (ctypes.c_int, [_P, ctypes.c_int, _P, _I64, ctypes.c_int, _P, _I64, ctypes.c_double,
                                              ctypes.POINTER(_I64)]),
    "rs_server_submit_build": (ctypes.c_int, [_P, _P, _I64, ctypes.c_int, ctypes.POINTER(rs_params), ctypes.c_double,
                                              ctypes.c_int, ctypes.POINTER(_I64)]),
    "rs_server_wait": (ctypes.c_int, [_P, _I64, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int)]),
    "rs_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(rs_server_stats_t)]),
    "rs_server_reset_stats": (ctypes.c_int, [_P]),
    "rs_server_handle": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "rs_server_destroy": (ctypes.c_int, [_P]),
    "rs_set_path": (ctypes.c_int, [ctypes.c_char_p]),
    "rs_gmres_patches": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                        _P]),
    "rs_tc_selftest": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, ctypes.c_int]),
    "rs_probe_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "rs_path_counts": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "rs_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "rs_profile_ncat": (ctypes.c_int, []),
    "rs_launch_count": (ctypes.c_int64, []),
    "rs_profile_nrec": (ctypes.c_int, []),
    "rs_profile_record": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P]),
    "rs_profile_record_start": (ctypes.c_int, [ctypes.c_int, _P]),
    "rs_green": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, _P, ctypes.c_int64, _P]),
    "rs_profile_tiles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _P, _P, _P, _P,
                                         _P, _P, _P, _P]),
    "rs_profile_read": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_char_p)]),
    "rs_last_error": (ctypes.c_char_p, []),
    "rs_version": (ctypes.c_char_p, []),
}
EXPORTED = tuple(_PROTOS)

_lib = None


def load(path: str = LIB_PATH):
    """Load librs.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"librs.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != 0:
        raise RSError(rc, _lib.rs_last_error().decode())


def _ptr(a):
    """Data pointer and (rows, cols, ld, element size) of a 1D/2D column-major array."""
    if hasattr(a, "data_ptr"):   # torch tensor
        if a.dim() == 1:
            return a.data_ptr(), a.shape[0], 1, a.shape[0], a.element_size()
        if a.stride(0) != 1:
            raise ValueError("torch tensor must be column-major (stride(0) == 1)")
        return a.data_ptr(), a.shape[0], a.shape[1], a.stride(1), a.element_size()
    a = np.asarray(a)
    if a.ndim == 1:
        return a.ctypes.data, a.shape[0], 1, a.shape[0], a.itemsize
    if not a.flags["F_CONTIGUOUS"]:
        raise ValueError("numpy array must be Fortran (column-major) ordered")
    return a.ctypes.data, a.shape[0], a.shape[1], a.shape[0], a.itemsize


def _stream(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


class Handle:
    """Owns one rs_handle (compressed inverse on the current device)."""

    def __init__(self, ptr, n, complex_):
        self._h = ptr
        self.n = n
        self.complex = complex_

    @property
    def ptr(self):
        return self._h

    def free(self):
        if self._h:
            _lib.rs_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stats(self) -> dict:
        s = rs_stats_t()
        _check(_lib.rs_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in rs_stats_t._fields_}


ID_ARITH = {"fp64": 0, "dfloat": 1}


def rs_build(points, kernel: str, weight: float, eps: float, leaf: int, proxy_n: int,
             proxy_ratio: float = 1.5, k_wave: float = 0.0, stream=None, id_arith: str = "fp64",
             id_oversample: int = 0, id_seed: int = 0, normals=None, curvature=None) -> Handle:
    """points: (dim, N) array (any order numpy, or a column-major torch tensor).
    id_arith: "fp64" or "dfloat" (arithmetic of the ID's pivoted QR, rs_id_arith).
    id_oversample > 0: randomized ID with n + id_oversample sample rows (seed id_seed).
    normals (2, N) and curvature (N,): the double-layer kernel's geometry (host arrays)."""
    load()
    if hasattr(points, "data_ptr"):
        dim, n = points.shape
        pts = points.t().contiguous() if points.stride(1) != dim else points   # point-major
        ptr = pts.data_ptr()
        keep = pts
    else:
        pts = np.asfortranarray(np.asarray(points, dtype=np.float64))
        dim, n = pts.shape
        ptr = pts.ctypes.data
        keep = pts
    keep_dl, pn, pk = _dlayer(normals, curvature)
    p = rs_params(KERNELS[kernel], float(k_wave), float(weight), int(proxy_n), float(proxy_ratio),
                  ID_ARITH[id_arith], int(id_oversample), int(id_seed), pn, pk)
    out = ctypes.c_void_p()
    rc = _lib.rs_build(ptr, n, dim, ctypes.byref(p), float(eps), int(leaf), _stream(stream), ctypes.byref(out))
    del keep, keep_dl
    _check(rc)
    return Handle(out.value, n, kernel in COMPLEX_KERNELS)


def rs_solve(h: Handle, B, X, precision: int = RS_PREC_FP64, stream=None):
    pb, nb, rb, ldb, _ = _ptr(B)
    px, nx, rx, ldx, _ = _ptr(X)
    _check(_lib.rs_solve(h.ptr, precision, pb, ldb, rb, px, ldx, _stream(stream)))
    return X


def rs_solve_noalloc(h: Handle, B, X, precision: int = RS_PREC_FP64, stream=None):
    """rs_solve without any device allocation (B and X must be device tensors)."""
    pb, nb, rb, ldb, _ = _ptr(B)
    px, nx, rx, ldx, _ = _ptr(X)
    _check(_lib.rs_solve_noalloc(h.ptr, precision, pb, ldb, rb, px, ldx, _stream(stream)))
    return X


def rs_solve_refined(h: Handle, B, X, tol: float = 1e-10, max_it: int = 10, stream=None):
    pb, nb, rb, ldb, _ = _ptr(B)
    px, nx, rx, ldx, _ = _ptr(X)
    its = ctypes.c_int(0)
    rel = np.zeros(rb)
    _check(_lib.rs_solve_refined(h.ptr, pb, ldb, rb, px, ldx, float(tol), int(max_it), ctypes.byref(its),
                                 rel.ctypes.data, _stream(stream)))
    return its.value, rel


def rs_matvec(h: Handle, X, Y, stream=None):
    px, nx, rx, ldx, _ = _ptr(X)
    py, ny, ry, ldy, _ = _ptr(Y)
    _check(_lib.rs_matvec(h.ptr, px, ldx, rx, py, ldy, _stream(stream)))
    return Y


def rs_tree_perm(h: Handle) -> np.ndarray:
    out = np.zeros(h.n, dtype=np.int64)
    _check(_lib.rs_tree_perm(h.ptr, out.ctypes.data))
    return out


def rs_tree_level(h: Handle, level: int):
    nbox = ctypes.c_int(0)
    _check(_lib.rs_tree_level(h.ptr, level, ctypes.byref(nbox), None, None, None, None))
    nb = nbox.value
    begin = np.zeros(nb, dtype=np.int64)
    parent = np.zeros(nb, dtype=np.int32)
    ncoll = np.zeros(nb, dtype=np.int32)
    coll = np.zeros(nb * 27, dtype=np.int32)
    _check(_lib.rs_tree_level(h.ptr, level, ctypes.byref(nbox), begin.ctypes.data, parent.ctypes.data,
                              ncoll.ctypes.data, coll.ctypes.data))
    coll = coll.reshape(nb, 27)
    return dict(begin=begin, parent=parent, colleagues=[coll[b, :ncoll[b]].copy() for b in range(nb)])


def rs_box_ranks(h: Handle, level: int, nbox: int):
    n = np.zeros(nbox, dtype=np.int32)
    k = np.zeros(nbox, dtype=np.int32)
    _check(_lib.rs_box_ranks(h.ptr, level, n.ctypes.data, k.ctypes.data))
    return n, k


def rs_profile_enable(on=True):
    """True/1: time every launch; 2: also record tile timelines (rs_profile_tiles); False/0: off."""
    _check(load().rs_profile_enable(2 if on == 2 else (1 if on else 0)))


def rs_profile_read() -> dict:
    """{category: dict(ms, launches, bytes, flops)} of the recorded launches."""
    lib = load()
    out = {}
    for c in range(lib.rs_profile_ncat()):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        by = ctypes.c_double()
        fl = ctypes.c_double()
        name = ctypes.c_char_p()
        _check(lib.rs_profile_read(c, ctypes.addressof(ms), ctypes.addressof(n), ctypes.addressof(by),
                                   ctypes.addressof(fl), ctypes.byref(name)))
        if n.value:
            out[name.value.decode()] = dict(ms=ms.value, launches=n.value, bytes=by.value, flops=fl.value)
    return out


def rs_profile_records(with_start: bool = False) -> list:
    """[(category index, ms, bytes, flops[, start ms])] of the recorded launches, in order;
    start is measured from the start of the first record."""
    lib = load()
    out = []
    for i in range(lib.rs_profile_nrec()):
        cat = ctypes.c_int()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        fl = ctypes.c_double()
        _check(lib.rs_profile_record(i, ctypes.addressof(cat), ctypes.addressof(ms), ctypes.addressof(by),
                                     ctypes.addressof(fl)))
        rec = (cat.value, ms.value, by.value, fl.value)
        if with_start:
            t0 = ctypes.c_double()
            _check(lib.rs_profile_record_start(i, ctypes.addressof(t0)))
            rec = rec + (t0.value,)
        out.append(rec)
    return out


def rs_profile_tiles(h: "Handle", mode: int, nrhs: int) -> dict:
    """Tile timeline of the last profiled persistent launch of (mode, nrhs): numpy
    arrays kind, depth, row0, ncol, t_claim, t_start, t_end (microseconds)."""
    lib = load()
    cnt = ctypes.c_int64()
    _check(lib.rs_profile_tiles(h.ptr, int(mode), int(nrhs), 0, None, None, None, None, None, None, None,
                                ctypes.byref(cnt)))
    n = cnt.value
    out = {k: np.zeros(n, dtype=np.int32) for k in ("kind", "depth", "row0", "ncol")}
    out.update({k: np.zeros(n, dtype=np.float64) for k in ("t_claim", "t_start", "t_end")})
    _check(lib.rs_profile_tiles(h.ptr, int(mode), int(nrhs), n, out["kind"].ctypes.data, out["depth"].ctypes.data,
                                out["row0"].ctypes.data, out["ncol"].ctypes.data, out["t_claim"].ctypes.data,
                                out["t_start"].ctypes.data, out["t_end"].ctypes.data, ctypes.byref(cnt)))
    return out


def rs_green(kernel: str, s2, k_wave: float = 0.0) -> np.ndarray:
    """The device evaluation of G at squared distances s2 (no weight)."""
    lib = load()
    s2 = np.ascontiguousarray(np.asarray(s2, dtype=np.float64))
    cplx = kernel in COMPLEX_KERNELS
    out = np.zeros(2 * s2.size if cplx else s2.size, dtype=np.float64)
    _check(lib.rs_green(KERNELS[kernel], float(k_wave), s2.ctypes.data, s2.size, out.ctypes.data))
    return out.view(np.complex128) if cplx else out


def rs_probe_fma_peak(precision: int = RS_PREC_FP64) -> float:
    """Measured FMA throughput (GFLOP/s) of the current device."""
    out = ctypes.c_double()
    _check(load().rs_probe_fma_peak(int(precision), ctypes.byref(out)))
    return out.value


def rs_tc_selftest(kind: int, A, B, D):
    """D = A B^T on the tensor cores (kind 0 tf32, 1 bf16); CUDA float32 tensors."""
    _check(load().rs_tc_selftest(int(kind), A.data_ptr(), B.data_ptr(), D.data_ptr(), int(B.shape[0])))
    return D


def rs_gmres_patches(handles, points, B, X, tol: float = 1e-10, max_it: int = 500, restart: int = 50,
                     precondition: bool = True, stream=None):
    """Block-diagonal RS-preconditioned GMRES on the system coupling the
    patches (handles in patch order; points (dim, n) of all patches in the
    same order; B, X length-n vectors).  Returns (iterations, relres)."""
    lib = load()
    arr = (ctypes.c_void_p * len(handles))(*[h.ptr for h in handles])
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).T)   # point-major
    pb = B.data_ptr() if hasattr(B, "data_ptr") else np.asarray(B).ctypes.data
    px = X.data_ptr() if hasattr(X, "data_ptr") else np.asarray(X).ctypes.data
    its = ctypes.c_int()
    rel = ctypes.c_double()
    _check(lib.rs_gmres_patches(len(handles), arr, pts.ctypes.data, pb, px, float(tol), int(max_it), int(restart),
                                1 if precondition else 0, ctypes.byref(its), ctypes.byref(rel), _stream(stream)))
    return its.value, rel.value


def rs_launch_count() -> int:
    return int(load().rs_launch_count())


class Server:
    """Continuous-batching solve server over resident factorizations (rs_server_*)."""

    def __init__(self, max_cols: int = 256, hbm_budget_bytes: int = 0):
        load()
        out = ctypes.c_void_p()
        _check(_lib.rs_server_create(int(max_cols), int(hbm_budget_bytes), ctypes.byref(out)))
        self._s = out.value
        self._keep = {}          # ticket -> buffers kept alive until waited
        self._built = {}         # handle id -> Handle wrapper (not owned)

    def add(self, h: Handle) -> int:
        hid = ctypes.c_int()
        _check(_lib.rs_server_add_handle(self._s, h.ptr, ctypes.byref(hid)))
        return hid.value

    def submit(self, hid: int, B, X, tol: float = 1e-10) -> int:
        pb, nb, rb, ldb, _ = _ptr(B)
        px, nx, rx, ldx, _ = _ptr(X)
        t = ctypes.c_int64()
        _check(_lib.rs_server_submit_solve(self._s, int(hid), pb, ldb, rb, px, ldx, float(tol), ctypes.byref(t)))
        self._keep[t.value] = (B, X)
        return t.value

    def submit_build(self, points, kernel: str, weight: float, eps: float, leaf: int, proxy_n: int,
                     proxy_ratio: float = 1.5, k_wave: float = 0.0, id_arith: str = "fp64", normals=None,
                     curvature=None) -> int:
        pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).T)   # point-major
        n, dim = pts.shape
        keep_dl, pn, pk = _dlayer(normals, curvature)   # copied by the library at submission
        p = rs_params(KERNELS[kernel], float(k_wave), float(weight), int(proxy_n), float(proxy_ratio),
                      ID_ARITH[id_arith], 0, 0, pn, pk)
        t = ctypes.c_int64()
        _check(_lib.rs_server_submit_build(self._s, pts.ctypes.data, n, dim, ctypes.byref(p), float(eps), int(leaf),
                                           ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_s: float = 0.0) -> dict:
        st = ctypes.c_int()
        lat = ctypes.c_double()
        rel = ctypes.c_double()
        res = ctypes.c_int()
        _check(_lib.rs_server_wait(self._s, int(ticket), float(timeout_s), ctypes.byref(st), ctypes.byref(lat),
                                   ctypes.byref(rel), ctypes.byref(res)))
        self._keep.pop(ticket, None)
        return dict(status=st.value, latency_ms=lat.value, relres=rel.value, result=res.value)

    def handle(self, hid: int, n: int, complex_: bool = False) -> Handle:
        """Non-owning wrapper of the handle behind an id (e.g. one the server built)."""
        out = ctypes.c_void_p()
        _check(_lib.rs_server_handle(self._s, int(hid), ctypes.byref(out)))
        h = Handle(out.value, n, complex_)
        h.free = lambda: None   # the server owns it
        return h

    def stats(self) -> dict:
        s = rs_server_stats_t()
        _check(_lib.rs_server_stats(self._s, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in rs_server_stats_t._fields_}

    def reset_stats(self):
        _check(_lib.rs_server_reset_stats(self._s))

    def destroy(self):
        if self._s:
            _lib.rs_server_destroy(self._s)
            self._s = None
            self._keep.clear()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


PATH_NAMES = ("id_cta", "id_cluster", "id_coop", "id_step", "factor_smem", "factor_big", "factor_generic",
              "gj_cluster", "gj_blocked", "gj_coop", "gj_step")


def rs_set_path(spec):
    """Build-path override for tests: e.g. "id:step,gj:coop"; None or "off" restores the selection."""
    _check(load().rs_set_path(None if spec is None else spec.encode()))


def rs_path_counts(reset: bool = False) -> dict:
    """Level launches per build form since the last reset: {name: count}."""
    lib = load()
    out = np.zeros(len(PATH_NAMES), dtype=np.int64)
    n = lib.rs_path_counts(out.ctypes.data, len(PATH_NAMES), 1 if reset else 0)
    if n < 0:
        _check(n)
    return dict(zip(PATH_NAMES, (int(v) for v in out)))


def rs_set_fault(spec):
    """Arm host-side fault injection: "alloc:n", "wait" or "off"."""
    _check(load().rs_set_fault(None if spec is None else spec.encode()))


def rs_free(h: Handle):
    h.free()


def rs_version() -> str:
    return load().rs_version().decode()
