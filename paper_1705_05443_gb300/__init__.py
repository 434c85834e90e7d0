"""Python binding of libsmash.so, the GB300 CUDA library for SMASH H^2
matrices (construction of Section 3.3.2, matvec of Section 3.4).

The functions here carry the names of the C entry points in
``include/smash.h`` and only marshal arguments: every step of the build and of
the matvec runs in the library's CUDA kernels.  Arrays may be torch tensors
(CUDA or CPU) or numpy arrays; device tensors are passed to the library as
device pointers, host arrays as host pointers.

There is no CPU fallback: importing works without a GPU, but every call that
computes needs the compiled library and a CUDA device, and raises otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

__all__ = [
    "SmashError", "smash_build", "smash_build_xy", "smash_build_batch", "smash_matvec", "smash_matvec_ex",
    "smash_matvec_graph", "smash_matvec_graph_count", "smash_matvec_cauchy_like", "smash_matvec_kernel",
    "smash_matvec_double_layer", "SMASH_K_DLP1", "SMASH_K_DLP2", "smash_set_autotune", "smash_autotune_load",
    "smash_autotune_save", "smash_autotune_entries", "smash_autotune_clear", "smash_autotune_lookup",
    "smash_autotune_force",
    "smash_matvec_noalloc", "smash_near_fallback_leaves", "smash_build_taylor", "smash_matvec_complex",
    "smash_build_hss", "smash_export_hss",
    "SMASH_K_CAUCHY_C", "smash_measure_fma_peak", "smash_node_ranks", "smash_free",
    "smash_info", "smash_export", "smash_footprint_bytes", "smash_predict_footprint",
    "smash_suggest_rank", "smash_last_error", "smash_launch_count", "smash_set_profiling",
    "smash_last_profile", "H2Matrix", "SmashServer", "load_library", "library_path",
    "SMASH_K_LOG", "SMASH_K_INVR", "SMASH_K_YUKAWA", "SMASH_K_CAUCHY1D", "SMASH_PREC_F64", "SMASH_PREC_F32X2", "SMASH_PREC_F32",
    "SMASH_PREC_TF32", "SMASH_PREC_BF16", "SMASH_PREC_TF32X3",
    "PROFILE_PHASES",
]

SMASH_K_LOG, SMASH_K_INVR, SMASH_K_YUKAWA, SMASH_K_CAUCHY1D = 0, 1, 2, 3
SMASH_K_DLP1, SMASH_K_DLP2 = 4, 5
SMASH_K_CAUCHY_C = 6
SMASH_PREC_F64 = 0
SMASH_PREC_F32X2 = 1
SMASH_PREC_F32 = 2
SMASH_PREC_TF32 = 3
SMASH_PREC_BF16 = 4
SMASH_PREC_TF32X3 = 5
PROFILE_PHASES = ("geometry", "tree", "lists", "compression", "gather", "near", "upward", "coupling",
                  "downward", "scatter")
_STATUS = {0: "SMASH_OK", 1: "SMASH_EINVAL", 2: "SMASH_ENOMEM", 3: "SMASH_ECUDA", 4: "SMASH_ETIMEOUT",
           5: "SMASH_EDEPTH", 6: "SMASH_ENOTSUP"}


class SmashError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class smash_options(C.Structure):
    _fields_ = [("tau", C.c_double), ("f", C.c_double), ("stream", C.c_void_p)]


class smash_info_t(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("dim", C.c_int), ("kernel_id", C.c_int),
                ("leaf_size", C.c_int), ("order", C.c_int), ("r", C.c_int), ("same", C.c_int),
                ("levels", C.c_int), ("nnodes", C.c_int64), ("nadm", C.c_int64), ("nnear", C.c_int64),
                ("nleaves", C.c_int64), ("skel_row", C.c_int64), ("rest_row", C.c_int64),
                ("g_row", C.c_int64), ("skel_col", C.c_int64), ("rest_col", C.c_int64),
                ("g_col", C.c_int64), ("swaps", C.c_int64), ("swap_cap_hits", C.c_int64),
                ("coupling_pairs", C.c_int64), ("near_pairs", C.c_int64), ("lo", C.c_double * 3),
                ("s", C.c_double), ("tau", C.c_double), ("f", C.c_double), ("tol", C.c_double),
                ("footprint_bytes", C.c_size_t), ("nproblems", C.c_int64)]


_EXPORT_FIELDS = ["permx", "permy", "keyx", "keyy", "lvl_off", "level", "leaf", "parent", "child0",
                  "nchild", "rs", "rc", "cs", "cc", "cell", "adm_ptr", "adm_col", "near_ptr", "near_col",
                  "m_row", "k_row", "skel_row", "rest_row", "G_row", "m_col", "k_col", "skel_col",
                  "rest_col", "G_col", "node_problem", "problem_cube"]


class smash_export_t(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in _EXPORT_FIELDS]


_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build: bool = True):
    """Load libsmash.so (compiling it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"the SMASH CUDA library is missing ({_build.LIB}); build it with "
                           "paper_1705_05443_gb300._build.build()")
    lib = C.CDLL(_build.LIB)
    P, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    lib.smash_default_options.argtypes = [P]
    lib.smash_default_options.restype = None
    lib.smash_build.argtypes = [P, i32, i64, i32, i32, i32, dbl, C.POINTER(P)]
    lib.smash_build.restype = i32
    lib.smash_build_xy.argtypes = [P, i64, P, i64, i32, i32, i32, i32, dbl, P, C.POINTER(P)]
    lib.smash_build_xy.restype = i32
    lib.smash_build_batch.argtypes = [P, P, i32, i32, i32, i32, i32, dbl, P, C.POINTER(P)]
    lib.smash_build_batch.restype = i32
    lib.smash_build_taylor.argtypes = [P, i64, i32, i32, dbl, dbl, dbl, dbl, C.POINTER(P)]
    lib.smash_build_taylor.restype = i32
    lib.smash_matvec_complex.argtypes = [P, P, P, i32, P]
    lib.smash_matvec_complex.restype = i32
    lib.smash_build_hss.argtypes = [P, i64, P, i64, i32, i32, i32, dbl, dbl, P, C.POINTER(P)]
    lib.smash_build_hss.restype = i32
    lib.smash_export_hss.argtypes = [P, P, P, i64, P, P, C.POINTER(i64)]
    lib.smash_export_hss.restype = i32
    lib.smash_matvec_kernel.argtypes = [P, i32, P, P, i32, i32, P]
    lib.smash_matvec_kernel.restype = i32
    lib.smash_matvec_double_layer.argtypes = [P, P, P, P, P, P, i32, i32, P]
    lib.smash_matvec_double_layer.restype = i32
    lib.smash_matvec_cauchy_like.argtypes = [P, P, P, i32, P, P, i32, i32, P]
    lib.smash_matvec_cauchy_like.restype = i32
    lib.smash_matvec_graph.argtypes = [P, P, P, i32, i32, P]
    lib.smash_matvec_graph.restype = i32
    lib.smash_matvec_graph_count.argtypes = [P]
    lib.smash_matvec_graph_count.restype = i32
    lib.smash_set_autotune.argtypes = [i32]
    lib.smash_set_autotune.restype = None
    lib.smash_autotune_load.argtypes = [C.c_char_p]
    lib.smash_autotune_load.restype = i32
    lib.smash_autotune_save.argtypes = [C.c_char_p]
    lib.smash_autotune_save.restype = i32
    lib.smash_autotune_entries.argtypes = []
    lib.smash_autotune_entries.restype = i32
    lib.smash_autotune_clear.argtypes = []
    lib.smash_autotune_clear.restype = None
    lib.smash_autotune_lookup.argtypes = [C.c_char_p, C.POINTER(i32)]
    lib.smash_autotune_lookup.restype = i32
    lib.smash_autotune_force.argtypes = [C.c_char_p, i32]
    lib.smash_autotune_force.restype = None
    lib.smash_matvec.argtypes = [P, P, P, i32]
    lib.smash_matvec.restype = i32
    lib.smash_matvec_ex.argtypes = [P, P, P, i32, i32, P]
    lib.smash_matvec_ex.restype = i32
    lib.smash_matvec_noalloc.argtypes = [P, P, P, i32, P]
    lib.smash_matvec_noalloc.restype = i32
    lib.smash_free.argtypes = [P]
    lib.smash_free.restype = None
    lib.smash_info.argtypes = [P, P]
    lib.smash_info.restype = i32
    lib.smash_export.argtypes = [P, P]
    lib.smash_export.restype = i32
    lib.smash_near_fallback_leaves.argtypes = [P, P, i64, C.POINTER(i64)]
    lib.smash_near_fallback_leaves.restype = i32
    lib.smash_measure_fma_peak.argtypes = [i32, C.POINTER(dbl)]
    lib.smash_measure_fma_peak.restype = i32
    lib.smash_footprint_bytes.argtypes = [P]
    lib.smash_footprint_bytes.restype = C.c_size_t
    lib.smash_predict_footprint.argtypes = [i64, i32, i32, i32, i32]
    lib.smash_predict_footprint.restype = C.c_size_t
    lib.smash_suggest_rank.argtypes = [dbl, dbl]
    lib.smash_suggest_rank.restype = i32
    lib.smash_last_error.argtypes = []
    lib.smash_last_error.restype = C.c_char_p
    lib.smash_launch_count.argtypes = []
    lib.smash_launch_count.restype = C.c_uint64
    lib.smash_set_profiling.argtypes = [i32]
    lib.smash_set_profiling.restype = None
    lib.smash_last_profile.argtypes = [P, P, i32]
    lib.smash_last_profile.restype = i32
    lib.smash_server_create.argtypes = [i32, C.c_size_t, i32, C.POINTER(P)]
    lib.smash_server_create.restype = i32
    lib.smash_server_submit.argtypes = [P, P, i64, P, i64, i32, i32, i32, i32, dbl, P, i32, P, i32,
                                        C.POINTER(i64)]
    lib.smash_server_submit.restype = i32
    lib.smash_server_apply.argtypes = [P, i64, P, i32, P, C.POINTER(i64)]
    lib.smash_server_apply.restype = i32
    lib.smash_server_wait.argtypes = [P, i64, P]
    lib.smash_server_wait.restype = i32
    lib.smash_server_release.argtypes = [P, i64]
    lib.smash_server_release.restype = i32
    lib.smash_server_max_inflight_seen.argtypes = [P]
    lib.smash_server_max_inflight_seen.restype = i32
    lib.smash_server_destroy.argtypes = [P]
    lib.smash_server_destroy.restype = None
    _lib = lib
    return lib


# ------------------------------------------------------------------ marshalling
def _ptr(a):
    """Data pointer of a torch tensor or numpy array (None stays None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous() or str(a.dtype) != "torch.float64":
            raise ValueError("expected a contiguous float64 tensor")
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"] or a.dtype != np.float64:
            raise ValueError("expected a C-contiguous float64 array")
        return C.c_void_p(a.ctypes.data)
    if isinstance(a, int):
        return C.c_void_p(a)
    raise TypeError(f"unsupported array type {type(a)}")


def _rows(a) -> int:
    return int(a.shape[0])


def _check_shapes(h, X, Y, nrhs: int):
    """X must be ny x nrhs and Y nx x nrhs: the C ABI takes bare pointers and
    cannot check sizes, so an undersized buffer would be read or written out
    of bounds."""
    i = smash_info(h)
    for name, a, rows in (("X", X, i["ny"]), ("Y", Y, i["nx"])):
        shape = tuple(int(v) for v in a.shape)
        if len(shape) != 2 or shape[0] != rows or shape[1] < nrhs:
            raise ValueError(f"{name} must have shape ({rows}, {nrhs}), got {shape}")
        if shape[1] != nrhs:
            raise ValueError(f"{name} must have exactly nrhs = {nrhs} columns (rows are packed), got {shape}")


def _check(st: int):
    if st != 0:
        raise SmashError(st, load_library(False).smash_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# ------------------------------------------------------------------ entry points
def smash_build(points, kernel_id: int, leaf_size: int, order: int, tol: float):
    """smash_build(points, dim, n, ...) -> handle; points is n x dim float64."""
    lib = load_library()
    h = C.c_void_p()
    n, dim = int(points.shape[0]), int(points.shape[1])
    _check(lib.smash_build(_ptr(points), dim, n, kernel_id, leaf_size, order, float(tol), C.byref(h)))
    return h


def smash_build_xy(x, y, kernel_id: int, leaf_size: int, order: int, tol: float, tau: float = 0.7,
                   f: float = 2.0, stream=None):
    lib = load_library()
    h = C.c_void_p()
    opt = smash_options(tau, f, _stream_ptr(stream))
    nx, dim = int(x.shape[0]), int(x.shape[1])
    ny = 0 if y is None else int(y.shape[0])
    _check(lib.smash_build_xy(_ptr(x), nx, _ptr(y), ny, dim, kernel_id, leaf_size, order, float(tol),
                              C.byref(opt), C.byref(h)))
    return h


def smash_build_batch(points, offsets, kernel_id: int, leaf_size: int, order: int, tol: float,
                      tau: float = 0.7, f: float = 2.0, stream=None):
    """Independent problems points[offsets[t]:offsets[t+1]] in one representation (see smash.h)."""
    lib = load_library()
    h = C.c_void_p()
    opt = smash_options(tau, f, _stream_ptr(stream))
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    dim = int(points.shape[1])
    _check(lib.smash_build_batch(_ptr(points), C.c_void_p(off.ctypes.data), len(off) - 1, dim, kernel_id,
                                 leaf_size, order, float(tol), C.byref(opt), C.byref(h)))
    return h


def smash_build_taylor(points, leaf_size: int, r: int, tau: float = 0.65, tol: float = 1e-14,
                       dx: complex = 1.0 + 0.0j):
    """smash_build_taylor: the Taylor representation (2.4) of 1/(x - y) on C
    for n x 2 float64 points (x_0 + i x_1); see smash.h."""
    lib = load_library()
    h = C.c_void_p()
    dx = complex(dx)
    _check(lib.smash_build_taylor(_ptr(points), int(points.shape[0]), leaf_size, r, float(tau), float(tol),
                                  dx.real, dx.imag, C.byref(h)))
    return h


def _cptr(a):
    """Data pointer of a complex128 torch tensor or numpy array (interleaved)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous() or str(a.dtype) != "torch.complex128":
            raise ValueError("expected a contiguous complex128 tensor")
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"] or a.dtype != np.complex128:
            raise ValueError("expected a C-contiguous complex128 array")
        return C.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def smash_matvec_complex(h, X, Y, stream=None):
    """Y = A^ X on a Taylor representation; X, Y n x nrhs complex128."""
    lib = load_library()
    i = smash_info(h)
    nrhs = int(X.shape[1])
    for name, a in (("X", X), ("Y", Y)):
        if tuple(int(v) for v in a.shape) != (i["nx"], nrhs):
            raise ValueError(f"{name} must have shape ({i['nx']}, {nrhs}), got {tuple(a.shape)}")
    _check(lib.smash_matvec_complex(h, _cptr(X), _cptr(Y), nrhs, _stream_ptr(stream)))
    return Y


def smash_build_hss(x, y, kernel_id: int, leaf_size: int, order: int, tol: float, eps_svd: float,
                    tau: float = 0.6, f: float = 2.0, stream=None):
    """smash_build_hss: the HSS representation (Section 3.3.1) for points on
    a line (x: n x 1, y: m x 1 or None); see smash.h."""
    lib = load_library()
    for name, a in (("x", x), ("y", y)):
        if a is not None and (len(a.shape) != 2 or int(a.shape[1]) != 1):
            raise ValueError(f"{name} must be n x 1 (points on a line), got {tuple(a.shape)}")
    h = C.c_void_p()
    opt = smash_options(tau, f, _stream_ptr(stream))
    nx = int(x.shape[0])
    ny = 0 if y is None else int(y.shape[0])
    _check(lib.smash_build_hss(_ptr(x), nx, _ptr(y), ny, kernel_id, leaf_size, order, float(tol), float(eps_svd),
                               C.byref(opt), C.byref(h)))
    return h


def smash_export_hss(h) -> dict:
    """N_i (CSR by node) and the singular vectors per node of an HSS handle."""
    lib = load_library()
    nn = smash_info(h)["nnodes"]
    nnf = C.c_int64(0)
    _check(lib.smash_export_hss(h, None, None, 0, None, None, C.byref(nnf)))
    out = {"nf_ptr": np.empty(nn + 1, np.int64), "nf_col": np.empty(max(nnf.value, 1), np.int32),
           "svd_row": np.empty(nn, np.int32), "svd_col": np.empty(nn, np.int32)}
    _check(lib.smash_export_hss(h, C.c_void_p(out["nf_ptr"].ctypes.data), C.c_void_p(out["nf_col"].ctypes.data),
                                len(out["nf_col"]), C.c_void_p(out["svd_row"].ctypes.data),
                                C.c_void_p(out["svd_col"].ctypes.data), C.byref(nnf)))
    out["nf_col"] = out["nf_col"][: nnf.value].copy()
    return out


def smash_matvec(h, X, Y, nrhs: int | None = None):
    lib = load_library()
    nrhs = int(X.shape[1]) if nrhs is None else nrhs
    _check_shapes(h, X, Y, nrhs)
    _check(lib.smash_matvec(h, _ptr(X), _ptr(Y), nrhs))
    return Y


def smash_matvec_ex(h, X, Y, precision: int = SMASH_PREC_F64, stream=None, nrhs: int | None = None):
    lib = load_library()
    nrhs = int(X.shape[1]) if nrhs is None else nrhs
    _check_shapes(h, X, Y, nrhs)
    _check(lib.smash_matvec_ex(h, _ptr(X), _ptr(Y), nrhs, precision, _stream_ptr(stream)))
    return Y


def smash_matvec_noalloc(h, X, Y, stream=None, nrhs: int | None = None):
    """Y = A^ X without device allocation (X, Y device tensors); see smash.h."""
    lib = load_library()
    nrhs = int(X.shape[1]) if nrhs is None else nrhs
    _check_shapes(h, X, Y, nrhs)
    _check(lib.smash_matvec_noalloc(h, _ptr(X), _ptr(Y), nrhs, _stream_ptr(stream)))
    return Y


def smash_matvec_kernel(h, kernel_id: int, X, Y, precision: int = SMASH_PREC_F64, stream=None):
    """Y = A^_kappa X with another kernel on the same representation (see smash.h)."""
    lib = load_library()
    _check_shapes(h, X, Y, int(X.shape[1]))
    _check(lib.smash_matvec_kernel(h, kernel_id, _ptr(X), _ptr(Y), int(X.shape[1]), precision, _stream_ptr(stream)))
    return Y


def smash_matvec_double_layer(h, nu, wts, diag, X, Y, precision: int = SMASH_PREC_F64, stream=None):
    """Y = K X, the Nystrom double-layer matrix (6.7)/(6.9) on the handle's points (see smash.h)."""
    lib = load_library()
    _check(lib.smash_matvec_double_layer(h, _ptr(nu), _ptr(wts), _ptr(diag), _ptr(X), _ptr(Y), int(X.shape[1]),
                                         precision, _stream_ptr(stream)))
    return Y


def smash_matvec_cauchy_like(h, w, v, X, Y, precision: int = SMASH_PREC_F64, stream=None):
    """Y = sum_l diag(w[:, l]) C^ diag(v[:, l]) X, the Cauchy-like product (6.1)-(6.2)."""
    lib = load_library()
    p = int(w.shape[1])
    _check(lib.smash_matvec_cauchy_like(h, _ptr(w), _ptr(v), p, _ptr(X), _ptr(Y), int(X.shape[1]), precision,
                                        _stream_ptr(stream)))
    return Y


def smash_matvec_graph(h, X, Y, precision: int = SMASH_PREC_F64, stream=None, nrhs: int | None = None):
    """Y = A^ X replayed from a CUDA graph captured at the first call (device X, Y)."""
    lib = load_library()
    nrhs = int(X.shape[1]) if nrhs is None else nrhs
    _check_shapes(h, X, Y, nrhs)
    _check(lib.smash_matvec_graph(h, _ptr(X), _ptr(Y), nrhs, precision, _stream_ptr(stream)))
    return Y


def smash_matvec_graph_count(h) -> int:
    return int(load_library().smash_matvec_graph_count(h))


def smash_set_autotune(on: bool):
    load_library().smash_set_autotune(1 if on else 0)


def smash_autotune_load(path: str) -> int:
    return int(load_library().smash_autotune_load(str(path).encode()))


def smash_autotune_save(path: str):
    lib = load_library()
    _check(lib.smash_autotune_save(str(path).encode()))


def smash_autotune_entries() -> int:
    return int(load_library().smash_autotune_entries())


def smash_autotune_clear():
    load_library().smash_autotune_clear()


def smash_autotune_force(prefix: str, value: int):
    """Every tuned site whose key starts with prefix takes candidate value
    (when valid there); value < 0 removes the override."""
    load_library().smash_autotune_force(prefix.encode(), int(value))


def smash_autotune_lookup(key: str):
    v = C.c_int32(0)
    ok = load_library().smash_autotune_lookup(key.encode(), C.byref(v))
    return int(v.value) if ok else None


def smash_free(h):
    if h is not None and h.value:
        load_library(False).smash_free(h)


def smash_info(h) -> dict:
    lib = load_library()
    info = smash_info_t()
    _check(lib.smash_info(h, C.byref(info)))
    out = {name: getattr(info, name) for name, _ in smash_info_t._fields_}
    out["lo"] = list(info.lo)
    return out


def smash_export(h) -> dict:
    """Host copies of every array of the representation (layout in smash.h)."""
    lib = load_library()
    i = smash_info(h)
    nx, ny, nn, L = i["nx"], i["ny"], i["nnodes"], i["levels"]
    arrs = {
        "permx": np.empty(nx, np.int64), "permy": np.empty(ny, np.int64),
        "keyx": np.empty(nx, np.uint64), "keyy": np.empty(ny, np.uint64),
        "lvl_off": np.empty(L + 1, np.int64),
        "level": np.empty(nn, np.int32), "leaf": np.empty(nn, np.int32), "parent": np.empty(nn, np.int32),
        "child0": np.empty(nn, np.int32), "nchild": np.empty(nn, np.int32),
        "rs": np.empty(nn, np.int64), "rc": np.empty(nn, np.int64), "cs": np.empty(nn, np.int64),
        "cc": np.empty(nn, np.int64), "cell": np.empty((nn, 3), np.uint64),
        "adm_ptr": np.empty(nn + 1, np.int64), "adm_col": np.empty(i["nadm"], np.int32),
        "near_ptr": np.empty(nn + 1, np.int64), "near_col": np.empty(i["nnear"], np.int32),
        "node_problem": np.empty(nn, np.int32), "problem_cube": np.empty((i["nproblems"], 4), np.float64),
    }
    for tag in ("row", "col"):
        arrs[f"m_{tag}"] = np.empty(nn, np.int32)
        arrs[f"k_{tag}"] = np.empty(nn, np.int32)
        arrs[f"skel_{tag}"] = np.empty(i[f"skel_{tag}"], np.int64)
        arrs[f"rest_{tag}"] = np.empty(i[f"rest_{tag}"], np.int64)
        # a Taylor representation (kernel 6) has complex G
        arrs[f"G_{tag}"] = np.empty(i[f"g_{tag}"], np.complex128 if i["kernel_id"] == SMASH_K_CAUCHY_C else np.float64)
    ex = smash_export_t(*[C.c_void_p(arrs[name].ctypes.data) if arrs[name].size else None
                          for name in _EXPORT_FIELDS])
    _check(lib.smash_export(h, C.byref(ex)))
    arrs["L"] = L
    arrs["lo"] = np.array(i["lo"][: i["dim"]])
    arrs["s"] = i["s"]
    return arrs


def smash_near_fallback_leaves(h) -> np.ndarray:
    """Global ids of the leaves the double-float matvec's digit-split near
    field leaves to its double-float kernel (see smash.h)."""
    lib = load_library()
    cnt = C.c_int64(0)
    _check(lib.smash_near_fallback_leaves(h, None, 0, C.byref(cnt)))
    out = np.zeros(max(cnt.value, 1), np.int32)
    _check(lib.smash_near_fallback_leaves(h, C.c_void_p(out.ctypes.data), len(out), C.byref(cnt)))
    return out[: cnt.value].copy()


def smash_measure_fma_peak(fp64: bool) -> float:
    """Measured FMA peak of the current device in TFLOP/s (FP64 or FP32)."""
    v = C.c_double(0.0)
    _check(load_library().smash_measure_fma_peak(1 if fp64 else 0, C.byref(v)))
    return float(v.value)


def smash_node_ranks(h, side: str = "row") -> dict:
    """Per node: level, leaf flag, working-set size m and rank k (one side),
    through smash_export with every other array skipped."""
    lib = load_library()
    i = smash_info(h)
    nn = i["nnodes"]
    arrs = {"level": np.empty(nn, np.int32), "leaf": np.empty(nn, np.int32),
            f"m_{side}": np.empty(nn, np.int32), f"k_{side}": np.empty(nn, np.int32)}
    ex = smash_export_t(*[C.c_void_p(arrs[name].ctypes.data) if name in arrs and nn else None
                          for name in _EXPORT_FIELDS])
    _check(lib.smash_export(h, C.byref(ex)))
    return {"level": arrs["level"], "leaf": arrs["leaf"], "m": arrs[f"m_{side}"], "k": arrs[f"k_{side}"]}


def smash_footprint_bytes(h) -> int:
    return int(load_library().smash_footprint_bytes(h))


def smash_predict_footprint(n: int, dim: int, leaf_size: int, order: int, nrhs: int) -> int:
    return int(load_library().smash_predict_footprint(n, dim, leaf_size, order, nrhs))


def smash_suggest_rank(eps: float, tau: float) -> int:
    return int(load_library().smash_suggest_rank(eps, tau))


def smash_last_error() -> str:
    return load_library(False).smash_last_error().decode()


def smash_launch_count() -> int:
    return int(load_library().smash_launch_count())


def smash_set_profiling(on: bool):
    load_library().smash_set_profiling(1 if on else 0)


def smash_last_profile(h) -> dict:
    ms = np.zeros(len(PROFILE_PHASES))
    n = load_library().smash_last_profile(h, C.c_void_p(ms.ctypes.data), len(ms))
    return dict(zip(PROFILE_PHASES[:n], ms[:n].tolist()))


class smash_request_stats(C.Structure):
    _fields_ = [("queue_ms", C.c_double), ("service_ms", C.c_double), ("latency_ms", C.c_double),
                ("predicted_bytes", C.c_size_t), ("resident_id", C.c_int64), ("points", C.c_int64)]


class SmashServer:
    """The library's request server (smash_server_*): construct-and-apply
    requests admitted by in-flight slots and device-memory budget, run by
    worker threads on their own streams.  Buffers (numpy or torch, host or
    device) are not copied: this wrapper keeps references to them until the
    request has been waited on."""

    def __init__(self, max_inflight: int = 4, mem_budget_bytes: int = 0, precision: int = SMASH_PREC_F64):
        lib = load_library()
        self._s = C.c_void_p()
        _check(lib.smash_server_create(max_inflight, mem_budget_bytes, precision, C.byref(self._s)))
        self._live = {}

    def submit(self, x, kernel_id: int, leaf_size: int, order: int, tol: float, X, y=None, keep: bool = False,
               Y=None) -> int:
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float64)
            X = np.ascontiguousarray(X, dtype=np.float64)
            y = None if y is None else np.ascontiguousarray(y, dtype=np.float64)
        if Y is None:
            Y = X.new_empty((x.shape[0], X.shape[1])) if hasattr(X, "new_empty") else np.empty((x.shape[0], X.shape[1]))
        t = C.c_int64()
        _check(load_library().smash_server_submit(
            self._s, _ptr(x), int(x.shape[0]), _ptr(y), 0 if y is None else int(y.shape[0]), int(x.shape[1]),
            kernel_id, leaf_size, order, float(tol), _ptr(X), int(X.shape[1]), _ptr(Y), 1 if keep else 0,
            C.byref(t)))
        self._live[t.value] = (x, y, X, Y)
        return t.value

    def apply(self, resident_id: int, X, nx: int, Y=None) -> int:
        if isinstance(X, np.ndarray):
            X = np.ascontiguousarray(X, dtype=np.float64)
        if Y is None:
            Y = X.new_empty((nx, X.shape[1])) if hasattr(X, "new_empty") else np.empty((nx, X.shape[1]))
        t = C.c_int64()
        _check(load_library().smash_server_apply(self._s, resident_id, _ptr(X), int(X.shape[1]), _ptr(Y),
                                                 C.byref(t)))
        self._live[t.value] = (None, None, X, Y)
        return t.value

    def wait(self, ticket: int):
        """(Y, stats dict) of a finished request; raises SmashError on failure."""
        st = smash_request_stats()
        code = load_library().smash_server_wait(self._s, ticket, C.byref(st))
        bufs = self._live.pop(ticket, None)
        _check(code)
        return bufs[3], {name: getattr(st, name) for name, _ in smash_request_stats._fields_}

    def release(self, resident_id: int):
        _check(load_library().smash_server_release(self._s, resident_id))

    def max_inflight_seen(self) -> int:
        return int(load_library().smash_server_max_inflight_seen(self._s))

    def close(self):
        if getattr(self, "_s", None) is not None and self._s.value:
            load_library().smash_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class H2Matrix:
    """Owning wrapper: builds on construction, frees on close/garbage collection."""

    def __init__(self, x, kernel_id: int, leaf_size: int, order: int, tol: float, y=None,
                 tau: float = 0.7, f: float = 2.0, stream=None):
        self.nx = _rows(x)
        self.ny = self.nx if y is None else _rows(y)
        if y is None and tau == 0.7 and f == 2.0 and stream is None:
            self.h = smash_build(x, kernel_id, leaf_size, order, tol)
        else:
            self.h = smash_build_xy(x, y, kernel_id, leaf_size, order, tol, tau, f, stream)

    @classmethod
    def batch(cls, points, offsets, kernel_id: int, leaf_size: int, order: int, tol: float,
              tau: float = 0.7, f: float = 2.0, stream=None):
        """Independent problems points[offsets[t]:offsets[t+1]] (smash_build_batch)."""
        self = cls.__new__(cls)
        self.nx = self.ny = _rows(points)
        self.h = smash_build_batch(points, offsets, kernel_id, leaf_size, order, tol, tau, f, stream)
        return self

    def matvec(self, X, Y=None, precision: int = SMASH_PREC_F64, stream=None):
        if Y is None:
            if hasattr(X, "new_empty"):
                Y = X.new_empty((self.nx, X.shape[1]))
            else:
                Y = np.empty((self.nx, X.shape[1]))
        if precision == SMASH_PREC_F64 and stream is None:
            return smash_matvec(self.h, X, Y)
        return smash_matvec_ex(self.h, X, Y, precision, stream)

    def matvec_graph(self, X, Y, precision: int = SMASH_PREC_F64, stream=None):
        return smash_matvec_graph(self.h, X, Y, precision, stream)

    def info(self) -> dict:
        return smash_info(self.h)

    def export(self) -> dict:
        return smash_export(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            smash_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
