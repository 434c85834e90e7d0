"""CPU oracle for the SMASH H^2 path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``smash_oracle.c``, a plain
serial C implementation written from the paper, through ctypes.  It shares no
code with the CUDA library and never imports it.

Parity status of each part (what pins it is in ``tests/test_oracle_*.py``):
  dense product ............ pinned (numpy/scipy restatement, brute force)
  bounding cube / Morton ... pinned (per-point brute-force cell check)
  tree ..................... pinned (partition invariants, brute force)
  admissibility / lists .... pinned (exact cover, float geometry, perfect-tree counts)
  Lagrange basis ........... pinned (polynomial reproduction, (3.1))
  compr / SRRQR ............ pinned (ID identity rows, |G| <= f, Lemma 4.1,
                             singular-value bounds vs dense SVD, scipy QRCP)
  H^2 matvec ............... pinned (dense on small/trivial trees, symmetry,
                             telescoping form (3.21)-(3.26) on perfect trees,
                             error falling with the order)
  |H^2| row scales ......... pinned (dense sum |kappa||q| when nothing is
                             admissible; triangle inequality against the
                             matvec; not below the dense sum |kappa||q| by
                             more than the approximation error)
  parameter heuristic ...... pinned (the three worked values of Section 6.1)
  Taylor basis on C ........ pinned ((2.4) with the coefficients (2.5) within
                             the bound (2.6); eta, powers and factorials)
  complex compr ............ pinned (LAPACK's complex QRCP, rank, |A| <= f,
                             volume growth of each swap)
  complex H^2 matvec ....... pinned (dense when the root is a leaf,
                             antisymmetry of 1/(x-y), error falling with r,
                             the error magnitudes of Table 6.1)
  Jacobi truncated SVD ..... pinned (singular values and subspaces of
                             LAPACK's SVD, orthogonality)
  HSS construction ......... pinned (exact cover by (3.5), the bound on
                             |N_i| and the empty third case of Appendix A
                             for uniform points, dense when the root is a
                             leaf, |G| <= f, error falling with eps_svd,
                             antisymmetry of 1/(x-y))
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smash_oracle.c")
_OUT = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT, "liboracle.so")
# ORACLE_OPENMP=1 loads the same source built with -fopenmp (threads from
# OMP_NUM_THREADS): identical results, node and row loops on several cores;
# used only to report a multi-core CPU baseline beside the serial one
_OMP_PATH = os.path.join(_OUT, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None

KERNEL_LOG, KERNEL_INVR, KERNEL_YUKAWA, KERNEL_CAUCHY = 0, 1, 2, 3
KERNEL_DLP1, KERNEL_DLP2 = 4, 5  # y-gradient of -(1/2 pi) log|x - y| (Section 6.4), d = 2

_Q = dict(nx=0, ny=1, L=2, nnodes=3, nadm=4, nnear=5, same=6, skel_row=7, rest_row=8,
          g_row=9, skel_col=10, rest_col=11, g_col=12, r=13, swaps_row=14, swaps_col=15,
          badswap=16, nnf=17)


def _compile(path: str, extra, force: bool) -> str:
    if not force and os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", *extra,
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/_build:
    the serial library and its -fopenmp twin."""
    os.makedirs(_OUT, exist_ok=True)
    _compile(_OMP_PATH, ["-fopenmp"], force)
    return _compile(_LIB_PATH, [], force)


def openmp() -> bool:
    """True when this process loads the -fopenmp build (ORACLE_OPENMP=1)."""
    return os.environ.get("ORACLE_OPENMP", "0") == "1"


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_OMP_PATH if openmp() else _LIB_PATH)
        P = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int, C.c_double
        lib.orc_build.restype = P
        lib.orc_build.argtypes = [P, i64, P, i64, i32, i32, i32, i32, dbl, dbl, dbl]
        lib.orc_free.argtypes = [P]
        lib.orc_free.restype = None
        lib.orc_matvec.argtypes = [P, P, P, i32]
        lib.orc_matvec_leaves.argtypes = [P, P, P, i32, P, i64]
        lib.orc_matvec_leaves.restype = i32
        lib.orc_matvec_abs.argtypes = [P, P, P, i32, P, i64]
        lib.orc_matvec_abs.restype = i32
        lib.orc_dense_rows.argtypes = [P, i64, P, i64, i32, i32, P, i32, P, i64, P]
        lib.orc_dense_rows.restype = None
        lib.orc_query.restype = i64
        lib.orc_query.argtypes = [P, i32]
        lib.orc_kernel.restype = dbl
        lib.orc_kernel.argtypes = [i32, i32, P, P]
        lib.orc_suggest_rank.restype = i32
        lib.orc_suggest_rank.argtypes = [dbl, dbl]
        lib.orc_bits_per_dim.restype = i32
        lib.orc_bits_per_dim.argtypes = [i32]
        lib.orc_bounding_cube.argtypes = [P, i64, P, i64, i32, P, P]
        lib.orc_bounding_cube.restype = None
        lib.orc_morton_keys.argtypes = [P, i64, i32, P, dbl, P]
        lib.orc_morton_keys.restype = None
        lib.orc_admissible.restype = i32
        lib.orc_admissible.argtypes = [i32, i32, P, i32, P, dbl]
        lib.orc_chebyshev.argtypes = [i32, P]
        lib.orc_chebyshev.restype = None
        lib.orc_lagrange.restype = dbl
        lib.orc_lagrange.argtypes = [i32, P, P, i32, dbl]
        lib.orc_lagrange_weights.restype = None
        lib.orc_lagrange_weights.argtypes = [i32, P, P]
        lib.orc_basis_t.argtypes = [i32, i32, P, P, dbl, i32, P, P, i32, P]
        lib.orc_basis_t.restype = None
        lib.orc_compr.restype = i32
        lib.orc_compr.argtypes = [P, i32, i32, dbl, dbl, P, P, P, P]
        lib.orc_export_geometry.argtypes = [P, P, P, P, P, P, P]
        lib.orc_export_geometry.restype = None
        lib.orc_export_nodes.argtypes = [P] * 12
        lib.orc_export_nodes.restype = None
        lib.orc_export_lists.argtypes = [P] * 5
        lib.orc_export_lists.restype = None
        lib.orc_export_comp.argtypes = [P, i32, P, P, P, P, P]
        lib.orc_export_comp.restype = None
        lib.orc_taylor_coefficients.argtypes = [i32, P]
        lib.orc_taylor_coefficients.restype = None
        lib.orc_taylor_basis_t.argtypes = [i32, P, dbl, dbl, dbl, P, i32, P]
        lib.orc_taylor_basis_t.restype = None
        lib.orc_compr_c.argtypes = [P, i32, i32, dbl, dbl, P, P, P, P]
        lib.orc_compr_c.restype = i32
        lib.orc_build_taylor.restype = P
        lib.orc_build_taylor.argtypes = [P, i64, i32, i32, dbl, dbl, dbl, dbl, dbl]
        lib.orc_matvec_taylor.argtypes = [P, P, P, i32, i32]
        lib.orc_matvec_taylor.restype = i32
        lib.orc_dense_rows_taylor.argtypes = [P, i64, P, i32, P, i64, dbl, dbl, P]
        lib.orc_dense_rows_taylor.restype = None
        lib.orc_export_taylor.argtypes = [P] * 6
        lib.orc_export_taylor.restype = None
        lib.orc_build_hss.restype = P
        lib.orc_build_hss.argtypes = [P, i64, P, i64, i32, i32, i32, dbl, dbl, dbl, dbl]
        lib.orc_export_hss.argtypes = [P, P, P, P, P]
        lib.orc_export_hss.restype = None
        lib.orc_jacobi_rows.argtypes = [P, i32, i32, P, P]
        lib.orc_jacobi_rows.restype = i32
        lib.orc_truncated_svd_rows.argtypes = [P, i32, i32, dbl, P]
        lib.orc_truncated_svd_rows.restype = i32
        lib.orc_cauchy_c_entry.argtypes = [P, P, dbl, dbl, P]
        lib.orc_cauchy_c_entry.restype = dbl
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# building blocks (each a step of the paper, exposed for the pins)
# --------------------------------------------------------------------------

def kernel(kid: int, x, y) -> float:
    """kappa(x, y) with value 0 at coincident points ((2.1) with d_x = 0)."""
    x, y = _f64(x).ravel(), _f64(y).ravel()
    return _load().orc_kernel(kid, len(x), _ptr(x), _ptr(y))


def dense_rows(x, kid: int, q, rows=None, y=None) -> np.ndarray:
    """Brute-force rows of A q with Neumaier summation; A_ij = kappa(x_i, y_j)."""
    x = _f64(x)
    y = x if y is None else _f64(y)
    q = _f64(q)
    if q.ndim == 1:
        q = q[:, None]
    nrhs = q.shape[1]
    rows = np.arange(len(x), dtype=np.int64) if rows is None else np.ascontiguousarray(rows, np.int64)
    out = np.empty((len(rows), nrhs))
    _load().orc_dense_rows(_ptr(x), len(x), _ptr(y), len(y), x.shape[1], kid, _ptr(q), nrhs,
                           _ptr(rows), len(rows), _ptr(out))
    return out


def suggest_rank(eps: float, tau: float) -> int:
    """The farfield rank heuristic of Section 6.1."""
    return _load().orc_suggest_rank(eps, tau)


def bits_per_dim(d: int) -> int:
    return _load().orc_bits_per_dim(d)


def bounding_cube(x, y=None):
    x = _f64(x)
    d = x.shape[1]
    lo = np.zeros(3)
    s = np.zeros(1)
    yy = None if y is None else _f64(y)
    _load().orc_bounding_cube(_ptr(x), len(x), _ptr(yy), 0 if yy is None else len(yy), d,
                              _ptr(lo), _ptr(s))
    return lo[:d].copy(), float(s[0])


def morton_keys(pts, lo, s) -> np.ndarray:
    pts = _f64(pts)
    lo = _f64(np.concatenate([np.asarray(lo, np.float64), np.zeros(3)])[:3])
    keys = np.empty(len(pts), dtype=np.uint64)
    _load().orc_morton_keys(_ptr(pts), len(pts), pts.shape[1], _ptr(lo), float(s), _ptr(keys))
    return keys


def admissible(d: int, li: int, ci, lj: int, cj, tau: float) -> bool:
    ci = np.ascontiguousarray(list(ci) + [0] * (3 - len(ci)), dtype=np.uint64)
    cj = np.ascontiguousarray(list(cj) + [0] * (3 - len(cj)), dtype=np.uint64)
    return bool(_load().orc_admissible(d, li, _ptr(ci), lj, _ptr(cj), tau))


def chebyshev(p: int) -> np.ndarray:
    t = np.empty(p)
    _load().orc_chebyshev(p, _ptr(t))
    return t


def lagrange(p: int, m: int, t: float, anchors=None) -> float:
    anchors = chebyshev(p) if anchors is None else _f64(anchors)
    w = np.empty(p)
    _load().orc_lagrange_weights(p, _ptr(anchors), _ptr(w))
    return _load().orc_lagrange(p, _ptr(anchors), _ptr(w), m, float(t))


def basis_t(pts, p: int, lo, s: float, level: int, cell, anchors=None) -> np.ndarray:
    """U^^T (r x npts) of the cell (level, cell) of the cube [lo, lo+s]^d."""
    pts = _f64(pts)
    d = pts.shape[1]
    anchors = chebyshev(p) if anchors is None else _f64(anchors)
    lo3 = _f64(np.concatenate([np.asarray(lo, np.float64), np.zeros(3)])[:3])
    cell3 = np.ascontiguousarray(list(cell) + [0] * (3 - len(cell)), dtype=np.uint64)
    r = p ** d
    Mt = np.empty((r, len(pts)))
    _load().orc_basis_t(d, p, _ptr(anchors), _ptr(lo3), float(s), level, _ptr(cell3), _ptr(pts),
                        len(pts), _ptr(Mt))
    return Mt


def compr(Mt, tol: float, f: float = 2.0):
    """Strong RRQR / ID of the r x m matrix Mt (Theorem 2.4, (2.11)).

    Returns (perm, k, A, nswaps): perm[:k] are the selected columns, perm[k:]
    the others, A = R11^{-1} R12 (k x (m-k)), so that in exact arithmetic
    Mt[:, perm[k:]] ~= Mt[:, perm[:k]] @ A."""
    Mt = _f64(Mt)
    r, m = Mt.shape
    perm = np.empty(m, dtype=np.int32)
    kmax = min(r, m)
    A = np.zeros(max(kmax * max(m - 1, 0) + 1, 1))
    k = C.c_int(0)
    ns = C.c_int(0)
    _load().orc_compr(_ptr(Mt), r, m, tol, f, _ptr(perm), C.byref(k), _ptr(A), C.byref(ns))
    k = k.value
    return perm, k, A[: k * (m - k)].reshape(k, m - k).copy(), ns.value


# --------------------------------------------------------------------------
# the whole H^2 construction and matvec
# --------------------------------------------------------------------------

class H2:
    """Oracle H^2 approximation of A = [kappa(x_i, y_j)] (Section 3.3.2)."""

    def __init__(self, x, kernel: int, leaf: int, order: int, tol: float, y=None,
                 tau: float = 0.7, f: float = 2.0):
        lib = _load()
        self.x = _f64(x)
        self.y = None if y is None else _f64(y)
        self.d = self.x.shape[1]
        self.kernel, self.leaf, self.order, self.tol, self.tau, self.f = kernel, leaf, order, tol, tau, f
        ny = 0 if self.y is None else len(self.y)
        h = lib.orc_build(_ptr(self.x), len(self.x), _ptr(self.y), ny, self.d, kernel, leaf, order,
                          tau, tol, f)
        if not h:
            raise ValueError("oracle: invalid input")
        self._h = C.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_free(h)
            self._h = None

    def query(self, what: str) -> int:
        return int(_load().orc_query(self._h, _Q[what]))

    def matvec(self, q) -> np.ndarray:
        q = _f64(q)
        squeeze = q.ndim == 1
        if squeeze:
            q = q[:, None]
        q = np.ascontiguousarray(q)
        z = np.empty((self.query("nx"), q.shape[1]))
        _load().orc_matvec(self._h, _ptr(q), _ptr(z), q.shape[1])
        return z[:, 0] if squeeze else z

    def matvec_leaves(self, q, leaves) -> np.ndarray:
        """Rows of A^ q for the points of the given leaf gids (other rows NaN),
        computed exactly as matvec() computes them."""
        q = np.ascontiguousarray(_f64(q))
        if q.ndim == 1:
            q = q[:, None]
        leaves = np.ascontiguousarray(leaves, dtype=np.int32)
        z = np.full((self.query("nx"), q.shape[1]), np.nan)
        st = _load().orc_matvec_leaves(self._h, _ptr(q), _ptr(z), q.shape[1], _ptr(leaves), len(leaves))
        if st != 0:
            raise ValueError("matvec_leaves: not a leaf gid")
        return z

    def matvec_abs(self, q, leaves=None) -> np.ndarray:
        """Row scales of A^ q: the matvec with every factor (q, G, kappa)
        replaced by its magnitude, so each entry is the sum of |terms| that
        matvec() adds up for it -- the scale of its rounding error.  With
        leaves, only the rows of those leaf gids are computed (others NaN)."""
        q = np.ascontiguousarray(_f64(q))
        if q.ndim == 1:
            q = q[:, None]
        nx = self.query("nx")
        if leaves is None:
            z = np.empty((nx, q.shape[1]))
            _load().orc_matvec_abs(self._h, _ptr(q), _ptr(z), q.shape[1], None, 0)
            return z
        leaves = np.ascontiguousarray(leaves, dtype=np.int32)
        z = np.full((nx, q.shape[1]), np.nan)
        st = _load().orc_matvec_abs(self._h, _ptr(q), _ptr(z), q.shape[1], _ptr(leaves), len(leaves))
        if st != 0:
            raise ValueError("matvec_abs: not a leaf gid")
        return z

    def export(self) -> dict:
        """Every array of the representation, in the layout shared by the
        library's smash_export (documented in include/smash.h)."""
        e = self.export_structure()
        lib = _load()
        nn = self.query("nnodes")
        for side, tag in ((0, "row"), (1, "col")):
            e[f"m_{tag}"] = np.empty(nn, np.int32)
            e[f"k_{tag}"] = np.empty(nn, np.int32)
            e[f"skel_{tag}"] = np.empty(self.query(f"skel_{tag}"), np.int64)
            e[f"rest_{tag}"] = np.empty(self.query(f"rest_{tag}"), np.int64)
            e[f"G_{tag}"] = np.empty(self.query(f"g_{tag}"), np.float64)
            lib.orc_export_comp(self._h, side, _ptr(e[f"m_{tag}"]), _ptr(e[f"k_{tag}"]),
                                _ptr(e[f"skel_{tag}"]), _ptr(e[f"rest_{tag}"]), _ptr(e[f"G_{tag}"]))
        e["swaps_row"] = self.query("swaps_row")
        e["badswap"] = self.query("badswap")
        return e

    def export_structure(self) -> dict:
        """Points, tree and lists (the part shared by every representation)."""
        lib = _load()
        nx, ny, L, nn = (self.query(k) for k in ("nx", "ny", "L", "nnodes"))
        nadm, nnear = self.query("nadm"), self.query("nnear")
        e = {}
        lo = np.zeros(3)
        s = np.zeros(1)
        e["permx"] = np.empty(nx, np.int64)
        e["permy"] = np.empty(ny, np.int64)
        e["keyx"] = np.empty(nx, np.uint64)
        e["keyy"] = np.empty(ny, np.uint64)
        lib.orc_export_geometry(self._h, _ptr(lo), _ptr(s), _ptr(e["permx"]), _ptr(e["permy"]),
                                _ptr(e["keyx"]), _ptr(e["keyy"]))
        e["lo"], e["s"] = lo[: self.d].copy(), float(s[0])
        e["L"] = L
        e["lvl_off"] = np.empty(L + 1, np.int64)
        for name, dt in (("level", np.int32), ("leaf", np.int32), ("parent", np.int32),
                         ("child0", np.int32), ("nchild", np.int32), ("rs", np.int64),
                         ("rc", np.int64), ("cs", np.int64), ("cc", np.int64)):
            e[name] = np.empty(nn, dt)
        e["cell"] = np.empty((nn, 3), np.uint64)
        lib.orc_export_nodes(self._h, _ptr(e["lvl_off"]), _ptr(e["level"]), _ptr(e["leaf"]),
                             _ptr(e["parent"]), _ptr(e["child0"]), _ptr(e["nchild"]), _ptr(e["rs"]),
                             _ptr(e["rc"]), _ptr(e["cs"]), _ptr(e["cc"]), _ptr(e["cell"]))
        e["adm_ptr"] = np.empty(nn + 1, np.int64)
        e["near_ptr"] = np.empty(nn + 1, np.int64)
        e["adm_col"] = np.empty(nadm, np.int32)
        e["near_col"] = np.empty(nnear, np.int32)
        lib.orc_export_lists(self._h, _ptr(e["adm_ptr"]), _ptr(e["adm_col"]), _ptr(e["near_ptr"]),
                             _ptr(e["near_col"]))
        return e


# --------------------------------------------------------------------------
# Section 2.1: the Taylor expansion (2.4)-(2.5) of 1/(x - y) on C
# --------------------------------------------------------------------------

def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def cauchy_c(x, y, dx=1.0 + 0.0j) -> complex:
    """kappa of (2.1) on C: 1/(x - y), d_x where x = y (points as (re, im))."""
    x, y = _f64(x).ravel(), _f64(y).ravel()
    im = C.c_double(0.0)
    re = _load().orc_cauchy_c_entry(_ptr(x), _ptr(y), float(dx.real), float(dx.imag), C.byref(im))
    return complex(re, im.value)


def taylor_coefficients(r: int) -> np.ndarray:
    """cl[l] = (l/e) (2 pi r)^(1/(2r)), so that eta_{v,l} = (cl[l]/delta_v)^l (2.5)."""
    cl = np.empty(r)
    _load().orc_taylor_coefficients(r, _ptr(cl))
    return cl


def taylor_basis_t(pts, r: int, centre: complex, delta: float) -> np.ndarray:
    """phi_{a,l}(x - a) of (2.5) for l < r at the points (npts x 2, read as
    x_0 + i x_1): an r x npts complex matrix."""
    pts = _f64(pts)
    cl = taylor_coefficients(r)
    Mt = np.empty((r, len(pts)), np.complex128)
    _load().orc_taylor_basis_t(r, _ptr(cl), float(centre.real), float(centre.imag), float(delta), _ptr(pts),
                               len(pts), C.c_void_p(Mt.ctypes.data))
    return Mt


def compr_c(Mt, tol: float, f: float = 2.0):
    """Complex strong RRQR / ID of the r x m matrix Mt (Theorem 2.4, (2.11)):
    (perm, k, A, nswaps) with Mt[:, perm[k:]] ~= Mt[:, perm[:k]] @ A."""
    Mt = _c128(Mt)
    r, m = Mt.shape
    perm = np.empty(m, dtype=np.int32)
    kmax = min(r, m)
    A = np.zeros(max(kmax * max(m - 1, 0) + 1, 1), np.complex128)
    k = C.c_int(0)
    ns = C.c_int(0)
    _load().orc_compr_c(C.c_void_p(Mt.ctypes.data), r, m, tol, f, _ptr(perm), C.byref(k),
                        C.c_void_p(A.ctypes.data), C.byref(ns))
    k = k.value
    return perm, k, A[: k * (m - k)].reshape(k, m - k).copy(), ns.value


def dense_rows_taylor(x, q, rows=None, dx=1.0 + 0.0j) -> np.ndarray:
    """Brute-force rows of A q for kappa of (2.1) on C (Neumaier sums)."""
    x = _f64(x)
    q = _c128(q)
    if q.ndim == 1:
        q = q[:, None]
    nrhs = q.shape[1]
    rows = np.arange(len(x), dtype=np.int64) if rows is None else np.ascontiguousarray(rows, np.int64)
    out = np.empty((len(rows), nrhs), np.complex128)
    _load().orc_dense_rows_taylor(_ptr(x), len(x), C.c_void_p(q.ctypes.data), nrhs, _ptr(rows), len(rows),
                                  float(dx.real), float(dx.imag), C.c_void_p(out.ctypes.data))
    return out


class H2Taylor(H2):
    """Oracle H^2 approximation of A = [kappa(x_i, x_j)] with kappa of (2.1)
    on C (points n x 2 read as x_0 + i x_1, X = Y), bases from the Taylor
    expansion (2.4) with r terms (Sections 2.1 and 3.3.2)."""

    def __init__(self, x, leaf: int, r: int, tol: float, tau: float = 0.65, f: float = 2.0,
                 dx: complex = 1.0 + 0.0j):
        lib = _load()
        self.x = _f64(x)
        self.y = None
        self.d = 2
        self.kernel, self.leaf, self.order, self.tol, self.tau, self.f = None, leaf, r, tol, tau, f
        self.r, self.dx = r, complex(dx)
        h = lib.orc_build_taylor(_ptr(self.x), len(self.x), leaf, r, tau, tol, f, self.dx.real, self.dx.imag)
        if not h:
            raise ValueError("oracle: invalid input")
        self._h = C.c_void_p(h)

    def matvec(self, q) -> np.ndarray:
        q = _c128(q)
        squeeze = q.ndim == 1
        if squeeze:
            q = q[:, None]
        q = np.ascontiguousarray(q)
        z = np.empty((self.query("nx"), q.shape[1]), np.complex128)
        _load().orc_matvec_taylor(self._h, C.c_void_p(q.ctypes.data), C.c_void_p(z.ctypes.data), q.shape[1], 0)
        return z[:, 0] if squeeze else z

    def matvec_abs(self, q, leaves=None) -> np.ndarray:
        """Row scales (sums of |terms|) of the complex matvec."""
        q = _c128(q)
        if q.ndim == 1:
            q = q[:, None]
        q = np.ascontiguousarray(q)
        z = np.empty((self.query("nx"), q.shape[1]))
        _load().orc_matvec_taylor(self._h, C.c_void_p(q.ctypes.data), _ptr(z), q.shape[1], 1)
        return z

    def matvec_leaves(self, q, leaves):
        raise NotImplementedError("use matvec() on the Taylor representation")

    def export(self) -> dict:
        e = super().export_structure()
        nn = self.query("nnodes")
        e["m_row"] = np.empty(nn, np.int32)
        e["k_row"] = np.empty(nn, np.int32)
        e["skel_row"] = np.empty(self.query("skel_row"), np.int64)
        e["rest_row"] = np.empty(self.query("rest_row"), np.int64)
        e["G_row"] = np.empty(self.query("g_row"), np.complex128)
        _load().orc_export_taylor(self._h, _ptr(e["m_row"]), _ptr(e["k_row"]), _ptr(e["skel_row"]),
                                  _ptr(e["rest_row"]), C.c_void_p(e["G_row"].ctypes.data))
        return e


# --------------------------------------------------------------------------
# Section 3.3.1 and Appendix A: HSS construction (points on a line)
# --------------------------------------------------------------------------

def jacobi_rows(B):
    """One-sided Jacobi SVD of the rows of B (m x n): (JT, sig, sweeps) with
    B = JT^T B' for mutually orthogonal rows of B' of norms sig."""
    B = np.array(B, dtype=np.float64, order="C")
    m, n = B.shape
    JT = np.empty((m, m))
    sig = np.empty(m)
    sw = _load().orc_jacobi_rows(_ptr(B), m, n, _ptr(JT), _ptr(sig))
    return JT, sig, sw


def truncated_svd_rows(A, eps_svd: float) -> np.ndarray:
    """Left singular vectors of A (m x n) with singular values above eps_svd
    times the largest, descending, as the rows of an s x m array (3.7)."""
    A = np.array(A, dtype=np.float64, order="C")
    m, n = A.shape
    ST = np.empty((max(min(m, n), 1), m))
    s = _load().orc_truncated_svd_rows(_ptr(A), m, n, eps_svd, _ptr(ST))
    return ST[:s].copy()


class HSS(H2):
    """Oracle HSS approximation (Section 3.3.1) of A = [kappa(x_i, y_j)] for
    points on a line: the binary tree of Section 3.1, L and L^- of (3.5),
    the nearfield sets N_i of (A.1), the truncated SVD of each nearfield
    block row (3.7) joined with the interpolation basis and compressed by
    strong RRQR (3.9)/(3.13); matvec() is the Section 3.4 matvec with these
    lists."""

    def __init__(self, x, kernel: int, leaf: int, order: int, tol: float, eps_svd: float, y=None,
                 tau: float = 0.6, f: float = 2.0):
        lib = _load()
        self.x = _f64(x).reshape(-1, 1)
        self.y = None if y is None else _f64(y).reshape(-1, 1)
        self.d = 1
        self.kernel, self.leaf, self.order, self.tol, self.tau, self.f = kernel, leaf, order, tol, tau, f
        self.eps_svd = eps_svd
        ny = 0 if self.y is None else len(self.y)
        h = lib.orc_build_hss(_ptr(self.x), len(self.x), _ptr(self.y), ny, kernel, leaf, order, tau, tol,
                              eps_svd, f)
        if not h:
            raise ValueError("oracle: invalid input")
        self._h = C.c_void_p(h)

    def export(self) -> dict:
        e = super().export()
        nn = self.query("nnodes")
        e["nf_ptr"] = np.empty(nn + 1, np.int64)
        lib = _load()
        e["nf_col"] = np.empty(max(1, self.query("nnf")), np.int32)
        e["svd_row"] = np.empty(nn, np.int32)
        e["svd_col"] = np.empty(nn, np.int32)
        lib.orc_export_hss(self._h, _ptr(e["nf_ptr"]), _ptr(e["nf_col"]), _ptr(e["svd_row"]), _ptr(e["svd_col"]))
        e["nf_col"] = e["nf_col"][: e["nf_ptr"][-1]].copy()
        return e
