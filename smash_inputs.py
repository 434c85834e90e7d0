"""Seeded synthetic point clouds and right-hand sides.

This module is the only code shared by the CPU oracle tests, the GPU parity
tests and the benchmark.  It draws random numbers and nothing else: it holds
none of the method's arithmetic (no tree, no basis, no kernel evaluation).

The workloads mirror the shapes of the paper's test problems (Section 6):
points in the unit square/cube, points on a surface with clustered patches,
Gaussian mixtures, and the mixed 1D Cauchy point sets of Section 6.3, where
each y_j sits a small random offset to the right of x_j, as in (6.3).

Every generator takes an explicit seed; the convention used by the tests and
the benchmark is ``seed = config_index * 1000 + repetition``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "uniform_cube",
    "sphere_with_caps",
    "gaussian_mixture",
    "cauchy_1d",
    "jittered_grid",
    "cauchy_like_6_3",
    "curve_6_4",
    "rhs",
    "sample_rows",
    "batched_problems",
    "WORKLOADS",
    "make_workload",
    "grid_2d",
    "uniform_01",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def uniform_cube(n: int, d: int, seed: int) -> np.ndarray:
    """n points i.i.d. uniform in [0,1]^d, float64, shape (n, d), C order."""
    return np.ascontiguousarray(_rng(seed).random((n, d)), dtype=np.float64)


def sphere_with_caps(n: int, seed: int, frac_caps: float = 0.1, ncaps: int = 8,
                     sigma: float = 0.02) -> np.ndarray:
    """Points on the unit sphere S^2: (1-frac_caps) uniform (normalised
    Gaussian vectors) plus frac_caps spread over ncaps clustered caps, each
    point of cap m being normalise(c_m + sigma * N(0, I_3)) with c_m uniform
    on S^2."""
    g = _rng(seed)
    n_caps = int(round(frac_caps * n))
    n_uni = n - n_caps
    u = g.standard_normal((n_uni, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    c = g.standard_normal((ncaps, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    which = g.integers(0, ncaps, size=n_caps)
    v = c[which] + sigma * g.standard_normal((n_caps, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pts = np.concatenate([u, v], axis=0)
    pts = pts[g.permutation(n)]
    return np.ascontiguousarray(pts, dtype=np.float64)


def gaussian_mixture(n: int, d: int, seed: int, ncomp: int = 4,
                     sigma: float = 0.1) -> np.ndarray:
    """n points from an equal-weight mixture of ncomp isotropic Gaussians with
    means uniform in [0,1]^d and standard deviation sigma."""
    g = _rng(seed)
    means = g.random((ncomp, d))
    which = g.integers(0, ncomp, size=n)
    pts = means[which] + sigma * g.standard_normal((n, d))
    return np.ascontiguousarray(pts, dtype=np.float64)


def cauchy_1d(n: int, seed: int, offset: float = 1e-3):
    """Section 6.3-style interleaved 1D point sets: x_i uniform in [0,1] and
    y_j = x_j + offset * U(0,1).  Returns (x, y), each of shape (n, 1)."""
    g = _rng(seed)
    x = g.random((n, 1))
    y = x + offset * g.random((n, 1))
    return (np.ascontiguousarray(x, dtype=np.float64),
            np.ascontiguousarray(y, dtype=np.float64))


def cauchy_like_6_3(n: int, seed: int, offset: float = 1e-7, p: int = 2):
    """The first point sets of Section 6.3, (6.3): x_k = k/(n+1) and
    y_k = x_k + offset U(0,1), with generators w, v (n x p) of U(0,1) entries
    as the paper draws them.  Returns (x, y, w, v); x, y of shape (n, 1)."""
    g = _rng(seed)
    x = (np.arange(1, n + 1, dtype=np.float64) / (n + 1))[:, None]
    y = x + offset * g.random((n, 1))
    w = g.random((n, p))
    v = g.random((n, p))
    return tuple(np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, w, v))


def curve_6_4(name: str, n: int):
    """The boundary curves of Section 6.4 sampled for the trapezoidal rule at
    t_j = j/n: ram head (6.10) or sunflower (6.11).  Returns a dict with the
    points r(t_j) (n x 2), the unit outer normals (n x 2; both curves run
    counter-clockwise, so the outer normal is (r2', -r1')/|r'|), the speeds
    |r'(t_j)|, the signed curvatures and the weights |r'(t_j)|/n."""
    t = np.arange(n, dtype=np.float64) / n
    tp = 2.0 * np.pi
    if name == "ram_head":
        c4 = np.cos(2 * tp * t)
        r1 = 2.0 * np.cos(tp * t)
        r2 = 1.0 + np.sin(tp * t) - 1.4 * c4 ** 4
        d1 = -2.0 * tp * np.sin(tp * t)
        # d/dt cos^4(4 pi t) = -16 pi cos^3 sin
        d2 = tp * np.cos(tp * t) + 1.4 * 4 * c4 ** 3 * (2 * tp) * np.sin(2 * tp * t)
        dd1 = -2.0 * tp ** 2 * np.cos(tp * t)
        s4 = np.sin(2 * tp * t)
        dd2 = (-tp ** 2 * np.sin(tp * t)
               + 1.4 * 4 * (2 * tp) ** 2 * (c4 ** 3 * np.cos(2 * tp * t) - 3 * c4 ** 2 * s4 ** 2))
    elif name == "sunflower":
        rho = 1.3 + 1.25 * np.cos(20 * tp * t)
        drho = -1.25 * 20 * tp * np.sin(20 * tp * t)
        ddrho = -1.25 * (20 * tp) ** 2 * np.cos(20 * tp * t)
        c, s = np.cos(tp * t), np.sin(tp * t)
        r1, r2 = rho * c, rho * s
        d1 = drho * c - rho * tp * s
        d2 = drho * s + rho * tp * c
        dd1 = ddrho * c - 2 * drho * tp * s - rho * tp ** 2 * c
        dd2 = ddrho * s + 2 * drho * tp * c - rho * tp ** 2 * s
    else:
        raise ValueError(name)
    speed = np.sqrt(d1 ** 2 + d2 ** 2)
    return dict(x=np.ascontiguousarray(np.stack([r1, r2], axis=1)),
                nu=np.ascontiguousarray(np.stack([d2 / speed, -d1 / speed], axis=1)),
                speed=speed, curvature=(d1 * dd2 - d2 * dd1) / speed ** 3, w=speed / n)


def jittered_grid(cells_per_dim: int, d: int, seed: int, per_cell: int = 1) -> np.ndarray:
    """per_cell points drawn uniformly inside each cell of a regular grid with
    cells_per_dim cells along each axis of [0,1]^d.  With cells_per_dim a
    power of two and a leaf size that is a multiple of per_cell * 2^(d*j),
    the adaptive tree of these points is a perfect 2^d-tree, while the random
    positions avoid the exact ties of a regular lattice.  The first point is
    moved to the origin and the last to (1 - 2^-40, ...), which keeps them in
    their grid cells and makes the bounding cube exactly the unit cube."""
    g = _rng(seed)
    axes = [np.arange(cells_per_dim)] * d
    corners = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, d)
    corners = np.repeat(corners, per_cell, axis=0)
    pts = (corners + g.random(corners.shape)) / cells_per_dim
    # pin the bounding box to [0, 1 - 2^-40]^d so that the smallest cube
    # around the points is [0, 1]^d and its dyadic cells are the grid cells
    pts[0] = 0.0
    pts[-1] = 1.0 - 2.0 ** -40
    pts = pts[g.permutation(len(pts))]
    return np.ascontiguousarray(pts, dtype=np.float64)


def grid_2d(m: int) -> np.ndarray:
    """The uniform m x m grid of Section 6.2 in [0,1]^2: points ((i + 1/2)/m,
    (j + 1/2)/m), j fastest, shape (m*m, 2)."""
    t = (np.arange(m, dtype=np.float64) + 0.5) / m
    gx, gy = np.meshgrid(t, t, indexing="ij")
    return np.ascontiguousarray(np.stack([gx.ravel(), gy.ravel()], axis=1))


def uniform_01(n: int, nrhs: int, seed: int) -> np.ndarray:
    """n x nrhs entries U[0,1] (the rand([0,1]) vectors of Section 6.2)."""
    return np.ascontiguousarray(_rng(seed).random((n, nrhs)), dtype=np.float64)


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """n x nrhs standard normal right-hand sides, row-major float64."""
    return np.ascontiguousarray(_rng(seed).standard_normal((n, nrhs)), dtype=np.float64)


def sample_rows(n: int, count: int, seed: int) -> np.ndarray:
    """A sorted sample of `count` distinct row indices out of n (all rows when
    count >= n)."""
    if count >= n:
        return np.arange(n, dtype=np.int64)
    return np.sort(_rng(seed).choice(n, size=count, replace=False)).astype(np.int64)


def batched_problems(count: int, seed: int, n_lo: int = 1024, n_hi: int = 32768) -> list:
    """`count` independent problems of the batched-trees workload.  Per
    problem: N = floor(exp(U(ln n_lo, ln n_hi))) (log-uniform), dimension 2
    or 3 with probability 1/2 each (kernel log|x-y| in 2D, 1/|x-y| in 3D),
    points uniform in the unit cube or from a 4-component Gaussian mixture
    with sigma 0.1, with probability 1/2 each.  Returns a list of dicts with
    keys d, kernel, kind and x (N x d float64)."""
    g = _rng(seed)
    out = []
    for _ in range(count):
        n = int(np.floor(np.exp(g.uniform(np.log(n_lo), np.log(n_hi)))))
        n = min(max(n, n_lo), n_hi)
        d = 2 if g.random() < 0.5 else 3
        kind = "cube" if g.random() < 0.5 else "mixture"
        sub = int(g.integers(0, 2 ** 31 - 1))
        x = uniform_cube(n, d, sub) if kind == "cube" else gaussian_mixture(n, d, sub, ncomp=4, sigma=0.1)
        out.append(dict(d=d, kernel=KERNEL_LOG if d == 2 else KERNEL_INVR, kind=kind, x=x))
    return out


def group_by_dimension(problems: list) -> dict:
    """Concatenates the problems of each dimension: {d: (points, offsets,
    kernel, indices into `problems`)}, problems kept in their order."""
    groups = {}
    for i, p in enumerate(problems):
        groups.setdefault(p["d"], []).append(i)
    out = {}
    for d, idx in sorted(groups.items()):
        xs = [problems[i]["x"] for i in idx]
        off = np.zeros(len(xs) + 1, dtype=np.int64)
        off[1:] = np.cumsum([len(x) for x in xs])
        out[d] = (np.ascontiguousarray(np.concatenate(xs, axis=0)), off, problems[idx[0]]["kernel"], idx)
    return out


# Kernel identifiers shared by convention (the C-ABI header and the oracle
# each define their own copy of these numbers).
KERNEL_LOG, KERNEL_INVR, KERNEL_YUKAWA, KERNEL_CAUCHY = 0, 1, 2, 3
KERNEL_DLP1, KERNEL_DLP2 = 4, 5

# The named workloads: point-cloud recipe plus method parameters.
WORKLOADS = {
    # 2D plain FP64, full dense check
    "2d_log_4096": dict(kind="cube", n=4096, d=2, kernel=KERNEL_LOG, leaf=64, order=5,
                        tol=1e-8, nrhs=4, index=0),
    # 3D plain FP64, 1024 sampled rows
    "3d_invr_65536": dict(kind="cube", n=65536, d=3, kernel=KERNEL_INVR, leaf=128, order=4,
                          tol=1e-8, nrhs=16, index=1),
    # the headline workload: the 3D 1/r configuration at N = 2^20
    "3d_invr_1m": dict(kind="cube", n=1 << 20, d=3, kernel=KERNEL_INVR, leaf=128, order=4,
                       tol=1e-8, nrhs=16, index=1),
    # 3D mixed precision on the sphere with clustered caps
    "sphere_yukawa_1m": dict(kind="sphere", n=1 << 20, d=3, kernel=KERNEL_YUKAWA, leaf=128,
                             order=5, tol=1e-8, nrhs=32, index=2),
    # 512 independent problems (batched_problems), FP32 matvec with 8 RHS each
    "batched_512": dict(kind="batch", count=512, leaf=64, order=4, tol=1e-8, nrhs=8, index=3),
}


def make_workload(name: str, rep: int = 0, n: int | None = None):
    """Points and right-hand sides of a named workload.  `n` overrides the
    point count (same recipe, smaller or larger cloud).  Returns a dict with
    x, y (None when Y = X), q and the method parameters."""
    w = dict(WORKLOADS[name])
    if n is not None:
        w["n"] = int(n)
    seed = w["index"] * 1000 + rep
    if w["kind"] == "batch":
        # `n` overrides the number of problems
        if n is not None:
            w["count"] = int(n)
        w["problems"] = batched_problems(w["count"], seed)
        w["groups"] = group_by_dimension(w["problems"])
        w["n"] = sum(len(p["x"]) for p in w["problems"])
        w["q"] = {d: rhs(len(g[0]), w["nrhs"], seed + 500 + d) for d, g in w["groups"].items()}
        return w
    if w["kind"] == "cube":
        x = uniform_cube(w["n"], w["d"], seed)
        y = None
    elif w["kind"] == "sphere":
        x = sphere_with_caps(w["n"], seed)
        y = None
    elif w["kind"] == "cauchy":
        x, y = cauchy_1d(w["n"], seed)
    else:
        raise ValueError(w["kind"])
    ny = w["n"] if y is None else len(y)
    w["x"], w["y"] = x, y
    w["q"] = rhs(ny, w["nrhs"], seed + 500)
    return w
