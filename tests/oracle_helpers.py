"""Independent restatements used by the oracle pins (numpy / exact arithmetic).

Nothing here calls into the oracle's arithmetic: these helpers recompute the
paper's definitions a second, different way so that the oracle can be checked
against them.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def kernel_matrix(kid: int, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Dense kappa(x_i, y_j) via broadcasting, value 0 where the points coincide."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    if kid == 3:
        D = X[:, 0][:, None] - Y[:, 0][None, :]
        with np.errstate(divide="ignore"):
            K = np.where(D == 0.0, 0.0, 1.0 / np.where(D == 0.0, 1.0, D))
        return K
    diff = X[:, None, :] - Y[None, :, :]
    R = np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
    zero = R == 0.0
    Rs = np.where(zero, 1.0, R)
    if kid == 0:
        K = np.log(Rs)
    elif kid == 1:
        K = 1.0 / Rs
    elif kid == 2:
        K = np.exp(-Rs) / Rs
    else:
        raise ValueError(kid)
    return np.where(zero, 0.0, K)


def cell_geometry(lo, s: float, level: int, cell, d: int):
    """Centre and radius of a node cell from its corners (float):
    centre = midpoint of the box, radius = max distance to the 2^d corners."""
    h = float(s) * 2.0 ** (1 - int(level))
    lo = np.asarray(lo, np.float64)[:d]
    c = np.asarray(cell, np.float64)[:d]
    corner0 = lo + c * h
    corners = np.array([[corner0[a] + h * ((bits >> a) & 1) for a in range(d)]
                        for bits in range(1 << d)])
    centre = corner0 + 0.5 * h
    radius = float(np.max(np.linalg.norm(corners - centre, axis=1)))
    return centre, radius


def well_separated(lo, s, d, li, ci, lj, cj, tau) -> bool:
    """Definition 2.1, (2.3), on the two cells in exact rational arithmetic,
    with tau read as its decimal value: (delta_i + delta_j)^2 <= tau^2 |a-b|^2,
    delta = sqrt(d) h / 2, a = lo + (c + 1/2) h.  Equality counts as
    well separated, as the inequality of (2.3) says."""
    t = Fraction(repr(float(tau)))
    S = Fraction(float(s))
    hi = S * Fraction(2) ** (1 - int(li))
    hj = S * Fraction(2) ** (1 - int(lj))
    dist2 = Fraction(0)
    for a in range(d):
        ca = (int(ci[a]) + Fraction(1, 2)) * hi
        cb = (int(cj[a]) + Fraction(1, 2)) * hj
        dist2 += (ca - cb) ** 2
    return Fraction(d) * (hi + hj) ** 2 / 4 <= t * t * dist2


def point_in_cell(pt, lo, s, level, cell, d, slack_ulps: float = 8.0) -> bool:
    """Exact-rational containment of a point in the half-open cell box, with a
    slack of a few ulps of s for values that sit on a bisection plane."""
    level = int(level)
    h = Fraction(float(s)) * Fraction(2) ** (1 - level)
    eps = Fraction(float(s)) * Fraction(slack_ulps) * Fraction(2) ** -52
    for a in range(d):
        lo_a = Fraction(float(lo[a])) + int(cell[a]) * h
        x = Fraction(float(pt[a]))
        if x < lo_a - eps or x >= lo_a + h + eps:
            return False
    return True


def lattice_counts(d: int, tau: float):
    """Closed-form interior counts on a perfect tree: same-level integer cell
    offsets D are well separated iff d <= tau^2 |D|^2 (exact rationals)."""
    t2 = Fraction(tau) ** 2

    def sep(D):
        return Fraction(d) <= t2 * sum(Fraction(x * x) for x in D)

    import itertools
    near_offsets = [D for D in itertools.product(range(-3, 4), repeat=d) if not sep(D)]
    near = len(near_offsets)
    # far partners of a node = children of the parent's near neighbours that
    # are well separated from the node; average over the 2^d child positions
    counts = set()
    for pos in itertools.product((0, 1), repeat=d):
        cnt = 0
        for P in near_offsets:
            for ch in itertools.product((0, 1), repeat=d):
                D = tuple(2 * P[a] + ch[a] - pos[a] for a in range(d))
                if sep(D):
                    cnt += 1
        counts.add(cnt)
    assert len(counts) == 1
    return counts.pop(), near


def local_positions(e: dict, side: str):
    """Working set ibar of every node rebuilt from an export: leaves own their
    point range, parents concatenate their children's skeletons (3.6)/(3.18).
    Returns per node (ibar, skel, rest, G) with G of shape (m-k, k)."""
    nn = len(e["level"])
    m, k = e[f"m_{side}"], e[f"k_{side}"]
    so = np.concatenate([[0], np.cumsum(k)])
    ro = np.concatenate([[0], np.cumsum(m - k)])
    go = np.concatenate([[0], np.cumsum((m - k).astype(np.int64) * k)])
    start = e["rs"] if side == "row" else e["cs"]
    count = e["rc"] if side == "row" else e["cc"]
    skel = [e[f"skel_{side}"][so[g]:so[g + 1]] for g in range(nn)]
    rest = [e[f"rest_{side}"][ro[g]:ro[g + 1]] for g in range(nn)]
    G = [e[f"G_{side}"][go[g]:go[g + 1]].reshape(m[g] - k[g], k[g]) for g in range(nn)]
    ibar = [None] * nn
    for g in range(nn):
        if e["level"][g] == 1:
            ibar[g] = np.zeros(0, np.int64)
        elif e["leaf"][g]:
            ibar[g] = np.arange(start[g], start[g] + count[g], dtype=np.int64)
        else:
            c0, nc = e["child0"][g], e["nchild"][g]
            ibar[g] = np.concatenate([skel[c] for c in range(c0, c0 + nc)])
    return ibar, skel, rest, G


def dense_transfer(ibar, skel, rest, G):
    """P [I; G] as an m x k matrix with rows in working-set order (2.11)."""
    m, k = len(ibar), len(skel)
    U = np.zeros((m, k))
    pos = {int(v): i for i, v in enumerate(ibar)}
    for t in range(k):
        U[pos[int(skel[t])], t] = 1.0
    for u in range(m - k):
        U[pos[int(rest[u])], :] = G[u]
    return U


def rel(a, b) -> float:
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def log_floor(x: float) -> int:
    return math.floor(x)
