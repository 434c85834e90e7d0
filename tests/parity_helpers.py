"""Element-wise parity bar of the GPU matvec tests.

Every GPU matvec result z is compared with the oracle's H^2 matvec z_o entry
by entry, against that entry's own rounding scale

    s_i = sum over the terms t that the matvec adds up for entry i of |t|,

which the oracle computes by running the same passes with every factor
replaced by its magnitude (oracle.H2.matvec_abs).  A floating-point sum of
terms t_1..t_n differs from the exact one by at most a small multiple of the
unit roundoff times sum |t_j|, and so does every rounding of a term; so two
correct evaluations of the same approximant A^ q differ entry by entry by a
modest multiple of u * s_i, whatever the cancellation in the entry.  The
bars, from the arithmetic of each precision (u = unit roundoff of the format
the products are rounded to):

  FP64                 1e-12   u = 2^-53: a row adds up to ~10^4 terms, and
                               naive FP64 sums of n terms are within
                               (n - 1) u sum|t| of the exact sum.  Four
                               orders inside the 1e-8 parity bar.
  double-float         1e-11   each double-float operation (a kernel entry,
                               a transfer product, a digit-split fold) errs
                               by up to a few 2^-44 of its operands'
                               magnitudes, and a value passes through up to
                               2L + 1 of them (L up and L down the tree, one
                               coupling): with L <= 20 and 4 * 2^-44 per
                               operation, 41 * 4 * 2^-44 < 1e-11.
  FP32, split TF32     1e-5    u = 2^-24, entries and FP32 sums; the
                               mixed-precision bar of the method.
  TF32                 2^-9    products of two TF32-rounded factors carry
                               <= 2 u = 2^-10 each, plus FP32 sums.
  BF16                 2^-6    likewise with u = 2^-8.

Zero scale means every term is zero, so the entry must be exactly zero.  The
relative 2-norm over all compared entries is reported beside the worst entry.
"""
from __future__ import annotations

import os

import numpy as np

TOL_F64 = 1e-12
TOL_F32X2 = 1e-11
TOL_F32 = 1e-5
TOL_TF32X3 = 1e-5
TOL_TF32 = 2.0 ** -9
TOL_BF16 = 2.0 ** -6


def worst_entry(z, zo, scale, rows=None):
    """(worst |z - zo| / scale over the compared entries, its flat index,
    relative 2-norm).  rows: only those rows (all when None)."""
    z = np.asarray(z, np.float64)
    zo = np.asarray(zo, np.float64)
    scale = np.asarray(scale, np.float64)
    if rows is not None:
        z, zo, scale = z[rows], zo[rows], scale[rows]
    assert z.shape == zo.shape == scale.shape, (z.shape, zo.shape, scale.shape)
    assert np.all(np.isfinite(zo)) and np.all(np.isfinite(scale)), "oracle rows missing"
    d = np.abs(z - zo)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), np.where(d == 0, 0.0, np.inf))
    ratio = np.where(np.isfinite(z), ratio, np.inf)
    k = int(np.argmax(ratio)) if ratio.size else 0
    worst = float(ratio.ravel()[k]) if ratio.size else 0.0
    nz = np.linalg.norm(zo)
    rel2 = float(np.linalg.norm(z - zo) / nz) if nz > 0 else float(np.linalg.norm(z - zo))
    return worst, k, rel2


def assert_entrywise(z, zo, scale, tol, rows=None, what=""):
    """Assert max_i |z_i - zo_i| / s_i <= tol (see the module docstring);
    returns (worst, rel2)."""
    worst, k, rel2 = worst_entry(z, zo, scale, rows)
    log = os.environ.get("SMASH_PARITY_LOG")
    if log:  # margins of every comparison, for the record
        with open(log, "a") as f:
            f.write(f"{os.environ.get('PYTEST_CURRENT_TEST', '?').split(' ')[0]}\t{what}\t"
                    f"worst {worst:.3e}\tbar {tol:.1e}\trel2 {rel2:.3e}\n")
    assert worst <= tol, (f"{what}: entry {k} off by {worst:.3e} of its scale sum|terms| "
                          f"(bar {tol:.1e}); relative 2-norm {rel2:.3e}")
    return worst, rel2


def oracle_reference(ho, q, leaves=None):
    """(z_o, s) of the oracle's H^2 matvec on all rows, or on the rows of the
    given leaf gids (others NaN)."""
    if leaves is None:
        return ho.matvec(q), ho.matvec_abs(q)
    return ho.matvec_leaves(q, leaves), ho.matvec_abs(q, leaves)


def leaf_rows(e, leaves):
    """Caller-order rows of the points of the given leaves (an export)."""
    return np.concatenate([e["permx"][e["rs"][g]:e["rs"][g] + e["rc"][g]] for g in leaves])


def sample_leaves(e, x, count=64, seed=0, extra=()):
    """At least `count` leaf gids of an export: the leaves holding the point
    nearest to each corner of the bounding box and to the centre of each of
    its faces, every leaf in `extra`, and the rest drawn at random (seeded).
    Returns a sorted int32 array."""
    leaf_ids = np.flatnonzero(e["leaf"])
    # leaf of each sorted position
    owner = np.empty(len(e["permx"]), np.int64)
    for g in leaf_ids:
        owner[e["rs"][g]:e["rs"][g] + e["rc"][g]] = g
    inv = np.empty_like(e["permx"])
    inv[e["permx"]] = np.arange(len(e["permx"]))
    d = x.shape[1]
    lo, hi = x.min(axis=0), x.max(axis=0)
    mid = 0.5 * (lo + hi)
    targets = []
    for bits in range(1 << d):
        targets.append([hi[a] if (bits >> a) & 1 else lo[a] for a in range(d)])
    for a in range(d):
        for v in (lo[a], hi[a]):
            t = mid.copy()
            t[a] = v
            targets.append(t)
    chosen = set(int(g) for g in extra)
    for t in targets:
        i = int(np.argmin(np.sum((x - np.asarray(t)) ** 2, axis=1)))
        chosen.add(int(owner[inv[i]]))
    rng = np.random.default_rng(seed)
    rest = np.setdiff1d(leaf_ids, np.fromiter(chosen, np.int64, len(chosen)))
    need = max(0, count - len(chosen))
    if need and len(rest):
        chosen.update(int(g) for g in rng.choice(rest, size=min(need, len(rest)), replace=False))
    return np.array(sorted(chosen), np.int32)
