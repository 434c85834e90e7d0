"""The geometric entry bounds behind the digit-split coupling, on the oracle's tree.

The tensor-core coupling scales the entries of a target point's row by a power
of two taken from a bound on 1/|x - y| over the row's admissible partners
(Def. 2.1, (2.3)): the distance from x to the partner's cell, and
|c_i - c_j| - r_i - r_j from the cell centres and half-diagonals.  Both rest
on the cell frame of the tree: the root (level 1) is the unit cube
[lo, lo + s)^d, a level-l cell has width 2^(1-l) in units of s, and its
integer coordinates c place it at lo + c 2^(1-l) s.  This test checks, on
trees the oracle builds (the library's trees are identical, see the parity
tests), that every point of a node lies in its cell and that every entry of
every admissible pair obeys both bounds.

The near field's digit split has no geometric bound (its pairs are not
admissible); it scales a row by its nearest source, found from the float32
hi parts of the normalised coordinates with a margin.  The last tests check
that this distance is a lower bound of every distance of the row.
"""
import numpy as np
import pytest

import oracle
import smash_inputs as si


def _frame(e):
    lo, s = np.asarray(e["lo"]), float(e["s"])
    lev = np.asarray(e["level"])
    return lo, s, lev, np.asarray(e["cell"]).reshape(-1, 3)


def _check(x, y, kernel, leaf, order, tol):
    h = oracle.H2(x, kernel, leaf, order, tol, y=y)
    e = h.export()
    lo, s, lev, cell = _frame(e)
    d = x.shape[1]
    ys = x if y is None else y
    xn = (x[np.asarray(e["permx"])] - lo[:d]) / s
    yn = (ys[np.asarray(e["permy"] if y is not None else e["permx"])] - lo[:d]) / s
    rs, rc = np.asarray(e["rs"]), np.asarray(e["rc"])
    cs, cc = np.asarray(e["cs"]), np.asarray(e["cc"])
    ptr, col = np.asarray(e["adm_ptr"]), np.asarray(e["adm_col"])
    assert lev.min() >= 1 and lev[0] == 1  # the root is level 1
    w = 2.0 ** (1 - lev)
    # points of every node lie in its cell
    for g in range(len(lev)):
        c0 = cell[g, :d] * w[g]
        for P in (xn[rs[g]:rs[g] + rc[g]], yn[cs[g]:cs[g] + cc[g]]):
            assert np.all(P >= c0 - 1e-15) and np.all(P <= c0 + w[g] + 1e-15)
    checked = 0
    for g in range(len(lev)):
        if ptr[g] == ptr[g + 1] or rc[g] == 0:
            continue
        P = xn[rs[g]:rs[g] + rc[g]]
        for j in col[ptr[g]:ptr[g + 1]]:
            Q = yn[cs[j]:cs[j] + cc[j]]
            if len(Q) == 0:
                continue
            dist = np.sqrt(((P[:, None, :] - Q[None, :, :]) ** 2).sum(2))
            kmax = (1.0 / dist).max(1)
            # distance from each target point to the partner's cell
            blo = cell[j, :d] * w[j]
            gap = np.maximum(np.maximum(blo - P, P - (blo + w[j])), 0.0)
            kb_point = 1.0 / np.sqrt((gap ** 2).sum(1))
            assert np.all(kmax <= kb_point * (1 + 1e-12))
            # centres and half-diagonals, in units of half a level-m cell
            m = max(lev[g], lev[j])
            Ci = (2 * cell[g, :d] + 1) * 2.0 ** (m - lev[g])
            Cj = (2 * cell[j, :d] + 1) * 2.0 ** (m - lev[j])
            gapc = np.sqrt(((Ci - Cj) ** 2).sum()) - np.sqrt(d) * (2.0 ** (m - lev[g]) + 2.0 ** (m - lev[j]))
            assert gapc > 0
            assert kmax.max() <= 2.0 ** m / gapc * (1 + 1e-12)
            checked += 1
    assert checked > 0


@pytest.mark.parametrize("d,n,leaf,seed", [(3, 4000, 32, 8100), (2, 3000, 32, 8101), (1, 1500, 16, 8102)])
def test_entry_bounds_hold_on_uniform_points(d, n, leaf, seed):
    _check(si.uniform_cube(n, d, seed), None, 1, leaf, 3, 1e-6)


def test_entry_bounds_hold_on_clustered_sphere():
    _check(si.sphere_with_caps(3000, 8103), None, 1, 32, 3, 1e-6)


def test_entry_bounds_hold_for_rectangular_cauchy():
    x, y = si.cauchy_1d(2000, 8104)
    _check(x, y, 3, 32, 8, 1e-8)


def _near_check(x, d, leaf, seed_kernel=1):
    """The near field's row bound: from the hi parts of the normalised
    coordinates x'' = 1 + (x - lo)/s (float32), the kernel takes
    dlo = sqrt(min hi-part r^2) (1 - 2^-20) - 2^-22 as a lower bound of every
    distance |x'' - y''| of the row (the target's own point skipped)."""
    h = oracle.H2(x, seed_kernel, leaf, 3, 1e-6)
    e = h.export()
    lo, s = np.asarray(e["lo"])[:d], float(e["s"])
    xs = x[np.asarray(e["permx"])]
    xn = 1.0 + (xs - lo) / s                         # FP64 normalised coordinates
    xh = xn.astype(np.float32)                       # their hi parts
    rs, rc, cs, cc = (np.asarray(e[k]) for k in ("rs", "rc", "cs", "cc"))
    ptr, col = np.asarray(e["near_ptr"]), np.asarray(e["near_col"])
    leaves = np.flatnonzero(np.asarray(e["leaf"]))
    checked = 0
    for g in leaves:
        if rc[g] == 0 or ptr[g] == ptr[g + 1]:
            continue
        tgt = np.arange(rs[g], rs[g] + rc[g])
        src = np.concatenate([np.arange(cs[j], cs[j] + cc[j]) for j in col[ptr[g]:ptr[g + 1]]])
        dh = xh[tgt][:, None, :].astype(np.float32) - xh[src][None, :, :]   # exact (Sterbenz)
        r2 = np.zeros(dh.shape[:2], dtype=np.float32)
        for a in range(d):                                                 # the kernel's fma chain
            r2 = (dh[:, :, a].astype(np.float64) ** 2 + r2.astype(np.float64)).astype(np.float32)
        true = np.sqrt(((xn[tgt][:, None, :] - xn[src][None, :, :]) ** 2).sum(2))
        self_pair = tgt[:, None] == src[None, :]
        r2 = np.where(self_pair, np.inf, r2)
        dlo = np.sqrt(r2.min(1).astype(np.float64)).astype(np.float32) * np.float32(1 - 2.0 ** -20) \
            - np.float32(2.0 ** -22)
        mtrue = np.where(self_pair, np.inf, true).min(1)
        assert np.all(dlo <= mtrue), g
        checked += 1
    assert checked > 0


@pytest.mark.parametrize("d,n,leaf,seed", [(3, 3000, 32, 8200), (2, 2500, 32, 8201), (1, 1500, 16, 8202)])
def test_near_field_row_bound_is_a_lower_bound(d, n, leaf, seed):
    _near_check(si.uniform_cube(n, d, seed), d, leaf)


def test_near_field_row_bound_on_clustered_sphere():
    _near_check(si.sphere_with_caps(2500, 8203), 3, 32)
