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
