"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks one part of the oracle against something other than the
oracle itself: values printed in the paper (tests/golden), closed forms,
invariants of the construction, exact or brute-force restatements, and
library routines (numpy/scipy) in the special cases where the method reduces
to them.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import smash_inputs as si
from oracle_helpers import (dense_transfer, kernel_matrix, lattice_counts, local_positions,
                            point_in_cell, rel, well_separated)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# Section 6.1 heuristic: the three printed worked values
# --------------------------------------------------------------------------

def test_suggest_rank_matches_section_6_1_worked_values():
    for eps, tau, r in _golden("section6_1_rank.txt"):
        assert oracle.suggest_rank(float(eps), float(tau)) == int(r)


def test_suggest_rank_floor_of_five():
    # the 'otherwise' branch never goes below 5
    assert oracle.suggest_rank(0.5, 0.6) == 5


# --------------------------------------------------------------------------
# kernels and the dense product (the plain definition of A q)
# --------------------------------------------------------------------------

def test_kernel_special_values():
    e = np.e
    assert oracle.kernel(1, [0, 0, 0], [0, 0, 2]) == pytest.approx(0.5, rel=1e-15)
    assert oracle.kernel(0, [0, 0], [e, 0]) == pytest.approx(1.0, rel=1e-15)
    assert oracle.kernel(2, [0, 0, 0], [1, 0, 0]) == pytest.approx(np.exp(-1.0), rel=1e-15)
    assert oracle.kernel(3, [1.0], [3.0]) == pytest.approx(-0.5, rel=1e-15)
    assert oracle.kernel(3, [3.0], [1.0]) == pytest.approx(0.5, rel=1e-15)
    for kid, d in ((0, 2), (1, 3), (2, 3), (3, 1)):
        x = np.full(d, 0.25)
        assert oracle.kernel(kid, x, x) == 0.0   # diagonal value d_x = 0


@pytest.mark.parametrize("kid,d", [(0, 2), (1, 3), (2, 3), (3, 1), (0, 1), (1, 2)])
def test_dense_rows_vs_numpy(kid, d):
    x = si.uniform_cube(300, d, 11)
    x[7] = x[3]          # a duplicate point: kappa = 0 there too
    q = si.rhs(300, 3, 12)
    ref = kernel_matrix(kid, x, x) @ q
    got = oracle.dense_rows(x, kid, q)
    assert rel(got, ref) < 1e-13


def test_dense_rows_rectangular_and_sampled():
    x, y = si.cauchy_1d(400, 5)
    q = si.rhs(400, 2, 6)
    rows = np.array([0, 17, 399], dtype=np.int64)
    ref = (kernel_matrix(3, x, y) @ q)[rows]
    got = oracle.dense_rows(x, 3, q, rows=rows, y=y)
    assert rel(got, ref) < 1e-13


# --------------------------------------------------------------------------
# Section 3.1: cube, Morton order, adaptive tree
# --------------------------------------------------------------------------

def test_bounding_cube_is_a_cube_holding_all_points():
    x = si.gaussian_mixture(500, 3, 2)
    lo, s = oracle.bounding_cube(x)
    assert np.all(x >= lo)
    assert np.all(x < lo + s)
    ext = (x.max(0) - x.min(0)).max()
    assert ext < s <= ext * (1 + 1e-11)
    lo2, s2 = oracle.bounding_cube(np.zeros((4, 2)))
    assert s2 == 1.0 and np.all(lo2 == 0.0)


def _check_tree(h, x, y, leaf, d):
    e = h.export()
    b = oracle.bits_per_dim(d)
    nn = len(e["level"])
    xs = x[e["permx"]]
    ys = (x if y is None else y)[e["permy"]]
    nx, ny = len(xs), len(ys)
    # permutations, keys sorted, ties in original order (stable)
    assert sorted(e["permx"].tolist()) == list(range(nx))
    kx = e["keyx"]
    assert np.all(kx[1:] >= kx[:-1])
    same = kx[1:] == kx[:-1]
    assert np.all(e["permx"][1:][same] > e["permx"][:-1][same])
    # levels
    assert e["level"][0] == 1 and e["parent"][0] == -1
    for l in range(1, e["L"] + 1):
        assert np.all(e["level"][e["lvl_off"][l - 1]:e["lvl_off"][l]] == l)
    covered_r = np.zeros(nx, int)
    covered_c = np.zeros(ny, int)
    for g in range(nn):
        rs, rc, cs, cc = e["rs"][g], e["rc"][g], e["cs"][g], e["cc"][g]
        assert rc + cc > 0                                     # empty boxes discarded
        big = max(rc, cc)
        if e["leaf"][g]:
            assert big <= leaf or e["level"][g] == b + 1       # depth cap
            covered_r[rs:rs + rc] += 1
            covered_c[cs:cs + cc] += 1
        else:
            assert big > leaf
            c0, ncd = e["child0"][g], e["nchild"][g]
            assert 1 <= ncd <= 2 ** d
            kids = range(c0, c0 + ncd)
            assert all(e["parent"][c] == g and e["level"][c] == e["level"][g] + 1 for c in kids)
            # children partition the parent's ranges, in order
            assert e["rs"][c0] == rs and e["cs"][c0] == cs
            assert sum(e["rc"][c] for c in kids) == rc and sum(e["cc"][c] for c in kids) == cc
            for c in list(kids)[1:]:
                assert e["rs"][c] == e["rs"][c - 1] + e["rc"][c - 1]
                assert e["cs"][c] == e["cs"][c - 1] + e["cc"][c - 1]
            # child cells: distinct sub-cubes of the parent cell, in Morton digit order
            digits = []
            for c in kids:
                off = e["cell"][c][:d] - 2 * e["cell"][g][:d]
                assert np.all((off == 0) | (off == 1))
                digits.append(int(sum(int(off[a]) << (d - 1 - a) for a in range(d))))
            assert digits == sorted(set(digits))
        # brute force: every point of the node lies inside the node's cell
        for p_ in range(rs, rs + rc):
            assert point_in_cell(xs[p_], e["lo"], e["s"], e["level"][g], e["cell"][g], d)
        for p_ in range(cs, cs + cc):
            assert point_in_cell(ys[p_], e["lo"], e["s"], e["level"][g], e["cell"][g], d)
    assert np.all(covered_r == 1) and np.all(covered_c == 1)   # one leaf per point
    return e


@pytest.mark.parametrize("d,leaf", [(1, 4), (2, 8), (3, 8)])
def test_tree_invariants_uniform(d, leaf):
    x = si.uniform_cube(700, d, 20 + d)
    h = oracle.H2(x, 1 if d > 1 else 0, leaf, 3, 1e-8)
    _check_tree(h, x, None, leaf, d)


def test_tree_invariants_clustered_and_rectangular():
    x = si.gaussian_mixture(600, 2, 3, sigma=0.02)
    _check_tree(oracle.H2(x, 0, 6, 3, 1e-8), x, None, 6, 2)
    xx, yy = si.cauchy_1d(500, 4)
    _check_tree(oracle.H2(xx, 3, 5, 4, 1e-8, y=yy), xx, yy, 5, 1)


def test_tree_depth_cap_on_duplicates():
    x = np.concatenate([np.full((20, 2), 0.3), si.uniform_cube(30, 2, 1)])
    h = oracle.H2(x, 0, 4, 2, 1e-8)
    e = _check_tree(h, x, None, 4, 2)
    b = oracle.bits_per_dim(2)
    deep = [g for g in range(len(e["level"])) if e["leaf"][g] and e["rc"][g] > 4]
    assert deep and all(e["level"][g] == b + 1 for g in deep)


def test_morton_order_is_lexicographic_in_cells():
    # sorted by key == sorted by the sequence of cell indices from the root down
    x = si.uniform_cube(300, 3, 9)
    lo, s = oracle.bounding_cube(x)
    keys = oracle.morton_keys(x, lo, s)
    b = oracle.bits_per_dim(3)
    from fractions import Fraction
    def path(pt):
        out = []
        for l in range(1, 12):
            q = [int(Fraction(float(pt[a]) - float(lo[a])) / Fraction(s) * 2 ** l) for a in range(3)]
            out.append(tuple(q))
        return out
    order_keys = np.argsort(keys, kind="stable")
    order_paths = sorted(range(300), key=lambda i: (path(x[i]), i))
    assert order_keys.tolist() == order_paths
    assert b == 21


# --------------------------------------------------------------------------
# (3.3) / (3.4): admissible and inadmissible leaves
# --------------------------------------------------------------------------

def _cover_and_lists(h, d, tau):
    e = h.export()
    nn = len(e["level"])
    nx, ny = len(e["permx"]), len(e["permy"])
    cover = np.zeros((nx, ny), np.int32)
    adm = set()
    near = set()
    for g in range(nn):
        for t in range(e["adm_ptr"][g], e["adm_ptr"][g + 1]):
            adm.add((g, int(e["adm_col"][t])))
        for t in range(e["near_ptr"][g], e["near_ptr"][g + 1]):
            near.add((g, int(e["near_col"][t])))
        # CSR rows sorted by (level, node id) = gid
        assert np.all(np.diff(e["adm_col"][e["adm_ptr"][g]:e["adm_ptr"][g + 1]]) > 0)
        assert np.all(np.diff(e["near_col"][e["near_ptr"][g]:e["near_ptr"][g + 1]]) > 0)
    for (i, j) in adm | near:
        cover[e["rs"][i]:e["rs"][i] + e["rc"][i], e["cs"][j]:e["cs"][j] + e["cc"][j]] += 1
    assert np.all(cover == 1), "L and L^- must cover every matrix entry exactly once"
    # brute force over all node pairs: membership in (3.3) and (3.4)
    lv, par, leaf = e["level"], e["parent"], e["leaf"]
    def ws(i, j):
        return well_separated(e["lo"], e["s"], d, lv[i], e["cell"][i], lv[j], e["cell"][j], tau)
    want_adm, want_near = set(), set()
    for i in range(nn):
        if e["rc"][i] == 0:
            continue
        for j in range(nn):
            if e["cc"][j] == 0:
                continue
            if leaf[i] and leaf[j] and not ws(i, j):
                want_near.add((i, j))
            if not ws(i, j):
                continue
            if lv[i] == lv[j] and lv[i] > 1 and not ws(par[i], par[j]):
                want_adm.add((i, j))
            elif leaf[i] and lv[j] > lv[i] and not ws(i, par[j]):
                want_adm.add((i, j))
            elif leaf[j] and lv[i] > lv[j] and not ws(par[i], j):
                want_adm.add((i, j))
    assert adm == want_adm
    assert near == want_near
    return e


@pytest.mark.parametrize("d,n,leaf", [(1, 200, 3), (2, 500, 6), (3, 500, 8)])
def test_lists_match_definitions_uniform(d, n, leaf):
    x = si.uniform_cube(n, d, 40 + d)
    _cover_and_lists(oracle.H2(x, 1 if d > 1 else 3, leaf, 2, 1e-8), d, 0.7)


def test_lists_match_definitions_adaptive_and_rectangular():
    x = si.gaussian_mixture(400, 2, 8, sigma=0.05)
    _cover_and_lists(oracle.H2(x, 0, 5, 2, 1e-8), 2, 0.7)
    xx, yy = si.cauchy_1d(300, 9)
    _cover_and_lists(oracle.H2(xx, 3, 4, 3, 1e-8, y=yy), 1, 0.7)
    x3 = si.sphere_with_caps(400, 10)
    _cover_and_lists(oracle.H2(x3, 2, 8, 2, 1e-8, tau=0.6), 3, 0.6)


def test_perfect_tree_interior_counts():
    golden = {int(d): (int(far), int(near)) for d, tau, far, near in _golden("perfect_tree_counts.txt")}
    for d, cells in ((1, 64), (2, 32), (3, 16)):
        assert lattice_counts(d, 0.7) == golden[d]
        x = si.jittered_grid(cells, d, 70 + d)
        h = oracle.H2(x, 1 if d > 1 else 3, 1, 1, 1.0)
        e = h.export()
        L = e["L"]
        assert 2 ** (d * (L - 1)) == cells ** d       # perfect tree
        far, near = golden[d]
        lo_c, hi_c = 6, cells - 7
        for g in range(e["lvl_off"][L - 1], e["lvl_off"][L]):
            c = e["cell"][g][:d]
            if np.all(c >= lo_c) and np.all(c <= hi_c):
                assert e["adm_ptr"][g + 1] - e["adm_ptr"][g] == far
                assert e["near_ptr"][g + 1] - e["near_ptr"][g] == near


def test_admissibility_never_self_or_ancestor():
    for d in (1, 2, 3):
        for l in range(1, 6):
            c = [min(3, 2 ** (l - 1) - 1)] * d
            assert not oracle.admissible(d, l, c, l, c, 0.7)
            # an ancestor cell contains the cell
            for la in range(1, l):
                ca = [ci >> (l - la) for ci in c]
                assert not oracle.admissible(d, la, ca, l, c, 0.7)
                assert not oracle.admissible(d, l, c, la, ca, 0.7)


# --------------------------------------------------------------------------
# (2.2) / (3.1): Lagrange interpolation at Chebyshev anchors
# --------------------------------------------------------------------------

def test_chebyshev_points_are_roots_of_T_p():
    for p in (1, 2, 5, 8, 16):
        t = oracle.chebyshev(p)
        Tp = np.polynomial.chebyshev.Chebyshev.basis(p)
        assert np.max(np.abs(Tp(t))) < 1e-13
        assert len(set(np.round(t, 14))) == p


def test_lagrange_cardinal_property():
    for p in (2, 4, 7):
        t = oracle.chebyshev(p)
        for m in range(p):
            for n in range(p):
                assert oracle.lagrange(p, m, t[n]) == pytest.approx(1.0 if m == n else 0.0, abs=1e-14)


@pytest.mark.parametrize("d,p", [(1, 2), (1, 9), (2, 3), (2, 5), (3, 2), (3, 4)])
def test_basis_reproduces_polynomials(d, p):
    """Sum_k ell_k(x) P(x_k) = P(x) for every tensor polynomial of degree < p
    per axis: the identity behind the nested basis (3.1)."""
    g = np.random.default_rng(100 + 10 * d + p)
    lo = g.random(d) - 0.5
    s = 1.0 + g.random()
    level = 3
    cell = [int(v) for v in g.integers(0, 4, size=d)]
    h = s * 2.0 ** (1 - level)
    corner = lo + np.array(cell) * h
    pts = corner + h * g.random((25, d))
    Ut = oracle.basis_t(pts, p, lo, s, level, cell)     # r x npts
    anchors1d = oracle.chebyshev(p)
    centre = corner + 0.5 * h
    idx = list(itertools.product(range(p), repeat=d))   # lexicographic, last fastest
    X_anchor = np.array([[centre[a] + 0.5 * h * anchors1d[k[a]] for a in range(d)] for k in idx])
    for alpha in itertools.product(range(p), repeat=d):
        coef = g.standard_normal()
        P = lambda X: coef * np.prod([X[:, a] ** alpha[a] for a in range(d)], axis=0)
        got = Ut.T @ P(X_anchor)
        want = P(pts)
        assert np.max(np.abs(got - want)) <= 1e-11 * max(1.0, np.max(np.abs(want)))
    # at the anchors themselves the basis is the identity matrix
    assert np.max(np.abs(oracle.basis_t(X_anchor, p, lo, s, level, cell) - np.eye(p ** d))) < 1e-12


# --------------------------------------------------------------------------
# Theorem 2.4 and (2.11): strong RRQR and the interpolative decomposition
# --------------------------------------------------------------------------

def _id_checks(Mt, tol, f=2.0):
    r, m = Mt.shape
    perm, k, A, ns = oracle.compr(Mt, tol, f)
    assert sorted(perm.tolist()) == list(range(m))
    assert ns >= 0
    sel, rest = perm[:k], perm[k:]
    # |R11^{-1} R12|_max <= f  (Theorem 2.4)
    if A.size:
        assert np.max(np.abs(A)) <= f * (1 + 1e-12)
    # Lemma 4.1: ||P [I; G]||_F <= f sqrt(m k)
    PIG = np.vstack([np.eye(k), A.T]) if k else np.zeros((m, 0))
    assert np.linalg.norm(PIG) <= f * np.sqrt(m * max(k, 1)) + 1e-12
    # ID: U^ = P [I; G] U^|_sel, i.e. Mt[:, rest] ~= Mt[:, sel] A
    if k and m > k:
        resid = np.linalg.norm(Mt[:, rest] - Mt[:, sel] @ A)
        assert resid <= 10 * np.sqrt(m) * max(tol, 1e-14) * np.linalg.norm(Mt) * (1 + np.sqrt(k * (m - k)) * f)
    return perm, k, A, ns


def test_compr_reduces_to_lapack_qrcp_when_no_swaps_needed():
    g = np.random.default_rng(5)
    hits = 0
    for trial in range(40):
        r, m = int(g.integers(3, 12)), int(g.integers(3, 30))
        Mt = g.standard_normal((r, m))
        perm, k, A, ns = _id_checks(Mt, 1e-13)
        assert k == min(r, m)
        if ns == 0:
            _, _, P = scipy.linalg.qr(Mt, pivoting=True)
            assert perm[:k].tolist() == P[:k].tolist()
            hits += 1
    assert hits > 20


def test_compr_numerical_rank():
    g = np.random.default_rng(6)
    for rank in (1, 3, 7):
        Mt = g.standard_normal((12, rank)) @ g.standard_normal((rank, 40))
        perm, k, A, ns = _id_checks(Mt, 1e-8)
        assert k == rank
    perm, k, A, ns = oracle.compr(np.zeros((4, 6)), 1e-8)
    assert k == 0


def test_compr_singular_value_bounds_vs_dense_svd():
    """Gu-Eisenstat bounds on tiny inputs: sigma_i(R11) >= sigma_i(M)/q and
    sigma_j(R22) <= sigma_{k+j}(M) q with q = sqrt(1 + f^2 k (m-k))."""
    g = np.random.default_rng(7)
    f = 2.0
    for trial in range(30):
        r, m = int(g.integers(4, 10)), int(g.integers(8, 25))
        # decaying spectrum so that the tolerance cuts the rank
        U, _ = np.linalg.qr(g.standard_normal((r, r)))
        V, _ = np.linalg.qr(g.standard_normal((m, r)))
        sv = 10.0 ** -np.arange(r) * 3.0
        Mt = U @ np.diag(sv) @ V.T
        perm, k, A, ns = _id_checks(Mt, 2e-3, f)
        sig = np.linalg.svd(Mt, compute_uv=False)
        q = np.sqrt(1 + f * f * k * (m - k))
        Q, R = np.linalg.qr(Mt[:, perm[:k]])
        s11 = np.linalg.svd(R, compute_uv=False)
        assert np.all(s11 >= sig[:k] / q * (1 - 1e-10))
        R22 = Mt[:, perm[k:]] - Q @ (Q.T @ Mt[:, perm[k:]])
        s22 = np.linalg.svd(R22, compute_uv=False)[: max(0, min(r, m) - k)]
        assert np.all(s22 <= sig[k:k + len(s22)] * q * (1 + 1e-8) + 1e-14)


def test_compr_swaps_grow_the_volume():
    """Each Gu-Eisenstat swap multiplies |det R11| by more than f, starting
    from the column-pivoted QR selection (LAPACK's, via scipy)."""
    g = np.random.default_rng(8)
    seen = 0
    for trial in range(240):
        d, p = 3, int(g.integers(2, 5))
        m = int(g.integers(p ** d, 4 * p ** d))
        pts = g.random((m, d)) ** int(g.integers(1, 4))      # clustered toward a corner
        Mt = oracle.basis_t(pts, p, [0.0, 0.0, 0.0], 1.0, 1, [0, 0, 0])
        perm, k, A, ns = _id_checks(Mt, 1e-8)
        if ns > 0:
            _, R0, P = scipy.linalg.qr(Mt, pivoting=True)
            vol0 = np.prod(np.abs(np.diag(R0)[:k]))
            vol1 = abs(np.linalg.det(np.linalg.qr(Mt[:, perm[:k]])[1]))
            assert vol1 >= vol0 * 2.0 ** ns * (1 - 1e-9)
            seen += 1
    assert seen >= 3


# --------------------------------------------------------------------------
# the whole construction and the matvec of Section 3.4
# --------------------------------------------------------------------------

def test_h2_equals_dense_when_root_is_a_leaf():
    x = si.uniform_cube(120, 3, 1)
    q = si.rhs(120, 3, 2)
    h = oracle.H2(x, 1, 128, 4, 1e-8)
    assert h.query("nadm") == 0 and h.query("nnear") == 1
    assert rel(h.matvec(q), kernel_matrix(1, x, x) @ q) < 1e-14


def test_h2_equals_dense_when_nothing_is_admissible():
    x = si.uniform_cube(800, 2, 3)
    q = si.rhs(800, 2, 4)
    h = oracle.H2(x, 0, 16, 4, 1e-8, tau=0.01)
    assert h.query("nadm") == 0
    assert rel(h.matvec(q), kernel_matrix(0, x, x) @ q) < 1e-13


def test_h2_symmetric_kernel_gives_symmetric_operator():
    x = si.uniform_cube(3000, 3, 5)
    h = oracle.H2(x, 1, 32, 3, 1e-8)
    v, w = si.rhs(3000, 1, 6)[:, 0], si.rhs(3000, 1, 7)[:, 0]
    a, b = v @ h.matvec(w), w @ h.matvec(v)
    assert abs(a - b) <= 1e-13 * (abs(a) + np.linalg.norm(v) * np.linalg.norm(h.matvec(w)))


@pytest.mark.parametrize("kid,d", [(0, 2), (1, 3)])
def test_h2_error_falls_with_order(kid, d):
    n = 3000 if d == 2 else 4000
    x = si.uniform_cube(n, d, 30 + d)
    q = si.rhs(n, 2, 31)
    rows = si.sample_rows(n, 300, 32)
    ref = kernel_matrix(kid, x[rows], x) @ q
    errs = []
    for p in ((2, 3, 4, 6, 8) if d == 2 else (2, 3, 4, 5)):
        z = oracle.H2(x, kid, 32, p, 1e-12).matvec(q)
        errs.append(rel(z[rows], ref))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < errs[0] * 1e-2


def test_h2_id_structure_at_every_node():
    x = si.uniform_cube(4000, 2, 50)
    h = oracle.H2(x, 0, 40, 6, 1e-8)
    e = h.export()
    ibar, skel, rest, G = local_positions(e, "row")
    for g in range(len(e["level"])):
        if e["level"][g] == 1:
            continue
        assert np.all(np.diff(skel[g]) > 0) and np.all(np.diff(rest[g]) > 0)
        assert sorted(np.concatenate([skel[g], rest[g]]).tolist()) == sorted(ibar[g].tolist())
        if G[g].size:
            assert np.max(np.abs(G[g])) <= 2.0 * (1 + 1e-12)
        U = dense_transfer(ibar[g], skel[g], rest[g], G[g])
        pos = {int(v): i for i, v in enumerate(ibar[g])}
        rows_sel = [pos[int(v)] for v in skel[g]]
        assert np.array_equal(U[rows_sel], np.eye(len(skel[g])))   # identity rows (2.11)
        assert np.linalg.norm(U) <= 2.0 * np.sqrt(len(ibar[g]) * max(1, len(skel[g])))


def _telescoping_matvec(e, x, kid, q, absval=False):
    """(3.24)-(3.26) on a perfect tree, written with dense block-diagonal
    U^(l) (3.22) and dense coupling blocks B^(l) from the skeleton indices.
    absval: the same products with every generator, kernel entry and q
    replaced by its magnitude."""
    L = e["L"]
    xs = x[e["permx"]]
    ibar, skel, rest, G = local_positions(e, "row")
    if absval:
        G = [np.abs(g) for g in G]
        q = np.abs(q)
        kmat = lambda k, a, b: np.abs(kernel_matrix(k, a, b))
    else:
        kmat = kernel_matrix
    lvl = lambda l: range(e["lvl_off"][l - 1], e["lvl_off"][l])
    Ublk = {}
    for l in range(2, L + 1):
        Ublk[l] = scipy.linalg.block_diag(*[dense_transfer(ibar[g], skel[g], rest[g], G[g])
                                            for g in lvl(l)])
    qs = q[e["permy"]]
    # (3.24)
    qhat = {}
    v = qs
    for l in range(L, 1, -1):
        v = Ublk[l].T @ v
        qhat[l] = v
    # (3.25): B^(l-1) has blocks B_ij for (i,j) in L at level l
    def skel_offsets(l):
        offs, acc = {}, 0
        for g in lvl(l):
            offs[g] = acc
            acc += len(skel[g])
        return offs, acc
    zhat = {}
    for l in range(2, L + 1):
        offs, tot = skel_offsets(l)
        B = np.zeros((tot, tot))
        for i in lvl(l):
            for t in range(e["adm_ptr"][i], e["adm_ptr"][i + 1]):
                j = int(e["adm_col"][t])
                assert e["level"][j] == l
                B[offs[i]:offs[i] + len(skel[i]), offs[j]:offs[j] + len(skel[j])] = \
                    kmat(kid, xs[skel[i]], xs[skel[j]])
        zhat[l] = B @ qhat[l]
    # B^(L): near field
    n = len(xs)
    BL = np.zeros((n, n))
    for i in lvl(L):
        for t in range(e["near_ptr"][i], e["near_ptr"][i + 1]):
            j = int(e["near_col"][t])
            BL[e["rs"][i]:e["rs"][i] + e["rc"][i], e["cs"][j]:e["cs"][j] + e["cc"][j]] = \
                kmat(kid, xs[e["rs"][i]:e["rs"][i] + e["rc"][i]], xs[e["cs"][j]:e["cs"][j] + e["cc"][j]])
    # (3.26)
    w = Ublk[2] @ zhat[2]
    for l in range(3, L + 1):
        w = Ublk[l] @ (w + zhat[l])
    zs = BL @ qs + w
    z = np.empty_like(zs)
    z[e["permx"]] = zs
    return z


@pytest.mark.parametrize("d,cells,per_cell,p,kid", [(2, 16, 16, 3, 0), (1, 64, 8, 5, 3), (3, 4, 16, 2, 1)])
def test_h2_nodewise_matvec_equals_telescoping_form(d, cells, per_cell, p, kid):
    x = si.jittered_grid(cells, d, 90 + d, per_cell=per_cell)
    q = si.rhs(len(x), 2, 91)
    h = oracle.H2(x, kid, per_cell, p, 1e-10)
    e = h.export()
    assert e["leaf"][e["lvl_off"][e["L"] - 1]:].all() and not e["leaf"][:e["lvl_off"][e["L"] - 1]].any()
    assert e["G_row"].size > 0
    z_tel = _telescoping_matvec(e, x, kid, q)
    z = h.matvec(q)
    assert rel(z, z_tel) < 1e-12
    # and the approximation is a real one
    assert 0 < rel(z, kernel_matrix(kid, x, x) @ q) < 1e-2


# ---------------------------------------------------------------- row scales of A^ q
def test_h2_abs_matvec_is_dense_abs_when_root_is_a_leaf():
    x = si.uniform_cube(120, 2, 121)
    q = si.rhs(120, 3, 122)
    h = oracle.H2(x, 0, 128, 4, 1e-8)
    assert h.query("nadm") == 0
    assert rel(h.matvec_abs(q), np.abs(kernel_matrix(0, x, x)) @ np.abs(q)) < 1e-14


@pytest.mark.parametrize("d,cells,per_cell,p,kid", [(2, 16, 16, 3, 0), (1, 64, 8, 5, 3), (3, 4, 16, 2, 1)])
def test_h2_abs_matvec_equals_telescoping_form_of_magnitudes(d, cells, per_cell, p, kid):
    """On perfect trees the node-wise sums of |terms| equal (3.24)-(3.26)
    written with |U^(l)|, |B^(l)| and |q|: both expand to the same sum over
    paths of products of nonnegative factors."""
    x = si.jittered_grid(cells, d, 90 + d, per_cell=per_cell)
    q = si.rhs(len(x), 2, 91)
    h = oracle.H2(x, kid, per_cell, p, 1e-10)
    e = h.export()
    za = h.matvec_abs(q)
    assert rel(za, _telescoping_matvec(e, x, kid, q, absval=True)) < 1e-12
    assert rel(za, _telescoping_matvec(e, x, kid, q)) > 1e-2   # not the signed sums


@pytest.mark.parametrize("kid,d,n", [(0, 2, 3000), (1, 3, 4000), (2, 3, 3000)])
def test_h2_abs_matvec_bounds(kid, d, n):
    """Triangle inequality: |(A^ q)_i| <= (|A^| |q|)_i, row by row.  And
    (|A^| |q|)_i >= sum_j |A_ij| |q_j| - sum_j |E_ij| |q_j| with E = A^ - A,
    so it is not below the dense sum of magnitudes by more than the
    approximation error (here ~1e-3 per entry at order 4)."""
    x = si.gaussian_mixture(n, d, 3, sigma=0.1) if kid == 2 else si.uniform_cube(n, d, 130 + kid)
    q = si.rhs(n, 3, 131)
    h = oracle.H2(x, kid, 32, 4, 1e-8)
    assert h.query("nadm") > 0
    za, z = h.matvec_abs(q), h.matvec(q)
    assert np.all(za >= np.abs(z) * (1 - 1e-13))
    rows = si.sample_rows(n, 200, 132)
    dense_abs = np.abs(kernel_matrix(kid, x[rows], x)) @ np.abs(q)
    assert np.all(za[rows] >= 0.99 * dense_abs)
    # a sampled leaf set gives the same rows
    e = h.export()
    leaves = np.flatnonzero(e["leaf"])[[0, 3, -1]].astype(np.int32)
    zs = h.matvec_abs(q, leaves)
    sel = np.concatenate([e["permx"][e["rs"][g]:e["rs"][g] + e["rc"][g]] for g in leaves])
    assert np.array_equal(zs[sel], za[sel])


def test_h2_rectangular_cauchy_close_to_dense():
    x, y = si.cauchy_1d(3000, 60)
    q = si.rhs(3000, 2, 61)
    h = oracle.H2(x, 3, 32, 16, 1e-10, y=y)
    ref = kernel_matrix(3, x, y) @ q
    assert rel(h.matvec(q), ref) < 1e-6


def test_h2_matvec_on_selected_leaves_equals_full_matvec():
    x = si.uniform_cube(5000, 3, 77)
    q = si.rhs(5000, 3, 78)
    h = oracle.H2(x, 1, 64, 3, 1e-8)
    e = h.export()
    leaves = np.flatnonzero(e["leaf"])[[0, 5, -1]].astype(np.int32)
    zsel = h.matvec_leaves(q, leaves)
    zall = h.matvec(q)
    rows = np.concatenate([e["permx"][e["rs"][g]:e["rs"][g] + e["rc"][g]] for g in leaves])
    assert np.array_equal(zsel[rows], zall[rows])
    others = np.setdiff1d(np.arange(5000), rows)
    assert np.all(np.isnan(zsel[others]))


# ---------------------------------------------------------------- Section 6.4 kernels
def _double_layer_dense(c, pts, rows=None):
    """sum_a kernel_a(x, y_j) nu_a(y_j) w_j for the oracle's gradient kernels."""
    x, nu, w = c["x"], c["nu"], c["w"]
    q1 = np.ascontiguousarray((nu[:, 0] * w)[:, None])
    q2 = np.ascontiguousarray((nu[:, 1] * w)[:, None])
    return (oracle.dense_rows(pts, 4, q1, rows=rows, y=x) + oracle.dense_rows(pts, 5, q2, rows=rows, y=x)).ravel()


@pytest.mark.parametrize("name,inside,n", [("ram_head", (0.1, 0.1), 2000), ("sunflower", (1.5, 0.0), 40000)])
def test_gradient_kernels_satisfy_gauss_integral(name, inside, n):
    """Gauss's integral for the double layer of Section 6.4 with
    Phi = -(1/2 pi) log|x - y| and outer normals: int_Gamma dPhi/dnu_y ds_y is
    -1 inside the domain, 0 outside and -1/2 on the (smooth) boundary.  The
    trapezoidal rule on these periodic curves converges spectrally; on the
    curve the Nystrom diagonal is the kernel's limit -curvature/(4 pi) times
    the weight.  A wrong sign, factor or component of the kernels fails."""
    c = si.curve_6_4(name, n)
    v_in = _double_layer_dense(c, np.array([inside]))
    v_out = _double_layer_dense(c, np.array([[5.0, 5.0]]))
    assert abs(v_in[0] + 1.0) < 1e-12
    assert abs(v_out[0]) < 1e-12
    rows = np.arange(0, n, n // 50)
    on = _double_layer_dense(c, c["x"], rows=rows) - c["curvature"][rows] / (4 * np.pi) * c["w"][rows]
    assert np.max(np.abs(on + 0.5)) < 1e-7


def test_gradient_kernels_are_antisymmetric_and_h2_converges():
    """kernel_a(x, y) = -kernel_a(y, x) (the gradient of a symmetric function
    of x - y), and the oracle's H^2 matrix of a gradient kernel converges to
    the dense product as the order rises."""
    a, b = np.array([0.3, -0.2]), np.array([-1.1, 0.7])
    for kid in (4, 5):
        assert oracle.kernel(kid, a, b) == -oracle.kernel(kid, b, a)
        assert oracle.kernel(kid, a, a) == 0.0
    c = si.curve_6_4("ram_head", 3000)
    q = si.rhs(3000, 2, 7000)
    zd = oracle.dense_rows(c["x"], 4, q)
    errs = [rel(oracle.H2(c["x"], 4, 50, p, 1e-14).matvec(q), zd) for p in (4, 6, 8)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-12, errs
