"""Pins of the oracle's HSS construction (Section 3.3.1, Appendix A) and of
its truncated SVD, against LAPACK (numpy/scipy), dense kernel matrices, the
statements the paper makes about the nearfield sets N_i, and identities of
the representation."""
import numpy as np
import pytest

import oracle
import smash_inputs as si
from oracle_helpers import kernel_matrix


def test_jacobi_matches_lapack_singular_values_and_is_orthogonal():
    rng = np.random.default_rng(3)
    for m, n in ((7, 20), (16, 16), (30, 12), (5, 1)):
        A = rng.standard_normal((m, n)) * np.logspace(0, -9, n)[None, :]
        JT, sig, sweeps = oracle.jacobi_rows(A)
        ref = np.linalg.svd(A, compute_uv=False)
        assert np.allclose(np.sort(sig)[::-1][: len(ref)], ref, rtol=1e-12, atol=1e-15 * ref[0])
        assert np.allclose(JT @ JT.T, np.eye(m), atol=1e-14)
        assert sweeps < 60


def test_truncated_svd_spans_lapacks_leading_left_subspace():
    rng = np.random.default_rng(4)
    U0, _ = np.linalg.qr(rng.standard_normal((24, 24)))
    V0, _ = np.linalg.qr(rng.standard_normal((40, 24)))
    s0 = np.logspace(0, -14, 24)
    A = U0 @ np.diag(s0) @ V0.T
    for eps in (1e-4, 1e-8, 1e-11):
        ST = oracle.truncated_svd_rows(A, eps)
        keep = int(np.sum(s0 > eps * s0[0]))
        assert ST.shape == (keep, 24)
        assert np.allclose(ST @ ST.T, np.eye(keep), atol=1e-13)
        # principal angles with the exact leading subspace
        cosines = np.linalg.svd(ST @ U0[:, :keep], compute_uv=False)
        assert np.all(cosines > 1 - 1e-10)


def _hss(x, y=None, kid=3, leaf=32, p=12, eps=1e-10, tau=0.6):
    return oracle.HSS(x, kid, leaf, p, 1e-12, eps, y=y, tau=tau)


def test_hss_lists_are_3_5_and_cover_the_matrix_once():
    x, y = si.cauchy_1d(2000, 20)
    h = _hss(x, y)
    e = h.export()
    nn = len(e["level"])
    cover = 0
    for g in range(nn):
        sib = set(range(e["child0"][e["parent"][g]], e["child0"][e["parent"][g]] + e["nchild"][e["parent"][g]])) \
            - {g} if e["parent"][g] >= 0 else set()
        assert set(e["adm_col"][e["adm_ptr"][g]:e["adm_ptr"][g + 1]].tolist()) == sib
        near = e["near_col"][e["near_ptr"][g]:e["near_ptr"][g + 1]].tolist()
        assert near == ([g] if e["leaf"][g] else [])
        for j in e["adm_col"][e["adm_ptr"][g]:e["adm_ptr"][g + 1]]:
            cover += int(e["rc"][g]) * int(e["cc"][j])
        for j in near:
            cover += int(e["rc"][g]) * int(e["cc"][j])
    assert cover == 2000 * 2000


def test_nearfield_sets_of_uniform_points_at_tau_one_half():
    """Appendix A: for uniform points on [0, 1] (a perfect binary tree) and
    tau = 0.5, N_i holds at most two nodes, and its third case (leaves of
    N_{p_i}) is empty."""
    x = (np.arange(4096) + 0.5) / 4096
    h = _hss(x[:, None], kid=1, leaf=16, tau=0.5)
    e = h.export()
    sizes = np.diff(e["nf_ptr"])
    assert sizes[1:].max() <= 2 and sizes[0] == 0
    for g in range(1, len(sizes)):
        for k in e["nf_col"][e["nf_ptr"][g]:e["nf_ptr"][g + 1]]:
            assert e["level"][k] == e["level"][g]       # no coarser leaf (third case)


def test_hss_is_dense_when_the_root_is_a_leaf():
    x = si.uniform_cube(40, 1, 31)
    q = si.rhs(40, 2, 32)
    h = _hss(x, kid=0, leaf=64)
    assert h.query("nadm") == 0
    A = kernel_matrix(0, x, x)
    assert np.linalg.norm(h.matvec(q) - A @ q) <= 1e-14 * np.linalg.norm(A @ q)


@pytest.mark.parametrize("kid", [0, 1, 3])
def test_hss_error_falls_with_the_svd_tolerance(kid):
    if kid == 3:
        x, y = si.cauchy_1d(3000, 40)
    else:
        x, y = si.uniform_cube(3000, 1, 41 + kid), None
    q = si.rhs(3000, 2, 42)
    A = kernel_matrix(kid, x, x if y is None else y)
    errs = []
    for eps in (1e-2, 1e-5, 1e-9):
        h = _hss(x, y, kid=kid, p=6, eps=eps)
        e = h.export()
        assert np.abs(e["G_row"]).max() <= 2.0 * (1 + 1e-12)
        assert e["svd_row"].max() > 0
        errs.append(np.linalg.norm(h.matvec(q) - A @ q) / np.linalg.norm(A @ q))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 1e-7, errs


def test_hss_cauchy_kernel_is_antisymmetric():
    x = si.uniform_cube(2500, 1, 51)
    h = _hss(x, kid=3, leaf=32, p=12, eps=1e-12)
    rng = np.random.default_rng(52)
    v, w = rng.standard_normal(2500), rng.standard_normal(2500)
    a, b = v @ h.matvec(w), w @ h.matvec(v)
    assert abs(a + b) <= 1e-12 * np.linalg.norm(v) * np.linalg.norm(h.matvec(w))
