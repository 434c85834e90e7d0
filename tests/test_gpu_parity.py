"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Bars, each with the reason it holds:
  - partition, Morton keys, permutations, tree arrays, L and L^- lists:
    bit-exact (integer work);
  - ranks, skeleton and rest index sets: bit-exact;
  - G matrices: bit-exact -- the compression kernel evaluates every basis
    value, dot product and norm in the oracle's operation order without FMA
    contraction, so identical inputs give identical bits;
  - FP64 matvec: entry by entry against the oracle's H^2 matvec, each
    difference within 1e-12 of that entry's sum of |terms| (only the
    summation order and the rounding of the entries differ; see
    parity_helpers), four orders inside the 1e-8 parity bar.  At N = 2^20
    the rows of 64 sampled leaves (box corners and faces included) are
    compared.
"""
import numpy as np
import pytest

import oracle
import smash_inputs as si
from parity_helpers import TOL_F64, assert_entrywise, leaf_rows, oracle_reference, sample_leaves

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

DEV = torch.device("cuda:0")

TREE_KEYS = ["permx", "permy", "keyx", "keyy", "lvl_off", "level", "leaf", "parent", "child0", "nchild",
             "rs", "rc", "cs", "cc", "cell"]
LIST_KEYS = ["adm_ptr", "adm_col", "near_ptr", "near_col"]


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _gpu_build(x, kid, leaf, order, tol, y=None):
    if y is None:
        return sm.H2Matrix(_dev(x), kid, leaf, order, tol)
    return sm.H2Matrix(_dev(x), kid, leaf, order, tol, y=_dev(y))


def _compare_exports(eg, eo, sides=("row",)):
    for k in TREE_KEYS:
        assert np.array_equal(np.asarray(eg[k]), np.asarray(eo[k])), f"tree array {k} differs"
    for k in LIST_KEYS:
        assert np.array_equal(eg[k], eo[k]), f"list array {k} differs"
    for tag in sides:
        for k in (f"m_{tag}", f"k_{tag}", f"skel_{tag}", f"rest_{tag}"):
            assert np.array_equal(eg[k], eo[k]), f"{k} differs"
        gg, go = eg[f"G_{tag}"], eo[f"G_{tag}"]
        if not np.array_equal(gg, go):
            diff = np.max(np.abs(gg - go)) if gg.size else 0.0
            pytest.fail(f"G_{tag} not bit-identical: max |diff| {diff:.3e}")


CASES = {
    "2d_log_4096": dict(x=lambda: si.uniform_cube(4096, 2, 0), kid=0, leaf=64, order=5, tol=1e-8, nrhs=4),
    "3d_invr_20000": dict(x=lambda: si.uniform_cube(20000, 3, 1), kid=1, leaf=128, order=4, tol=1e-8, nrhs=16),
    "sphere_yukawa_8192": dict(x=lambda: si.sphere_with_caps(8192, 2), kid=2, leaf=128, order=5, tol=1e-8,
                               nrhs=32),
    "2d_mixture_6000": dict(x=lambda: si.gaussian_mixture(6000, 2, 3, sigma=0.05), kid=0, leaf=32, order=6,
                            tol=1e-10, nrhs=3),
    "1d_invr_3000": dict(x=lambda: si.uniform_cube(3000, 1, 4), kid=1, leaf=16, order=12, tol=1e-12, nrhs=1),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    c = CASES[request.param]
    x = c["x"]()
    q = si.rhs(len(x), c["nrhs"], 99)
    ho = oracle.H2(x, c["kid"], c["leaf"], c["order"], c["tol"])
    hg = _gpu_build(x, c["kid"], c["leaf"], c["order"], c["tol"])
    params = {k: v for k, v in c.items() if k != "x"}
    yield dict(name=request.param, x=x, q=q, ho=ho, hg=hg, **params)
    hg.close()


def test_build_is_bit_exact(case):
    eg, eo = case["hg"].export(), case["ho"].export()
    _compare_exports(eg, eo)
    assert case["hg"].info()["swaps"] == eo["swaps_row"]


def test_matvec_fp64_parity(case):
    zo, sc = oracle_reference(case["ho"], case["q"])
    zg = case["hg"].matvec(_dev(case["q"])).cpu().numpy()
    assert_entrywise(zg, zo, sc, TOL_F64, what=case["name"])


def test_matvec_host_buffers_equal_device_buffers(case):
    q = case["q"]
    zd = case["hg"].matvec(_dev(q)).cpu().numpy()
    zh = case["hg"].matvec(np.ascontiguousarray(q))
    assert np.array_equal(zd, zh)


def test_rectangular_cauchy_bit_exact_and_parity():
    x, y = si.cauchy_1d(5000, 40)
    q = si.rhs(5000, 5, 41)
    ho = oracle.H2(x, 3, 64, 16, 1e-10, y=y)
    hg = _gpu_build(x, 3, 64, 16, 1e-10, y=y)
    _compare_exports(hg.export(), ho.export(), sides=("row", "col"))
    zo, sc = oracle_reference(ho, q)
    zg = hg.matvec(_dev(q)).cpu().numpy()
    assert_entrywise(zg, zo, sc, TOL_F64, what="cauchy x != y")
    hg.close()


@pytest.mark.parametrize("nrhs", [1, 3, 17, 33, 64])
def test_ragged_rhs_counts(nrhs):
    x = si.uniform_cube(6000, 3, 50)
    q = si.rhs(6000, nrhs, 51)
    ho = oracle.H2(x, 1, 64, 3, 1e-8)
    hg = _gpu_build(x, 1, 64, 3, 1e-8)
    zo, sc = oracle_reference(ho, q)
    zg = hg.matvec(_dev(q)).cpu().numpy()
    assert_entrywise(zg, zo, sc, TOL_F64, what=f"nrhs={nrhs}")
    hg.close()


def test_root_leaf_is_dense():
    x = si.uniform_cube(100, 3, 60)
    q = si.rhs(100, 2, 61)
    hg = _gpu_build(x, 1, 128, 4, 1e-8)
    info = hg.info()
    assert info["nadm"] == 0 and info["nnear"] == 1 and info["levels"] == 1
    z = hg.matvec(_dev(q)).cpu().numpy()
    zd = oracle.dense_rows(x, 1, q)
    assert np.linalg.norm(z - zd) / np.linalg.norm(zd) < 1e-13
    # here A^ = A, so the dense sums of magnitudes are the row scales
    sc = oracle.dense_rows(x, 1, np.abs(q))
    assert_entrywise(z, zd, sc, TOL_F64, what="root leaf")
    hg.close()


def test_single_point_and_duplicates():
    x1 = np.array([[0.3, 0.4, 0.5]])
    hg = _gpu_build(x1, 1, 8, 2, 1e-8)
    z = hg.matvec(_dev(np.ones((1, 1)))).cpu().numpy()
    assert z[0, 0] == 0.0                      # kappa(x, x) = 0
    hg.close()
    x = np.concatenate([np.full((40, 2), 0.25), si.uniform_cube(200, 2, 62)])
    q = si.rhs(240, 2, 63)
    ho = oracle.H2(x, 0, 8, 3, 1e-8)
    hg = _gpu_build(x, 0, 8, 3, 1e-8)
    _compare_exports(hg.export(), ho.export())
    zo, sc = oracle_reference(ho, q)
    zg = hg.matvec(_dev(q)).cpu().numpy()
    assert_entrywise(zg, zo, sc, TOL_F64, what="duplicates")
    hg.close()


def test_error_vs_dense_small_configs():
    """The approximation error at the configs' orders (reported, loosely bounded)."""
    x = si.uniform_cube(4096, 2, 0)
    q = si.rhs(4096, 4, 500)
    hg = _gpu_build(x, 0, 64, 5, 1e-8)
    z = hg.matvec(_dev(q)).cpu().numpy()
    zd = oracle.dense_rows(x, 0, q)
    err = np.linalg.norm(z - zd) / np.linalg.norm(zd)
    assert err < 1e-4, err
    hg.close()


def test_full_size_headline_workload(headline_oracle):
    """The 3D 1/r workload at N = 2^20 in the launch configuration the
    benchmark times: the whole build is compared with the oracle's build
    array by array, and the matvec entry by entry on the rows of 64 sampled
    leaves (the leaves at the corners and face centres of the box, the leaves
    the double-float near field leaves to its fallback, the rest at random)
    with the oracle's H^2 matvec on the same leaves."""
    w, ho, eo = headline_oracle
    x, q = w["x"], w["q"]
    hg = _gpu_build(x, w["kernel"], w["leaf"], w["order"], w["tol"])
    eg = hg.export()
    _compare_exports(eg, eo)
    zg = hg.matvec(_dev(q)).cpu().numpy()
    fb = sm.smash_near_fallback_leaves(hg.h)
    pick = sample_leaves(eo, x, 64, seed=1, extra=fb)
    assert len(pick) >= 64 and set(fb.tolist()) <= set(pick.tolist())
    zo, sc = oracle_reference(ho, q, pick)
    rows = leaf_rows(eo, pick)
    worst, rel2 = assert_entrywise(zg, zo, sc, TOL_F64, rows=rows, what="N=2^20 sampled leaves")
    # approximation error against the dense product on the same rows
    zd = oracle.dense_rows(x, w["kernel"], q, rows=rows[:256])
    err = np.linalg.norm(zg[rows[:256]] - zd) / np.linalg.norm(zd)
    assert err < 1e-3, err
    hg.close()
