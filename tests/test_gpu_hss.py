"""GPU parity of the HSS construction (Section 3.3.1, Appendix A) against the
CPU oracle, for points on a line: the Cauchy kernel 1/(x - y) with the
interlaced X != Y of the serving configuration, and 1/|x - y| with X = Y.

Bars: the lists of (3.5), the nearfield sets N_i of (A.1), the numbers of
singular vectors, ranks, skeletons and every G entry bit-identical (the
nearfield blocks are evaluated with IEEE division and square root, the
Jacobi SVD and the compression run the oracle's operations in its order);
the matvec entry by entry within 1e-12 of each entry's sum of |terms|
(FP64) and 1e-5 (FP32); the approximation error against the dense product
falling with eps_svd.  For the log kernel the nearfield entries come from
the device's log, so bits may differ from the oracle's; there the matvec is
checked against the dense product.
"""
import numpy as np
import pytest

import oracle
import smash_inputs as si
from oracle_helpers import kernel_matrix
from parity_helpers import TOL_F32, TOL_F64, assert_entrywise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

DEV = torch.device("cuda:0")
KEYS = ["permx", "permy", "lvl_off", "level", "leaf", "parent", "child0", "nchild", "rs", "rc", "cs", "cc", "cell",
        "adm_ptr", "adm_col", "near_ptr", "near_col"]


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _compare(h, ho, sides):
    eg, eo = sm.smash_export(h), ho.export()
    for k in KEYS:
        assert np.array_equal(np.asarray(eg[k]), np.asarray(eo[k])), k
    xg = sm.smash_export_hss(h)
    assert np.array_equal(xg["nf_ptr"], eo["nf_ptr"]) and np.array_equal(xg["nf_col"], eo["nf_col"])
    assert np.array_equal(xg["svd_row"], eo["svd_row"])
    if "col" in sides:
        assert np.array_equal(xg["svd_col"], eo["svd_col"])
    for tag in sides:
        for k in (f"m_{tag}", f"k_{tag}", f"skel_{tag}", f"rest_{tag}"):
            assert np.array_equal(eg[k], eo[k]), k
        assert np.array_equal(eg[f"G_{tag}"], eo[f"G_{tag}"]), f"G_{tag} not bit-identical"


@pytest.mark.parametrize("n,leaf,p,eps", [(3000, 32, 12, 1e-10), (20000, 64, 16, 1e-12)])
def test_hss_cauchy_rectangular(n, leaf, p, eps):
    x, y = si.cauchy_1d(n, 900 + n)
    q = si.rhs(n, 3, 901)
    ho = oracle.HSS(x, 3, leaf, p, 1e-12, eps, y=y, tau=0.6)
    h = sm.smash_build_hss(_dev(x), _dev(y), sm.SMASH_K_CAUCHY1D, leaf, p, 1e-12, eps, tau=0.6)
    _compare(h, ho, ("row", "col"))
    zo, sc = ho.matvec(q), ho.matvec_abs(q)
    for prec, bar in ((sm.SMASH_PREC_F64, TOL_F64), (sm.SMASH_PREC_F32, TOL_F32)):
        z = np.empty_like(q)
        sm.smash_matvec_ex(h, q, z, prec)
        assert_entrywise(z, zo, sc, bar, what=f"n={n} precision {prec}")
    with pytest.raises(sm.SmashError):
        sm.smash_matvec_ex(h, q, np.empty_like(q), sm.SMASH_PREC_F32X2)
    sm.smash_free(h)


def test_hss_symmetric_kernel_same_points():
    x = si.uniform_cube(8000, 1, 910)
    q = si.rhs(8000, 2, 911)
    ho = oracle.HSS(x, 1, 32, 10, 1e-12, 1e-10, tau=0.6)
    h = sm.smash_build_hss(_dev(x), None, sm.SMASH_K_INVR, 32, 10, 1e-12, 1e-10, tau=0.6)
    _compare(h, ho, ("row",))
    zo, sc = ho.matvec(q), ho.matvec_abs(q)
    z = np.empty_like(q)
    sm.smash_matvec_ex(h, q, z)
    assert_entrywise(z, zo, sc, TOL_F64, what="1/r")
    sm.smash_free(h)


def test_hss_log_kernel_against_dense_and_errors_fall():
    x = si.uniform_cube(4000, 1, 920)
    q = si.rhs(4000, 2, 921)
    A = kernel_matrix(0, x, x)
    errs = []
    for eps in (1e-3, 1e-6, 1e-10):
        h = sm.smash_build_hss(_dev(x), None, sm.SMASH_K_LOG, 32, 8, 1e-12, eps, tau=0.6)
        z = np.empty_like(q)
        sm.smash_matvec_ex(h, q, z)
        errs.append(np.linalg.norm(z - A @ q) / np.linalg.norm(A @ q))
        sm.smash_free(h)
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 1e-8, errs


def test_hss_root_leaf_and_invalid_input():
    x = si.uniform_cube(50, 1, 930)
    q = si.rhs(50, 1, 931)
    h = sm.smash_build_hss(x, None, sm.SMASH_K_INVR, 64, 8, 1e-12, 1e-10)
    z = np.empty_like(q)
    sm.smash_matvec_ex(h, q, z)
    zd = oracle.dense_rows(x, 1, q)
    assert np.linalg.norm(z - zd) <= 1e-14 * np.linalg.norm(zd)
    sm.smash_free(h)
    # points in the plane are refused (by the binding: the C ABI sees n doubles)
    with pytest.raises(ValueError):
        sm.smash_build_hss(si.uniform_cube(100, 2, 932), None, sm.SMASH_K_INVR, 16, 4, 1e-8, 1e-8)
    # and the library refuses the kernels it does not take, and a bad eps_svd
    with pytest.raises(sm.SmashError):
        sm.smash_build_hss(si.uniform_cube(100, 1, 933), None, sm.SMASH_K_DLP1, 16, 4, 1e-8, 1e-8)
    with pytest.raises(sm.SmashError):
        sm.smash_build_hss(si.uniform_cube(100, 1, 934), None, sm.SMASH_K_INVR, 16, 4, 1e-8, 0.0)
