"""GPU parity of the mixed-precision matvec (SMASH_PREC_F32) against FP64.

Bar: relative 2-norm error <= 1e-5 against the FP64 H^2 matvec of the same
representation (the mixed-precision bar).  Budget: an FP32 kernel entry is
within a few ulps (~2e-7 relative; differences are taken from two-float
coordinates, so close pairs lose nothing before the rounding to FP32), the
products and the coupling sums are FP32 (errors of random sign: ~1e-7 times
the row's scale), the near field is Kahan-compensated, the transfers are FP64.
Observed errors are ~1e-7..1e-6, one to two orders inside the bar.  Every
comparison with the oracle is entry by entry: each difference within 1e-5 of
the entry's sum of |terms| (parity_helpers); the relative 2-norm is a second
line.
"""
import numpy as np
import pytest

import oracle
import smash_inputs as si
from parity_helpers import (TOL_BF16, TOL_F32, TOL_F64, TOL_TF32, TOL_TF32X3, assert_entrywise, leaf_rows,
                            oracle_reference, sample_leaves)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

DEV = torch.device("cuda:0")
RTOL = 1e-5
F32 = sm.SMASH_PREC_F32


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    ("2d_log", lambda: si.uniform_cube(8000, 2, 400), None, sm.SMASH_K_LOG, 64, 5, 1e-8, 4),
    ("3d_invr", lambda: si.uniform_cube(20000, 3, 401), None, sm.SMASH_K_INVR, 128, 4, 1e-8, 16),
    ("sphere_yukawa", lambda: si.sphere_with_caps(12000, 402), None, sm.SMASH_K_YUKAWA, 128, 5, 1e-8, 32),
    ("mixture_2d_invr", lambda: si.gaussian_mixture(8000, 2, 403, sigma=0.05), None, sm.SMASH_K_INVR, 32, 6,
     1e-10, 3),
]


@pytest.mark.parametrize("name,xf,yf,kid,leaf,order,tol,nrhs", CASES, ids=[c[0] for c in CASES])
def test_f32_matches_oracle(name, xf, yf, kid, leaf, order, tol, nrhs):
    x = xf()
    q = si.rhs(len(x), nrhs, 404)
    zo, sc = oracle_reference(oracle.H2(x, kid, leaf, order, tol), q)
    H = sm.H2Matrix(_dev(x), kid, leaf, order, tol)
    z = H.matvec(_dev(q), precision=F32).cpu().numpy()
    assert_entrywise(z, zo, sc, TOL_F32, what=name)
    err = _rel(z, zo)
    assert err <= RTOL, f"{name}: {err:.3e}"
    H.close()


def test_f32_cauchy_rectangular():
    x, y = si.cauchy_1d(6000, 405)
    q = si.rhs(6000, 4, 406)
    zo, sc = oracle_reference(oracle.H2(x, sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10, y=y), q)
    H = sm.H2Matrix(_dev(x), sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10, y=_dev(y))
    z = H.matvec(_dev(q), precision=F32).cpu().numpy()
    assert_entrywise(z, zo, sc, TOL_F32, what="cauchy x != y")
    assert _rel(z, zo) <= RTOL
    H.close()


def test_sphere_yukawa_full_size_against_the_oracle(sphere_oracle):
    """The mixed-precision workload at N = 2^20 (sphere with caps, Yukawa,
    order 5, 32 RHS): every precision against the FP64 oracle entry by entry
    on the rows of 64 sampled leaves (about 4100 rows: box corners, face
    centres, the rest at random), against the FP64 GPU matvec on all rows,
    and the FP64 result against the dense product on sampled rows."""
    w, ho, eo = sphere_oracle
    x, q = w["x"], w["q"]
    H = sm.H2Matrix(_dev(x), w["kernel"], w["leaf"], w["order"], w["tol"])
    qd = _dev(q)
    z64 = H.matvec(qd).cpu().numpy()
    pick = sample_leaves(eo, x, 64, seed=4)
    rows = leaf_rows(eo, pick)
    assert len(rows) >= 3000
    zo, sc = oracle_reference(ho, q, pick)
    assert_entrywise(z64, zo, sc, TOL_F64, rows=rows, what="f64")
    for p, etol, rtol in ((F32, TOL_F32, RTOL), (sm.SMASH_PREC_TF32X3, TOL_TF32X3, 1e-5),
                          (sm.SMASH_PREC_TF32, TOL_TF32, 1e-3), (sm.SMASH_PREC_BF16, TOL_BF16, 8e-3)):
        z = H.matvec(qd, precision=p).cpu().numpy()
        assert_entrywise(z, zo, sc, etol, rows=rows, what=f"precision {p}")
        assert _rel(z[rows], zo[rows]) <= rtol, p
        assert _rel(z, z64) <= rtol, p
    sel = si.sample_rows(len(x), 128, 407)
    zd = oracle.dense_rows(x, w["kernel"], q, rows=sel)
    err = _rel(z64[sel], zd)
    assert err < 1e-3, err
    H.close()
