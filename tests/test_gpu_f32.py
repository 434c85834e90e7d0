"""GPU parity of the mixed-precision matvec (SMASH_PREC_F32) against FP64.

Bar: relative 2-norm error <= 1e-5 against the FP64 H^2 matvec of the same
representation (the mixed-precision bar).  Budget: an FP32 kernel entry is
within a few ulps (~2e-7 relative; differences are taken from two-float
coordinates, so close pairs lose nothing before the rounding to FP32), the
products and the coupling sums are FP32 (errors of random sign: ~1e-7 times
the row's scale), the near field is Kahan-compensated, the transfers are FP64.
Observed errors are ~1e-7..1e-6, one to two orders inside the bar.
"""
import numpy as np
import pytest

import oracle
import smash_inputs as si

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
    zo = oracle.H2(x, kid, leaf, order, tol).matvec(q)
    H = sm.H2Matrix(_dev(x), kid, leaf, order, tol)
    z = H.matvec(_dev(q), precision=F32).cpu().numpy()
    err = _rel(z, zo)
    assert err <= RTOL, f"{name}: {err:.3e}"
    H.close()


def test_f32_cauchy_rectangular():
    x, y = si.cauchy_1d(6000, 405)
    q = si.rhs(6000, 4, 406)
    zo = oracle.H2(x, sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10, y=y).matvec(q)
    H = sm.H2Matrix(_dev(x), sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10, y=_dev(y))
    z = H.matvec(_dev(q), precision=F32).cpu().numpy()
    assert _rel(z, zo) <= RTOL
    H.close()


def test_f32_sphere_yukawa_full_size():
    """The mixed-precision workload at N = 2^20 (sphere with caps, Yukawa,
    order 5, 32 RHS): FP32 against the FP64 matvec of the same handle on all
    rows (the FP64 path is bit-exact to the oracle's build and within 1e-11 of
    its matvec), and against the dense product on sampled rows."""
    w = si.make_workload("sphere_yukawa_1m")
    x, q = w["x"], w["q"]
    H = sm.H2Matrix(_dev(x), w["kernel"], w["leaf"], w["order"], w["tol"])
    qd = _dev(q)
    z32 = H.matvec(qd, precision=F32).cpu().numpy()
    z64 = H.matvec(qd).cpu().numpy()
    assert _rel(z32, z64) <= RTOL
    rows = si.sample_rows(len(x), 128, 407)
    zd = oracle.dense_rows(x, w["kernel"], q, rows=rows)
    err = _rel(z64[rows], zd)
    assert err < 1e-3, err
    H.close()
