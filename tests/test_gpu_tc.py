"""Mixed-precision matvecs with the coupling products on the tensor cores
(SMASH_PREC_TF32, SMASH_PREC_BF16, SMASH_PREC_TF32X3) against the oracle's
FP64 H^2 matvec.

Bars, from the product formats: an entry and a q^ value are rounded to a
unit roundoff u (TF32 2^-11, BF16 2^-8), so a product carries <= 2u relative
error; on random right-hand sides the errors average and the relative error
of the result stays well inside 2u.  The split TF32 mode carries the low
parts too (error ~u^2 per product) and is held to the FP32 bar 1e-5.  The
near field is FP32 with compensated sums in all three modes.
  TF32 <= 1e-3, BF16 <= 8e-3, TF32X3 <= 1e-5 in relative 2-norm; and the
  split mode must beat plain TF32, which must beat BF16.
Entry by entry (parity_helpers), each difference is held to twice the
per-product bound times the entry's sum of |terms|: TF32 2^-9, BF16 2^-6,
split TF32 1e-5.
"""
import numpy as np
import pytest

import oracle
import smash_inputs as si
from parity_helpers import TOL_BF16, TOL_TF32, TOL_TF32X3, assert_entrywise, worst_entry

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

DEV = torch.device("cuda:0")
BARS = {sm.SMASH_PREC_TF32: 1e-3, sm.SMASH_PREC_BF16: 8e-3, sm.SMASH_PREC_TF32X3: 1e-5}
ENTRY_BARS = {sm.SMASH_PREC_TF32: TOL_TF32, sm.SMASH_PREC_BF16: TOL_BF16, sm.SMASH_PREC_TF32X3: TOL_TF32X3}


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


CASES = {
    "sphere_yukawa_8192": dict(x=lambda: si.sphere_with_caps(8192, 5100), y=None, kid=2, leaf=128, order=5,
                               tol=1e-8, nrhs=32),
    "3d_invr_20000": dict(x=lambda: si.uniform_cube(20000, 3, 5101), y=None, kid=1, leaf=128, order=4, tol=1e-8,
                          nrhs=16),
    "2d_log_6000": dict(x=lambda: si.gaussian_mixture(6000, 2, 5102), y=None, kid=0, leaf=64, order=5, tol=1e-8,
                        nrhs=5),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    c = CASES[request.param]
    x = c["x"]()
    q = si.rhs(len(x), c["nrhs"], 5200)
    ho = oracle.H2(x, c["kid"], c["leaf"], c["order"], c["tol"])
    hg = sm.H2Matrix(_dev(x), c["kid"], c["leaf"], c["order"], c["tol"])
    yield dict(name=request.param, q=q, zo=ho.matvec(q), sc=ho.matvec_abs(q), hg=hg)
    hg.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_tensor_core_modes_meet_their_bars(case):
    errs = {}
    for p, bar in BARS.items():
        z = case["hg"].matvec(_dev(case["q"]), precision=p).cpu().numpy()
        errs[p] = _rel(z, case["zo"])
        assert_entrywise(z, case["zo"], case["sc"], ENTRY_BARS[p], what=f"{case['name']} precision {p}")
        assert errs[p] <= bar, (case["name"], p, errs[p])
    assert errs[sm.SMASH_PREC_TF32X3] < errs[sm.SMASH_PREC_TF32] < errs[sm.SMASH_PREC_BF16], errs


@pytest.mark.parametrize("nrhs", [1, 3, 8, 9, 33, 64])
def test_tensor_core_ragged_rhs(nrhs):
    x = si.uniform_cube(9000, 3, 5300)
    q = si.rhs(9000, nrhs, 5301)
    ho = oracle.H2(x, 1, 64, 4, 1e-8)
    zo, sc = ho.matvec(q), ho.matvec_abs(q)
    hg = sm.H2Matrix(_dev(x), 1, 64, 4, 1e-8)
    for p, bar in BARS.items():
        z = hg.matvec(_dev(q), precision=p).cpu().numpy()
        assert_entrywise(z, zo, sc, ENTRY_BARS[p], what=f"nrhs={nrhs} precision {p}")
        assert _rel(z, zo) <= bar, (nrhs, p)
    hg.close()


def test_tensor_core_rectangular_cauchy_and_batch():
    x, y = si.cauchy_1d(6000, 5400)
    q = si.rhs(6000, 4, 5401)
    ho = oracle.H2(x, 3, 64, 16, 1e-10, y=y)
    zo, sc = ho.matvec(q), ho.matvec_abs(q)
    hg = sm.H2Matrix(_dev(x), 3, 64, 16, 1e-10, y=_dev(y))
    for p, bar in BARS.items():
        z = hg.matvec(_dev(q), precision=p).cpu().numpy()
        assert_entrywise(z, zo, sc, ENTRY_BARS[p], what=f"cauchy precision {p}")
        assert _rel(z, zo) <= bar, p
    hg.close()
    probs = si.batched_problems(6, 5402, n_lo=400, n_hi=4000)
    for d, (xb, off, kid, idx) in si.group_by_dimension(probs).items():
        qb = si.rhs(len(xb), 8, 5403)
        hb = sm.H2Matrix.batch(_dev(xb), off, kid, 64, 4, 1e-8)
        z = hb.matvec(_dev(qb), precision=sm.SMASH_PREC_TF32X3).cpu().numpy()
        for t, i in enumerate(idx):
            o0, o1 = off[t], off[t + 1]
            ho = oracle.H2(probs[i]["x"], kid, 64, 4, 1e-8)
            qt = np.ascontiguousarray(qb[o0:o1])
            zo = ho.matvec(qt)
            assert worst_entry(z[o0:o1], zo, ho.matvec_abs(qt))[0] <= TOL_TF32X3, (d, t)
            assert _rel(z[o0:o1], zo) <= 1e-5, (d, t)
        hb.close()


@pytest.mark.slow
def test_tensor_core_sphere_full_size_against_fp64():
    """The sphere Yukawa workload at N = 2^20 against the FP64 GPU matvec
    (itself within 1e-11 of the oracle)."""
    w = si.make_workload("sphere_yukawa_1m")
    hg = sm.H2Matrix(_dev(w["x"]), w["kernel"], w["leaf"], w["order"], w["tol"])
    q = _dev(w["q"])
    z64 = hg.matvec(q).cpu().numpy()
    for p, bar in BARS.items():
        z = hg.matvec(q, precision=p).cpu().numpy()
        assert _rel(z, z64) <= bar, p
    hg.close()
