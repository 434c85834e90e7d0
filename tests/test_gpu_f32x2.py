"""GPU parity of the double-float matvec (SMASH_PREC_F32X2) against the oracle.

The coupling and near field run as double-float (hi + lo float) arithmetic
with error-free transformations on the FP32 pipe.  Bar: relative 2-norm
difference <= 1e-11 against the oracle's FP64 H^2 matvec -- the same bar as the
FP64 path.  Error budget: coordinates carry ~2^-48 relative precision in the
unit-cube frame (~1e-13 relative in a difference at leaf distances), the
reciprocal square root one Newton step from a 2-ulp seed (< 3e-14), products
and sums are error-free up to the renormalisation of the accumulators once per
128 sources (~1e-13 over the longest rows).  Compared entry by entry: each
difference within 1e-11 of the entry's sum of |terms| (parity_helpers); the
relative 2-norm stays a second line at 1e-11.
"""
import numpy as np
import pytest

import oracle
import smash_inputs as si
from parity_helpers import TOL_F32X2, assert_entrywise, leaf_rows, oracle_reference, sample_leaves

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

DEV = torch.device("cuda:0")
RTOL = 1e-11
F32X2 = sm.SMASH_PREC_F32X2


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("d,n,leaf,order,nrhs", [(3, 20000, 128, 4, 16), (2, 8000, 64, 5, 4),
                                                 (1, 4000, 32, 10, 3), (3, 6000, 32, 3, 33)])
def test_invr_f32x2_matches_oracle(d, n, leaf, order, nrhs):
    x = si.uniform_cube(n, d, 300 + d)
    q = si.rhs(n, nrhs, 301)
    zo, sc = oracle_reference(oracle.H2(x, sm.SMASH_K_INVR, leaf, order, 1e-8), q)
    H = sm.H2Matrix(_dev(x), sm.SMASH_K_INVR, leaf, order, 1e-8)
    z = H.matvec(_dev(q), precision=F32X2).cpu().numpy()
    assert_entrywise(z, zo, sc, TOL_F32X2, what=f"d={d} nrhs={nrhs}")
    assert _rel(z, zo) <= RTOL
    H.close()


def test_clustered_sphere_f32x2_matches_oracle():
    x = si.sphere_with_caps(12000, 310)
    q = si.rhs(12000, 8, 311)
    zo, sc = oracle_reference(oracle.H2(x, sm.SMASH_K_INVR, 64, 4, 1e-8), q)
    H = sm.H2Matrix(_dev(x), sm.SMASH_K_INVR, 64, 4, 1e-8)
    z = H.matvec(_dev(q), precision=F32X2).cpu().numpy()
    assert_entrywise(z, zo, sc, TOL_F32X2, what="sphere")
    assert _rel(z, zo) <= RTOL
    H.close()


def test_cauchy_rectangular_f32x2_matches_oracle():
    x, y = si.cauchy_1d(6000, 320)
    q = si.rhs(6000, 4, 321)
    zo, sc = oracle_reference(oracle.H2(x, sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10, y=y), q)
    H = sm.H2Matrix(_dev(x), sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10, y=_dev(y))
    z = H.matvec(_dev(q), precision=F32X2).cpu().numpy()
    assert_entrywise(z, zo, sc, TOL_F32X2, what="cauchy x != y")
    assert _rel(z, zo) <= RTOL
    H.close()


def test_unsupported_kernel_is_rejected():
    x = si.uniform_cube(500, 2, 330)
    H = sm.H2Matrix(_dev(x), sm.SMASH_K_LOG, 32, 3, 1e-8)
    with pytest.raises(sm.SmashError) as ei:
        H.matvec(_dev(si.rhs(500, 1, 331)), precision=F32X2)
    assert ei.value.status == 1
    H.close()


def test_full_size_headline_workload_f32x2(headline_oracle):
    """N = 2^20: the double-float matvec entry by entry on the rows of 64
    sampled leaves (box corners and faces, every leaf the digit-split near
    field leaves to its fallback, the rest at random) against the oracle's
    H^2 matvec on the same leaves, and against the library's FP64 matvec on
    all rows."""
    w, ho, eo = headline_oracle
    x, q = w["x"], w["q"]
    H = sm.H2Matrix(_dev(x), w["kernel"], w["leaf"], w["order"], w["tol"])
    z2 = H.matvec(_dev(q), precision=F32X2).cpu().numpy()
    z64 = H.matvec(_dev(q)).cpu().numpy()
    assert _rel(z2, z64) <= RTOL
    fb = sm.smash_near_fallback_leaves(H.h)
    pick = sample_leaves(eo, x, 64, seed=2, extra=fb)
    assert len(pick) >= 64 and set(fb.tolist()) <= set(pick.tolist())
    zo, sc = oracle_reference(ho, q, pick)
    rows = leaf_rows(eo, pick)
    assert_entrywise(z2, zo, sc, TOL_F32X2, rows=rows, what="N=2^20 sampled leaves")
    # the same with the coupling pinned to its tcgen05 form (a tuning
    # candidate the headline does not take by default)
    try:
        sm.smash_autotune_force("coupling_dd/", 2)
        z5 = H.matvec(_dev(q), precision=F32X2).cpu().numpy()
    finally:
        sm.smash_autotune_force("coupling_dd/", -1)
    assert_entrywise(z5, zo, sc, TOL_F32X2, rows=rows, what="N=2^20 sampled leaves, tcgen05 coupling")
    assert _rel(z5, z64) <= RTOL
    assert _rel(z5, z2) <= 1e-12
    H.close()


def test_full_size_with_coincident_points_f32x2():
    """N = 2^18 with 200 points duplicated: the leaves holding them are left
    by the digit-split near field to the double-float kernel; all of them,
    and random others, are compared entry by entry with the oracle."""
    x = si.uniform_cube(1 << 18, 3, 340)
    x = np.concatenate([x, x[:200]])
    q = si.rhs(len(x), 16, 341)
    ho = oracle.H2(x, sm.SMASH_K_INVR, 128, 4, 1e-8)
    eo = ho.export()
    H = sm.H2Matrix(_dev(x), sm.SMASH_K_INVR, 128, 4, 1e-8)
    z = H.matvec(_dev(q), precision=F32X2).cpu().numpy()
    fb = sm.smash_near_fallback_leaves(H.h)
    assert len(fb) > 0, "coincident points must take the fallback"
    pick = sample_leaves(eo, x, len(fb) + 32, seed=3, extra=fb)
    zo, sc = oracle_reference(ho, q, pick)
    assert_entrywise(z, zo, sc, TOL_F32X2, rows=leaf_rows(eo, pick), what="fallback leaves")
    H.close()
