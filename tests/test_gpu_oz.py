"""GPU parity of the coupling with exact digit-split products on the tensor cores.

The double-float matvec (SMASH_PREC_F32X2) computes the coupling (3.19) in one
of three ways, chosen per launch shape by the tuner (untuned default: the first
from 8 columns per pass, else the second):
  0. entries in double-float, entries and q^ split into 8-bit digits whose
     products are summed exactly on the tensor cores (warp MMAs), the digit
     levels combined in double-float;
  1. every operation in double-float on the FP32 pipe;
  2. as 0, with the digit products issued as tcgen05.mma and the level sums
     in tensor memory.
All carry ~2^-46 relative precision per entry, so all meet the FP64 bar
(entry by entry within 1e-11 of each entry's sum of |terms| against the
oracle's FP64 H^2 matvec, parity_helpers; relative 2-norm 1e-11 as a second
line) and agree with each other far below it.  Blocks the digit split does not cover (more than
16 right-hand sides per pass; trees on the exact three-float coordinates)
take the second way.
"""
import json

import numpy as np
import pytest

import oracle
import smash_inputs as si
from parity_helpers import TOL_F32X2, assert_entrywise, oracle_reference

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

DEV = torch.device("cuda:0")
F32X2 = sm.SMASH_PREC_F32X2
RTOL = 1e-11


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture
def clean_table():
    sm.smash_set_autotune(False)
    sm.smash_autotune_clear()
    yield
    sm.smash_set_autotune(False)
    sm.smash_autotune_clear()


def _coupling_keys(h, q, tmp_path):
    sm.smash_set_autotune(True)
    h.matvec(_dev(q), precision=F32X2)
    sm.smash_set_autotune(False)
    path = tmp_path / "t.json"
    sm.smash_autotune_save(str(path))
    table = json.loads(path.read_text())["entries"]
    return table, [k for k in table if k.startswith("coupling_dd/")], path


def _forced(h, q, table, keys, path, choice):
    forced = dict(table)
    forced.update({k: choice for k in keys})
    path.write_text(json.dumps({"smash_autotune": 1, "entries": forced}))
    sm.smash_autotune_clear()
    sm.smash_autotune_load(str(path))
    return h.matvec(_dev(q), precision=F32X2).cpu().numpy()


@pytest.mark.parametrize("d,n,leaf,order,nrhs", [(3, 20000, 128, 4, 16), (3, 12000, 128, 5, 16), (3, 9000, 64, 3, 5),
                                                 (2, 8000, 64, 5, 8),
                                                 (2, 6000, 32, 6, 16), (1, 4000, 32, 10, 1), (1, 5000, 64, 8, 12)])
def test_both_couplings_match_the_oracle(clean_table, tmp_path, d, n, leaf, order, nrhs):
    x = si.uniform_cube(n, d, 6100 + d)
    q = si.rhs(n, nrhs, 6101)
    zo, sc = oracle_reference(oracle.H2(x, sm.SMASH_K_INVR, leaf, order, 1e-8), q)
    h = sm.H2Matrix(_dev(x), sm.SMASH_K_INVR, leaf, order, 1e-8)
    table, keys, path = _coupling_keys(h, q, tmp_path)
    assert keys, "the digit-split coupling is offered for this tree"
    z0 = _forced(h, q, table, keys, path, 0)
    z1 = _forced(h, q, table, keys, path, 1)
    z2 = _forced(h, q, table, keys, path, 2)
    for z, what in ((z0, "warp MMAs"), (z1, "FP32 pipe"), (z2, "tcgen05")):
        assert_entrywise(z, zo, sc, TOL_F32X2, what=what)
        assert _rel(z, zo) <= RTOL, what
    # the ways differ only by roundings of the double-float arithmetic (the
    # digit products' level sums are exact in both tensor-core variants)
    assert _rel(z0, z1) <= 1e-12
    assert _rel(z0, z2) <= 1e-12
    # the tcgen05 variant is deterministic
    assert np.array_equal(z2, _forced(h, q, table, keys, path, 2))
    h.close()


def test_default_matvec_takes_the_digit_split_coupling(clean_table):
    """With tuning off and an empty table the default (0) is used; the result
    is deterministic (fixed reduction order) and meets the bar."""
    x = si.sphere_with_caps(12000, 6200)
    q = si.rhs(12000, 16, 6201)
    zo, sc = oracle_reference(oracle.H2(x, sm.SMASH_K_INVR, 64, 4, 1e-8), q)
    h = sm.H2Matrix(_dev(x), sm.SMASH_K_INVR, 64, 4, 1e-8)
    za = h.matvec(_dev(q), precision=F32X2).cpu().numpy()
    zb = h.matvec(_dev(q), precision=F32X2).cpu().numpy()
    assert np.array_equal(za, zb)
    assert_entrywise(za, zo, sc, TOL_F32X2)
    assert _rel(za, zo) <= RTOL
    h.close()


def test_cauchy_rectangular_digit_split(clean_table, tmp_path):
    x, y = si.cauchy_1d(6000, 6300)
    q = si.rhs(6000, 4, 6301)
    zo, sc = oracle_reference(oracle.H2(x, sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10, y=y), q)
    h = sm.H2Matrix(_dev(x), sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10, y=_dev(y))
    table, keys, path = _coupling_keys(h, q, tmp_path)
    assert keys
    for choice in (0, 1, 2):
        z = _forced(h, q, table, keys, path, choice)
        assert_entrywise(z, zo, sc, TOL_F32X2, what=f"choice {choice}")
        assert _rel(z, zo) <= RTOL, choice
    h.close()


def test_wide_scales_of_q_columns(clean_table, tmp_path):
    """Columns scaled by 2^-40 .. 2^40 and a zero column: every column keeps
    its own exponent, so each meets the bar on its own."""
    x = si.uniform_cube(10000, 3, 6400)
    q = si.rhs(10000, 8, 6401)
    q = q * (2.0 ** np.array([-40, -13, 0, 7, 19, 40, 0, 3]))[None, :]
    q[:, 6] = 0.0
    zo, sc = oracle_reference(oracle.H2(x, sm.SMASH_K_INVR, 64, 4, 1e-8), q)
    h = sm.H2Matrix(_dev(x), sm.SMASH_K_INVR, 64, 4, 1e-8)
    table, keys, path = _coupling_keys(h, q, tmp_path)
    for choice in (0, 2):
        z = _forced(h, q, table, keys, path, choice)
        for c in range(8):
            if c == 6:
                assert not np.any(z[:, c])
            else:
                assert_entrywise(z[:, c], zo[:, c], sc[:, c], TOL_F32X2, what=f"choice {choice} column {c}")
                assert _rel(z[:, c], zo[:, c]) <= RTOL, (choice, c)
    h.close()


@pytest.mark.parametrize("nrhs", [17, 40])
def test_wide_blocks_take_the_double_float_coupling(clean_table, tmp_path, nrhs):
    """More than 16 right-hand sides exceed one pass of the digit-split
    kernel: no digit-split key is offered and the double-float coupling meets
    the bar."""
    x = si.uniform_cube(8000, 3, 6500)
    q = si.rhs(8000, nrhs, 6501)
    zo, sc = oracle_reference(oracle.H2(x, sm.SMASH_K_INVR, 64, 4, 1e-8), q)
    h = sm.H2Matrix(_dev(x), sm.SMASH_K_INVR, 64, 4, 1e-8)
    _, keys, _ = _coupling_keys(h, q, tmp_path)
    assert not keys
    z = h.matvec(_dev(q), precision=F32X2).cpu().numpy()
    assert_entrywise(z, zo, sc, TOL_F32X2, what=f"nrhs={nrhs}")
    assert _rel(z, zo) <= RTOL
    h.close()


# ------------------------------------------------------------------ near field
def _near_keys(h, q, tmp_path):
    sm.smash_set_autotune(True)
    h.matvec(_dev(q), precision=F32X2)
    sm.smash_set_autotune(False)
    path = tmp_path / "n.json"
    sm.smash_autotune_save(str(path))
    table = json.loads(path.read_text())["entries"]
    return table, [k for k in table if k.startswith("near_dd/")], path


@pytest.mark.parametrize("case", ["cube3", "sphere", "plane2", "line1", "cauchy"])
def test_both_near_fields_match_the_oracle(clean_table, tmp_path, case):
    """The near field (3.20) by digit-split products on the tensor cores
    (rows scaled by their nearest source, nodes with coincident points or a
    wide spread of distances left to the double-float kernel) and all in
    double-float: both meet the bar and agree far below it."""
    y = None
    if case == "cube3":
        x, kern, leaf, order, tol = si.uniform_cube(12000, 3, 6600), sm.SMASH_K_INVR, 64, 4, 1e-8
    elif case == "sphere":
        x, kern, leaf, order, tol = si.sphere_with_caps(12000, 6601), sm.SMASH_K_INVR, 64, 4, 1e-8
    elif case == "plane2":
        x, kern, leaf, order, tol = si.uniform_cube(8000, 2, 6602), sm.SMASH_K_INVR, 64, 5, 1e-8
    elif case == "line1":
        x, kern, leaf, order, tol = si.uniform_cube(5000, 1, 6603), sm.SMASH_K_INVR, 64, 8, 1e-8
    else:
        (x, y), kern, leaf, order, tol = si.cauchy_1d(6000, 6604), sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10
    n = len(x) if y is None else len(y)
    q = si.rhs(n, 16, 6605)
    zo, sc = oracle_reference(oracle.H2(x, kern, leaf, order, tol, y=y), q)
    h = sm.H2Matrix(_dev(x), kern, leaf, order, tol, y=None if y is None else _dev(y))
    table, keys, path = _near_keys(h, q, tmp_path)
    assert keys, "the digit-split near field is offered"
    z0 = _forced(h, q, table, keys, path, 0)
    z1 = _forced(h, q, table, keys, path, 1)
    assert_entrywise(z0, zo, sc, TOL_F32X2)
    assert _rel(z0, zo) <= RTOL
    assert_entrywise(z1, zo, sc, TOL_F32X2)
    assert _rel(z1, zo) <= RTOL
    assert _rel(z0, z1) <= 1e-12
    h.close()


def test_coincident_points_take_the_double_float_near_field(clean_table, tmp_path):
    """Duplicated points (distinct indices, equal coordinates) have entry 0 and
    no positive nearest distance: their leaves fall back to the double-float
    kernel inside the digit-split path, and the result meets the bar."""
    x = si.uniform_cube(8000, 3, 6700)
    x = np.concatenate([x, x[:300]])  # 300 coincident pairs
    q = si.rhs(len(x), 16, 6701)
    zo, sc = oracle_reference(oracle.H2(x, sm.SMASH_K_INVR, 64, 4, 1e-8), q)
    h = sm.H2Matrix(_dev(x), sm.SMASH_K_INVR, 64, 4, 1e-8)
    table, keys, path = _near_keys(h, q, tmp_path)
    assert keys
    z0 = _forced(h, q, table, keys, path, 0)
    assert np.all(np.isfinite(z0))
    assert_entrywise(z0, zo, sc, TOL_F32X2)
    assert _rel(z0, zo) <= RTOL
    h.close()


def test_forced_coupling_prefix(clean_table, tmp_path):
    """smash_autotune_force pins every coupling site to one candidate ahead of
    the table: the tcgen05 variant forced by prefix gives the bits of the
    same variant chosen through the table, and removing the override returns
    to the table's choice."""
    x = si.uniform_cube(9000, 3, 6800)
    q = si.rhs(9000, 16, 6801)
    h = sm.H2Matrix(_dev(x), sm.SMASH_K_INVR, 64, 4, 1e-8)
    table, keys, path = _coupling_keys(h, q, tmp_path)
    z_table = _forced(h, q, table, keys, path, 2)
    z_warp = _forced(h, q, table, keys, path, 0)
    try:
        sm.smash_autotune_force("coupling_dd/", 2)
        z_force = h.matvec(_dev(q), precision=F32X2).cpu().numpy()
    finally:
        sm.smash_autotune_force("coupling_dd/", -1)
    assert np.array_equal(z_force, z_table)
    # the table (all coupling keys at 0) rules again
    assert np.array_equal(h.matvec(_dev(q), precision=F32X2).cpu().numpy(), z_warp)
    h.close()
