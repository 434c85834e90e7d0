"""The Cauchy-like matvec of Section 6.3 against the oracle: (6.2) applied
with the oracle's H^2 matvec of the Cauchy matrix and numpy diagonal
scalings (parity), and against the dense entries (6.1) (approximation).

Bars: the scalings are exact multiplications and the recombination sums p
terms, so parity inherits the bar of the matvec precision, entry by entry
against the entry's sum of |terms| (parity_helpers: FP64 1e-12, double-float
1e-11, FP32 1e-5; relative 2-norm 1e-11 / 1e-5 as a second line); against
(6.1) the bar is the H^2 approximation error at order 16, tol 1e-10 (1e-7
with margin).
"""
import numpy as np
import pytest

import oracle
import smash_inputs as si
from parity_helpers import TOL_F32, TOL_F32X2, TOL_F64, assert_entrywise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

DEV = torch.device("cuda:0")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle_cauchy_like(ho, w, v, X):
    """(6.2) with the oracle's H^2 matvec, and each entry's sum of |terms|."""
    p, nrhs = w.shape[1], X.shape[1]
    Xp = np.ascontiguousarray(np.concatenate([v[:, l:l + 1] * X for l in range(p)], axis=1))
    Yp = ho.matvec(Xp)
    Sp = ho.matvec_abs(Xp)
    zo = sum(w[:, l:l + 1] * Yp[:, l * nrhs:(l + 1) * nrhs] for l in range(p))
    sc = sum(np.abs(w[:, l:l + 1]) * Sp[:, l * nrhs:(l + 1) * nrhs] for l in range(p))
    return zo, sc


@pytest.mark.parametrize("offset", [1e-7, 1e-3])
def test_cauchy_like_parity_with_the_oracle(offset):
    x, y, w, v = si.cauchy_like_6_3(6000, 6100, offset=offset)
    X = si.rhs(6000, 3, 6101)
    ho = oracle.H2(x, 3, 50, 16, 1e-10, y=y)
    zo, sc = _oracle_cauchy_like(ho, w, v, X)
    hg = sm.H2Matrix(_dev(x), 3, 50, 16, 1e-10, y=_dev(y))
    for prec, bar, ebar in ((sm.SMASH_PREC_F64, 1e-11, TOL_F64), (sm.SMASH_PREC_F32X2, 1e-11, TOL_F32X2),
                            (sm.SMASH_PREC_F32, 1e-5, TOL_F32)):
        Y = torch.empty((6000, 3), dtype=torch.float64, device=DEV)
        sm.smash_matvec_cauchy_like(hg.h, _dev(w), _dev(v), _dev(X), Y, prec)
        assert_entrywise(Y.cpu().numpy(), zo, sc, ebar, what=f"offset {offset} precision {prec}")
        assert _rel(Y.cpu().numpy(), zo) <= bar, prec
    # host buffers give the same result as device buffers
    Yh = np.empty((6000, 3))
    sm.smash_matvec_cauchy_like(hg.h, w, v, X, Yh, sm.SMASH_PREC_F64)
    Yd = torch.empty((6000, 3), dtype=torch.float64, device=DEV)
    sm.smash_matvec_cauchy_like(hg.h, _dev(w), _dev(v), _dev(X), Yd, sm.SMASH_PREC_F64)
    assert np.array_equal(Yh, Yd.cpu().numpy())
    hg.close()


def test_cauchy_like_against_the_dense_entries():
    n = 2000
    x, y, w, v = si.cauchy_like_6_3(n, 6200)
    X = si.rhs(n, 2, 6201)
    A = (1.0 / (x - y.T)) * (w @ v.T)   # (6.1)
    zd = A @ X
    hg = sm.H2Matrix(_dev(x), 3, 50, 16, 1e-10, y=_dev(y))
    Y = torch.empty((n, 2), dtype=torch.float64, device=DEV)
    sm.smash_matvec_cauchy_like(hg.h, _dev(w), _dev(v), _dev(X), Y, sm.SMASH_PREC_F64)
    assert _rel(Y.cpu().numpy(), zd) <= 1e-7
    hg.close()


def test_unit_generators_reduce_to_the_plain_matvec():
    x, y, _, _ = si.cauchy_like_6_3(3000, 6300, offset=1e-3)
    X = _dev(si.rhs(3000, 4, 6301))
    hg = sm.H2Matrix(_dev(x), 3, 64, 16, 1e-10, y=_dev(y))
    ones = torch.ones((3000, 1), dtype=torch.float64, device=DEV)
    Y = torch.empty_like(X)
    sm.smash_matvec_cauchy_like(hg.h, ones, ones, X, Y, sm.SMASH_PREC_F64)
    assert torch.equal(Y, hg.matvec(X))
    with pytest.raises(sm.SmashError, match="p \\* nrhs"):
        big = torch.ones((3000, 17), dtype=torch.float64, device=DEV)
        sm.smash_matvec_cauchy_like(hg.h, big, big, X, Y, sm.SMASH_PREC_F64)
    hg.close()
