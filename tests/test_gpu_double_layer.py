"""The double-layer (Nystrom) matvec of Section 6.4 and the kernel override
on the GPU.

Parity: K X by smash_matvec_double_layer against the oracle's H^2 matvecs of
the two gradient kernels (6.9) combined in numpy, entry by entry at the bars
of the matvec precisions against each entry's sum of |terms| (parity_helpers:
FP64 1e-12; FP32 and split TF32 1e-5; relative 2-norm 1e-11 / 1e-5 as a
second line).  Physics: with sigma = 1
the discretised double layer on the curve is -1/2 (Gauss), to the H^2
approximation error.  The representation is kernel-independent: applying a
kernel by override equals a handle built for that kernel, bit for bit.
"""
import numpy as np
import pytest

import oracle
import smash_inputs as si
from parity_helpers import TOL_F32, TOL_F64, TOL_TF32X3, assert_entrywise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

DEV = torch.device("cuda:0")
LEAF, ORDER, TOL = 50, 8, 1e-12


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", params=["ram_head", "sunflower"])
def curve(request):
    # the sunflower's narrow petals need about 40000 trapezoidal points
    n = 3000 if request.param == "ram_head" else 40000
    c = si.curve_6_4(request.param, n)
    c["diag"] = -c["curvature"] / (4 * np.pi) * c["w"]
    c["h"] = sm.H2Matrix(_dev(c["x"]), sm.SMASH_K_DLP1, LEAF, ORDER, TOL)
    yield c
    c["h"].close()


def _oracle_double_layer(c, X):
    """K X from the oracle's H^2 matvecs of the two gradient kernels, and each
    entry's sum of |terms|."""
    nu, w = c["nu"], c["w"]
    z = np.zeros_like(X)
    sc = np.zeros_like(X)
    for a, kid in ((0, 4), (1, 5)):
        ho = oracle.H2(c["x"], kid, LEAF, ORDER, TOL)
        qa = np.ascontiguousarray((nu[:, a] * w)[:, None] * X)
        z += ho.matvec(qa)
        sc += ho.matvec_abs(qa)
    return z + c["diag"][:, None] * X, sc + np.abs(c["diag"][:, None] * X)


def test_double_layer_parity_with_the_oracle(curve):
    X = si.rhs(len(curve["x"]), 3, 7100)
    zo, sc = _oracle_double_layer(curve, X)
    for prec, bar, ebar in ((sm.SMASH_PREC_F64, 1e-11, TOL_F64), (sm.SMASH_PREC_F32, 1e-5, TOL_F32),
                            (sm.SMASH_PREC_TF32X3, 1e-5, TOL_TF32X3)):
        Y = torch.empty_like(_dev(X))
        sm.smash_matvec_double_layer(curve["h"].h, _dev(curve["nu"]), _dev(curve["w"]), _dev(curve["diag"]),
                                     _dev(X), Y, prec)
        assert_entrywise(Y.cpu().numpy(), zo, sc, ebar, what=f"precision {prec}")
        assert _rel(Y.cpu().numpy(), zo) <= bar, prec


def test_double_layer_of_a_constant_density_is_minus_one_half(curve):
    """K 1 = -1/2 on the curve up to the quadrature error (ram head: 1e-6;
    the sunflower's inner petal tips keep a 3.4e-4 trapezoidal error even at
    40000 points, the same for the dense Nystrom sum), and K 1 equals the
    dense Nystrom sum of the oracle on sampled rows to the H^2 error (order
    8: ~1e-11 on the ram head, 2.3e-7 at the sunflower's petals)."""
    n = len(curve["x"])
    Y = torch.empty((n, 1), dtype=torch.float64, device=DEV)
    sm.smash_matvec_double_layer(curve["h"].h, curve["nu"], curve["w"], curve["diag"], np.ones((n, 1)), Y,
                                 sm.SMASH_PREC_F64)
    y = Y.cpu().numpy().ravel()
    rows = np.arange(0, n, 97)
    x, nu, w = curve["x"], curve["nu"], curve["w"]
    dense = (oracle.dense_rows(x, 4, np.ascontiguousarray((nu[:, 0] * w)[:, None]), rows=rows) +
             oracle.dense_rows(x, 5, np.ascontiguousarray((nu[:, 1] * w)[:, None]), rows=rows)).ravel()
    dense += curve["diag"][rows]
    assert np.max(np.abs(y[rows] - dense)) < 1e-6
    assert np.max(np.abs(y + 0.5)) < (1e-6 if n == 3000 else 1e-3)


def test_kernel_override_equals_a_handle_built_for_the_kernel():
    c = si.curve_6_4("ram_head", 4000)
    X = _dev(si.rhs(4000, 4, 7200))
    h_log = sm.H2Matrix(_dev(c["x"]), sm.SMASH_K_LOG, LEAF, ORDER, TOL)
    h_dlp = sm.H2Matrix(_dev(c["x"]), sm.SMASH_K_DLP2, LEAF, ORDER, TOL)
    for prec in (sm.SMASH_PREC_F64, sm.SMASH_PREC_F32):
        Y1 = torch.empty_like(X)
        sm.smash_matvec_kernel(h_log.h, sm.SMASH_K_DLP2, X, Y1, prec)
        assert torch.equal(Y1, h_dlp.matvec(X, precision=prec)), prec
    with pytest.raises(sm.SmashError, match="dim == 1"):
        sm.smash_matvec_kernel(h_log.h, sm.SMASH_K_CAUCHY1D, X, torch.empty_like(X))
    with pytest.raises(sm.SmashError, match="F32X2"):
        sm.smash_matvec_kernel(h_log.h, sm.SMASH_K_DLP1, X, torch.empty_like(X), sm.SMASH_PREC_F32X2)
    h_log.close()
    h_dlp.close()
    x3 = _dev(si.uniform_cube(500, 3, 7201))
    with pytest.raises(sm.SmashError, match="dim == 2"):
        sm.H2Matrix(x3, sm.SMASH_K_DLP1, LEAF, ORDER, TOL)
