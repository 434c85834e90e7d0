"""GPU parity of the Taylor-expansion representation (Section 2.1, (2.4)-(2.5);
construction of Section 3.3.2; matvec of Section 3.4) of kappa(x, y) =
1/(x - y) on C against the CPU oracle, on the workload of Section 6.2: an
m x m grid in [0,1]^2, leaves of at most 50 points, r = 22, tau = 0.65,
d_x = 1.

Bars: tree, lists, ranks and skeletons bit-exact; every complex G entry
bit-identical (the complex compression runs the oracle's operations in the
oracle's order without contraction); the complex matvec entry by entry
within 1e-12 of each entry's sum of |terms| (parity_helpers); against the
dense product the magnitude Table 6.1 prints (~1e-12).
"""
import numpy as np
import pytest

import oracle
import smash_inputs as si
from parity_helpers import TOL_F64, assert_entrywise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

DEV = torch.device("cuda:0")
TREE_KEYS = ["permx", "lvl_off", "level", "leaf", "parent", "child0", "nchild", "rs", "rc", "cell", "adm_ptr",
             "adm_col", "near_ptr", "near_col", "m_row", "k_row", "skel_row", "rest_row"]


def _rhs(n, nrhs, seed):
    return np.ascontiguousarray(si.uniform_01(n, nrhs, seed) + 1j * si.uniform_01(n, nrhs, seed + 1))


@pytest.mark.parametrize("m,nrhs", [(40, 1), (80, 3), (160, 2)])
def test_taylor_build_bit_exact_and_matvec_parity(m, nrhs):
    x = si.grid_2d(m)
    n = m * m
    ho = oracle.H2Taylor(x, 50, 22, 1e-14, tau=0.65, dx=1.0)
    h = sm.smash_build_taylor(torch.from_numpy(x).to(DEV), 50, 22, tau=0.65, tol=1e-14, dx=1.0)
    eg, eo = sm.smash_export(h), ho.export()
    for k in TREE_KEYS:
        assert np.array_equal(np.asarray(eg[k]), np.asarray(eo[k])), k
    assert eg["G_row"].dtype == np.complex128
    assert np.array_equal(eg["G_row"].view(np.float64), eo["G_row"].view(np.float64)), "complex G not bit-identical"
    q = _rhs(n, nrhs, 70 + m)
    zo, sc = ho.matvec(q), ho.matvec_abs(q)
    Y = torch.empty((n, nrhs), dtype=torch.complex128, device=DEV)
    sm.smash_matvec_complex(h, torch.from_numpy(q).to(DEV), Y)
    z = Y.cpu().numpy()
    for part in (np.real, np.imag):
        assert_entrywise(part(z), part(zo), sc, TOL_F64, what=f"m={m} {part.__name__}")
    # host buffers give the device result
    Yh = np.empty((n, nrhs), np.complex128)
    sm.smash_matvec_complex(h, q, Yh)
    assert np.array_equal(Yh, z)
    sm.smash_free(h)


def test_taylor_table_6_1_sizes_against_dense():
    """The four sizes of Table 6.1 (n = 1600 .. 102400): the relative error of
    the GPU matvec against the dense product on sampled rows is of the
    printed magnitude (within a factor of 4 of tests/golden/table6_1.txt)."""
    printed = {1600: 6.69e-13, 6400: 2.00e-12, 25600: 3.65e-12, 102400: 4.87e-12}
    for n, ref_err in printed.items():
        m = int(round(n ** 0.5))
        x = si.grid_2d(m)
        u = si.uniform_01(n, 1, 61).astype(np.complex128)
        h = sm.smash_build_taylor(torch.from_numpy(x).to(DEV), 50, 22, tau=0.65, tol=1e-14, dx=1.0)
        Y = torch.empty((n, 1), dtype=torch.complex128, device=DEV)
        sm.smash_matvec_complex(h, torch.from_numpy(u).to(DEV), Y)
        rows = si.sample_rows(n, 512, 62)
        zd = oracle.dense_rows_taylor(x, u, rows=rows)
        err = np.linalg.norm(Y.cpu().numpy()[rows] - zd) / np.linalg.norm(zd)
        assert ref_err / 4 <= err <= ref_err * 4, (n, err, ref_err)
        sm.smash_free(h)


def test_taylor_root_leaf_and_complex_diagonal():
    x = si.grid_2d(6)                        # 36 points: the root is a leaf
    q = _rhs(36, 2, 80)
    h = sm.smash_build_taylor(x, 50, 22, dx=2.0 - 0.5j)
    Y = np.empty((36, 2), np.complex128)
    sm.smash_matvec_complex(h, q, Y)
    z = x[:, 0] + 1j * x[:, 1]
    D = z[:, None] - z[None, :]
    A = np.where(D == 0, 2.0 - 0.5j, 1.0 / np.where(D == 0, 1.0, D))
    assert np.linalg.norm(Y - A @ q) <= 1e-14 * np.linalg.norm(A @ q)
    # the real entry points refuse a complex representation
    with pytest.raises(sm.SmashError):
        sm.smash_matvec_ex(h, np.zeros((36, 1)), np.zeros((36, 1)))
    sm.smash_free(h)
