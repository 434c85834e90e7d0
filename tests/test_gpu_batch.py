"""GPU parity of batched problems (smash_build_batch) against the oracle run
on every problem alone.

Bars: each problem's partition, lists, ranks, skeletons and G are
bit-identical to the oracle's for that problem alone (the batch keeps one
bounding cube and one root per problem); the matvec of each problem is
compared entry by entry with the oracle's H^2 matvec of that problem, each
difference within a bar times the entry's sum of |terms| (parity_helpers):
1e-12 for FP64, 1e-11 for double-float (1/r), 1e-5 for FP32.
"""
import numpy as np
import pytest

import oracle
import smash_inputs as si
from batch_helpers import split_batch_export
from parity_helpers import TOL_F32, TOL_F32X2, TOL_F64, worst_entry

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

DEV = torch.device("cuda:0")
LEAF, ORDER, TOL = 64, 4, 1e-8
TREE_KEYS = ["permx", "keyx", "lvl_off", "level", "leaf", "parent", "child0", "nchild", "rs", "rc", "cs", "cc",
             "cell"]
LIST_KEYS = ["adm_ptr", "adm_col", "near_ptr", "near_col"]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def batch():
    # small problems of the batched recipe: both dimensions, cube and mixture
    probs = si.batched_problems(16, 3100, n_lo=150, n_hi=3000)
    groups = si.group_by_dimension(probs)
    out = {}
    for d, (x, off, kid, idx) in groups.items():
        h = sm.H2Matrix.batch(_dev(x), off, kid, LEAF, ORDER, TOL)
        q = si.rhs(len(x), 8, 3200 + d)
        orc = [oracle.H2(probs[i]["x"], kid, LEAF, ORDER, TOL) for i in idx]
        out[d] = dict(x=x, off=off, kid=kid, h=h, q=q, orc=orc)
    yield out
    for g in out.values():
        g["h"].close()


def test_batch_has_both_dimensions(batch):
    assert sorted(batch) == [2, 3]
    for g in batch.values():
        assert g["h"].info()["nproblems"] == len(g["off"]) - 1 >= 2


def test_batch_build_is_bit_exact_per_problem(batch):
    for d, g in batch.items():
        parts = split_batch_export(g["h"].export(), g["off"])
        for t, (eg, ho) in enumerate(zip(parts, g["orc"])):
            eo = ho.export()
            assert np.array_equal(eg["cube"][:d], eo["lo"]) and eg["cube"][3] == eo["s"], (d, t)
            assert eg["L"] == eo["L"]
            for k in TREE_KEYS:
                assert np.array_equal(np.asarray(eg[k]), np.asarray(eo[k])), (d, t, k)
            for k in LIST_KEYS:
                assert np.array_equal(eg[k], eo[k]), (d, t, k)
            for k in ("m_row", "k_row", "skel_row", "rest_row"):
                assert np.array_equal(eg[k], eo[k]), (d, t, k)
            assert np.array_equal(eg["G_row"], eo["G_row"]), (d, t, "G")


def _per_problem_worst(g, z):
    """Per problem: (worst entry / its sum of |terms|, relative 2-norm)."""
    out = []
    for t, ho in enumerate(g["orc"]):
        o0, o1 = g["off"][t], g["off"][t + 1]
        qt = np.ascontiguousarray(g["q"][o0:o1])
        worst, _, rel2 = worst_entry(z[o0:o1], ho.matvec(qt), ho.matvec_abs(qt))
        out.append((worst, rel2))
    return np.array(out)


def test_batch_matvec_fp64_parity(batch):
    for d, g in batch.items():
        z = g["h"].matvec(_dev(g["q"])).cpu().numpy()
        r = _per_problem_worst(g, z)
        assert r[:, 0].max() <= TOL_F64, (d, r[:, 0].max())
        assert r[:, 1].max() <= 1e-11, (d, r[:, 1].max())


def test_batch_matvec_double_float_parity(batch):
    g = batch[3]  # 1/r
    z = g["h"].matvec(_dev(g["q"]), precision=sm.SMASH_PREC_F32X2).cpu().numpy()
    r = _per_problem_worst(g, z)
    assert r[:, 0].max() <= TOL_F32X2, r[:, 0].max()
    assert r[:, 1].max() <= 1e-11, r[:, 1].max()


def test_batch_matvec_fp32_parity(batch):
    for d, g in batch.items():
        z = g["h"].matvec(_dev(g["q"]), precision=sm.SMASH_PREC_F32).cpu().numpy()
        r = _per_problem_worst(g, z)
        assert r[:, 0].max() <= TOL_F32, (d, r[:, 0].max())


def test_batch_equals_problems_built_alone(batch):
    """The batch applies diag(A^_0, ..., A^_{T-1}): each block equals the same
    problem built and applied alone on the GPU."""
    g = batch[2]
    zb = g["h"].matvec(_dev(g["q"])).cpu().numpy()
    for t in range(len(g["off"]) - 1):
        o0, o1 = g["off"][t], g["off"][t + 1]
        h1 = sm.H2Matrix(_dev(g["x"][o0:o1]), g["kid"], LEAF, ORDER, TOL)
        z1 = h1.matvec(_dev(g["q"][o0:o1])).cpu().numpy()
        h1.close()
        assert np.linalg.norm(zb[o0:o1] - z1) <= 1e-13 * np.linalg.norm(z1), t


def test_batch_of_one_point_problems_and_a_root_leaf():
    """Degenerate members: single points and a problem that is one leaf."""
    rng = np.random.default_rng(3300)
    xs = [rng.random((1, 3)), rng.random((40, 3)), rng.random((1, 3)), rng.random((700, 3))]
    off = np.concatenate([[0], np.cumsum([len(x) for x in xs])])
    x = np.concatenate(xs)
    q = si.rhs(len(x), 2, 3301)
    h = sm.H2Matrix.batch(_dev(x), off, 1, LEAF, ORDER, TOL)
    z = h.matvec(_dev(q)).cpu().numpy()
    for t in range(len(xs)):
        o0, o1 = off[t], off[t + 1]
        zd = oracle.dense_rows(xs[t], 1, np.ascontiguousarray(q[o0:o1]))
        if o1 - o0 == 1:
            assert np.all(z[o0:o1] == 0.0)
        else:
            assert np.linalg.norm(z[o0:o1] - zd) <= 1e-6 * np.linalg.norm(zd)
    h.close()


@pytest.mark.slow
def test_full_batched_workload_sampled_problems():
    """The full 512-problem workload, FP32 matvec with 8 RHS; the smallest
    and the largest problem of each dimension against the oracle."""
    w = si.make_workload("batched_512")
    for d, (x, off, kid, idx) in w["groups"].items():
        h = sm.H2Matrix.batch(_dev(x), off, kid, w["leaf"], w["order"], w["tol"])
        assert h.info()["nproblems"] == len(idx)
        q = w["q"][d]
        z = h.matvec(_dev(q), precision=sm.SMASH_PREC_F32).cpu().numpy()
        sizes = np.diff(off)
        for t in (int(np.argmin(sizes)), int(np.argmax(sizes))):
            o0, o1 = off[t], off[t + 1]
            ho = oracle.H2(x[o0:o1], kid, w["leaf"], w["order"], w["tol"])
            qt = np.ascontiguousarray(q[o0:o1])
            worst, _, _ = worst_entry(z[o0:o1], ho.matvec(qt), ho.matvec_abs(qt))
            assert worst <= TOL_F32, (d, t, worst)
        h.close()
