"""The autotuner and the CUDA-graph matvec on the GPU.

- Every candidate CTA size of the compression gives the oracle's bits, so a
  tuned build is still bit-exact; a tuned matvec stays within the FP64 parity
  bar; a saved and reloaded table reproduces the tuned build and matvec.
- A matvec replayed from its CUDA graph equals the plain matvec bit for bit
  (same kernels, same choices) and follows new contents of X.
"""
import json

import numpy as np
import pytest

import oracle
import smash_inputs as si
from parity_helpers import TOL_F32, TOL_F32X2, TOL_F64, TOL_TF32, assert_entrywise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

DEV = torch.device("cuda:0")
KEYS = ["permx", "lvl_off", "level", "leaf", "parent", "rs", "rc", "adm_ptr", "adm_col", "near_ptr", "near_col",
        "m_row", "k_row", "skel_row", "rest_row", "G_row"]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _same(ea, eb):
    for k in KEYS:
        assert np.array_equal(np.asarray(ea[k]), np.asarray(eb[k])), k


@pytest.fixture
def clean_table():
    sm.smash_set_autotune(False)
    sm.smash_autotune_clear()
    yield
    sm.smash_set_autotune(False)
    sm.smash_autotune_clear()


def test_tuned_build_and_matvec_keep_parity(clean_table, tmp_path):
    x = si.uniform_cube(30000, 3, 4100)
    q = si.rhs(30000, 16, 4101)
    ho = oracle.H2(x, 1, 128, 4, 1e-8)
    eo = ho.export()
    zo, sc = ho.matvec(q), ho.matvec_abs(q)
    sm.smash_set_autotune(True)
    h = sm.H2Matrix(_dev(x), 1, 128, 4, 1e-8)
    z = {p: h.matvec(_dev(q), precision=p).cpu().numpy()
         for p in (sm.SMASH_PREC_F64, sm.SMASH_PREC_F32X2, sm.SMASH_PREC_F32)}
    sm.smash_set_autotune(False)
    assert sm.smash_autotune_entries() >= 4
    e1 = h.export()
    _same(e1, eo)
    for p, tol, etol in ((sm.SMASH_PREC_F64, 1e-11, TOL_F64), (sm.SMASH_PREC_F32X2, 1e-11, TOL_F32X2),
                         (sm.SMASH_PREC_F32, 1e-5, TOL_F32)):
        assert_entrywise(z[p], zo, sc, etol, what=f"tuned precision {p}")
        assert np.linalg.norm(z[p] - zo) / np.linalg.norm(zo) <= tol, p
    path = tmp_path / "tune.json"
    sm.smash_autotune_save(str(path))
    table = json.loads(path.read_text())["entries"]
    assert any(k.startswith("compress/") for k in table) and any(k.startswith("ksum_") for k in table)
    # a fresh process state with the saved table reproduces build and matvec exactly
    sm.smash_autotune_clear()
    assert sm.smash_autotune_load(str(path)) == len(table)
    h2 = sm.H2Matrix(_dev(x), 1, 128, 4, 1e-8)
    _same(h2.export(), e1)
    for p in z:
        assert np.array_equal(h2.matvec(_dev(q), precision=p).cpu().numpy(), z[p]), p
    h.close()
    h2.close()


@pytest.mark.parametrize("nt", [64, 128, 256, 512])
def test_every_compression_cta_size_gives_the_oracle_bits(clean_table, tmp_path, nt):
    x = si.sphere_with_caps(12000, 4200)
    ho = oracle.H2(x, 2, 64, 4, 1e-9)
    # record the keys of this build, then force every one of them to nt
    sm.smash_set_autotune(True)
    h = sm.H2Matrix(_dev(x), 2, 64, 4, 1e-9)
    sm.smash_set_autotune(False)
    h.close()
    path = tmp_path / "t.json"
    sm.smash_autotune_save(str(path))
    table = json.loads(path.read_text())["entries"]
    forced = {k: nt for k in table if k.startswith("compress/")}
    assert forced
    path.write_text(json.dumps({"smash_autotune": 1, "entries": forced}))
    sm.smash_autotune_clear()
    assert sm.smash_autotune_load(str(path)) == len(forced)
    h = sm.H2Matrix(_dev(x), 2, 64, 4, 1e-9)
    _same(h.export(), ho.export())
    h.close()


def test_graph_matvec_equals_plain_and_follows_x(clean_table):
    x = si.uniform_cube(20000, 3, 4300)
    h = sm.H2Matrix(_dev(x), 1, 128, 4, 1e-8)
    s = torch.cuda.Stream(DEV)
    X = _dev(si.rhs(20000, 16, 4301))
    Y = torch.empty_like(X)
    for prec in (sm.SMASH_PREC_F32X2, sm.SMASH_PREC_F64, sm.SMASH_PREC_F32):
        ref = h.matvec(X, precision=prec, stream=s)
        torch.cuda.synchronize()
        ref = ref.clone()
        n0 = sm.smash_launch_count()
        h.matvec_graph(X, Y, precision=prec, stream=s)
        torch.cuda.synchronize()
        assert torch.equal(Y, ref), prec
        n1 = sm.smash_launch_count()
        h.matvec_graph(X, Y, precision=prec, stream=s)
        torch.cuda.synchronize()
        n2 = sm.smash_launch_count()
        assert n2 - n1 > 5            # the replay's kernels are counted
        assert torch.equal(Y, ref)
        assert n1 > n0
    assert sm.smash_matvec_graph_count(h.h) == 3
    # new contents of the same buffer: the replay reads them
    with torch.cuda.stream(s):
        X.copy_(_dev(si.rhs(20000, 16, 4302)))
    h.matvec_graph(X, Y, precision=sm.SMASH_PREC_F32X2, stream=s)
    ref = h.matvec(X, precision=sm.SMASH_PREC_F32X2, stream=s)
    torch.cuda.synchronize()
    assert torch.equal(Y, ref)
    assert sm.smash_matvec_graph_count(h.h) == 3
    # a batch representation replays too
    probs = si.batched_problems(6, 4310, n_lo=500, n_hi=4000)
    for d, (xb, off, kid, _) in si.group_by_dimension(probs).items():
        hb = sm.H2Matrix.batch(_dev(xb), off, kid, 64, 4, 1e-8)
        Xb = _dev(si.rhs(len(xb), 8, 4311))
        Yb = torch.empty_like(Xb)
        hb.matvec_graph(Xb, Yb, precision=sm.SMASH_PREC_F32)
        assert torch.equal(Yb, hb.matvec(Xb, precision=sm.SMASH_PREC_F32))
        hb.close()
    h.close()


def test_graph_matvec_rejects_host_buffers(clean_table):
    x = si.uniform_cube(2000, 3, 4400)
    h = sm.H2Matrix(_dev(x), 1, 128, 4, 1e-8)
    X = si.rhs(2000, 2, 4401)
    with pytest.raises(sm.SmashError, match="device buffers"):
        h.matvec_graph(X, np.empty_like(X))
    h.close()


def test_tcgen05_coupling_candidate_keeps_the_tf32_bar(clean_table, tmp_path):
    """The TF32 coupling has two kernels: warp MMAs over staged tiles and the
    tcgen05 kernel with its accumulator in tensor memory.  Forcing the tcgen05
    candidate through the tuning table gives the same bar against the oracle
    (1e-3) as the default."""
    x = si.sphere_with_caps(10000, 4500)
    q = si.rhs(10000, 32, 4501)
    ho = oracle.H2(x, 2, 128, 5, 1e-8)
    zo, sc = ho.matvec(q), ho.matvec_abs(q)
    sm.smash_set_autotune(True)
    h = sm.H2Matrix(_dev(x), 2, 128, 5, 1e-8)
    h.matvec(_dev(q), precision=sm.SMASH_PREC_TF32)
    sm.smash_set_autotune(False)
    path = tmp_path / "t.json"
    sm.smash_autotune_save(str(path))
    table = json.loads(path.read_text())["entries"]
    keys = [k for k in table if k.startswith("ksum_tc/") and "/m0/" in k]
    assert keys
    for choice in (1, 64):  # 1 = the tcgen05 kernel, 64 = a warp-MMA tile
        forced = dict(table)
        forced.update({k: choice for k in keys})
        path.write_text(json.dumps({"smash_autotune": 1, "entries": forced}))
        sm.smash_autotune_clear()
        sm.smash_autotune_load(str(path))
        z = h.matvec(_dev(q), precision=sm.SMASH_PREC_TF32).cpu().numpy()
        assert_entrywise(z, zo, sc, TOL_TF32, what=f"tf32 choice {choice}")
        assert np.linalg.norm(z - zo) / np.linalg.norm(zo) <= 1e-3, choice
    h.close()
