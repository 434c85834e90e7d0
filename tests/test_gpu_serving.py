"""The request server: continuous batching of construct-and-apply requests.

Each request's result must be the same whether it runs alone through the
plain path (smash_build_xy + smash_matvec) or in the mix with other requests
in flight: the kernels are deterministic and every request owns its
representation and vectors, so the bar is 1e-12 relative (observed: equal).
"""
import numpy as np
import pytest

import smash_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

RTOL = 1e-12


def _requests(count, seed):
    g = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(2 ** g.uniform(10, 14))
        x, y = si.cauchy_1d(n, seed * 100 + i)
        X = si.rhs(n, int(g.integers(1, 9)), seed * 100 + i + 50)
        out.append((x, y, X))
    return out


def _plain(x, y, X, prec=sm.SMASH_PREC_F64):
    H = sm.H2Matrix(x, sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10, y=y)
    Z = H.matvec(np.ascontiguousarray(X), precision=prec)
    H.close()
    return Z


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [sm.SMASH_PREC_F64, sm.SMASH_PREC_F32X2])
def test_results_are_the_same_alone_and_in_the_mix(prec):
    reqs = _requests(12, 1)
    srv = sm.SmashServer(max_inflight=4, precision=prec)
    tickets = [srv.submit(x, sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10, X, y=y) for x, y, X in reqs]
    mixed = [srv.wait(t) for t in tickets]
    assert srv.max_inflight_seen() >= 2            # requests really overlapped
    srv.close()
    for (x, y, X), (Z, st) in zip(reqs, mixed):
        assert _rel(Z, _plain(x, y, X, prec)) <= RTOL
        assert st["latency_ms"] >= st["service_ms"] > 0 and st["points"] == len(x)


def test_admission_by_memory_budget_serialises():
    reqs = _requests(5, 2)
    srv = sm.SmashServer(max_inflight=4, mem_budget_bytes=1)   # nothing fits: one at a time
    tickets = [srv.submit(x, sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10, X, y=y) for x, y, X in reqs]
    res = [srv.wait(t) for t in tickets]
    assert srv.max_inflight_seen() == 1
    srv.close()
    for (x, y, X), (Z, _) in zip(reqs, res):
        assert _rel(Z, _plain(x, y, X)) <= RTOL


def test_resident_representation_is_reused():
    (x, y, X), = _requests(1, 3)
    srv = sm.SmashServer(max_inflight=2)
    Z0, st = srv.wait(srv.submit(x, sm.SMASH_K_CAUCHY1D, 64, 16, 1e-10, X, y=y, keep=True))
    rid = st["resident_id"]
    assert rid > 0
    X2 = si.rhs(len(y), 3, 99)
    Z1, st1 = srv.wait(srv.apply(rid, X2, len(x)))
    assert st1["points"] == 0
    assert _rel(Z0, _plain(x, y, X)) <= RTOL
    assert _rel(Z1, _plain(x, y, X2)) <= RTOL
    srv.release(rid)
    with pytest.raises(sm.SmashError):
        srv.apply(rid, X2, len(x))
    srv.close()


def test_failed_request_reports_its_error():
    srv = sm.SmashServer(max_inflight=1)
    x = si.uniform_cube(100, 2, 4)
    t = srv.submit(x, sm.SMASH_K_CAUCHY1D, 16, 4, 1e-8, si.rhs(100, 1, 5))   # Cauchy needs dim 1
    with pytest.raises(sm.SmashError) as ei:
        srv.wait(t)
    assert ei.value.status == 1
    with pytest.raises(sm.SmashError):
        srv.wait(12345)
    srv.close()
