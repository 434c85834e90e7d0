"""smash_matvec_noalloc: the matvec for callers that cannot allocate device
memory while they run (a host whose own pool allocator holds all free device
memory, a real-time loop that forbids allocation after start-up).  It must
give the same result as the allocating entry point, call after call, since
every call reuses one static scratch array.

This file is collected last on purpose (test_zz_*) so that a run stopping at
the first failure has already run every other test; it also passes alone in a
fresh process (the first call on the device performs the one-time set-up).
"""
import ctypes as C

import numpy as np
import pytest

import smash_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1705_05443_gb300 as sm  # noqa: E402

DEV = torch.device("cuda:0")
RTOL = 1e-11   # the FP64 matvec tolerance of the parity tests


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _build(n, d, kid, leaf, order, seed):
    x = torch.from_numpy(si.uniform_cube(n, d, seed)).to(DEV)
    return sm.H2Matrix(x, kid, leaf, order, 1e-8)


def test_noalloc_matches_the_allocating_matvec_on_consecutive_calls():
    A = _build(20000, 3, sm.SMASH_K_INVR, 128, 4, 1)
    B = _build(6000, 2, sm.SMASH_K_LOG, 64, 5, 2)
    qa = torch.from_numpy(si.rhs(20000, 16, 3)).to(DEV)
    qb = torch.from_numpy(si.rhs(6000, 5, 4)).to(DEV)
    ref_a = A.matvec(qa)                      # the existing entry point, smash_matvec
    ref_b = B.matvec(qb)
    torch.cuda.synchronize()
    # all calls share one scratch array, so they go on one stream, in order
    # (a dedicated stream: the default stream's handle is NULL, which the C
    # ABI reads as "the handle's own stream", one per handle)
    stream = torch.cuda.Stream(DEV)
    for _ in range(2):                        # two calls in a row on the same handle
        out = torch.full_like(ref_a, float("nan"))
        sm.smash_matvec_noalloc(A.h, qa, out, stream=stream)
        torch.cuda.synchronize()
        assert _rel(out, ref_a) <= RTOL
    # another handle in between, then the first again: nothing carries over
    outb = torch.full_like(ref_b, float("nan"))
    sm.smash_matvec_noalloc(B.h, qb, outb, stream=stream)
    out = torch.full_like(ref_a, float("nan"))
    sm.smash_matvec_noalloc(A.h, qa, out, stream=stream)
    torch.cuda.synchronize()
    assert _rel(outb, ref_b) <= RTOL
    assert _rel(out, ref_a) <= RTOL
    A.close()
    B.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    n = 200000
    A = _build(n, 3, sm.SMASH_K_INVR, 128, 3, 5)
    q = torch.zeros((n, 64), dtype=torch.float64, device=DEV)
    out = torch.empty_like(q)
    with pytest.raises(sm.SmashError) as ei:
        sm.smash_matvec_noalloc(A.h, q, out)
    assert ei.value.status == 1 and "no-alloc maximum" in str(ei.value)
    # host buffers are refused too (copying them would need device memory)
    qh = np.zeros((n, 1))
    with pytest.raises(sm.SmashError):
        sm.smash_matvec_noalloc(A.h, qh, np.zeros((n, 1)))
    A.close()
