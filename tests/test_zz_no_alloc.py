"""smash_matvec_noalloc: the matvec for callers that cannot allocate device
memory while they run (a host whose own pool allocator holds all free device
memory, a real-time loop that forbids allocation after start-up).  It must
give the same result as the allocating entry point, call after call, since
every call reuses one static scratch array.

This file is collected last on purpose (test_zz_*) so that a run stopping at
the first failure has already run every other test; it also passes alone in a
fresh process (the first build on the device commits the static scratch).
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


class _DefaultPool:
    """Usage counters of the device's default stream-ordered memory pool, the
    one the library's allocating paths draw from, read through the CUDA
    driver API (libcuda is part of every GPU driver install)."""

    USED_CURRENT, USED_HIGH, RESERVED_CURRENT = 7, 8, 5   # CUmemPool_attribute

    def __init__(self, ordinal):
        self.cu = C.CDLL("libcuda.so.1")
        assert self.cu.cuInit(0) == 0
        dev = C.c_int()
        assert self.cu.cuDeviceGet(C.byref(dev), ordinal) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def get(self, attr):
        v = C.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, C.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = C.c_uint64(0)      # setting the high-water mark resets it to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_HIGH, C.byref(zero)) == 0


def test_noalloc_calls_allocate_nothing():
    """After the builds, no call of the no-alloc entry point takes device
    memory: neither from the stream-ordered pool (its high-water mark stays at
    the use before the calls) nor from cudaMalloc (the device's free memory
    stays the same), on one handle and on a second one."""
    A = _build(20000, 3, sm.SMASH_K_INVR, 128, 4, 11)
    B = _build(6000, 2, sm.SMASH_K_LOG, 64, 5, 12)
    qa = torch.from_numpy(si.rhs(20000, 16, 13)).to(DEV)
    qb = torch.from_numpy(si.rhs(6000, 5, 14)).to(DEV)
    oa, ob = torch.empty_like(qa), torch.empty_like(qb)
    stream = torch.cuda.Stream(DEV)
    # one call per handle first: the runtime loads a module's kernels lazily
    # at their first launch (and may grow the local-memory reserve then),
    # which is the set-up of the process, not an allocation of the calls
    sm.smash_matvec_noalloc(A.h, qa, oa, stream=stream)
    sm.smash_matvec_noalloc(B.h, qb, ob, stream=stream)
    torch.cuda.synchronize()
    pool = _DefaultPool(DEV.index or 0)
    used0, reserved0 = pool.get(pool.USED_CURRENT), pool.get(pool.RESERVED_CURRENT)
    free0 = torch.cuda.mem_get_info(DEV)[0]
    pool.reset_high()
    for h, q, o in ((A.h, qa, oa), (B.h, qb, ob), (A.h, qa, oa), (B.h, qb, ob)):
        sm.smash_matvec_noalloc(h, q, o, stream=stream)
    torch.cuda.synchronize()
    assert pool.get(pool.USED_HIGH) == used0, "a no-alloc call drew memory from the stream-ordered pool"
    assert pool.get(pool.RESERVED_CURRENT) == reserved0
    assert torch.cuda.mem_get_info(DEV)[0] == free0, "device free memory changed across no-alloc calls"
    # the results are still the allocating entry point's
    assert _rel(oa, A.matvec(qa)) <= RTOL and _rel(ob, B.matvec(qb)) <= RTOL
    A.close()
    B.close()


def test_noalloc_rejects_wrong_shapes_before_the_call():
    A = _build(5000, 3, sm.SMASH_K_INVR, 64, 3, 15)
    q = torch.zeros((5000, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError):
        sm.smash_matvec_noalloc(A.h, q, torch.empty((4999, 4), dtype=torch.float64, device=DEV))
    with pytest.raises(ValueError):
        sm.smash_matvec_noalloc(A.h, q[:4000], torch.empty((5000, 4), dtype=torch.float64, device=DEV))
    A.close()


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
