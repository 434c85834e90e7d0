// noalloc.cu -- smash_matvec_noalloc: the H^2 matvec without any device
// allocation, for callers that cannot allocate device memory while they run
// (for instance a host that has handed all free device memory to its own
// pool allocator up front, or a real-time loop that forbids allocation after
// start-up).  Its scratch is one static device array of this file; the
// caller passes the built handle and its own device input and output.
#include <mutex>

#include "internal.cuh"

namespace smash {

namespace {

constexpr size_t kScratchBytes = (size_t)SMASH_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch of every smash_matvec_noalloc call on a device.  Each GPU that
// loads this library holds it until the process exits.  Host code must not
// use this name as an address: its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this set-up).
void *scratch_address(int dev) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(SMASH_ECUDA, "cudaGetSymbolAddress of the no-alloc scratch failed: %s", cudaGetErrorString(e));
        }
        g_addr[dev] = p;
    }
    return g_addr[dev];
}

}  // namespace

// Looks the scratch up on device dev (the current device) so that the module
// holding it is loaded and its 64 MiB committed now.  The CUDA runtime loads a
// module lazily, at its first use; without this the first
// smash_matvec_noalloc call would be the one to commit the array, possibly
// after a caller's own pool allocator has taken the free memory.  The build
// calls this once per device; a failure here is left for that first
// smash_matvec_noalloc call to report.
void noalloc_prepare(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return;
    try {
        scratch_address(dev);
    } catch (const Error &) {
    }
}

namespace {

bool on_device(const void *p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace smash

using namespace smash;

extern "C" smash_status smash_matvec_noalloc(smash_handle h, const double *X, double *Y, int nrhs, void *stream) {
    try {
        if (!h) fail(SMASH_EINVAL, "handle is NULL");
        if (!X || !Y) fail(SMASH_EINVAL, "X or Y is NULL");
        if (nrhs < 1 || nrhs > kMaxNrhs) fail(SMASH_EINVAL, "nrhs must be in [1, %d]", kMaxNrhs);
        int dev = -1;
        CK(cudaGetDevice(&dev));
        if (dev != h->device) fail(SMASH_EINVAL, "the handle's device (%d) must be the current device (%d)",
                                   h->device, dev);
        if (dev < 0 || dev >= kMaxDevices) fail(SMASH_ENOTSUP, "device index %d out of range", dev);
        if (!on_device(X) || !on_device(Y)) fail(SMASH_EINVAL, "X and Y must be device memory");
        size_t need = matvec_f64_scratch_bytes(h, nrhs);
        if (need > kScratchBytes)
            fail(SMASH_EINVAL, "problem needs %zu bytes of scratch, more than the %zu-byte no-alloc maximum "
                 "(use smash_matvec_ex)", need, kScratchBytes);
        void *scratch = scratch_address(dev);
        cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
        matvec_f64_scratch(h, X, Y, nrhs, s, scratch, kScratchBytes);
        return SMASH_OK;
    } catch (const Error &e) {
        set_last_error(e.msg.c_str());
        return e.status;
    }
}
