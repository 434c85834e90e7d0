// util.cu -- errors, stream-ordered arena, device scan, LSD radix sort.
#include <cstdarg>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace smash {

std::atomic<uint64_t> g_launches{0};

void fail(smash_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    throw Error{st, std::string(buf)};
}

void check_cuda(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    const char *base = strrchr(file, '/');
    base = base ? base + 1 : file;
    if (e == cudaErrorMemoryAllocation)
        fail(SMASH_ENOMEM, "%s: %s (%s:%d)", what, cudaGetErrorString(e), base, line);
    fail(SMASH_ECUDA, "%s: %s (%s:%d)", what, cudaGetErrorString(e), base, line);
}

// ---------------------------------------------------------------- arena
void *Arena::raw(size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, stream_);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(SMASH_ENOMEM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    blocks_.push_back({p, bytes});
    bytes_ += bytes;
    return p;
}

void Arena::free(void *p) {
    if (!p) return;
    for (size_t i = 0; i < blocks_.size(); ++i)
        if (blocks_[i].p == p) {
            cudaFreeAsync(p, stream_);
            bytes_ -= blocks_[i].n;
            blocks_[i] = blocks_.back();
            blocks_.pop_back();
            return;
        }
}

void Arena::release() {
    for (auto &b : blocks_) cudaFreeAsync(b.p, stream_);
    blocks_.clear();
    bytes_ = 0;
}

// ---------------------------------------------------------------- kernel attributes
void allow_max_dynamic_smem(const void *func) {
    static std::mutex mu;
    static std::vector<const void *> done;
    std::lock_guard<std::mutex> lock(mu);
    for (const void *f : done)
        if (f == func) return;
    int dev = 0, optin = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    CK(cudaFuncGetAttributes(&fa, func));
    int dyn = optin - (int)fa.sharedSizeBytes;  // static shared memory counts against the same limit
    CK(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    done.push_back(func);
}

// ---------------------------------------------------------------- timing
static std::atomic<int> g_prof{0};
bool profiling_enabled() { return g_prof.load() != 0; }

void PhaseTimer::mark() {
    if (!p || !p->on || n >= 11) return;
    CK(cudaEventCreate(&ev[n]));
    CK(cudaEventRecord(ev[n], s));
    ++n;
}

void PhaseTimer::finish(int first_slot) {
    if (!p || !p->on || n < 2) return;
    CK(cudaEventSynchronize(ev[n - 1]));
    for (int i = 0; i + 1 < n && first_slot + i < 10; ++i) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
        p->ms[first_slot + i] = ms;
    }
}

PhaseTimer::~PhaseTimer() {
    for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]);
}

// ---------------------------------------------------------------- scan
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__global__ void __launch_bounds__(kScanThreads)
scan_tile_kernel(const T *__restrict__ in, int64_t *__restrict__ out, int64_t n, int64_t *__restrict__ bsum) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t run = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        int64_t x = idx < n ? (int64_t)in[idx] : 0;
        v[i] = run;
        run += x;
    }
    // inclusive scan of per-thread totals
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        int64_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;  // exclusive
        if (lane == kScanThreads / 32 - 1 && bsum) bsum[blockIdx.x] = ti;
    }
    __syncthreads();
    int64_t off = warp_tot[w] + incl - run;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = v[i] + off;
    }
}

__global__ void scan_add_kernel(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ boff,
                                const int64_t *__restrict__ base_dev) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    int64_t b = boff ? boff[idx / kScanTile] : 0;
    if (base_dev) b += *base_dev;
    out[idx] += b;
}

template <class T>
__global__ void scan_total_typed(const int64_t *__restrict__ out, const T *__restrict__ in, int64_t n,
                                 int64_t *total, const int64_t *base_dev) {
    int64_t b = base_dev ? *base_dev : 0;
    *total = n ? out[n - 1] + (int64_t)in[n - 1] : b;
}

template <class T>
void exclusive_scan(const T *in, int64_t *out, int64_t n, const int64_t *base_dev, int64_t *total_dev,
                    cudaStream_t s, Arena &scratch) {
    if (n > 0) {
        int64_t nb = (n + kScanTile - 1) / kScanTile;
        int64_t *bsum = nullptr, *boff = nullptr;
        if (nb > 1) {
            bsum = scratch.alloc<int64_t>(nb);
            boff = scratch.alloc<int64_t>(nb);
        }
        scan_tile_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, bsum);
        LAUNCHED();
        if (nb > 1) exclusive_scan<int64_t>(bsum, boff, nb, nullptr, nullptr, s, scratch);
        if (nb > 1 || base_dev) {
            scan_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, boff, base_dev);
            LAUNCHED();
        }
    }
    if (total_dev) {
        scan_total_typed<T><<<1, 1, 0, s>>>(out, in, n, total_dev, base_dev);
        LAUNCHED();
    }
}

template void exclusive_scan<int32_t>(const int32_t *, int64_t *, int64_t, const int64_t *, int64_t *,
                                      cudaStream_t, Arena &);
template void exclusive_scan<int64_t>(const int64_t *, int64_t *, int64_t, const int64_t *, int64_t *,
                                      cudaStream_t, Arena &);
template void exclusive_scan<uint32_t>(const uint32_t *, int64_t *, int64_t, const int64_t *, int64_t *,
                                       cudaStream_t, Arena &);

// ---------------------------------------------------------------- max
__global__ void max_kernel(const int64_t *__restrict__ in, int64_t n, unsigned long long *out) {
    int64_t m = INT64_MIN;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, in[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    // values are non-negative sizes: compare as unsigned after clamping
    if ((threadIdx.x & 31) == 0 && m >= 0) atomicMax(out, (unsigned long long)m);
}

void reduce_max(const int64_t *in, int64_t n, int64_t *out_dev, cudaStream_t s) {
    CK(cudaMemsetAsync(out_dev, 0, sizeof(int64_t), s));
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
    max_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(in, n, reinterpret_cast<unsigned long long *>(out_dev));
    LAUNCHED();
}

// ---------------------------------------------------------------- radix sort
constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;

__global__ void __launch_bounds__(kRsThreads)
rs_hist_kernel(const uint64_t *__restrict__ keys, int64_t n, int shift, uint32_t *__restrict__ hist, int nblk) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t t0 = (int64_t)blockIdx.x * kRsTile;
    for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
        int64_t idx = t0 + i;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: elements of a tile are ranked in their original order,
// 256 at a time, with warp match masks and per-warp digit counts.
__global__ void __launch_bounds__(kRsThreads)
rs_scatter_kernel(const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin, uint64_t *__restrict__ kout,
                  int32_t *__restrict__ vout, int64_t n, int shift, const int64_t *__restrict__ offs, int nblk) {
    __shared__ int64_t run[256];
    __shared__ uint32_t wcnt[kRsThreads / 32][256];
    int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    run[tid] = offs[(int64_t)tid * nblk + blockIdx.x];
    int64_t t0 = (int64_t)blockIdx.x * kRsTile;
    unsigned lt = (1u << lane) - 1u;
    for (int round = 0; round < kRsItems; ++round) {
        int64_t idx = t0 + (int64_t)round * kRsThreads + tid;
        bool valid = idx < n;
        uint64_t key = valid ? kin[idx] : 0;
        int32_t val = (valid && vin) ? vin[idx] : 0;
        unsigned dig = valid ? (unsigned)((key >> shift) & 255u) : 256u;
#pragma unroll
        for (int ww = 0; ww < kRsThreads / 32; ++ww) wcnt[ww][tid] = 0;
        __syncthreads();
        unsigned peers = __match_any_sync(0xffffffffu, dig);
        int rank = __popc(peers & lt);
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcnt[w][dig] = (uint32_t)__popc(peers);
        __syncthreads();
        if (valid) {
            int64_t off = run[dig] + rank;
            for (int ww = 0; ww < w; ++ww) off += wcnt[ww][dig];
            kout[off] = key;
            if (vout) vout[off] = val;
        }
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (int ww = 0; ww < kRsThreads / 32; ++ww) tot += wcnt[ww][tid];
        run[tid] += tot;
        __syncthreads();
    }
}

void radix_sort(uint64_t *keys, int32_t *vals, int64_t n, int bits, cudaStream_t s, Arena &scratch) {
    if (n <= 1 || bits <= 0) return;
    int nblk = (int)((n + kRsTile - 1) / kRsTile);
    uint64_t *kb = scratch.alloc<uint64_t>(n);
    int32_t *vb = vals ? scratch.alloc<int32_t>(n) : nullptr;
    uint32_t *hist = scratch.alloc<uint32_t>((size_t)256 * nblk);
    int64_t *offs = scratch.alloc<int64_t>((size_t)256 * nblk);
    uint64_t *ka = keys, *kb2 = kb;
    int32_t *va = vals, *vb2 = vb;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        rs_hist_kernel<<<nblk, kRsThreads, 0, s>>>(ka, n, shift, hist, nblk);
        LAUNCHED();
        exclusive_scan<uint32_t>(hist, offs, (int64_t)256 * nblk, nullptr, nullptr, s, scratch);
        rs_scatter_kernel<<<nblk, kRsThreads, 0, s>>>(ka, va, kb2, vb2, n, shift, offs, nblk);
        LAUNCHED();
        std::swap(ka, kb2);
        std::swap(va, vb2);
    }
    if (ka != keys) {
        CK(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        if (vals) CK(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    scratch.free(kb);
    if (vb) scratch.free(vb);
    scratch.free(hist);
    scratch.free(offs);
}

}  // namespace smash

extern "C" void smash_set_profiling(int on) { smash::g_prof.store(on ? 1 : 0); }
extern "C" uint64_t smash_launch_count(void) { return smash::g_launches.load(); }
