// probe.cu -- measured arithmetic peaks of the device, the denominators of
// the roofline fractions of the ALU-bound kernels (kernel sums: FP32 pipe;
// compression and the FP64 matvec: FP64 pipe).  Each thread runs kChains
// independent chains of fused multiply-adds, enough to cover the pipe's
// latency at full occupancy; the grid is a multiple of the SM count.
#include <vector>

#include "internal.cuh"

namespace smash {

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, T b, T c, T *sink) {
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    // b = 1 and c = 0 at run time keep every value finite; the store keeps
    // the chains alive
    if (s == (T)-1.2345) sink[blockIdx.x] = s;
}

template <typename T>
double measure(int iters, int reps) {
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * kBlocksPerSm;
    cudaStream_t s;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    T *sink = nullptr;
    cudaEvent_t e0, e1;
    double best = 0.0;
    try {
        CK(cudaMallocAsync(&sink, sizeof(T) * (size_t)blocks, s));
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        fma_chain_kernel<T><<<blocks, kThreads, 0, s>>>(iters / 8, (T)1, (T)0, sink);  // warm-up
        LAUNCHED();
        for (int r = 0; r < reps; ++r) {
            CK(cudaEventRecord(e0, s));
            fma_chain_kernel<T><<<blocks, kThreads, 0, s>>>(iters, (T)1, (T)0, sink);
            LAUNCHED();
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            const double flops = 2.0 * kChains * (double)iters * kThreads * blocks;
            best = std::max(best, flops / (ms * 1e-3) / 1e12);
        }
    } catch (...) {
        if (sink) cudaFreeAsync(sink, s);
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
        throw;
    }
    CK(cudaFreeAsync(sink, s));
    CK(cudaStreamSynchronize(s));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    return best;
}

}  // namespace

}  // namespace smash

using namespace smash;

extern "C" smash_status smash_measure_fma_peak(int fp64, double *tflops) {
    try {
        if (!tflops) fail(SMASH_EINVAL, "tflops is NULL");
        // about 30 ms per launch at the nominal rates (80 TFLOP/s FP32, 1.2 TFLOP/s FP64)
        *tflops = fp64 ? measure<double>(1 << 14, 3) : measure<float>(1 << 20, 3);
        return SMASH_OK;
    } catch (const Error &e) {
        set_last_error(e.msg.c_str());
        return e.status;
    }
}
