// graph.cu -- matvecs captured once into a CUDA graph and replayed.
//
// A resident representation applied again and again to the same device
// buffers (an iterative solver, a served apply loop) repeats the same
// sequence of per-level launches.  smash_matvec_graph records that sequence
// -- gather, near field, the upward levels, coupling, the downward levels,
// scatter, with their stream-ordered scratch allocations -- into one CUDA
// graph per (X, Y, nrhs, precision) and replays it with a single launch.
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace smash {

struct GraphCache {
    struct Entry {
        const double *X;
        double *Y;
        int nrhs, precision;
        cudaGraphExec_t exec;
        uint64_t kernels;  // kernel launches of one replay
    };
    std::mutex mu;
    std::vector<Entry> entries;
    cudaStream_t capture = nullptr;
};

void destroy_graphs(smash_h2 *h) {
    if (!h || !h->graphs) return;
    for (auto &e : h->graphs->entries) cudaGraphExecDestroy(e.exec);
    if (h->graphs->capture) cudaStreamDestroy(h->graphs->capture);
    delete h->graphs;
    h->graphs = nullptr;
}

static bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static GraphCache::Entry &capture_entry(smash_h2 *h, GraphCache &gc, const double *X, double *Y, int nrhs,
                                        int precision, cudaStream_t s) {
    for (auto &e : gc.entries)
        if (e.X == X && e.Y == Y && e.nrhs == nrhs && e.precision == precision) return e;
    if (!gc.capture) CK(cudaStreamCreateWithFlags(&gc.capture, cudaStreamNonBlocking));
    // one plain run first, after the work queued on s: sets the kernels'
    // shared-memory attributes and settles every tuned choice, neither of
    // which may happen under capture
    cudaEvent_t ready;
    CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    CK(cudaEventRecord(ready, s));
    CK(cudaStreamWaitEvent(gc.capture, ready, 0));
    cudaEventDestroy(ready);
    run_matvec(h, X, Y, nrhs, precision, gc.capture, nullptr);
    CK(cudaStreamSynchronize(gc.capture));
    const uint64_t before = g_launches.load();
    CK(cudaStreamBeginCapture(gc.capture, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t graph = nullptr;
    try {
        run_matvec(h, X, Y, nrhs, precision, gc.capture, nullptr);
    } catch (...) {
        cudaStreamEndCapture(gc.capture, &graph);
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        throw;
    }
    CK(cudaStreamEndCapture(gc.capture, &graph));
    const uint64_t kernels = g_launches.load() - before;
    g_launches.fetch_sub(kernels);  // counted again at every replay
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    gc.entries.push_back({X, Y, nrhs, precision, exec, kernels});
    return gc.entries.back();
}

}  // namespace smash

using namespace smash;

extern "C" {

smash_status smash_matvec_graph(smash_handle h, const double *X, double *Y, int nrhs, int precision,
                                void *stream) {
    try {
        check_matvec_args(h, X, Y, nrhs, precision);
        if (!on_device(X) || !on_device(Y)) fail(SMASH_EINVAL, "smash_matvec_graph needs device buffers X and Y");
        cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
        GraphCache *gc = nullptr;
        {
            static std::mutex create_mu;
            std::lock_guard<std::mutex> lock(create_mu);
            if (!h->graphs) h->graphs = new GraphCache();
            gc = h->graphs;
        }
        std::lock_guard<std::mutex> lock(gc->mu);
        GraphCache::Entry &e = capture_entry(h, *gc, X, Y, nrhs, precision, s);
        CK(cudaGraphLaunch(e.exec, s));
        g_launches.fetch_add(e.kernels);
        if (!stream) CK(cudaStreamSynchronize(s));
        return SMASH_OK;
    } catch (const Error &err) {
        set_last_error(err.msg.c_str());
        return err.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return SMASH_ENOMEM;
    }
}

int smash_matvec_graph_count(smash_handle h) {
    if (!h || !h->graphs) return 0;
    std::lock_guard<std::mutex> lock(h->graphs->mu);
    return (int)h->graphs->entries.size();
}

}  // extern "C"
