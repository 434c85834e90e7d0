// serve.cu -- a continuous-batching request server for construct-and-apply
// requests (host runtime around smash_build_xy / smash_matvec_ex).
//
// Requests are admitted in arrival order as in-flight slots and the device
// memory budget allow: a request is admitted when fewer than max_inflight
// requests run and its predicted footprint fits the unreserved budget (a
// request that does not fit runs alone once nothing else is in flight).
// Each worker thread owns a CUDA stream, so admitted requests build and apply
// concurrently and their kernels overlap on the device.  A request may keep
// its H^2 representation resident for later apply requests.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t id = 0;
    bool apply = false;       // apply to a resident representation
    int64_t resident_id = 0;  // for apply requests
    bool keep = false;
    const double *x = nullptr, *y = nullptr, *X = nullptr;  // caller memory
    double *Y = nullptr;                                     // caller memory
    int64_t nx = 0, ny = 0;
    int dim = 0, kernel_id = 0, leaf = 0, order = 0, nrhs = 0;
    double tol = 0;
    size_t predicted = 0;
    double t_submit = 0, t_start = 0, t_end = 0;
    smash_status status = SMASH_OK;
    std::string error;
    bool done = false;
    int64_t kept_id = 0;
};

}  // namespace

struct smash_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<int64_t, std::unique_ptr<Request>> requests;
    std::unordered_map<int64_t, smash_handle> resident;
    std::unordered_map<int64_t, size_t> resident_bytes;
    size_t budget = 0, reserved = 0;
    int max_inflight = 1, inflight = 0, max_seen = 0;
    int precision = SMASH_PREC_F64;
    int64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

bool admissible(const smash_server *s, const Request *r) {
    if (s->inflight >= s->max_inflight) return false;
    return s->reserved + r->predicted <= s->budget || s->inflight == 0;
}

void run_request(smash_server *s, Request *r, cudaStream_t stream) {
    smash_handle h = nullptr;
    smash_status st = SMASH_OK;
    if (r->apply) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            auto it = s->resident.find(r->resident_id);
            if (it != s->resident.end()) h = it->second;
        }
        if (!h) {
            r->status = SMASH_EINVAL;
            r->error = "no resident representation with this id";
            return;
        }
    } else {
        smash_options opt;
        smash_default_options(&opt);
        // a representation kept resident gets a stream of its own, which
        // outlives this worker; otherwise it builds on the worker's stream
        opt.stream = r->keep ? nullptr : stream;
        st = smash_build_xy(r->x, r->nx, r->y, r->ny, r->dim, r->kernel_id, r->leaf, r->order, r->tol, &opt, &h);
        if (st != SMASH_OK) {
            r->status = st;
            r->error = smash_last_error();
            return;
        }
    }
    st = smash_matvec_ex(h, r->X, r->Y, r->nrhs, s->precision, stream);
    if (st == SMASH_OK && r->Y && r->X) {
        // device buffers: wait for the queued work before the request counts as done
        cudaError_t e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            st = SMASH_ECUDA;
            r->error = cudaGetErrorString(e);
        }
    }
    if (st != SMASH_OK) {
        r->status = st;
        r->error = smash_last_error();
    }
    if (!r->apply) {
        if (r->keep && st == SMASH_OK) {
            std::lock_guard<std::mutex> lock(s->mu);
            r->kept_id = s->next_id++;
            s->resident[r->kept_id] = h;
            s->resident_bytes[r->kept_id] = smash_footprint_bytes(h);
            s->reserved += s->resident_bytes[r->kept_id];
        } else {
            smash_free(h);
        }
    }
}

void worker_main(smash_server *s) {
    cudaStream_t stream = nullptr;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_work.wait(lock, [&] {
                return (s->stop && s->queue.empty()) || (!s->queue.empty() && admissible(s, s->queue.front()));
            });
            if (s->queue.empty()) break;  // stopping and drained
            r = s->queue.front();
            s->queue.pop_front();
            s->inflight++;
            s->max_seen = std::max(s->max_seen, s->inflight);
            s->reserved += r->predicted;
            r->t_start = now_ms();
        }
        run_request(s, r, stream);
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->reserved -= r->predicted;
            s->inflight--;
            r->t_end = now_ms();
            r->done = true;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    if (stream) cudaStreamDestroy(stream);
}

smash_status server_fail(smash_status st, const char *msg) {
    smash::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" {

smash_status smash_server_create(int max_inflight, size_t mem_budget_bytes, int precision, smash_server_t *out) {
    if (!out) return server_fail(SMASH_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_inflight < 1 || max_inflight > 64) return server_fail(SMASH_EINVAL, "max_inflight must be in [1, 64]");
    if (precision < SMASH_PREC_F64 || precision > SMASH_PREC_TF32X3) return server_fail(SMASH_EINVAL, "bad precision");
    auto *s = new smash_server();
    s->max_inflight = max_inflight;
    s->precision = precision;
    if (mem_budget_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return server_fail(SMASH_ECUDA, "cudaMemGetInfo failed");
        }
        mem_budget_bytes = (size_t)(0.8 * (double)free_b);
    }
    s->budget = mem_budget_bytes;
    int dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < max_inflight; ++i)
        s->workers.emplace_back([s, dev]() {
            cudaSetDevice(dev);
            worker_main(s);
        });
    *out = s;
    return SMASH_OK;
}

static smash_status enqueue(smash_server_t s, std::unique_ptr<Request> r, int64_t *ticket) {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return server_fail(SMASH_EINVAL, "server is shutting down");
    r->id = s->next_id++;
    r->t_submit = now_ms();
    *ticket = r->id;
    s->queue.push_back(r.get());
    s->requests[r->id] = std::move(r);
    s->cv_work.notify_all();
    return SMASH_OK;
}

smash_status smash_server_submit(smash_server_t s, const double *x, int64_t nx, const double *y, int64_t ny, int dim,
                                 int kernel_id, int leaf_size, int order, double tol, const double *X, int nrhs,
                                 double *Y, int keep, int64_t *ticket) {
    if (!s || !x || !X || !Y || !ticket) return server_fail(SMASH_EINVAL, "NULL argument");
    if (nx < 1 || dim < 1 || dim > 3 || nrhs < 1 || nrhs > smash::kMaxNrhs)
        return server_fail(SMASH_EINVAL, "bad sizes");
    try {
        auto r = std::make_unique<Request>();
        r->nx = nx;
        r->ny = y ? ny : nx;
        r->dim = dim; r->kernel_id = kernel_id; r->leaf = leaf_size; r->order = order; r->tol = tol;
        r->nrhs = nrhs;
        r->keep = keep != 0;
        r->x = x;
        r->y = y;
        r->X = X;
        r->Y = Y;
        r->predicted = smash_predict_footprint(nx + (y ? ny : 0), dim, leaf_size, order, nrhs) +
                       sizeof(double) * (size_t)(r->nx + r->ny) * (dim + nrhs);
        return enqueue(s, std::move(r), ticket);
    } catch (const std::bad_alloc &) {
        return server_fail(SMASH_ENOMEM, "host allocation failed");
    }
}

smash_status smash_server_apply(smash_server_t s, int64_t resident_id, const double *X, int nrhs, double *Y,
                                int64_t *ticket) {
    if (!s || !X || !Y || !ticket) return server_fail(SMASH_EINVAL, "NULL argument");
    if (nrhs < 1 || nrhs > smash::kMaxNrhs) return server_fail(SMASH_EINVAL, "bad nrhs");
    int64_t ny = 0;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->resident.find(resident_id);
        if (it == s->resident.end()) return server_fail(SMASH_EINVAL, "no resident representation with this id");
        smash_info_t info;
        smash_info(it->second, &info);
        ny = info.ny;
    }
    try {
        auto r = std::make_unique<Request>();
        r->apply = true;
        r->resident_id = resident_id;
        r->nrhs = nrhs;
        r->X = X;
        r->Y = Y;
        r->predicted = sizeof(double) * (size_t)ny * 4 * 64;
        return enqueue(s, std::move(r), ticket);
    } catch (const std::bad_alloc &) {
        return server_fail(SMASH_ENOMEM, "host allocation failed");
    }
}

smash_status smash_server_wait(smash_server_t s, int64_t ticket, smash_request_stats *stats) {
    if (!s) return server_fail(SMASH_EINVAL, "server is NULL");
    std::unique_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lock(s->mu);
        auto it = s->requests.find(ticket);
        if (it == s->requests.end()) return server_fail(SMASH_EINVAL, "unknown ticket");
        Request *rp = it->second.get();
        s->cv_done.wait(lock, [&] { return rp->done; });
        r = std::move(it->second);
        s->requests.erase(it);
    }
    if (stats) {
        stats->queue_ms = r->t_start - r->t_submit;
        stats->service_ms = r->t_end - r->t_start;
        stats->latency_ms = r->t_end - r->t_submit;
        stats->predicted_bytes = r->predicted;
        stats->resident_id = r->kept_id;
        stats->points = r->apply ? 0 : r->nx;
    }
    if (r->status != SMASH_OK) return server_fail(r->status, r->error.c_str());
    return SMASH_OK;
}

smash_status smash_server_release(smash_server_t s, int64_t resident_id) {
    if (!s) return server_fail(SMASH_EINVAL, "server is NULL");
    smash_handle h = nullptr;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->resident.find(resident_id);
        if (it == s->resident.end()) return server_fail(SMASH_EINVAL, "no resident representation with this id");
        h = it->second;
        s->reserved -= s->resident_bytes[resident_id];
        s->resident.erase(it);
        s->resident_bytes.erase(resident_id);
    }
    smash_free(h);
    s->cv_work.notify_all();
    return SMASH_OK;
}

int smash_server_max_inflight_seen(smash_server_t s) {
    if (!s) return 0;
    std::lock_guard<std::mutex> lock(s->mu);
    return s->max_seen;
}

void smash_server_destroy(smash_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto &kv : s->resident) smash_free(kv.second);
    delete s;
}

}  // extern "C"
