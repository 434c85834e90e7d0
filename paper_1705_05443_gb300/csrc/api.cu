// api.cu -- the extern "C" boundary of include/smash.h: validation, handle
// life cycle, host/device buffer handling, statistics and export.
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

namespace smash {

static thread_local std::string t_last_error;

static smash_status record(const Error &e) {
    t_last_error = e.msg;
    return e.status;
}

void set_last_error(const char *msg) { t_last_error = msg ? msg : ""; }

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static int bits_per_dim(int d) { return d == 1 ? 62 : (d == 2 ? 31 : 21); }

// Chebyshev points of the first kind on [-1, 1]: cos((2m+1) pi / (2p)).
static void chebyshev(int p, double *t) {
    const double pi = 3.14159265358979323846;
    for (int m = 0; m < p; ++m) t[m] = cos((double)(2 * m + 1) * pi / (double)(2 * p));
}

// Keep freed stream-ordered allocations cached in the device's default pool.
static void init_pool_once(int dev) {
    static std::once_flag once;
    std::call_once(once, [dev]() {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    });
}

// ---------------------------------------------------------------- statistics
__global__ void side_stats_kernel(int64_t nn, const int32_t *__restrict__ m, const int32_t *__restrict__ k,
                                  const int32_t *__restrict__ nsw, unsigned long long *acc) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nn) return;
    int mk = m[g] - k[g];
    atomicAdd(acc + 0, (unsigned long long)mk);
    atomicAdd(acc + 1, (unsigned long long)mk * (unsigned long long)k[g]);
    if (nsw[g] > 0) atomicAdd(acc + 2, (unsigned long long)nsw[g]);
    if (nsw[g] < 0) atomicAdd(acc + 3, 1ull);
}

// sum over the CSR of |i| |j| with per-node sizes ti (rows) and sj (columns)
__global__ void pair_work_kernel(int64_t nn, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                 const int32_t *__restrict__ ti, const int32_t *__restrict__ sj,
                                 unsigned long long *acc) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nn) return;
    unsigned long long s = 0;
    for (int64_t e = ptr[g]; e < ptr[g + 1]; ++e) s += (unsigned long long)sj[col[e]];
    if (s) atomicAdd(acc, s * (unsigned long long)ti[g]);
}

void build_stats(smash_h2 *h, Arena &scratch) {
    cudaStream_t s = h->stream;
    unsigned long long *acc = scratch.alloc<unsigned long long>(10);
    CK(cudaMemsetAsync(acc, 0, 10 * 8, s));
    unsigned blocks = (unsigned)((h->nnodes + 255) / 256);
    side_stats_kernel<<<blocks, 256, 0, s>>>(h->nnodes, h->row.m, h->row.k, h->row.nswaps, acc);
    LAUNCHED();
    if (!h->same) {
        side_stats_kernel<<<blocks, 256, 0, s>>>(h->nnodes, h->colside.m, h->colside.k, h->colside.nswaps, acc + 4);
        LAUNCHED();
    }
    pair_work_kernel<<<blocks, 256, 0, s>>>(h->nnodes, h->adm_ptr, h->adm_col, h->row.k, h->col->k, acc + 8);
    LAUNCHED();
    pair_work_kernel<<<blocks, 256, 0, s>>>(h->nnodes, h->near_ptr, h->near_col, h->rc, h->cc, acc + 9);
    LAUNCHED();
    unsigned long long v[10];
    CK(cudaMemcpyAsync(v, acc, sizeof(v), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->rest_row = (int64_t)v[0];
    h->g_row = (int64_t)v[1];
    h->rest_col = h->same ? h->rest_row : (int64_t)v[4];
    h->g_col = h->same ? h->g_row : (int64_t)v[5];
    h->swaps = (int64_t)(v[2] + v[6]);
    h->swap_cap_hits = (int64_t)(v[3] + v[7]);
    h->coupling_pairs = (int64_t)v[8];
    h->near_pairs = (int64_t)v[9];
    scratch.free(acc);
}

static void destroy(smash_h2 *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    h->mem.release();
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // namespace smash

using namespace smash;

template <class T>
static std::vector<T> fetch(const T *p, int64_t n, cudaStream_t s) {
    std::vector<T> v((size_t)std::max<int64_t>(n, 0));
    if (n > 0) CK(cudaMemcpyAsync(v.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    return v;
}

static void export_side(const smash_h2 *h, const Side &S, bool rows, int32_t *m_out, int32_t *k_out,
                        int64_t *skel_out, int64_t *rest_out, double *G_out) {
    cudaStream_t s = h->stream;
    int64_t nn = h->nnodes;
    auto m = fetch(S.m, nn, s);
    auto k = fetch(S.k, nn, s);
    auto in_off = fetch(S.in_off, nn, s);
    auto loc_off = fetch(S.loc_off, nn, s);
    auto g_off = fetch(S.g_off, nn, s);
    auto leaf = fetch(h->leaf, nn, s);
    auto start = fetch(rows ? h->rs : h->cs, nn, s);
    auto loc = fetch(S.loc, S.total_loc, s);
    auto skg = fetch(S.skel_gidx, S.total_skel, s);
    // a Taylor representation's G is complex: two doubles per entry
    const int gw = h->taylor ? 2 : 1;
    std::vector<double> G;
    if (G_out) G = fetch(S.G, S.total_g * gw, s);
    CK(cudaStreamSynchronize(s));
    int64_t ps = 0, pr = 0, pg = 0;
    for (int64_t g = 0; g < nn; ++g) {
        if (m_out) m_out[g] = m[g];
        if (k_out) k_out[g] = k[g];
        auto gid = [&](int pos) -> int64_t { return leaf[g] ? start[g] + pos : skg[in_off[g] + pos]; };
        int kk = k[g], mk = m[g] - k[g];
        for (int t = 0; t < kk; ++t, ++ps)
            if (skel_out) skel_out[ps] = gid(loc[loc_off[g] + t]);
        for (int u = 0; u < mk; ++u, ++pr)
            if (rest_out) rest_out[pr] = gid(loc[loc_off[g] + kk + u]);
        int64_t ng = (int64_t)mk * kk;
        if (G_out) std::memcpy(G_out + gw * pg, G.data() + gw * g_off[g], gw * ng * sizeof(double));
        pg += ng;
    }
}


extern "C" {

void smash_default_options(smash_options *opt) {
    if (!opt) return;
    opt->tau = 0.7;
    opt->f = 2.0;
    opt->stream = nullptr;
}

smash_status smash_build(const double *points, int dim, int64_t n, int kernel_id, int leaf_size, int order,
                         double tol, smash_handle *out) {
    return smash_build_xy(points, n, nullptr, 0, dim, kernel_id, leaf_size, order, tol, nullptr, out);
}

}  // extern "C"

// Shared by smash_build_xy and smash_build_batch: offsets == nullptr builds
// one problem (x, y); otherwise x holds nproblems independent problems with
// X = Y each, problem t owning rows [offsets[t], offsets[t+1]).
struct TaylorSpec {
    double dx_re, dx_im;
};

struct HssSpec {
    double eps_svd;
};

static smash_status build_impl(const double *x, int64_t nx, const double *y, int64_t ny, const int64_t *offsets,
                               int nproblems, int dim, int kernel_id, int leaf_size, int order, double tol,
                               const smash_options *opt, smash_handle *out, const TaylorSpec *taylor = nullptr,
                               const HssSpec *hss = nullptr) {
    if (out) *out = nullptr;
    smash_h2 *h = nullptr;
    try {
        smash_options o;
        smash_default_options(&o);
        if (opt) o = *opt;
        if (!out) fail(SMASH_EINVAL, "out is NULL");
        if (!x) fail(SMASH_EINVAL, "points are NULL");
        if (dim < 1 || dim > 3) fail(SMASH_EINVAL, "dim must be 1, 2 or 3 (got %d)", dim);
        if (nx < 1 || nx > INT32_MAX) fail(SMASH_EINVAL, "n must be in [1, 2^31) (got %lld)", (long long)nx);
        if (y && (ny < 1 || ny > INT32_MAX)) fail(SMASH_EINVAL, "ny must be in [1, 2^31)");
        if (leaf_size < 1) fail(SMASH_EINVAL, "leaf_size must be >= 1");
        if (order < 1 || order > kMaxP) fail(SMASH_EINVAL, "order must be in [1, %d]", kMaxP);
        int r = 1;
        for (int a = 0; a < dim; ++a) r *= order;
        if (taylor) r = order;  // r terms of the expansion (2.4)
        if (r > kMaxR) fail(SMASH_EINVAL, "order^dim = %d exceeds %d", r, kMaxR);
        if (!(tol > 0.0) || !std::isfinite(tol)) fail(SMASH_EINVAL, "tol must be positive and finite");
        if (taylor) {
            if (dim != 2 || y || offsets) fail(SMASH_EINVAL, "the Taylor representation takes one 2D point set");
            if (!std::isfinite(taylor->dx_re) || !std::isfinite(taylor->dx_im)) fail(SMASH_EINVAL, "d_x must be finite");
        } else {
            check_kernel(kernel_id, dim);
        }
        if (hss) {
            if (dim != 1 || offsets) fail(SMASH_EINVAL, "the HSS construction takes one point set on a line (dim 1)");
            if (kernel_id > SMASH_K_CAUCHY1D) fail(SMASH_EINVAL, "the HSS construction supports kernels 0..3");
            if (!(hss->eps_svd > 0.0) || !std::isfinite(hss->eps_svd)) fail(SMASH_EINVAL, "eps_svd must be positive");
        }
        if (!(o.tau > 0.0 && o.tau < 1.0)) fail(SMASH_EINVAL, "tau must be in (0, 1)");
        if (!(o.f > 1.0)) fail(SMASH_EINVAL, "f must be > 1");

        h = new smash_h2();
        if (offsets) {
            h->nroots = nproblems;
            h->tree_off.assign(offsets, offsets + nproblems + 1);
        }
        h->dim = dim; h->kernel_id = kernel_id; h->leaf_size = leaf_size; h->order = order; h->r = r;
        h->tau = o.tau; h->f = o.f; h->tol = tol;
        h->same = y == nullptr;
        h->nx = nx; h->ny = y ? ny : nx;
        h->bits = bits_per_dim(dim);
        chebyshev(order, h->anchors);
        if (hss) {
            h->hss = 1;
            h->eps_svd = hss->eps_svd;
        }
        if (taylor) {
            // the node-independent factors of (2.5): eta_{v,l} = (cl[l] / delta_v)^l
            const double pi = 3.14159265358979323846;
            h->taylor = 1;
            h->dx_re = taylor->dx_re;
            h->dx_im = taylor->dx_im;
            const double rho = pow(2.0 * pi * (double)r, 1.0 / (2.0 * (double)r));
            for (int l = 0; l < r; ++l) h->taylor_cl[l] = ((double)l / exp(1.0)) * rho;
        }
        CK(cudaGetDevice(&h->device));
        CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
        init_pool_once(h->device);
        noalloc_prepare(h->device);
        if (o.stream) {
            h->stream = (cudaStream_t)o.stream;
        } else {
            CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
            h->own_stream = true;
        }
        h->mem.set_stream(h->stream);
        h->prof_build.on = profiling_enabled();
        Arena scratch(h->stream);
        const double *xd = x, *yd = y;
        if (!is_device_ptr(x)) {
            double *t = scratch.alloc<double>((size_t)nx * dim);
            CK(cudaMemcpyAsync(t, x, (size_t)nx * dim * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            xd = t;
        }
        if (y && !is_device_ptr(y)) {
            double *t = scratch.alloc<double>((size_t)ny * dim);
            CK(cudaMemcpyAsync(t, y, (size_t)ny * dim * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            yd = t;
        }
        PhaseTimer tm(h->stream, &h->prof_build);
        tm.mark();
        if (h->nroots > 1) build_geometry_batch(h, xd, scratch);
        else build_geometry(h, xd, yd, scratch);
        tm.mark();
        build_tree(h, scratch);
        tm.mark();
        if (h->hss) build_lists_hss(h, scratch);
        else build_lists(h, scratch);
        tm.mark();
        if (h->hss) build_compression_hss(h, scratch);
        else build_compression(h, scratch);
        {
            // normalised two-float copies of the point and skeleton coordinates for
            // the SMASH_PREC_F32X2 and SMASH_PREC_F32 matvecs
            h->xs_dd = h->mem.alloc<float>((size_t)h->nx * 8);
            dd_coords(h->xs, h->nx, h->lo, h->s, h->xs_dd, h->stream);
            if (h->same) {
                h->ys_dd = h->xs_dd;
            } else {
                h->ys_dd = h->mem.alloc<float>((size_t)h->ny * 8);
                dd_coords(h->ys, h->ny, h->lo, h->s, h->ys_dd, h->stream);
            }
            h->row.skel_dd = h->mem.alloc<float>((size_t)std::max<int64_t>(h->row.total_skel, 1) * 8);
            dd_coords(h->row.skel_xyz, h->row.total_skel, h->lo, h->s, h->row.skel_dd, h->stream);
            if (!h->same) {
                h->colside.skel_dd = h->mem.alloc<float>((size_t)std::max<int64_t>(h->colside.total_skel, 1) * 8);
                dd_coords(h->colside.skel_xyz, h->colside.total_skel, h->lo, h->s, h->colside.skel_dd, h->stream);
            }
        }
        {
            // exact three-float copies of the points: the near field of the
            // double-float matvec, and the close pairs of the FP32 near field
            h->dd_e = dd_exact_exponent(h->s);
            h->xs_x3 = h->mem.alloc<float>((size_t)h->nx * 12);
            dd_coords3(h->xs, h->nx, h->dd_e, h->xs_x3, h->stream);
            if (h->same) {
                h->ys_x3 = h->xs_x3;
            } else {
                h->ys_x3 = h->mem.alloc<float>((size_t)h->ny * 12);
                dd_coords3(h->ys, h->ny, h->dd_e, h->ys_x3, h->stream);
            }
        }
        if (dd_supported(h->kernel_id)) {
            // and, for deep trees, of the skeletons
            if (dd_exact_coupling(h)) {
                h->row.skel_x3 = h->mem.alloc<float>((size_t)std::max<int64_t>(h->row.total_skel, 1) * 12);
                dd_coords3(h->row.skel_xyz, h->row.total_skel, h->dd_e, h->row.skel_x3, h->stream);
                if (!h->same) {
                    h->colside.skel_x3 =
                        h->mem.alloc<float>((size_t)std::max<int64_t>(h->colside.total_skel, 1) * 12);
                    dd_coords3(h->colside.skel_xyz, h->colside.total_skel, h->dd_e, h->colside.skel_x3, h->stream);
                }
            }
        }
        tm.mark();
        tm.finish(0);
        build_stats(h, scratch);
        scratch.release();
        CK(cudaStreamSynchronize(h->stream));
        *out = h;
        return SMASH_OK;
    } catch (const Error &e) {
        smash_status st = record(e);
        destroy(h);
        return st;
    } catch (const std::bad_alloc &) {
        destroy(h);
        t_last_error = "host allocation failed";
        return SMASH_ENOMEM;
    }
}

extern "C" {

smash_status smash_build_xy(const double *x, int64_t nx, const double *y, int64_t ny, int dim, int kernel_id,
                            int leaf_size, int order, double tol, const smash_options *opt, smash_handle *out) {
    return build_impl(x, nx, y, ny, nullptr, 1, dim, kernel_id, leaf_size, order, tol, opt, out);
}

smash_status smash_build_taylor(const double *points, int64_t n, int leaf_size, int r, double tau, double tol,
                                double dx_re, double dx_im, smash_handle *out) {
    smash_options o;
    smash_default_options(&o);
    o.tau = tau;
    TaylorSpec spec{dx_re, dx_im};
    return build_impl(points, n, nullptr, 0, nullptr, 1, 2, SMASH_K_CAUCHY_C, leaf_size, r, tol, &o, out, &spec);
}

smash_status smash_build_hss(const double *x, int64_t nx, const double *y, int64_t ny, int kernel_id, int leaf_size,
                             int order, double tol, double eps_svd, const smash_options *opt, smash_handle *out) {
    smash_options o;
    smash_default_options(&o);
    if (opt) o = *opt;
    HssSpec spec{eps_svd};
    return build_impl(x, nx, y, ny, nullptr, 1, 1, kernel_id, leaf_size, order, tol, &o, out, nullptr, &spec);
}

smash_status smash_export_hss(smash_handle h, int64_t *nf_ptr, int32_t *nf_col, int64_t cap, int32_t *svd_row,
                              int32_t *svd_col, int64_t *nnf) {
    try {
        if (!h || !nnf) fail(SMASH_EINVAL, "NULL argument");
        if (!h->hss) fail(SMASH_EINVAL, "not an HSS representation");
        *nnf = h->nnf;
        cudaStream_t s = h->stream;
        CK(cudaStreamSynchronize(s));
        if (nf_ptr) CK(cudaMemcpy(nf_ptr, h->nf_ptr, sizeof(int64_t) * (h->nnodes + 1), cudaMemcpyDeviceToHost));
        if (nf_col && cap >= h->nnf && h->nnf > 0)
            CK(cudaMemcpy(nf_col, h->nf_col, sizeof(int32_t) * h->nnf, cudaMemcpyDeviceToHost));
        if (svd_row) CK(cudaMemcpy(svd_row, h->svd_row, sizeof(int32_t) * h->nnodes, cudaMemcpyDeviceToHost));
        if (svd_col) CK(cudaMemcpy(svd_col, h->svd_col, sizeof(int32_t) * h->nnodes, cudaMemcpyDeviceToHost));
        return SMASH_OK;
    } catch (const Error &e) {
        return record(e);
    }
}

smash_status smash_matvec_complex(smash_handle h, const double *X, double *Y, int nrhs, void *stream) {
    try {
        if (!h) fail(SMASH_EINVAL, "handle is NULL");
        if (!h->taylor) fail(SMASH_EINVAL, "smash_matvec_complex needs a handle from smash_build_taylor");
        if (!X || !Y) fail(SMASH_EINVAL, "X or Y is NULL");
        if (nrhs < 1 || nrhs > kMaxNrhs) fail(SMASH_EINVAL, "nrhs must be in [1, %d]", kMaxNrhs);
        cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
        Arena io(s);
        const size_t bytes = sizeof(double) * 2 * (size_t)h->nx * nrhs;
        const double *Xd = X;
        double *Yd = Y;
        const bool yhost = !is_device_ptr(Y);
        if (!is_device_ptr(X)) {
            double *t = io.alloc<double>(2 * (size_t)h->nx * nrhs);
            CK(cudaMemcpyAsync(t, X, bytes, cudaMemcpyHostToDevice, s));
            Xd = t;
        }
        if (yhost) Yd = io.alloc<double>(2 * (size_t)h->nx * nrhs);
        h->prof_mv.on = profiling_enabled();
        matvec_taylor(h, Xd, Yd, nrhs, s, &h->prof_mv);
        if (yhost) CK(cudaMemcpyAsync(Y, Yd, bytes, cudaMemcpyDeviceToHost, s));
        io.release();
        if (yhost || !stream) CK(cudaStreamSynchronize(s));
        return SMASH_OK;
    } catch (const Error &e) {
        return record(e);
    } catch (const std::bad_alloc &) {
        t_last_error = "host allocation failed";
        return SMASH_ENOMEM;
    }
}

smash_status smash_build_batch(const double *points, const int64_t *offsets, int nproblems, int dim, int kernel_id,
                               int leaf_size, int order, double tol, const smash_options *opt, smash_handle *out) {
    if (out) *out = nullptr;
    if (!offsets || nproblems < 1) {
        t_last_error = "offsets is NULL or nproblems < 1";
        return SMASH_EINVAL;
    }
    if (offsets[0] != 0) {
        t_last_error = "offsets[0] must be 0";
        return SMASH_EINVAL;
    }
    for (int t = 0; t < nproblems; ++t)
        if (offsets[t + 1] <= offsets[t]) {
            t_last_error = "every problem needs at least one point (offsets strictly increasing)";
            return SMASH_EINVAL;
        }
    const int64_t n = offsets[nproblems];
    if (nproblems == 1) return build_impl(points, n, nullptr, 0, nullptr, 1, dim, kernel_id, leaf_size, order, tol,
                                          opt, out);
    return build_impl(points, n, nullptr, 0, offsets, nproblems, dim, kernel_id, leaf_size, order, tol, opt, out);
}

}  // extern "C"

namespace smash {

void check_kernel(int kernel_id, int dim) {
    if (kernel_id < 0 || kernel_id > SMASH_K_DLP2) fail(SMASH_EINVAL, "unknown kernel_id %d", kernel_id);
    if (kernel_id == SMASH_K_CAUCHY1D && dim != 1) fail(SMASH_EINVAL, "the Cauchy kernel needs dim == 1");
    if ((kernel_id == SMASH_K_DLP1 || kernel_id == SMASH_K_DLP2) && dim != 2)
        fail(SMASH_EINVAL, "the double-layer kernels need dim == 2");
}

void check_matvec_args(const smash_h2 *h, const double *X, const double *Y, int nrhs, int precision, int kid) {
    if (!h) fail(SMASH_EINVAL, "handle is NULL");
    if (h->taylor) fail(SMASH_EINVAL, "a Taylor representation is complex: use smash_matvec_complex");
    if (kid < 0) kid = h->kernel_id;
    check_kernel(kid, h->dim);
    if (!X || !Y) fail(SMASH_EINVAL, "X or Y is NULL");
    if (nrhs < 1 || nrhs > kMaxNrhs) fail(SMASH_EINVAL, "nrhs must be in [1, %d]", kMaxNrhs);
    if (precision < SMASH_PREC_F64 || precision > SMASH_PREC_TF32X3)
        fail(SMASH_EINVAL, "unknown precision %d", precision);
    if (precision == SMASH_PREC_F32X2 && !dd_supported(kid))
        fail(SMASH_EINVAL, "SMASH_PREC_F32X2 supports the kernels 1/|x-y| and 1/(x-y) only");
    if (precision == SMASH_PREC_F32X2 && !dd_supported(h->kernel_id))
        fail(SMASH_EINVAL, "SMASH_PREC_F32X2 needs a handle built for 1/|x-y| or 1/(x-y)");
    // the digit-split kernel sums scale entries by bounds that hold for
    // well-separated pairs; HSS sibling pairs need not be
    if (precision == SMASH_PREC_F32X2 && h->hss)
        fail(SMASH_EINVAL, "SMASH_PREC_F32X2 is not available on an HSS representation");
}

void run_matvec(const smash_h2 *h, const double *X, double *Y, int nrhs, int precision, cudaStream_t s,
                Profile *prof, int kid) {
    if (kid < 0) kid = h->kernel_id;
    if (precision == SMASH_PREC_F32X2)
        matvec_dd(h, X, Y, nrhs, s, prof, kid);
    else if (precision >= SMASH_PREC_F32)
        matvec_f32(h, X, Y, nrhs, s, prof, precision, kid);
    else
        matvec_f64(h, X, Y, nrhs, s, prof, kid);
}

}  // namespace smash

extern "C" {

static smash_status matvec_impl(smash_handle h, int kid, const double *X, double *Y, int nrhs, int precision,
                                void *stream) {
    try {
        check_matvec_args(h, X, Y, nrhs, precision, kid);
        cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
        Arena io(s);
        const double *Xd = X;
        double *Yd = Y;
        bool yhost = !is_device_ptr(Y);
        if (!is_device_ptr(X)) {
            double *t = io.alloc<double>((size_t)h->ny * nrhs);
            CK(cudaMemcpyAsync(t, X, (size_t)h->ny * nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
            Xd = t;
        }
        if (yhost) Yd = io.alloc<double>((size_t)h->nx * nrhs);
        h->prof_mv.on = profiling_enabled();
        run_matvec(h, Xd, Yd, nrhs, precision, s, &h->prof_mv, kid);
        if (yhost) CK(cudaMemcpyAsync(Y, Yd, (size_t)h->nx * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        io.release();
        if (yhost || !stream) {
            CK(cudaStreamSynchronize(s));
            if ((precision == SMASH_PREC_TF32 && tc05_take_timeouts() > 0) ||
                (precision == SMASH_PREC_F32X2 && oz5_take_timeouts() > 0))
                fail(SMASH_ETIMEOUT, "a tensor-core wait gave up; the result is not valid");
        }
        return SMASH_OK;
    } catch (const Error &e) {
        return record(e);
    } catch (const std::bad_alloc &) {
        t_last_error = "host allocation failed";
        return SMASH_ENOMEM;
    }
}

smash_status smash_matvec_ex(smash_handle h, const double *X, double *Y, int nrhs, int precision, void *stream) {
    return matvec_impl(h, -1, X, Y, nrhs, precision, stream);
}

smash_status smash_matvec_kernel(smash_handle h, int kernel_id, const double *X, double *Y, int nrhs, int precision,
                                 void *stream) {
    if (kernel_id < 0) {
        t_last_error = "kernel_id must be >= 0";
        return SMASH_EINVAL;
    }
    return matvec_impl(h, kernel_id, X, Y, nrhs, precision, stream);
}

smash_status smash_matvec(smash_handle h, const double *X, double *Y, int nrhs) {
    return smash_matvec_ex(h, X, Y, nrhs, SMASH_PREC_F64, nullptr);
}

void smash_free(smash_handle h) { destroy(h); }

smash_status smash_info(smash_handle h, smash_info_t *info) {
    if (!h || !info) {
        t_last_error = "NULL argument";
        return SMASH_EINVAL;
    }
    std::memset(info, 0, sizeof(*info));
    info->nx = h->nx; info->ny = h->ny;
    info->dim = h->dim; info->kernel_id = h->kernel_id; info->leaf_size = h->leaf_size;
    info->order = h->order; info->r = h->r; info->same = h->same;
    info->levels = h->L;
    info->nnodes = h->nnodes; info->nadm = h->nadm; info->nnear = h->nnear; info->nleaves = h->nleaves;
    info->skel_row = h->row.total_skel; info->rest_row = h->rest_row; info->g_row = h->g_row;
    info->skel_col = h->col->total_skel; info->rest_col = h->rest_col; info->g_col = h->g_col;
    info->swaps = h->swaps; info->swap_cap_hits = h->swap_cap_hits;
    info->coupling_pairs = h->coupling_pairs; info->near_pairs = h->near_pairs;
    for (int a = 0; a < 3; ++a) info->lo[a] = h->lo[a];
    info->s = h->s; info->tau = h->tau; info->f = h->f; info->tol = h->tol;
    info->footprint_bytes = h->mem.bytes();
    info->nproblems = h->nroots;
    return SMASH_OK;
}

smash_status smash_export(smash_handle h, const smash_export_t *o) {
    try {
        if (!h || !o) fail(SMASH_EINVAL, "NULL argument");
        cudaStream_t s = h->stream;
        CK(cudaStreamSynchronize(s));
        int64_t nn = h->nnodes;
        auto put = [&](auto *dst, const auto *src, int64_t n) {
            if (dst && n > 0) CK(cudaMemcpyAsync(dst, src, n * sizeof(*dst), cudaMemcpyDeviceToHost, s));
        };
        put(o->permx, h->permx, h->nx);
        put(o->permy, h->permy, h->ny);
        put(o->keyx, h->keyx, h->nx);
        put(o->keyy, h->keyy, h->ny);
        if (o->lvl_off) std::memcpy(o->lvl_off, h->lvl_off.data(), (h->L + 1) * sizeof(int64_t));
        put(o->level, h->level, nn);
        put(o->leaf, h->leaf, nn);
        put(o->parent, h->parent, nn);
        put(o->child0, h->child0, nn);
        put(o->nchild, h->nchild, nn);
        put(o->rs, h->rs, nn);
        put(o->cs, h->cs, nn);
        put(o->cell, h->cell, nn * 3);
        put(o->adm_ptr, h->adm_ptr, nn + 1);
        put(o->adm_col, h->adm_col, h->nadm);
        put(o->near_ptr, h->near_ptr, nn + 1);
        put(o->near_col, h->near_col, h->nnear);
        put(o->node_problem, h->node_tree, nn);
        if (o->problem_cube)
            std::memcpy(o->problem_cube, h->tree_geo_host.data(), h->tree_geo_host.size() * sizeof(double));
        CK(cudaStreamSynchronize(s));
        if (o->rc || o->cc) {
            auto rc = fetch(h->rc, nn, s);
            auto cc = fetch(h->cc, nn, s);
            CK(cudaStreamSynchronize(s));
            for (int64_t g = 0; g < nn; ++g) {
                if (o->rc) o->rc[g] = rc[g];
                if (o->cc) o->cc[g] = cc[g];
            }
        }
        export_side(h, h->row, true, o->m_row, o->k_row, o->skel_row, o->rest_row, o->G_row);
        export_side(h, *h->col, h->same ? true : false, o->m_col, o->k_col, o->skel_col, o->rest_col, o->G_col);
        return SMASH_OK;
    } catch (const Error &e) {
        return record(e);
    } catch (const std::bad_alloc &) {
        t_last_error = "host allocation failed";
        return SMASH_ENOMEM;
    }
}

size_t smash_footprint_bytes(smash_handle h) { return h ? h->mem.bytes() : 0; }

size_t smash_predict_footprint(int64_t n, int dim, int leaf_size, int order, int nrhs) {
    if (n < 1 || dim < 1 || dim > 3 || leaf_size < 1 || order < 1) return 0;
    double r = 1;
    for (int a = 0; a < dim; ++a) r *= order;
    double nd = (double)(1 << dim);
    double leaves = std::max(1.0, 2.0 * (double)n / leaf_size);
    double nodes = leaves * nd / (nd - 1.0) + 1.0;
    double far = dim == 3 ? 600 : (dim == 2 ? 44 : 4);
    double near = dim == 3 ? 90 : (dim == 2 ? 15 : 4);
    int ldq = nrhs <= 32 ? 1 : 32;
    while (ldq < nrhs) ldq *= 2;
    double pts = (double)n * (32 + 8 + 8 + 4);
    double tree = nodes * 80;
    double lists = (nodes * far + leaves * near) * (4 + 16) + nodes * 16;
    double gen = 8.0 * (double)n * r * 1.5 + 40.0 * n;
    double mv = 8.0 * ldq * ((double)n * 2 + 2.4 * (double)n) + 16.0 * n * nrhs;
    return (size_t)(1.25 * (pts + tree + lists + gen + mv)) + (64u << 20);
}

int smash_suggest_rank(double eps, double tau) {
    double v = log(eps) / log(tau);
    if (eps < 1e-8) return (int)floor(v - 20.0);
    if (eps < 1e-6) return (int)floor(v - 15.0);
    int r = (int)floor(v - 10.0);
    return r > 5 ? r : 5;
}

const char *smash_last_error(void) { return t_last_error.c_str(); }

int smash_last_profile(smash_handle h, double *ms, int n) {
    if (!h || !ms) return 0;
    int c = 0;
    for (int i = 0; i < 4 && c < n; ++i) ms[c++] = h->prof_build.ms[i];
    for (int i = 4; i < 10 && c < n; ++i) ms[c++] = h->prof_mv.ms[i];
    return c;
}

}  // extern "C"
