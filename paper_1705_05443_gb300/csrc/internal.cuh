// internal.cuh -- shared declarations of the CUDA library behind include/smash.h.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <functional>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/smash.h"

namespace smash {

// one point (or a padded 4-vector), 32-byte aligned for vector loads
struct __align__(32) P4 {
    double x, y, z, w;
};

constexpr int kMaxR = 512;     // largest order^dim
constexpr int kMaxP = 64;      // largest order
constexpr int kMaxNrhs = 64;
constexpr int kMaxSwaps = 1000;  // cap of the Gu-Eisenstat swap loop per node

// ---------------------------------------------------------------- errors
struct Error {
    smash_status status;
    std::string msg;
};
[[noreturn]] void fail(smash_status st, const char *fmt, ...);
void check_cuda(cudaError_t e, const char *what, const char *file, int line);
#define CK(x) ::smash::check_cuda((x), #x, __FILE__, __LINE__)

extern std::atomic<uint64_t> g_launches;
#define LAUNCHED() \
    do { ::smash::g_launches.fetch_add(1, std::memory_order_relaxed); CK(cudaGetLastError()); } while (0)

// ---------------------------------------------------------------- memory
// Stream-ordered device allocations owned by one object; freed on release().
class Arena {
  public:
    explicit Arena(cudaStream_t s = nullptr) : stream_(s) {}
    ~Arena() { release(); }
    Arena(const Arena &) = delete;
    Arena &operator=(const Arena &) = delete;
    void set_stream(cudaStream_t s) { stream_ = s; }
    template <class T>
    T *alloc(size_t n) {
        return static_cast<T *>(raw(n * sizeof(T)));
    }
    void *raw(size_t bytes);
    void free(void *p);
    void release();
    size_t bytes() const { return bytes_; }

  private:
    struct Blk { void *p; size_t n; };
    cudaStream_t stream_;
    std::vector<Blk> blocks_;
    size_t bytes_ = 0;
};

// ---------------------------------------------------------------- primitives
// Exclusive scan of n values; out[i] = base + sum_{j<i} in[j] (base read from
// device memory when base_dev != nullptr); *total_dev = base + sum, if given.
template <class T>
void exclusive_scan(const T *in, int64_t *out, int64_t n, const int64_t *base_dev, int64_t *total_dev,
                    cudaStream_t s, Arena &scratch);

// Stable LSD radix sort of 64-bit keys on their low `bits` bits, carrying
// optional int32 values.  Sorts in place (keys, vals) using scratch buffers.
void radix_sort(uint64_t *keys, int32_t *vals, int64_t n, int bits, cudaStream_t s, Arena &scratch);

// Device maximum of an int64 array into *out_dev (n >= 1).
void reduce_max(const int64_t *in, int64_t n, int64_t *out_dev, cudaStream_t s);

// ---------------------------------------------------------------- representation
struct Side {
    // per node
    int32_t *m = nullptr;      // |i_bar|
    int32_t *k = nullptr;      // |i_hat|
    int64_t *in_off = nullptr; // leaf: first point (sorted); parent: skeleton slot of child0
    int64_t *sk_off = nullptr; // first skeleton slot of the node
    int64_t *loc_off = nullptr;// offset into loc (upper-bound prefix of m)
    int64_t *g_off = nullptr;  // offset into G (upper-bound prefix of max (m-k)k)
    int32_t *nswaps = nullptr;
    // flat
    int32_t *loc = nullptr;    // per node: k skeleton positions in i_bar, then m-k rest positions
    int64_t *skg_tmp = nullptr;// per node at loc_off: skeleton point indices before compaction
    double *G = nullptr;
    int64_t *skel_gidx = nullptr; // per skeleton slot: sorted point index
    double *skel_xyz = nullptr;   // per skeleton slot: coordinates, stride 4
    float *skel_dd = nullptr;     // per skeleton slot: double-float normalised coordinates, 8 floats
    float *skel_x3 = nullptr;     // per skeleton slot: exact three-float coordinates, 12 floats (deep trees)
    int64_t total_skel = 0, total_loc = 0, total_g = 0, skel_cap = 0;
    std::vector<int64_t> mub_max;  // per level, upper bound of m
};

struct Profile {
    bool on = false;
    double ms[10] = {0};
};

}  // namespace smash

namespace smash {
struct GraphCache;
}

struct smash_h2 {
    int dim = 0, kernel_id = 0, leaf_size = 0, order = 0, r = 0, same = 1, bits = 0;
    double tau = 0.7, f = 2.0, tol = 1e-8;
    int64_t nx = 0, ny = 0;
    // bounding cube of all points; for a batch of problems it is the frame of
    // the matvec coordinates only, each problem keeping its own cube below
    double lo[3] = {0, 0, 0}, s = 1.0;
    // batch of independent problems (X = Y each): problem t owns the sorted
    // points [tree_off[t], tree_off[t+1]) and the root node t; one problem
    // otherwise (nroots = 1, tree_geo = node_tree = nullptr)
    int64_t nroots = 1;
    std::vector<int64_t> tree_off;
    std::vector<double> tree_geo_host;  // nroots x {lo0, lo1, lo2, s}
    double *tree_geo = nullptr;         // device copy
    int32_t *node_tree = nullptr;       // problem of each node
    double anchors[smash::kMaxP];
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, num_sms = 0;
    smash::Arena mem;
    // sorted points
    int64_t *permx = nullptr, *permy = nullptr;
    uint64_t *keyx = nullptr, *keyy = nullptr;
    double *xs = nullptr, *ys = nullptr;  // stride 4
    float *xs_dd = nullptr, *ys_dd = nullptr;  // double-float x'' = 1 + (x - lo)/s, 8 floats per point
    float *xs_x3 = nullptr, *ys_x3 = nullptr;  // exact three-float x 2^-dd_e, 12 floats per point
    int dd_e = 0;
    // tree
    int L = 0;
    std::vector<int64_t> lvl_off;  // host copy, L + 1 entries
    int64_t nnodes = 0, nleaves = 0;
    int32_t *level = nullptr, *leaf = nullptr, *parent = nullptr, *child0 = nullptr, *nchild = nullptr;
    int64_t *rs = nullptr, *cs = nullptr;
    int32_t *rc = nullptr, *cc = nullptr;
    uint64_t *cell = nullptr;  // nnodes x 3
    int32_t *leaf_list = nullptr;
    int32_t *nonroot_list = nullptr;
    // lists
    int64_t nadm = 0, nnear = 0;
    int64_t *adm_ptr = nullptr, *near_ptr = nullptr;
    int32_t *adm_col = nullptr, *near_col = nullptr;
    // compression
    smash::Side row, colside;
    smash::Side *col = nullptr;  // == &row when same
    // statistics
    int64_t swaps = 0, swap_cap_hits = 0, coupling_pairs = 0, near_pairs = 0;
    int64_t rest_row = 0, g_row = 0, rest_col = 0, g_col = 0;  // exact sums of m-k and (m-k)k
    // the Taylor-expansion representation of 1/(x - y) on C (smash_build_taylor):
    // complex G and vectors, r = order terms, cl[l] = (l/e)(2 pi r)^(1/(2r)),
    // kappa(x, x) = d_x
    int taylor = 0;
    double taylor_cl[smash::kMaxP] = {0};
    double dx_re = 0.0, dx_im = 0.0;
    // the HSS representation (smash_build_hss, d = 1): L and L^- of (3.5), the
    // nearfield sets N_i of (A.1) in CSR, the truncated-SVD tolerance of (3.8)
    // and the singular vectors appended to each node's basis (rows, columns)
    int hss = 0;
    double eps_svd = 0.0;
    int64_t nnf = 0;
    int64_t *nf_ptr = nullptr;
    int32_t *nf_col = nullptr;
    int32_t *svd_row = nullptr, *svd_col = nullptr;
    smash::Profile prof_build, prof_mv;
    smash::GraphCache *graphs = nullptr;  // captured matvecs (smash_matvec_graph)
};

namespace smash {

// phases of the build (each in its own translation unit)
void build_geometry(smash_h2 *h, const double *x_dev, const double *y_dev, Arena &scratch);
void build_geometry_batch(smash_h2 *h, const double *x_dev, Arena &scratch);
void build_tree(smash_h2 *h, Arena &scratch);
void build_lists(smash_h2 *h, Arena &scratch);
void build_lists_hss(smash_h2 *h, Arena &scratch);
void build_compression_hss(smash_h2 *h, Arena &scratch);
void build_compression(smash_h2 *h, Arena &scratch);
void build_stats(smash_h2 *h, Arena &scratch);

// matvec in FP64: X_dev (ny x nrhs), Y_dev (nx x nrhs), both device
void matvec_f64(const smash_h2 *h, const double *X_dev, double *Y_dev, int nrhs, cudaStream_t s,
                Profile *prof, int kid);
// matvec with double-float kernel sums (kernels 1/|x-y| and 1/(x-y))
void matvec_dd(const smash_h2 *h, const double *X_dev, double *Y_dev, int nrhs, cudaStream_t s, Profile *prof,
               int kid);
bool dd_supported(int kernel_id);
// mixed-precision matvec: FP32 kernel sums (Kahan-compensated near field), FP64 transfers
// (precision SMASH_PREC_F32, or SMASH_PREC_TF32/BF16/TF32X3 for tensor-core coupling products)
void matvec_f32(const smash_h2 *h, const double *X_dev, double *Y_dev, int nrhs, cudaStream_t s, Profile *prof,
                int precision, int kid);
// tensor-core coupling over L: FP32 entries of the normalised two-float coordinates
// times q^ (FP32, ldq per slot) in TF32/BF16/split TF32, written to zhat (FP64) x scale
void coupling_tc(const smash_h2 *h, int precision, const float *qhat, double *zhat, int ldq, cudaStream_t s,
                 int kid);
// the TF32 coupling on tcgen05 (tensor-memory accumulator); tc05_take_timeouts
// returns and clears the count of CTAs whose bounded mbarrier waits gave up
void coupling_tc05(const smash_h2 *h, const float *qhat, double *zhat, int ldq, cudaStream_t s, int kid);
int tc05_take_timeouts();
// the double-float coupling with its products on the tensor cores (exact
// 8-bit digit splits of the entries and of q^, FP64 q^ in, FP64 zhat out);
// supported for one problem of at most 10 levels, tau < 1, ldq <= 16
// (warp MMAs); with tc05 true the same digit products are issued as tcgen05.mma
// with the level sums in tensor memory (9..16 columns).  oz5_take_timeouts
// returns and clears the count of CTAs of that variant whose bounded mbarrier
// waits gave up.
bool coupling_oz_supported(const smash_h2 *h, int kid, int ldq);
void coupling_oz(const smash_h2 *h, int kid, const double *qhat, double *zhat, int ldq, cudaStream_t s,
                 bool tc05 = false);
int oz5_take_timeouts();
// the near field with the same digit-split products (normalised two-float
// coordinates, exact three-float ones for close pairs, FP64 q in, zs out);
// nodes it cannot take get fallback[i] = 1
// (i indexes the leaf list) and must be run by the double-float kernel
bool near_oz_supported(const smash_h2 *h, int kid, int ldq);
void near_oz(const smash_h2 *h, int kid, const double *qs, double *zs, int ldq, int *fallback, cudaStream_t s);
void dd_coords(const double *pts, int64_t n, const double *lo, double s, float *out, cudaStream_t st);
void dd_coords3(const double *pts, int64_t n, int e, float *out, cudaStream_t st);
int dd_exact_exponent(double s);
// the double-float coupling uses normalised two-float coordinates up to this depth
constexpr int kDdNormalisedMaxLevels = 10;
// whether the double-float coupling takes the exact three-float coordinates:
// deep trees, and batches (whose cells are finer than the frame's levels)
inline bool dd_exact_coupling(const smash_h2 *h) { return h->L > kDdNormalisedMaxLevels || h->nroots > 1; }
// pass helpers shared by the matvec variants
void matvec_gather(const smash_h2 *h, const double *X, int nrhs, int ldq, double *qs, cudaStream_t s);
void matvec_upward(const smash_h2 *h, const double *qs, double *qhat, int ldq, cudaStream_t s);
void matvec_downward(const smash_h2 *h, double *zhat, double *zs, int ldq, cudaStream_t s);
void matvec_scatter(const smash_h2 *h, const double *zs, int ldq, int nrhs, double *Y, cudaStream_t s);

// The same matvec with caller-provided device scratch (no allocation):
// matvec_f64_scratch_bytes is the scratch it needs for nrhs right-hand sides.
size_t matvec_f64_scratch_bytes(const smash_h2 *h, int nrhs);
void matvec_f64_scratch(const smash_h2 *h, const double *X_dev, double *Y_dev, int nrhs, cudaStream_t s,
                        void *scratch, size_t scratch_bytes);
// The complex matvec of a Taylor representation (X, Y: nx x nrhs complex,
// interleaved, device memory).
void matvec_taylor(const smash_h2 *h, const double *X, double *Y, int nrhs, cudaStream_t s, Profile *prof);

// Commits the static scratch of smash_matvec_noalloc on device dev (the
// current device); called by every build.
void noalloc_prepare(int dev);

bool profiling_enabled();

// argument checks of the matvec entry points (fail() on bad input) and the
// precision dispatch they share
// (kid < 0: the kernel the handle was built for; the bases depend only on the
// points and cells, so any kernel valid for the dimension applies)
void check_kernel(int kernel_id, int dim);
void check_matvec_args(const smash_h2 *h, const double *X, const double *Y, int nrhs, int precision, int kid = -1);
void run_matvec(const smash_h2 *h, const double *X, double *Y, int nrhs, int precision, cudaStream_t s,
                Profile *prof, int kid = -1);
void destroy_graphs(smash_h2 *h);

// ---------------------------------------------------------------- autotuning
// tune_choose launches the recorded choice of `key` (or `dflt`); with tuning
// on and no record, it first times launch(c) for every candidate c on stream
// s (launch must be idempotent), records the fastest and launches it.
bool tune_active(cudaStream_t s);
bool tune_find(const std::string &key, int &value);
void tune_put(const std::string &key, int value);
int tune_choose(const std::string &key, const std::vector<int> &cands, int dflt, cudaStream_t s,
                const std::function<void(int)> &launch);
inline long long pow2_at_least(long long v) {
    long long p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Raises a kernel's dynamic shared-memory limit to the device's opt-in
// maximum, once per kernel.  The limit is a per-function setting shared by all
// host threads, so it is only ever raised, never set per launch.
void allow_max_dynamic_smem(const void *func);

// Message returned by smash_last_error() on this host thread.
void set_last_error(const char *msg);

// Helper for event-timed phases.
struct PhaseTimer {
    cudaStream_t s;
    Profile *p;
    cudaEvent_t ev[11];
    int n = 0;
    PhaseTimer(cudaStream_t s_, Profile *p_) : s(s_), p(p_) {}
    void mark();
    void finish(int first_slot);
    ~PhaseTimer();
};

}  // namespace smash
