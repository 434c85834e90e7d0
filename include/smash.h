/*
 * smash.h -- C ABI of the GB300 SMASH H^2 library (libsmash.so).
 *
 * SMASH (Cai, Chow, Saad, Xi): an H^2 approximation A^ of the dense kernel
 * matrix A = [kappa(x_i, y_j)] built level by level from an adaptive tree,
 * interpolation bases and a strong rank-revealing QR, then applied with the
 * upward / coupling / downward / near-field passes of Section 3.4.
 *
 * Conventions for every entry point
 *  - Pointers to point coordinates, right-hand sides and results may be host
 *    or device memory; the library asks the CUDA runtime which one it is
 *    and copies host data to and from the device itself.
 *  - Point arrays are float64, n x dim, row-major (point i at p[i*dim]).
 *    Right-hand sides X are float64 ny x nrhs row-major in the caller's point
 *    order; results Y are float64 nx x nrhs row-major, overwritten.
 *  - The caller keeps ownership of every buffer it passes.  A handle owns all
 *    device memory of the representation until smash_free.
 *  - A handle is immutable after the build.  smash_matvec_ex calls on
 *    different streams may run concurrently on one handle; each allocates
 *    its own scratch from the stream-ordered pool.
 *  - Calls without _ex are synchronous.  No C++ exception crosses the ABI:
 *    every failure is a status code, with a message in smash_last_error().
 *  - Invalid input returns SMASH_EINVAL and leaves *out = NULL.  Invalid is:
 *    dim not in {1,2,3}; n < 1; leaf_size < 1; order < 1 or order^dim > 512;
 *    tol <= 0 or not finite; a non-finite coordinate; a kernel_id unknown or
 *    not valid for dim (SMASH_K_CAUCHY1D needs dim == 1); nrhs < 1 or > 64.
 */
#ifndef SMASH_H
#define SMASH_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SMASH_API __attribute__((visibility("default")))
#else
#define SMASH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smash_h2 *smash_handle;

typedef enum {
    SMASH_OK = 0,
    SMASH_EINVAL = 1,   /* invalid argument */
    SMASH_ENOMEM = 2,   /* device or host allocation failed */
    SMASH_ECUDA = 3,    /* a CUDA runtime error (message has the detail) */
    SMASH_ETIMEOUT = 4, /* a bounded device wait ran out (the tcgen05 kernels wait on
                           their MMA commits with an iteration limit).  The next
                           synchronous matvec reports it and clears it; until then the
                           tcgen05 digit-split coupling skips its work, so results of
                           calls on caller streams in between are not valid */
    SMASH_EDEPTH = 5,   /* tree depth limit exceeded */
    SMASH_ENOTSUP = 6   /* option not supported on this device */
} smash_status;

/* Kernels kappa(x, y); kappa = 0 wherever x and y coincide ((2.1) with d_x = 0). */
enum {
    SMASH_K_LOG = 0,     /* log |x - y|                 */
    SMASH_K_INVR = 1,    /* 1 / |x - y|                 */
    SMASH_K_YUKAWA = 2,  /* exp(-|x - y|) / |x - y|     */
    SMASH_K_CAUCHY1D = 3, /* 1 / (x - y), dim = 1, (6.1) */
    /* The y-gradient of the fundamental solution Phi = -(1/2 pi) log|x - y| of
     * Section 6.4, component by component (dim = 2):
     * -(1/2 pi) (y_a - x_a) / |x - y|^2, 0 at coincident points.  The double-layer
     * kernel (6.9) is sum_a of these times nu_a(y) |r'(t)| (smash_matvec_double_layer). */
    SMASH_K_DLP1 = 4,
    SMASH_K_DLP2 = 5,
    /* 1/(x - y) on the complex plane, points (x_0, x_1) read as x_0 + i x_1,
     * complex values, d_x where the points coincide ((2.1)); only in the
     * Taylor representation of smash_build_taylor */
    SMASH_K_CAUCHY_C = 6
};

/* Arithmetic of the matvec (Section 3.4).  The build is always FP64. */
enum {
    SMASH_PREC_F64 = 0,   /* FP64 kernel evaluation, transfers and sums */
    SMASH_PREC_F32X2 = 1, /* coupling, near field and transfers in double-float arithmetic
                             on the FP32 pipe (each value hi + lo floats, error-free products
                             and sums).  From 8 right-hand sides per pass the coupling and
                             near-field products run on the tensor cores instead, as exact
                             products of 8-bit digits of the double-float entries and
                             vectors (Section 3.4, (3.19)-(3.20)).  ~1e-12 relative to FP64
                             either way.  Kernels 1/|x-y| and 1/(x-y) only. */
    SMASH_PREC_F32 = 2,   /* mixed precision: coupling and near field in FP32 (kernel entries,
                             products, sums; the near field with Kahan-compensated sums),
                             differences from two-float coordinates; transfers FP64.
                             ~1e-7..1e-6 relative to FP64.  All kernels. */
    /* As SMASH_PREC_F32, with the coupling products (3.19) on the tensor cores: each
     * coupling block is evaluated in FP32 straight into the operand registers of
     * warp-level MMAs and multiplied with q^ in the stated format, accumulating in FP32.
     * The near field stays FP32 with compensated sums.  All kernels. */
    SMASH_PREC_TF32 = 3,  /* TF32 products (10-bit mantissas); ~1e-4 relative to FP64 */
    SMASH_PREC_BF16 = 4,  /* BF16 products (7-bit mantissas); ~1e-3 relative to FP64 */
    SMASH_PREC_TF32X3 = 5 /* split TF32 (hi*hi + hi*lo + lo*hi): FP32-level, ~1e-6 */
};

typedef struct {
    double tau;     /* separation ratio of (2.3); default 0.7, must be in (0, 1) */
    double f;       /* strong-RRQR bound s of Theorem 2.4; default 2, must be > 1 */
    void *stream;   /* cudaStream_t for the build; NULL = a stream owned by the handle */
} smash_options;

/* Fills *opt with the defaults above. */
SMASH_API void smash_default_options(smash_options *opt);

/*
 * smash_build -- H^2 construction of Section 3.3.2 with X = Y = points.
 *
 * Adaptive partition of the bounding cube (Section 3.1), admissible leaves
 * L (3.3) and inadmissible leaves L^- (3.4) under Definition 2.1, then for
 * levels L..2 the interpolation basis (2.2) of each node, compr (2.14) by
 * strong RRQR (Theorem 2.4, f = 2) with rank cut |R_kk| <= tol |R_11|, and
 * the nested generators (3.17)/(3.18).  Coupling and near-field blocks
 * ((3.19)/(3.20)) are kept as index sets and evaluated on the fly.
 *   points    n x dim float64 (host or device), not retained
 *   kernel_id SMASH_K_*;  leaf_size: a box splits while it holds more points
 *   order     interpolation points per axis (order^dim anchors per node)
 *   tol       relative rank tolerance of the RRQR
 *   out       receives the handle (NULL on failure)
 * Synchronous.  Errors: SMASH_EINVAL, SMASH_ENOMEM, SMASH_ECUDA.
 */
SMASH_API smash_status smash_build(const double *points, int dim, int64_t n, int kernel_id, int leaf_size,
                         int order, double tol, smash_handle *out);

/*
 * smash_build_xy -- as smash_build for a rectangular A with X != Y: the tree
 * partitions X and Y jointly (a box splits while it holds more than
 * leaf_size points of X or of Y), and rows and columns get separate
 * generators (P, G) and (F, H) of (3.16)/(3.17).  y == NULL means Y = X.
 * opt == NULL means smash_default_options.
 */
SMASH_API smash_status smash_build_xy(const double *x, int64_t nx, const double *y, int64_t ny, int dim,
                            int kernel_id, int leaf_size, int order, double tol,
                            const smash_options *opt, smash_handle *out);

/*
 * smash_build_batch -- many independent problems in one representation.
 * Problem t is the point set points[offsets[t] .. offsets[t+1]) (rows of the
 * n x dim float64 array, host or device; n = offsets[nproblems]) with X = Y.
 * Each problem is partitioned in its own bounding cube exactly as
 * smash_build would partition it alone (Section 3.1), so its tree, lists
 * (3.3)/(3.4), skeletons and generators (3.17) are those of the problem
 * built alone; problems never interact.  The nodes of one level of all
 * problems are processed by the same launches, and smash_matvec* applies
 * the block-diagonal matrix diag(A^_0, ..., A^_{T-1}) to X (n x nrhs, rows
 * in the order of points).  The paper treats one problem at a time; the
 * batch is an extension of this library.
 *   offsets  host array of nproblems + 1 int64, offsets[0] = 0, strictly
 *            increasing (every problem has at least one point)
 * Synchronous.  Errors: SMASH_EINVAL (also for bad offsets), SMASH_ENOMEM,
 * SMASH_ECUDA.
 */
SMASH_API smash_status smash_build_batch(const double *points, const int64_t *offsets, int nproblems, int dim,
                                         int kernel_id, int leaf_size, int order, double tol,
                                         const smash_options *opt, smash_handle *out);

/*
 * smash_build_taylor -- H^2 construction of Section 3.3.2 for the kernel of
 * (2.1) on C, kappa(x, y) = 1/(x - y) with kappa(x, x) = d_x, with the
 * farfield basis from the Taylor expansion (2.4)-(2.5) instead of
 * interpolation: for node i with cell centre a and radius delta (half the
 * cell diagonal, Definition 2.1 on the cell), U^_i = [phi_{a,l}(x - a)],
 * phi_{a,l}(t) = eta_{a,l} t^l / l!, l = 0..r-1, eta of (2.5).  compr (2.14)
 * is the complex strong RRQR (Theorem 2.4, f = 2, Householder reflectors
 * with real R_jj) with rank cut |R_kk| <= tol |R_11|; G is complex.  X = Y.
 *   points  n x 2 float64 (host or device): x_0 + i x_1
 *   r       terms of the expansion (1..64); Section 6.2 uses r = 22
 *   tau     separation ratio of (2.3), in (0, 1); Section 6.2 uses 0.65
 *   dx_re, dx_im  the diagonal value d_x of (2.1) (Section 6.2: 1)
 * The tree, lists and skeleton layout are those of smash_build with dim 2;
 * smash_export returns G_row as complex entries (two doubles each: the
 * array must hold 2 g_row doubles).  Apply with smash_matvec_complex; the
 * real matvec entry points reject the handle.  Synchronous.
 * Errors: SMASH_EINVAL, SMASH_ENOMEM, SMASH_ECUDA.
 */
SMASH_API smash_status smash_build_taylor(const double *points, int64_t n, int leaf_size, int r, double tau,
                                          double tol, double dx_re, double dx_im, smash_handle *out);

/*
 * smash_matvec_complex -- Y = A^ X on a Taylor representation (Section 3.4
 * with complex vectors, generators and kernel entries, FP64).
 *   X, Y  n x nrhs complex, interleaved (re, im) float64, caller's point
 *         order (2 n nrhs doubles each; host or device); Y overwritten
 *   stream  as smash_matvec_ex
 * Errors: SMASH_EINVAL (not a Taylor handle, NULL, nrhs outside [1, 64]),
 * SMASH_ENOMEM, SMASH_ECUDA.
 */
SMASH_API smash_status smash_matvec_complex(smash_handle h, const double *X, double *Y, int nrhs, void *stream);

/*
 * smash_build_hss -- HSS construction of Section 3.3.1 for points on a line
 * (dim = 1, where the partition of Section 3.1 is a binary tree).
 *   L  = the sibling pairs of every level and L^- = the leaves with
 *        themselves (3.5);
 *   N_i = the nearfield sets of (A.1) (siblings, children of the nodes of
 *        N_{p_i} and leaves of N_{p_i} that are not well separated from i
 *        with ratio opt->tau, Definition 2.1 on the cells);
 *   for levels L..2 and each node: the nearfield block row
 *        [A|_{i_bar^row x j_bar^col}]_{j in N_i} (3.7) and block column (3.11),
 *        their left singular vectors above eps_svd times the largest
 *        singular value (one-sided Jacobi), joined with the interpolation
 *        basis (2.2) of `order` points and compressed by strong RRQR (3.9),
 *        (3.13); rank cut |R_kk| <= tol |R_11|, f = opt->f.
 *   B_i and D_i of (3.15) are kept as index sets and evaluated on the fly.
 * Arguments as smash_build_xy with dim = 1 (y == NULL: Y = X); kernel_id in
 * 0..3.  At most 64 singular vectors per node (SMASH_ENOTSUP above that).
 * Apply with smash_matvec / smash_matvec_ex in every precision except
 * SMASH_PREC_F32X2 (its digit scaling needs well-separated pairs).
 * Synchronous.  Errors: SMASH_EINVAL, SMASH_ENOMEM, SMASH_ECUDA, SMASH_ENOTSUP.
 */
SMASH_API smash_status smash_build_hss(const double *x, int64_t nx, const double *y, int64_t ny, int kernel_id,
                                       int leaf_size, int order, double tol, double eps_svd,
                                       const smash_options *opt, smash_handle *out);

/*
 * smash_export_hss -- the nearfield sets N_i of an HSS representation in
 * CSR by global node id (nf_ptr: nnodes + 1 entries; nf_col: *nnf entries,
 * written only if cap >= *nnf) and the number of singular vectors appended
 * to each node's row and column basis (svd_row, svd_col: nnodes entries).
 * Host memory; NULL skips an array; *nnf is always written.
 * Errors: SMASH_EINVAL (not an HSS handle), SMASH_ECUDA.
 */
SMASH_API smash_status smash_export_hss(smash_handle h, int64_t *nf_ptr, int32_t *nf_col, int64_t cap,
                                        int32_t *svd_row, int32_t *svd_col, int64_t *nnf);

/*
 * smash_matvec -- Y = A^ X by the node-wise algorithm of Section 3.4:
 * upward pass (q^_i = V_i^T q, then W_c^T), coupling over L with kernel
 * blocks on skeleton pairs, downward pass (R_c, then U_i), near field over L^-.
 *   X  ny x nrhs float64, caller's point order (host or device)
 *   Y  nx x nrhs float64, overwritten (host or device)
 *   nrhs in [1, 64]
 * Synchronous; FP64.  Errors: SMASH_EINVAL, SMASH_ENOMEM, SMASH_ECUDA.
 */
SMASH_API smash_status smash_matvec(smash_handle h, const double *X, double *Y, int nrhs);

/*
 * smash_matvec_ex -- as smash_matvec with a precision mode (SMASH_PREC_*)
 * and a cudaStream_t.  stream == NULL: runs on the handle's stream and
 * returns when Y is complete (like smash_matvec).  An explicit stream: the
 * work is queued on it and the call returns without waiting when X and Y are
 * device memory; with host buffers it returns after Y has been copied back.
 */
SMASH_API smash_status smash_matvec_ex(smash_handle h, const double *X, double *Y, int nrhs, int precision,
                             void *stream);

/*
 * smash_matvec_kernel -- smash_matvec_ex with another kernel on the same
 * representation.  The bases and generators of Section 3 depend only on the
 * points and the cells (the interpolation basis (2.2) and its compression),
 * not on kappa; only the coupling (3.19) and near-field (3.20) entries do.
 * So one build serves every kernel valid for its dimension.
 *   kernel_id  SMASH_K_*, valid for the handle's dim
 * Errors: as smash_matvec_ex; SMASH_EINVAL for a kernel the dimension does
 * not allow, and for SMASH_PREC_F32X2 on a handle built for a kernel other
 * than 1/|x-y| or 1/(x-y).
 */
SMASH_API smash_status smash_matvec_kernel(smash_handle h, int kernel_id, const double *X, double *Y, int nrhs,
                                           int precision, void *stream);

/*
 * smash_matvec_double_layer -- Y = K X for the Nystrom discretisation of the
 * double-layer operator (6.7) with kernel (6.9) on the points of h (X = Y,
 * dim = 2): K_ij = grad_y Phi(x_i, x_j) . nu_j w_j for i != j, K_ii = diag_i,
 * with Phi = -(1/2 pi) log|x - y|.  Evaluated as
 * K X = A_1 diag(nu_1 w) X + A_2 diag(nu_2 w) X + diag(diag) X, where A_a is
 * the H^2 matrix of SMASH_K_DLP1/2 on the same representation.
 *   nu    n x 2 unit normals at the points (row-major), w  n quadrature
 *         weights (|r'(t_j)| h for the trapezoidal rule), diag  n diagonal
 *         entries (the kernel's limit at coincident points) or NULL for 0;
 *         host or device memory
 *   X, Y  n x nrhs, precision and stream as smash_matvec_ex (not F32X2)
 * Errors: SMASH_EINVAL (NULL normals or weights, dim != 2, nx != ny, the
 * errors of smash_matvec_ex), SMASH_ENOMEM, SMASH_ECUDA.
 */
SMASH_API smash_status smash_matvec_double_layer(smash_handle h, const double *nu, const double *wts,
                                                 const double *diag, const double *X, double *Y, int nrhs,
                                                 int precision, void *stream);

/*
 * smash_matvec_cauchy_like -- Y = A X for the Cauchy-like matrix of (6.1):
 * a_ij = kappa(x_i, y_j) sum_{l<p} w_il v_jl, i.e. (6.2)
 * A = sum_l diag(w_l) C diag(v_l) with C the matrix that h approximates
 * (Section 6.3 takes kappa = 1/(x - y), SMASH_K_CAUCHY1D; any kernel works).
 * The p scaled copies of X run through the H^2 matvec as one block of
 * p * nrhs right-hand sides and are recombined row by row in the order of l.
 *   w  nx x p float64, row-major (host or device);  v  ny x p likewise
 *   X  ny x nrhs, Y  nx x nrhs (caller point order), as smash_matvec_ex
 *   precision, stream: as smash_matvec_ex
 * Errors: SMASH_EINVAL (NULL pointers, p < 1, p * nrhs outside [1, 64],
 * the errors of smash_matvec_ex), SMASH_ENOMEM, SMASH_ECUDA.
 */
SMASH_API smash_status smash_matvec_cauchy_like(smash_handle h, const double *w, const double *v, int p,
                                                const double *X, double *Y, int nrhs, int precision,
                                                void *stream);

/*
 * smash_matvec_noalloc -- the FP64 matvec of smash_matvec_ex that allocates
 * no device memory, for callers that cannot allocate while they run (a host
 * that gives all free device memory to its own pool allocator up front, or a
 * real-time loop that forbids allocation after start-up).  The paper has no
 * counterpart: this is a deployment variant of the same computation.
 *   X  ny x nrhs float64 DEVICE memory, caller's point order
 *   Y  nx x nrhs float64 DEVICE memory, overwritten
 *   stream  cudaStream_t, NULL = the handle's stream; asynchronous
 * Its scratch (the q, z, q^ and z^ vectors) lives in one static device array
 * of SMASH_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library
 * holds until the process exits; problems whose scratch does not fit, i.e.
 * 8 * ldq * (nx + ny + skeleton slots of rows and columns) bytes beyond that
 * maximum (ldq = nrhs rounded up to a power of two, or to a multiple of 32
 * above 32), are rejected with SMASH_EINVAL and a message.  The array is
 * committed on a device by the first build on it (smash_build*, which looks
 * up its device address with cudaGetSymbolAddress with that device current),
 * so a caller that builds before handing the remaining device memory to its
 * own allocator finds the array already in place; if that lookup failed, the
 * first smash_matvec_noalloc call on the device repeats it (make that call
 * before any stream capture).  The handle's device must be the current
 * device.  Every call overwrites each scratch region before reading it, so
 * no state carries over between calls, but all calls share the one array:
 * calls whose GPU work overlaps race and must be ordered by the caller.  That
 * includes the default: stream == NULL means each handle's own stream, so
 * NULL-stream calls on two different handles run on two streams and race;
 * pass one stream to all of them.  Errors: SMASH_EINVAL, SMASH_ECUDA.
 */
#define SMASH_NOALLOC_SCRATCH_BYTES (64u << 20)
SMASH_API smash_status smash_matvec_noalloc(smash_handle h, const double *X, double *Y, int nrhs, void *stream);

/*
 * smash_matvec_graph -- smash_matvec_ex for device buffers X and Y, replayed
 * from a CUDA graph: the first call with a given (X, Y, nrhs, precision)
 * runs the matvec once, then captures its launches and stream-ordered
 * scratch allocations into a graph kept by the handle; every call launches
 * that graph on `stream` (NULL: the handle's stream, and the call waits for
 * completion).  The paper has no counterpart; this serves repeated applies
 * of a resident representation.  Results equal smash_matvec_ex's with the
 * same precision.  Errors: as smash_matvec_ex; SMASH_EINVAL for host
 * buffers.  smash_matvec_graph_count returns the graphs a handle holds.
 */
SMASH_API smash_status smash_matvec_graph(smash_handle h, const double *X, double *Y, int nrhs, int precision,
                                          void *stream);
SMASH_API int smash_matvec_graph_count(smash_handle h);

/* Releases the handle and its device memory; NULL-safe; waits for the
 * handle's pending work first. */
SMASH_API void smash_free(smash_handle h);

/*
 * Request server (host runtime around smash_build_xy and smash_matvec_ex).
 * Construct-and-apply requests are admitted in arrival order as in-flight
 * slots and device memory allow: a request starts when fewer than
 * max_inflight requests run and its predicted footprint
 * (smash_predict_footprint plus its vectors) fits the unreserved budget; a
 * request that does not fit runs alone once nothing else is in flight.  Each
 * of the max_inflight worker threads owns a CUDA stream, so admitted requests
 * build and apply concurrently and their kernels overlap on the device.  A
 * request may keep its representation resident (counted against the budget
 * until released) and later apply requests reuse it.  Buffers are not
 * copied: points, X and Y (host or device memory) must stay valid until
 * smash_server_wait has returned for the request; Y is complete then.  The
 * paper has no counterpart (deployment runtime).
 */
typedef struct smash_server *smash_server_t;

typedef struct {
    double queue_ms;        /* submission to admission */
    double service_ms;      /* admission to completion */
    double latency_ms;      /* submission to completion */
    size_t predicted_bytes; /* admission estimate */
    int64_t resident_id;    /* id of the kept representation (0 if none) */
    int64_t points;         /* nx of a construct request, 0 for apply */
} smash_request_stats;

/* mem_budget_bytes == 0: 80 % of the free device memory at creation.
 * precision: SMASH_PREC_* of the served matvecs.  Errors: SMASH_EINVAL, SMASH_ECUDA. */
SMASH_API smash_status smash_server_create(int max_inflight, size_t mem_budget_bytes, int precision,
                                           smash_server_t *out);
/* Queues build(x[, y]) + Y = A^ X; arguments as smash_build_xy / smash_matvec.
 * keep != 0 keeps the representation resident. */
SMASH_API smash_status smash_server_submit(smash_server_t s, const double *x, int64_t nx, const double *y,
                                           int64_t ny, int dim, int kernel_id, int leaf_size, int order,
                                           double tol, const double *X, int nrhs, double *Y, int keep,
                                           int64_t *ticket);
/* Queues Y = A^ X on a resident representation (X: ny x nrhs, Y: nx x nrhs). */
SMASH_API smash_status smash_server_apply(smash_server_t s, int64_t resident_id, const double *X, int nrhs,
                                          double *Y, int64_t *ticket);
/* Blocks until the request completes and fills *stats (may be NULL).
 * Returns the request's status. */
SMASH_API smash_status smash_server_wait(smash_server_t s, int64_t ticket, smash_request_stats *stats);
/* Frees a resident representation. */
SMASH_API smash_status smash_server_release(smash_server_t s, int64_t resident_id);
/* Largest number of requests that were in flight at the same time. */
SMASH_API int smash_server_max_inflight_seen(smash_server_t s);
/* Finishes the queued requests, joins the workers, frees resident representations. */
SMASH_API void smash_server_destroy(smash_server_t s);

/* Sizes and statistics of a built representation. */
typedef struct {
    int64_t nx, ny;
    int dim, kernel_id, leaf_size, order, r, same;
    int levels;                 /* L; the root is level 1 */
    int64_t nnodes, nadm, nnear, nleaves;
    int64_t skel_row, rest_row, g_row; /* sum k, sum (m-k), sum (m-k)k over nodes */
    int64_t skel_col, rest_col, g_col;
    int64_t swaps;              /* Gu-Eisenstat swaps over all nodes and sides */
    int64_t swap_cap_hits;      /* nodes whose swap loop hit its cap */
    int64_t coupling_pairs;     /* sum over (i,j) in L of k_i k_j */
    int64_t near_pairs;         /* sum over (i,j) in L^- of |i| |j| */
    double lo[3], s;            /* bounding cube [lo, lo + s]^dim (of all problems of a batch) */
    double tau, f, tol;
    size_t footprint_bytes;     /* device bytes held by the handle */
    int64_t nproblems;          /* 1, or the problems of smash_build_batch */
} smash_info_t;

SMASH_API smash_status smash_info(smash_handle h, smash_info_t *info);

/*
 * smash_export -- host copies of the representation for inspection and
 * parity tests.  Every pointer is caller-allocated host memory sized from
 * smash_info (NULL skips that array).  Layout (gid = global node id, nodes
 * ordered by level, then Morton order within the level; root gid 0):
 *   permx[nx], permy[ny]  sorted position -> caller index
 *   keyx[nx], keyy[ny]    Morton keys in sorted order
 *   lvl_off[levels+1]     nodes of level l are gids [lvl_off[l-1], lvl_off[l])
 *   level, leaf, parent, child0, nchild [nnodes]; rs, rc, cs, cc [nnodes]
 *                         row/column point ranges in sorted order
 *   cell[nnodes*3]        integer cell coordinates (unused axes 0)
 *   adm_ptr[nnodes+1], adm_col[nadm]     L in CSR by row node, columns ascending
 *   near_ptr[nnodes+1], near_col[nnear]  L^- likewise
 *   m_*, k_*[nnodes]      working-set size |i_bar| and rank |i_hat| per node
 *   skel_*[sum k]         skeleton point indices (sorted positions), per node
 *                         ascending, nodes in gid order
 *   rest_*[sum (m-k)]     the other working-set points, per node ascending
 *   G_*[sum (m-k)k]       per node the (m-k) x k row-major matrix G of (2.11):
 *                         rows follow rest_*, columns follow skel_*
 *   node_problem[nnodes]  problem of each node (0 for a single problem)
 *   problem_cube[nproblems*4]  per problem {lo0, lo1, lo2, s} of its cube
 * (*_col equals *_row when Y = X.  In a batch the roots of the problems are
 * the gids 0 .. nproblems-1, and the nodes of problem t, taken in gid order,
 * are the nodes of that problem built alone.)
 */
typedef struct {
    int64_t *permx, *permy;
    uint64_t *keyx, *keyy;
    int64_t *lvl_off;
    int32_t *level, *leaf, *parent, *child0, *nchild;
    int64_t *rs, *rc, *cs, *cc;
    uint64_t *cell;
    int64_t *adm_ptr;
    int32_t *adm_col;
    int64_t *near_ptr;
    int32_t *near_col;
    int32_t *m_row, *k_row;
    int64_t *skel_row, *rest_row;
    double *G_row;
    int32_t *m_col, *k_col;
    int64_t *skel_col, *rest_col;
    double *G_col;
    int32_t *node_problem;
    double *problem_cube;
} smash_export_t;

SMASH_API smash_status smash_export(smash_handle h, const smash_export_t *out);

/*
 * smash_near_fallback_leaves -- the leaves whose near-field rows (3.20) the
 * SMASH_PREC_F32X2 matvec does not take through the digit-split products but
 * through its double-float kernel: a row of the leaf meets a source at the
 * same coordinates (other than its own point), or its sources span more than
 * 2^12 in distance, so a per-row digit exponent would lose accuracy.  The
 * classification depends on the points only.  Writes up to cap global node
 * ids (ascending) to leaves (host memory) and the total to *count; *count = 0
 * when the handle's matvec has no digit-split near field (kernels other than
 * 1/|x-y| and 1/(x-y)).  Synchronous (runs the classification on the
 * handle's stream).  Errors: SMASH_EINVAL, SMASH_ENOMEM, SMASH_ECUDA.
 */
SMASH_API smash_status smash_near_fallback_leaves(smash_handle h, int32_t *leaves, int64_t cap, int64_t *count);

/* Device bytes held by a handle (0 for NULL). */
SMASH_API size_t smash_footprint_bytes(smash_handle h);

/* Upper estimate of the device bytes smash_build plus one smash_matvec with
 * nrhs right-hand sides need for n uniformly spread points; used for
 * admission before a build. */
SMASH_API size_t smash_predict_footprint(int64_t n, int dim, int leaf_size, int order, int nrhs);

/* The farfield-rank heuristic of Section 6.1 for tolerance eps and ratio tau. */
SMASH_API int smash_suggest_rank(double eps, double tau);

/*
 * Autotuning (an extension of this library; the paper has no counterpart).
 * Launch sites with several valid configurations -- the threads per node CTA
 * of the compression, the source tile and target block of the kernel sums --
 * look their choice up in a process-wide table keyed by the launch shape.
 * With smash_set_autotune(1), a shape without an entry is timed once for
 * every candidate (CUDA events on the launching stream; not while the stream
 * is being captured into a graph) and the fastest is recorded.  All
 * candidates compute the same results: the compression bit for bit, the
 * kernel sums up to the order of their partial sums.  The table is saved to
 * and loaded from a flat JSON file; the environment variable
 * SMASH_AUTOTUNE_CACHE names a file loaded at the first lookup.
 *   smash_autotune_load    returns the entries read, or -1 (file missing or
 *                          malformed; the table is unchanged)
 *   smash_autotune_save    SMASH_EINVAL if the file cannot be written
 *   smash_autotune_lookup  1 and *value if key has an entry, else 0
 *   smash_autotune_force   every site whose key starts with prefix takes
 *                          candidate value (when it is one of the site's
 *                          candidates), before the table and the timing; a
 *                          value < 0 removes the prefix's override.  Keys of
 *                          the double-float coupling start with "coupling_dd/"
 *                          (0 digit products by warp MMAs, 1 all on the FP32
 *                          pipe, 2 digit products by tcgen05.mma); of its near
 *                          field, "near_dd/" (0 digit split, 1 FP32 pipe).
 */
SMASH_API void smash_set_autotune(int on);
SMASH_API int smash_autotune_load(const char *path);
SMASH_API smash_status smash_autotune_save(const char *path);
SMASH_API int smash_autotune_entries(void);
SMASH_API void smash_autotune_clear(void);
SMASH_API int smash_autotune_lookup(const char *key, int *value);
SMASH_API void smash_autotune_force(const char *prefix, int value);

/*
 * smash_measure_fma_peak -- measured arithmetic peak of the current device in
 * TFLOP/s: a launch of independent fused multiply-add chains over every SM
 * (fp64 != 0: FP64, else FP32), best of three CUDA-event-timed runs, 2 flops
 * per FMA.  The paper has no counterpart: it is the denominator of the
 * roofline fractions this library reports for its ALU-bound kernels.
 * Synchronous, ~0.2 s.  Errors: SMASH_EINVAL, SMASH_ECUDA.
 */
SMASH_API smash_status smash_measure_fma_peak(int fp64, double *tflops);

/* Message of the last failed call on this host thread ("" if none). */
SMASH_API const char *smash_last_error(void);

/* Number of kernels this library has launched in this process. */
SMASH_API uint64_t smash_launch_count(void);

/*
 * Phase timing.  With profiling on, smash_build and smash_matvec_ex record
 * CUDA events on the stream they run on around each phase;
 * smash_last_profile copies the durations (ms) of the handle's last build
 * and last matvec into ms[0..n) in this order and returns the count written:
 *   build: 0 geometry (cube, keys, sort)  1 tree  2 lists  3 compression
 *   matvec: 4 gather  5 near field  6 upward  7 coupling  8 downward  9 scatter
 */
SMASH_API void smash_set_profiling(int on);
SMASH_API int smash_last_profile(smash_handle h, double *ms, int n);

#ifdef __cplusplus
}
#endif

#endif /* SMASH_H */
