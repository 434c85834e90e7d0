// compress.cu -- per-level batched node compression of Section 3.3.2:
// interpolation basis (2.2) at Chebyshev anchors of the node cell, then
// compr (2.14) = strong rank-revealing QR of U^_i^T (Theorem 2.4) giving the
// interpolative decomposition U^_i = P_i [I; G_i] U^_i|_i^ of (2.11), then
// the nested working sets (3.18).
//
// One CTA compresses one node at a time (persistent over the level's nodes).
// The r x m matrix W = U^_i^T lives row-major in shared memory when it fits
// and in a per-CTA global slot (L2-resident) otherwise.  Threads own columns
// (= points): every dot product and norm is summed sequentially in the same
// order as the CPU oracle, and the file is compiled with --fmad=false, so the
// pivots, ranks and G of a node are bit-identical to the oracle's whenever
// its inputs are.  All arithmetic is FP64.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace smash {

struct CompressArgs {
    int d, p, r, level;
    double tol, f;
    const double *geo4;       // per problem {lo0, lo1, lo2, s}: the bounding cube
    const int32_t *node_tree; // problem of each node
    double anchors[kMaxP];
    double weights[kMaxP];    // w_m = 1 / prod_{n != m} (t_m - t_n)
    int64_t n0, nl;
    const int32_t *leaf;
    const uint64_t *cell;
    const int64_t *start;
    const int32_t *count;
    const int32_t *child0;
    const int32_t *nchild;
    const double *pts;        // sorted coordinates, stride 4
    const int64_t *skel_gidx; // skeleton slot -> sorted point index (children's working sets)
    int32_t *m;
    int32_t *k;
    int64_t *in_off;
    int64_t *sk_off;
    const int64_t *loc_off;
    const int64_t *g_off;
    int32_t *loc;
    int64_t *skg_tmp;
    double *G;
    int32_t *nswaps;
    double *work;             // per-CTA slots of slot_doubles
    int64_t slot_doubles;
    int64_t x_off;            // R11^{-1} (r x r) at this offset in a slot
    int m_cap;
    int64_t w_smem_doubles;   // W region in shared memory (0: none); a node with
                              // r m above it keeps W in its global slot
    // the Taylor basis (2.4)-(2.5) on C (complex W, G): cl[l] = (l/e)(2 pi r)^(1/(2r))
    double cl[kMaxP];
    // HSS (3.9): extra_rows[g] rows of length m appended below the basis of
    // node g (the truncated-SVD vectors of its nearfield block), stored at
    // extra + (g - n0) * extra_stride; nullptr for H^2.  rcap bounds the rows
    // of W (r for H^2) and sizes v, rho and the R11^{-1} slot.
    const double *extra;
    const int32_t *extra_rows;
    int64_t extra_stride;
    int rcap;
};

// ---------------------------------------------------------------- setup
// m and the input offset of each node of the level: leaves own their point
// range (3.6); a parent's working set is its children's skeletons (3.18),
// which are contiguous skeleton slots starting at the first child's.
__global__ void level_setup_kernel(CompressArgs a) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nl) return;
    int64_t g = a.n0 + i;
    if (a.leaf[g]) {
        a.m[g] = a.count[g];
        a.in_off[g] = a.start[g];
    } else {
        int c0 = a.child0[g], nc = a.nchild[g];
        int s = 0;
        for (int c = 0; c < nc; ++c) s += a.k[c0 + c];
        a.m[g] = s;
        a.in_off[g] = a.sk_off[c0];
    }
}

// ---------------------------------------------------------------- helpers
template <int NT>
struct Smem {
    double *nrm2;   // m_cap
    double *v;      // r
    double *rho;    // r
    double *rval;   // NT/32
    int64_t *ridx;  // NT/32
    double *ctrl;   // 8
    int *perm;      // m_cap
    int *ex;        // m_cap
    int *chunk;     // NT
    double *W;      // r * m_cap when in shared memory
};

// a before b: larger value, ties to the lower index.  The values compared are
// non-negative finite doubles (squared norms, the swap test) or the sentinel
// -1, whose bit patterns order as signed 64-bit integers exactly as the values
// do (no -0 arises: every value is a sum of squares starting at +0), so the
// test runs on the integer pipe rather than GB300's narrow FP64 pipe.
__device__ __forceinline__ bool better(double a, int64_t ia, double b, int64_t ib) {
    const long long ka = __double_as_longlong(a), kb = __double_as_longlong(b);
    return ka > kb || (ka == kb && ia < ib);
}

// block-wide maximum of (value, index), ties to the lowest index
template <int NT>
__device__ void block_argmax(double v, int64_t idx, Smem<NT> &sh, double &ov, int64_t &oi) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int64_t i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (better(v2, i2, v, idx)) { v = v2; idx = i2; }
    }
    if (lane == 0) { sh.rval[w] = v; sh.ridx[w] = idx; }
    __syncthreads();
    if (w == 0) {
        v = lane < NT / 32 ? sh.rval[lane] : -1.0;
        idx = lane < NT / 32 ? sh.ridx[lane] : INT64_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double v2 = __shfl_xor_sync(0xffffffffu, v, o);
            int64_t i2 = __shfl_xor_sync(0xffffffffu, idx, o);
            if (better(v2, i2, v, idx)) { v = v2; idx = i2; }
        }
        if (lane == 0) { sh.rval[0] = v; sh.ridx[0] = idx; }
    }
    __syncthreads();
    ov = sh.rval[0];
    oi = sh.ridx[0];
    __syncthreads();
}

// ell_m(t) = prod_{n != m} (t - t_n) / (t_m - t_n) = w_m prod_{n != m} (t - t_n)
__device__ __forceinline__ double lagrange(int p, const double *anch, const double *w, int m, double t) {
    double v = w[m];
    for (int n = 0; n < p; ++n)
        if (n != m) v = v * (t - anch[n]);
    return v;
}

// column c of W = U^^T for the point at sorted index gid, in the cell of node g
template <int PMAX>
__device__ void basis_column(const CompressArgs &a, int64_t g, int64_t gid, double *W, int ld, int c) {
    const double *cube = a.geo4 + (int64_t)a.node_tree[g] * 4;
    double h = ldexp(cube[3], 1 - a.level);
    double half = 0.5 * h;
    double L[3][PMAX];
    for (int ax = 0; ax < a.d; ++ax) {
        double centre = cube[ax] + ((double)a.cell[g * 3 + ax] + 0.5) * h;
        double t = (a.pts[gid * 4 + ax] - centre) / half;
        for (int mm = 0; mm < a.p; ++mm) L[ax][mm] = lagrange(a.p, a.anchors, a.weights, mm, t);
    }
    for (int kk = 0; kk < a.r; ++kk) {
        int rem = kk, idx[3] = {0, 0, 0};
        for (int ax = a.d - 1; ax >= 0; --ax) { idx[ax] = rem % a.p; rem /= a.p; }
        double v = L[0][idx[0]];
        for (int ax = 1; ax < a.d; ++ax) v = v * L[ax][idx[ax]];
        W[(int64_t)kk * ld + c] = v;
    }
}

__device__ __forceinline__ int64_t working_gid(const CompressArgs &a, int64_t g, int pos) {
    return a.leaf[g] ? a.start[g] + pos : a.skel_gidx[a.in_off[g] + pos];
}

// Householder QR of W (r x m, row-major, leading dimension ld).  With pivot:
// largest remaining column norm (ties: lowest position), stop before step j
// when |R_jj| <= tol |R_00|; returns the number of steps.  Without pivot:
// exactly ksteps steps in the current column order.  Sums run over the rows
// in ascending order with fused multiply-adds; rows are loaded in chunks of
// kChunk so that several loads of a column are in flight.
constexpr int kChunk = 8;

template <int NT>
__device__ int qr_steps(double *W, int ld, int r, int m, Smem<NT> &sh, bool pivot, int ksteps, double tol) {
    const int tid = threadIdx.x;
    int kmax = pivot ? min(r, m) : ksteps;
    if (pivot) {
        for (int c = tid; c < m; c += NT) {
            double s2 = 0.0;
            for (int i0 = 0; i0 < r; i0 += kChunk) {
                double x[kChunk];
#pragma unroll
                for (int u = 0; u < kChunk; ++u) x[u] = i0 + u < r ? W[(int64_t)(i0 + u) * ld + c] : 0.0;
#pragma unroll
                for (int u = 0; u < kChunk; ++u)
                    if (i0 + u < r) s2 = __fma_rn(x[u], x[u], s2);
            }
            sh.nrm2[c] = s2;
        }
        __syncthreads();
    }
    double r00 = 0.0;
    for (int j = 0; j < kmax; ++j) {
        if (pivot) {
            double best = -1.0;
            int64_t bi = INT64_MAX;
            for (int c = j + tid; c < m; c += NT)
                if (better(sh.nrm2[c], c, best, bi)) { best = sh.nrm2[c]; bi = c; }
            double val;
            int64_t piv;
            block_argmax<NT>(best, bi, sh, val, piv);
            double nrm = sqrt(val);
            if (j == 0) {
                r00 = nrm;
                if (nrm == 0.0) return 0;
            } else if (nrm <= tol * r00) {
                return j;
            }
            if (piv != j) {
                for (int i = tid; i < r; i += NT) {
                    double t = W[(int64_t)i * ld + j];
                    W[(int64_t)i * ld + j] = W[(int64_t)i * ld + piv];
                    W[(int64_t)i * ld + piv] = t;
                }
                if (tid == 0) {
                    int tp = sh.perm[j];
                    sh.perm[j] = sh.perm[piv];
                    sh.perm[piv] = tp;
                }
                __syncthreads();
            }
        }
        if (tid == 0) {
            double alpha = W[(int64_t)j * ld + j];
            double sigma = 0.0;
            for (int i = j + 1; i < r; ++i) {
                double x = W[(int64_t)i * ld + j];
                sigma = __fma_rn(x, x, sigma);
            }
            if (sigma == 0.0) {
                sh.ctrl[0] = 1.0;  // skip: the column is already reduced
            } else {
                double nrm = sqrt(__fma_rn(alpha, alpha, sigma));
                double beta = alpha <= 0.0 ? nrm : -nrm;
                sh.ctrl[0] = 0.0;
                sh.ctrl[1] = (beta - alpha) / beta;  // tau
                sh.ctrl[2] = alpha - beta;           // divisor of v
                sh.ctrl[3] = beta;
            }
        }
        __syncthreads();
        const bool skip = sh.ctrl[0] != 0.0;
        const double tau = sh.ctrl[1], den = sh.ctrl[2], beta = sh.ctrl[3];
        if (!skip) {
            for (int i = j + 1 + tid; i < r; i += NT) sh.v[i] = W[(int64_t)i * ld + j] / den;
            __syncthreads();
        }
        for (int c = j + 1 + tid; c < m; c += NT) {
            double s2 = 0.0;
            if (!skip) {
                double w = W[(int64_t)j * ld + c];
                for (int i0 = j + 1; i0 < r; i0 += kChunk) {
                    double x[kChunk];
#pragma unroll
                    for (int u = 0; u < kChunk; ++u) x[u] = i0 + u < r ? W[(int64_t)(i0 + u) * ld + c] : 0.0;
#pragma unroll
                    for (int u = 0; u < kChunk; ++u)
                        if (i0 + u < r) w = __fma_rn(sh.v[i0 + u], x[u], w);
                }
                double tw = tau * w;
                W[(int64_t)j * ld + c] = W[(int64_t)j * ld + c] - tw;
                for (int i0 = j + 1; i0 < r; i0 += kChunk) {
                    double x[kChunk];
#pragma unroll
                    for (int u = 0; u < kChunk; ++u) x[u] = i0 + u < r ? W[(int64_t)(i0 + u) * ld + c] : 0.0;
#pragma unroll
                    for (int u = 0; u < kChunk; ++u)
                        if (i0 + u < r) {
                            double y = __fma_rn(-tw, sh.v[i0 + u], x[u]);
                            W[(int64_t)(i0 + u) * ld + c] = y;
                            s2 = __fma_rn(y, y, s2);
                        }
                }
            } else {
                for (int i0 = j + 1; i0 < r; i0 += kChunk) {
                    double x[kChunk];
#pragma unroll
                    for (int u = 0; u < kChunk; ++u) x[u] = i0 + u < r ? W[(int64_t)(i0 + u) * ld + c] : 0.0;
#pragma unroll
                    for (int u = 0; u < kChunk; ++u)
                        if (i0 + u < r) s2 = __fma_rn(x[u], x[u], s2);
                }
            }
            if (pivot) sh.nrm2[c] = s2;
        }
        __syncthreads();
        if (!skip) {
            if (tid == 0) W[(int64_t)j * ld + j] = beta;
            for (int i = j + 1 + tid; i < r; i += NT) W[(int64_t)i * ld + j] = 0.0;
        }
        __syncthreads();
    }
    return kmax;
}

// exclusive prefix of flag[0..m) into ex[0..m)
template <int NT>
__device__ void block_scan_flags(Smem<NT> &sh, int m) {
    const int tid = threadIdx.x;
    int per = (m + NT - 1) / NT;
    int b0 = tid * per, b1 = min(m, b0 + per);
    int cnt = 0;
    for (int i = b0; i < b1; ++i) cnt += sh.ex[i];
    sh.chunk[tid] = cnt;
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int t = 0; t < NT; ++t) { int c = sh.chunk[t]; sh.chunk[t] = run; run += c; }
    }
    __syncthreads();
    int run = sh.chunk[tid];
    for (int i = b0; i < b1; ++i) { int f = sh.ex[i]; sh.ex[i] = run; run += f; }
    __syncthreads();
}

template <int NT, int PMAX>
__global__ void __launch_bounds__(NT) compress_kernel(CompressArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem<NT> sh;
    {
        double *dp = reinterpret_cast<double *>(smraw);
        sh.nrm2 = dp; dp += a.m_cap;
        sh.v = dp; dp += a.rcap;
        sh.rho = dp; dp += a.rcap;
        sh.rval = dp; dp += NT / 32;
        sh.ctrl = dp; dp += 8;
        sh.ridx = reinterpret_cast<int64_t *>(dp); dp += NT / 32;
        sh.W = a.w_smem_doubles ? dp : nullptr;
        dp += a.w_smem_doubles;
        int *ip = reinterpret_cast<int *>(dp);
        sh.perm = ip; ip += a.m_cap;
        sh.ex = ip; ip += a.m_cap;
        sh.chunk = ip;
    }
    const int tid = threadIdx.x;
    double *slot = a.work + (int64_t)blockIdx.x * a.slot_doubles;
    double *X = slot + a.x_off;  // R11^{-1}, k x k
    const int r = a.r;

    for (int64_t ni = blockIdx.x; ni < a.nl; ni += gridDim.x) {
        const int64_t g = a.n0 + ni;
        const int m = a.m[g];
        if (m == 0) {
            if (tid == 0) { a.k[g] = 0; a.nswaps[g] = 0; }
            continue;
        }
        const int ld = m;
        // rows of W: the basis, then (HSS) the nearfield singular vectors
        const int rr = r + (a.extra ? a.extra_rows[g] : 0);
        const double *ex = a.extra ? a.extra + (g - a.n0) * a.extra_stride : nullptr;
        double *W = (int64_t)rr * m <= a.w_smem_doubles ? sh.W : slot;
        // 1. W = U^^T (and [U^, S]^T)
        for (int c = tid; c < m; c += NT) {
            basis_column<PMAX>(a, g, working_gid(a, g, c), W, ld, c);
            for (int t = r; t < rr; ++t) W[(int64_t)t * ld + c] = ex[(int64_t)(t - r) * m + c];
            sh.perm[c] = c;
        }
        __syncthreads();
        // 2. column-pivoted QR with the rank cut
        int k = qr_steps<NT>(W, ld, rr, m, sh, true, 0, a.tol);
        // 3. Gu-Eisenstat swaps until max (A_ij^2 + gamma_j^2 / omega_i^2) <= f^2
        int nsw = 0;
        for (;;) {
            if (k == 0 || k == m) break;
            const int mk = m - k;
            // the mk columns of R11^{-1} R12 and the k columns of X = R11^{-1},
            // one triangular solve per thread (one loop, so that no thread
            // takes two while others idle)
            for (int e = tid; e < mk + k; e += NT) {
                if (e < mk) {
                    const int u = e;
                    for (int t = k - 1; t >= 0; --t) {
                        double s = W[(int64_t)t * ld + k + u];
                        for (int q = t + 1; q < k; ++q)
                            s = __fma_rn(-W[(int64_t)t * ld + q], W[(int64_t)q * ld + k + u], s);
                        W[(int64_t)t * ld + k + u] = s / W[(int64_t)t * ld + t];
                    }
                } else {
                    const int c = e - mk;
                    for (int t = k - 1; t >= 0; --t) {
                        double s = (t == c) ? 1.0 : 0.0;
                        for (int q = t + 1; q < k; ++q)
                            s = __fma_rn(-W[(int64_t)t * ld + q], X[(int64_t)q * k + c], s);
                        X[(int64_t)t * k + c] = s / W[(int64_t)t * ld + t];
                    }
                }
            }
            __syncthreads();
            // rho_t (row norms of X) and gamma_u^2 (norms of the rest of the
            // columns of R22), again one per thread
            for (int e = tid; e < k + mk; e += NT) {
                double s = 0.0;
                if (e < k) {
                    for (int c = 0; c < k; ++c) {
                        double x = X[(int64_t)e * k + c];
                        s = __fma_rn(x, x, s);
                    }
                    sh.rho[e] = s;
                } else {
                    const int u = e - k;
                    for (int i = k; i < rr; ++i) {
                        double x = W[(int64_t)i * ld + k + u];
                        s = __fma_rn(x, x, s);
                    }
                    sh.nrm2[u] = s;  // gamma_u^2
                }
            }
            __syncthreads();
            double best = -1.0;
            int64_t bi = INT64_MAX;
            const int64_t tot = (int64_t)k * mk;
            for (int64_t e = tid; e < tot; e += NT) {
                int t = (int)(e / mk), u = (int)(e % mk);
                double av = W[(int64_t)t * ld + k + u];
                double val = __fma_rn(av, av, sh.nrm2[u] * sh.rho[t]);
                if (better(val, e, best, bi)) { best = val; bi = e; }
            }
            double bv;
            int64_t be;
            block_argmax<NT>(best, bi, sh, bv, be);
            if (bv <= a.f * a.f) break;
            if (nsw >= kMaxSwaps) { nsw = -1; break; }
            if (tid == 0) {
                int bt = (int)(be / mk), bu = (int)(be % mk);
                int tp = sh.perm[bt];
                sh.perm[bt] = sh.perm[k + bu];
                sh.perm[k + bu] = tp;
            }
            ++nsw;
            __syncthreads();
            for (int c = tid; c < m; c += NT) {
                basis_column<PMAX>(a, g, working_gid(a, g, sh.perm[c]), W, ld, c);
                for (int t = r; t < rr; ++t) W[(int64_t)t * ld + c] = ex[(int64_t)(t - r) * m + sh.perm[c]];
            }
            __syncthreads();
            qr_steps<NT>(W, ld, rr, m, sh, false, k, a.tol);
        }
        // 4. canonical form: skeleton and rest in ascending working-set order
        const int mk = m - k;
        for (int pos = tid; pos < m; pos += NT) sh.ex[pos] = 0;
        __syncthreads();
        for (int t = tid; t < k; t += NT) sh.ex[sh.perm[t]] = 1;
        __syncthreads();
        block_scan_flags<NT>(sh, m);
        const int64_t lo = a.loc_off[g];
        for (int t = tid; t < k; t += NT) {
            int pos = sh.perm[t];
            int tp = sh.ex[pos];
            a.loc[lo + tp] = pos;
            a.skg_tmp[lo + tp] = working_gid(a, g, pos);
        }
        for (int u = tid; u < mk; u += NT) {
            int pos = sh.perm[k + u];
            a.loc[lo + k + (pos - sh.ex[pos])] = pos;
        }
        const int64_t go = a.g_off[g];
        for (int64_t e = tid; e < (int64_t)k * mk; e += NT) {
            int t = (int)(e / mk), u = (int)(e % mk);
            int tp = sh.ex[sh.perm[t]];
            int pu = sh.perm[k + u];
            int up = pu - sh.ex[pu];
            a.G[go + (int64_t)up * k + tp] = W[(int64_t)t * ld + k + u];
        }
        if (tid == 0) { a.k[g] = k; a.nswaps[g] = nsw; }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- Taylor basis on C
// compr (2.14) of the complex basis phi_{a,l}(x - a) = eta_{a,l} (x - a)^l / l!
// of (2.5), l < r, at the cell centre a and radius delta = half the cell
// diagonal: complex Householder QR with column pivoting (reflectors in
// LAPACK's convention, real R_jj), the rank cut and the Gu-Eisenstat swaps,
// then the canonical skeleton order and the complex G ((m-k) x k,
// interleaved).  Every product, sum and division is written out in real
// arithmetic in the same order as the CPU oracle's complex path, so with
// --fmad=false the pivots, ranks and G are the oracle's bits.  W (r x m) and
// R11^{-1} live in the CTA's global slot (L2-resident).
struct Cx { double re, im; };

__device__ __forceinline__ Cx cx_mul(Cx a, Cx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Cx cx_mulc(Cx a, Cx b) { return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im}; }
__device__ __forceinline__ Cx cx_div(Cx a, Cx b) {
    double den = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}

// column c of the complex W for the point at sorted index gid
__device__ void taylor_column(const CompressArgs &a, int64_t g, int64_t gid, Cx *W, int ld, int c) {
    const double *cube = a.geo4 + (int64_t)a.node_tree[g] * 4;
    double h = ldexp(cube[3], 1 - a.level);
    double are = cube[0] + ((double)a.cell[g * 3 + 0] + 0.5) * h;
    double aim = cube[1] + ((double)a.cell[g * 3 + 1] + 0.5) * h;
    double delta = 0.5 * h * sqrt(2.0);
    Cx u = {(a.pts[gid * 4 + 0] - are) / delta, (a.pts[gid * 4 + 1] - aim) / delta};
    for (int l = 0; l < a.r; ++l) {
        Cx w = {a.cl[l] * u.re, a.cl[l] * u.im};
        Cx v = {1.0, 0.0};
        for (int j = 1; j <= l; ++j) {
            v = cx_mul(v, w);
            v.re = v.re / (double)j;
            v.im = v.im / (double)j;
        }
        W[(int64_t)l * ld + c] = v;
    }
}

template <int NT>
__device__ int qr_steps_c(Cx *W, int ld, int r, int m, Smem<NT> &sh, Cx *vv, bool pivot, int ksteps, double tol) {
    const int tid = threadIdx.x;
    int kmax = pivot ? min(r, m) : ksteps;
    if (pivot) {
        for (int c = tid; c < m; c += NT) {
            double s2 = 0.0;
            for (int i = 0; i < r; ++i) {
                Cx x = W[(int64_t)i * ld + c];
                s2 = __fma_rn(x.re, x.re, s2);
                s2 = __fma_rn(x.im, x.im, s2);
            }
            sh.nrm2[c] = s2;
        }
        __syncthreads();
    }
    double r00 = 0.0;
    for (int j = 0; j < kmax; ++j) {
        if (pivot) {
            double best = -1.0;
            int64_t bi = INT64_MAX;
            for (int c = j + tid; c < m; c += NT)
                if (better(sh.nrm2[c], c, best, bi)) { best = sh.nrm2[c]; bi = c; }
            double val;
            int64_t piv;
            block_argmax<NT>(best, bi, sh, val, piv);
            double nrm = sqrt(val);
            if (j == 0) {
                r00 = nrm;
                if (nrm == 0.0) return 0;
            } else if (nrm <= tol * r00) {
                return j;
            }
            if (piv != j) {
                for (int i = tid; i < r; i += NT) {
                    Cx t = W[(int64_t)i * ld + j];
                    W[(int64_t)i * ld + j] = W[(int64_t)i * ld + piv];
                    W[(int64_t)i * ld + piv] = t;
                }
                if (tid == 0) {
                    int tp = sh.perm[j];
                    sh.perm[j] = sh.perm[piv];
                    sh.perm[piv] = tp;
                }
                __syncthreads();
            }
        }
        if (tid == 0) {
            Cx alpha = W[(int64_t)j * ld + j];
            double sigma = 0.0;
            for (int i = j + 1; i < r; ++i) {
                Cx x = W[(int64_t)i * ld + j];
                sigma = __fma_rn(x.re, x.re, sigma);
                sigma = __fma_rn(x.im, x.im, sigma);
            }
            if (sigma == 0.0 && alpha.im == 0.0) {
                sh.ctrl[0] = 1.0;  // skip: already triangular with a real diagonal entry
            } else {
                double nrm = sqrt(__fma_rn(alpha.re, alpha.re, __fma_rn(alpha.im, alpha.im, sigma)));
                double beta = alpha.re <= 0.0 ? nrm : -nrm;
                sh.ctrl[0] = 0.0;
                sh.ctrl[1] = (beta - alpha.re) / beta;  // tau
                sh.ctrl[2] = -alpha.im / beta;
                sh.ctrl[3] = alpha.re - beta;           // divisor of v
                sh.ctrl[4] = alpha.im;
                sh.ctrl[5] = beta;
            }
        }
        __syncthreads();
        const bool skip = sh.ctrl[0] != 0.0;
        const Cx tau = {sh.ctrl[1], sh.ctrl[2]}, den = {sh.ctrl[3], sh.ctrl[4]};
        const double beta = sh.ctrl[5];
        if (!skip) {
            for (int i = j + 1 + tid; i < r; i += NT) vv[i] = cx_div(W[(int64_t)i * ld + j], den);
            __syncthreads();
        }
        for (int c = j + 1 + tid; c < m; c += NT) {
            double s2 = 0.0;
            if (!skip) {
                Cx w = W[(int64_t)j * ld + c];
                for (int i = j + 1; i < r; ++i) {
                    Cx x = W[(int64_t)i * ld + c];
                    const Cx v = vv[i];
                    w.re = __fma_rn(v.re, x.re, __fma_rn(v.im, x.im, w.re));
                    w.im = __fma_rn(v.re, x.im, __fma_rn(-v.im, x.re, w.im));
                }
                Cx tw = cx_mulc(w, tau);
                W[(int64_t)j * ld + c].re = W[(int64_t)j * ld + c].re - tw.re;
                W[(int64_t)j * ld + c].im = W[(int64_t)j * ld + c].im - tw.im;
                for (int i = j + 1; i < r; ++i) {
                    Cx y = cx_mul(tw, vv[i]);
                    Cx x = W[(int64_t)i * ld + c];
                    x.re = x.re - y.re;
                    x.im = x.im - y.im;
                    W[(int64_t)i * ld + c] = x;
                    s2 = __fma_rn(x.re, x.re, s2);
                    s2 = __fma_rn(x.im, x.im, s2);
                }
            } else {
                for (int i = j + 1; i < r; ++i) {
                    Cx x = W[(int64_t)i * ld + c];
                    s2 = __fma_rn(x.re, x.re, s2);
                    s2 = __fma_rn(x.im, x.im, s2);
                }
            }
            if (pivot) sh.nrm2[c] = s2;
        }
        __syncthreads();
        if (!skip) {
            if (tid == 0) W[(int64_t)j * ld + j] = {beta, 0.0};
            for (int i = j + 1 + tid; i < r; i += NT) W[(int64_t)i * ld + j] = {0.0, 0.0};
        }
        __syncthreads();
    }
    return kmax;
}

template <int NT>
__global__ void __launch_bounds__(NT) compress_taylor_kernel(CompressArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem<NT> sh;
    Cx *vv;
    {
        double *dp = reinterpret_cast<double *>(smraw);
        sh.nrm2 = dp; dp += a.m_cap;
        sh.v = dp; dp += a.r;
        sh.rho = dp; dp += a.r;
        sh.rval = dp; dp += NT / 32;
        sh.ctrl = dp; dp += 8;
        sh.ridx = reinterpret_cast<int64_t *>(dp); dp += NT / 32;
        vv = reinterpret_cast<Cx *>(dp); dp += 2 * a.r;
        sh.W = nullptr;
        int *ip = reinterpret_cast<int *>(dp);
        sh.perm = ip; ip += a.m_cap;
        sh.ex = ip; ip += a.m_cap;
        sh.chunk = ip;
    }
    const int tid = threadIdx.x;
    Cx *W = reinterpret_cast<Cx *>(a.work + (int64_t)blockIdx.x * a.slot_doubles);
    Cx *X = W + a.x_off;  // R11^{-1}, k x k
    const int r = a.r;

    for (int64_t ni = blockIdx.x; ni < a.nl; ni += gridDim.x) {
        const int64_t g = a.n0 + ni;
        const int m = a.m[g];
        if (m == 0) {
            if (tid == 0) { a.k[g] = 0; a.nswaps[g] = 0; }
            continue;
        }
        const int ld = m;
        for (int c = tid; c < m; c += NT) {
            taylor_column(a, g, working_gid(a, g, c), W, ld, c);
            sh.perm[c] = c;
        }
        __syncthreads();
        int k = qr_steps_c<NT>(W, ld, r, m, sh, vv, true, 0, a.tol);
        int nsw = 0;
        for (;;) {
            if (k == 0 || k == m) break;
            const int mk = m - k;
            // A = R11^{-1} R12 in place of R12 (rows from the last up)
            for (int u = tid; u < mk; u += NT)
                for (int t = k - 1; t >= 0; --t) {
                    Cx sacc = W[(int64_t)t * ld + k + u];
                    for (int q = t + 1; q < k; ++q) {
                        Cx y = cx_mul(W[(int64_t)t * ld + q], W[(int64_t)q * ld + k + u]);
                        sacc.re = sacc.re - y.re;
                        sacc.im = sacc.im - y.im;
                    }
                    W[(int64_t)t * ld + k + u] = cx_div(sacc, W[(int64_t)t * ld + t]);
                }
            for (int c = tid; c < k; c += NT)
                for (int t = k - 1; t >= 0; --t) {
                    Cx sacc = {(t == c) ? 1.0 : 0.0, 0.0};
                    for (int q = t + 1; q < k; ++q) {
                        Cx y = cx_mul(W[(int64_t)t * ld + q], X[(int64_t)q * k + c]);
                        sacc.re = sacc.re - y.re;
                        sacc.im = sacc.im - y.im;
                    }
                    X[(int64_t)t * k + c] = cx_div(sacc, W[(int64_t)t * ld + t]);
                }
            __syncthreads();
            for (int t = tid; t < k; t += NT) {
                double sacc = 0.0;
                for (int c = 0; c < k; ++c) {
                    sacc = __fma_rn(X[(int64_t)t * k + c].re, X[(int64_t)t * k + c].re, sacc);
                    sacc = __fma_rn(X[(int64_t)t * k + c].im, X[(int64_t)t * k + c].im, sacc);
                }
                sh.rho[t] = sacc;
            }
            for (int u = tid; u < mk; u += NT) {
                double sacc = 0.0;
                for (int i = k; i < r; ++i) {
                    sacc = __fma_rn(W[(int64_t)i * ld + k + u].re, W[(int64_t)i * ld + k + u].re, sacc);
                    sacc = __fma_rn(W[(int64_t)i * ld + k + u].im, W[(int64_t)i * ld + k + u].im, sacc);
                }
                sh.nrm2[u] = sacc;  // gamma_u^2
            }
            __syncthreads();
            double best = -1.0;
            int64_t bi = INT64_MAX;
            const int64_t tot = (int64_t)k * mk;
            for (int64_t e = tid; e < tot; e += NT) {
                int t = (int)(e / mk), u = (int)(e % mk);
                Cx av = W[(int64_t)t * ld + k + u];
                double val = __fma_rn(av.re, av.re, __fma_rn(av.im, av.im, sh.nrm2[u] * sh.rho[t]));
                if (better(val, e, best, bi)) { best = val; bi = e; }
            }
            double bv;
            int64_t be;
            block_argmax<NT>(best, bi, sh, bv, be);
            if (bv <= a.f * a.f) break;
            if (nsw >= kMaxSwaps) { nsw = -1; break; }
            if (tid == 0) {
                int bt = (int)(be / mk), bu = (int)(be % mk);
                int tp = sh.perm[bt];
                sh.perm[bt] = sh.perm[k + bu];
                sh.perm[k + bu] = tp;
            }
            ++nsw;
            __syncthreads();
            for (int c = tid; c < m; c += NT) taylor_column(a, g, working_gid(a, g, sh.perm[c]), W, ld, c);
            __syncthreads();
            qr_steps_c<NT>(W, ld, r, m, sh, vv, false, k, a.tol);
        }
        // canonical form: skeleton and rest in ascending working-set order
        const int mk = m - k;
        for (int pos = tid; pos < m; pos += NT) sh.ex[pos] = 0;
        __syncthreads();
        for (int t = tid; t < k; t += NT) sh.ex[sh.perm[t]] = 1;
        __syncthreads();
        block_scan_flags<NT>(sh, m);
        const int64_t lo = a.loc_off[g];
        for (int t = tid; t < k; t += NT) {
            int pos = sh.perm[t];
            int tp = sh.ex[pos];
            a.loc[lo + tp] = pos;
            a.skg_tmp[lo + tp] = working_gid(a, g, pos);
        }
        for (int u = tid; u < mk; u += NT) {
            int pos = sh.perm[k + u];
            a.loc[lo + k + (pos - sh.ex[pos])] = pos;
        }
        const int64_t go = a.g_off[g];
        Cx *Gc = reinterpret_cast<Cx *>(a.G);
        for (int64_t e = tid; e < (int64_t)k * mk; e += NT) {
            int t = (int)(e / mk), u = (int)(e % mk);
            int tp = sh.ex[sh.perm[t]];
            int pu = sh.perm[k + u];
            int up = pu - sh.ex[pu];
            Gc[go + (int64_t)up * k + tp] = W[(int64_t)t * ld + k + u];
        }
        if (tid == 0) { a.k[g] = k; a.nswaps[g] = nsw; }
        __syncthreads();
    }
}

// skeleton slots of the level, compacted in node order
__global__ void compact_skeleton_kernel(int64_t n0, int64_t nl, const int32_t *__restrict__ k,
                                        const int64_t *__restrict__ sk_off, const int64_t *__restrict__ loc_off,
                                        const int64_t *__restrict__ skg_tmp, const double *__restrict__ pts,
                                        int64_t *__restrict__ skel_gidx, double *__restrict__ skel_xyz) {
    int64_t g = n0 + blockIdx.x;
    int kk = k[g];
    for (int t = threadIdx.x; t < kk; t += blockDim.x) {
        int64_t gid = skg_tmp[loc_off[g] + t];
        int64_t slot = sk_off[g] + t;
        skel_gidx[slot] = gid;
        reinterpret_cast<P4 *>(skel_xyz)[slot] = reinterpret_cast<const P4 *>(pts)[gid];
    }
}

// upper bounds: k <= min(r, count), m <= leaf ? count : sum_children min(r, count_c),
// |G| <= max_{k <= min(r,m)} (m - k) k
__global__ void bounds_kernel(int64_t nn, int r, const int32_t *__restrict__ level,
                              const int32_t *__restrict__ leaf, const int32_t *__restrict__ cnt,
                              const int32_t *__restrict__ child0, const int32_t *__restrict__ nchild,
                              int64_t *__restrict__ kub, int64_t *__restrict__ mub, int64_t *__restrict__ gub) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nn) return;
    int64_t m;
    const bool root = level[g] == 1;
    if (root) {
        m = 0;  // a root is never compressed
    } else if (leaf[g]) {
        m = cnt[g];
    } else {
        m = 0;
        for (int c = 0; c < nchild[g]; ++c) m += min((int64_t)r, (int64_t)cnt[child0[g] + c]);
    }
    int64_t kmax = min((int64_t)r, m);
    int64_t kh = m / 2;
    int64_t kb = kh <= kmax ? kh : kmax;
    int64_t gb = (m - kb) * kb;
    if (kh + 1 <= kmax) gb = max(gb, (m - kh - 1) * (kh + 1));
    kub[g] = root ? 0 : min((int64_t)r, (int64_t)cnt[g]);
    mub[g] = m;
    gub[g] = gb;
}

static void compress_side(smash_h2 *h, Side &S, bool rows, Arena &scratch) {
    cudaStream_t st = h->stream;
    const int64_t nn = h->nnodes;
    const int32_t *cnt = rows ? h->rc : h->cc;
    const int64_t *start = rows ? h->rs : h->cs;
    const double *pts = rows ? h->xs : h->ys;
    S.m = h->mem.alloc<int32_t>(nn);
    S.k = h->mem.alloc<int32_t>(nn);
    S.in_off = h->mem.alloc<int64_t>(nn);
    S.sk_off = h->mem.alloc<int64_t>(nn);
    S.loc_off = h->mem.alloc<int64_t>(nn + 1);
    S.g_off = h->mem.alloc<int64_t>(nn + 1);
    S.nswaps = h->mem.alloc<int32_t>(nn);
    CK(cudaMemsetAsync(S.m, 0, nn * 4, st));
    CK(cudaMemsetAsync(S.k, 0, nn * 4, st));
    CK(cudaMemsetAsync(S.nswaps, 0, nn * 4, st));
    CK(cudaMemsetAsync(S.sk_off, 0, nn * 8, st));
    CK(cudaMemsetAsync(S.in_off, 0, nn * 8, st));
    int64_t *kub = scratch.alloc<int64_t>(nn), *mub = scratch.alloc<int64_t>(nn), *gub = scratch.alloc<int64_t>(nn);
    int64_t *tot = scratch.alloc<int64_t>(4);
    bounds_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(nn, h->r, h->level, h->leaf, cnt, h->child0, h->nchild, kub,
                                                                 mub, gub);
    LAUNCHED();
    int64_t *kub_off = scratch.alloc<int64_t>(nn);
    exclusive_scan<int64_t>(kub, kub_off, nn, nullptr, tot + 0, st, scratch);
    exclusive_scan<int64_t>(mub, S.loc_off, nn, nullptr, tot + 1, st, scratch);
    exclusive_scan<int64_t>(gub, S.g_off, nn, nullptr, tot + 2, st, scratch);
    // per-level maximum of the m bound
    std::vector<int64_t> lmax(h->L + 1, 0);
    int64_t *lm = scratch.alloc<int64_t>(h->L + 1);
    for (int l = 2; l <= h->L; ++l) {
        int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        reduce_max(mub + n0, nl, lm + l, st);
    }
    int64_t ht[3];
    CK(cudaMemcpyAsync(ht, tot, 3 * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(lmax.data(), lm, (h->L + 1) * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    S.skel_cap = std::max<int64_t>(ht[0], 1);
    S.total_loc = ht[1];
    S.total_g = ht[2];
    S.mub_max = lmax;
    S.loc = h->mem.alloc<int32_t>(std::max<int64_t>(S.total_loc, 1));
    S.skg_tmp = scratch.alloc<int64_t>(std::max<int64_t>(S.total_loc, 1));
    // complex G (Taylor basis): two doubles per entry
    S.G = h->mem.alloc<double>(std::max<int64_t>(S.total_g, 1) * (h->taylor ? 2 : 1));
    S.skel_gidx = h->mem.alloc<int64_t>(S.skel_cap);
    S.skel_xyz = h->mem.alloc<double>(S.skel_cap * 4);
    int64_t *base = tot + 3;
    CK(cudaMemsetAsync(base, 0, 8, st));

    // one persistent launch per level, deepest first
    double *work = nullptr;
    int64_t work_cap = 0;
    double weights[kMaxP] = {0};
    for (int m = 0; m < h->order; ++m) {
        double den = 1.0;
        for (int n = 0; n < h->order; ++n)
            if (n != m) den = den * (h->anchors[m] - h->anchors[n]);
        weights[m] = 1.0 / den;
    }
    for (int l = h->L; l >= 2; --l) {
        int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        int m_cap = (int)std::max<int64_t>(lmax[l], 1);
        CompressArgs a;
        a.d = h->dim; a.p = h->order; a.r = h->r; a.level = l;
        a.tol = h->tol; a.f = h->f;
        a.geo4 = h->tree_geo; a.node_tree = h->node_tree;
        for (int i = 0; i < kMaxP; ++i) {
            a.anchors[i] = i < h->order ? h->anchors[i] : 0.0;
            a.weights[i] = i < h->order ? weights[i] : 0.0;
        }
        a.n0 = n0; a.nl = nl;
        a.leaf = h->leaf; a.cell = h->cell; a.start = start; a.count = cnt;
        a.child0 = h->child0; a.nchild = h->nchild; a.pts = pts; a.skel_gidx = S.skel_gidx;
        a.m = S.m; a.k = S.k; a.in_off = S.in_off; a.sk_off = S.sk_off; a.loc_off = S.loc_off;
        a.g_off = S.g_off; a.loc = S.loc; a.skg_tmp = S.skg_tmp; a.G = S.G; a.nswaps = S.nswaps;
        a.m_cap = m_cap;
        for (int i = 0; i < kMaxP; ++i) a.cl[i] = i < h->r && h->taylor ? h->taylor_cl[i] : 0.0;
        a.extra = nullptr; a.extra_rows = nullptr; a.extra_stride = 0; a.rcap = h->r;
        level_setup_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(a);
        LAUNCHED();
        if (h->taylor) {
            // complex W and R11^{-1} in a global slot per CTA; one column per thread
            const int NT = m_cap <= 64 ? 64 : (m_cap <= 128 ? 128 : 256);
            const size_t smem = sizeof(double) * ((size_t)m_cap + 2 * h->r + NT / 32 + 8 + NT / 32 + 2 * h->r) +
                                sizeof(int) * ((size_t)2 * m_cap + NT) + 64;
            void (*kern)(CompressArgs) = NT == 64 ? compress_taylor_kernel<64>
                                                  : (NT == 128 ? compress_taylor_kernel<128> : compress_taylor_kernel<256>);
            allow_max_dynamic_smem((const void *)kern);
            int per_sm = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
            if (per_sm < 1) fail(SMASH_ENOTSUP, "complex compression kernel does not fit on an SM");
            const int64_t grid = std::min<int64_t>(nl, (int64_t)per_sm * h->num_sms);
            CompressArgs b = a;
            b.w_smem_doubles = 0;
            b.x_off = (int64_t)h->r * m_cap;                 // in complex entries
            b.slot_doubles = 2 * (b.x_off + (int64_t)h->r * h->r);
            const int64_t need = grid * b.slot_doubles;
            if (need > work_cap) {
                if (work) scratch.free(work);
                work = scratch.alloc<double>(need);
                work_cap = need;
            }
            b.work = work;
            kern<<<(unsigned)grid, NT, smem, st>>>(b);
            LAUNCHED();
            exclusive_scan<int32_t>(S.k + n0, S.sk_off + n0, nl, base, base, st, scratch);
            compact_skeleton_kernel<<<(unsigned)nl, 128, 0, st>>>(n0, nl, S.k, S.sk_off, S.loc_off, S.skg_tmp, pts,
                                                                   S.skel_gidx, S.skel_xyz);
            LAUNCHED();
            continue;
        }
        // The CTA size is a free choice: every candidate computes the same bits
        // (each column is reduced by one thread in the oracle's order).  The
        // default gives one column per thread up to 512 threads.
        const bool small_p = h->order <= 16;
        // W stays in shared memory up to the opt-in limit of one CTA (less a
        // margin); larger working sets use a global slot in the L2
        int optin = 0;
        CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
        const size_t w_smem_limit = (size_t)std::max(0, optin - 2048);
        struct Plan {
            void (*kern)(CompressArgs);
            size_t smem;
            int64_t grid;
            bool all_in_smem;
            int64_t w_smem_doubles, slot_doubles, x_off;
        };
        // a candidate is NT + kCpsUnit * c: NT threads per CTA and, for c > 1,
        // a W region of 1/c of the opt-in limit (c CTAs per SM, so that one
        // CTA's serial phases overlap another's column updates); nodes whose
        // W exceeds the region use the CTA's global slot
        constexpr int kCpsUnit = 4096;
        auto plan = [&](int cand, Plan &pl) -> bool {
            const int NT = cand % kCpsUnit, cps = std::max(1, cand / kCpsUnit);
            size_t base_smem = sizeof(double) * ((size_t)m_cap + 2 * h->r + NT / 32 + 8 + NT / 32) +
                               sizeof(int) * ((size_t)2 * m_cap + NT) + 64;
            size_t w_bytes = sizeof(double) * (size_t)h->r * m_cap;
            pl.all_in_smem = cps == 1 && (base_smem + w_bytes) <= w_smem_limit;
            if (pl.all_in_smem) {
                pl.w_smem_doubles = (int64_t)h->r * m_cap;
                pl.x_off = 0;
            } else {
                // as much of W as fits in 1/cps of the limit; the nodes above it use
                // the global slot
                const size_t lim = w_smem_limit / cps;
                int64_t room = base_smem < lim ? (int64_t)((lim - base_smem) / sizeof(double)) : 0;
                pl.w_smem_doubles = room >= h->r ? room : 0;
                pl.x_off = (int64_t)h->r * m_cap;
            }
            pl.smem = base_smem + sizeof(double) * (size_t)pl.w_smem_doubles;
            pl.slot_doubles = pl.x_off + (int64_t)h->r * h->r;
            if (NT == 64) pl.kern = small_p ? compress_kernel<64, 16> : compress_kernel<64, kMaxP>;
            else if (NT == 128) pl.kern = small_p ? compress_kernel<128, 16> : compress_kernel<128, kMaxP>;
            else if (NT == 256) pl.kern = small_p ? compress_kernel<256, 16> : compress_kernel<256, kMaxP>;
            else pl.kern = small_p ? compress_kernel<512, 16> : compress_kernel<512, kMaxP>;
            allow_max_dynamic_smem((const void *)pl.kern);
            int per_sm = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pl.kern, NT, pl.smem));
            if (per_sm < 1) return false;
            pl.grid = std::min<int64_t>(nl, (int64_t)per_sm * h->num_sms);
            // keep the concurrent node matrices of a global-slot level inside the L2
            if (!pl.all_in_smem) {
                int64_t fit = (int64_t)(64ll << 20) / (pl.slot_doubles * (int64_t)sizeof(double));
                pl.grid = std::max<int64_t>(1, std::min<int64_t>(pl.grid, std::max<int64_t>(fit, h->num_sms)));
            }
            return true;
        };
        const int NT_def = m_cap <= 64 ? 64 : (m_cap <= 128 ? 128 : (m_cap <= 256 ? 256 : 512));
        std::vector<int> cands;
        Plan pdef;
        if (!plan(NT_def, pdef)) fail(SMASH_ENOTSUP, "compression kernel does not fit on an SM (%zu B smem)", pdef.smem);
        for (int nt = 64; nt <= 512; nt *= 2) {
            Plan pl;
            if (!plan(nt, pl)) continue;
            cands.push_back(nt);
            for (int cps = 2; cps <= 8; cps *= 2) {
                if (nt * cps > 2048) break;  // threads per SM
                Plan p2;
                if (plan(nt + kCpsUnit * cps, p2)) cands.push_back(nt + kCpsUnit * cps);
            }
        }
        auto run = [&](int cand) {
            const int NT = cand % kCpsUnit;
            Plan pl;
            plan(cand, pl);
            CompressArgs b = a;
            b.w_smem_doubles = pl.w_smem_doubles;
            b.slot_doubles = pl.slot_doubles;
            b.x_off = pl.x_off;
            int64_t need = pl.grid * pl.slot_doubles;
            if (need > work_cap) {
                if (work) scratch.free(work);
                work = scratch.alloc<double>(need);
                work_cap = need;
            }
            b.work = work;
            pl.kern<<<(unsigned)pl.grid, NT, pl.smem, st>>>(b);
            LAUNCHED();
        };
        char key[128];
        std::snprintf(key, sizeof(key), "compress/sm%d/d%d/p%d/m%lld/n%lld", h->num_sms, h->dim, h->order,
                      pow2_at_least(m_cap), pow2_at_least(nl));
        tune_choose(key, cands, NT_def, st, run);
        exclusive_scan<int32_t>(S.k + n0, S.sk_off + n0, nl, base, base, st, scratch);
        compact_skeleton_kernel<<<(unsigned)nl, 128, 0, st>>>(n0, nl, S.k, S.sk_off, S.loc_off, S.skg_tmp, pts,
                                                               S.skel_gidx, S.skel_xyz);
        LAUNCHED();
    }
    int64_t total_skel = 0;
    CK(cudaMemcpyAsync(&total_skel, base, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    S.total_skel = total_skel;
    if (work) scratch.free(work);
    scratch.free(kub); scratch.free(mub); scratch.free(gub); scratch.free(kub_off);
    scratch.free(lm); scratch.free(tot); scratch.free(S.skg_tmp);
    S.skg_tmp = nullptr;
}

void build_compression(smash_h2 *h, Arena &scratch) {
    compress_side(h, h->row, true, scratch);
    if (h->same) {
        h->col = &h->row;
    } else {
        compress_side(h, h->colside, false, scratch);
        h->col = &h->colside;
    }
}

// ---------------------------------------------------------------- HSS (Section 3.3.1)
// The nearfield block row (side 0) or column (side 1) of each node of a level
// (3.7)/(3.11) and its truncated SVD by one-sided Jacobi on the rows, in the
// CPU oracle's order of operations: rounds of disjoint row pairs (the
// round-robin order of Brent and Luk).  A round runs in three phases: one
// thread per dot product (three per pair, on neighbouring lanes) sums it in
// ascending order; one thread per pair decides its rotation; then every
// thread applies the rotations element by element, a warp per pair and its
// lanes along the rows (each element is computed exactly as the oracle does,
// so the order of elements is free).  The dot products are the only
// sequential chains left.  The kept left singular vectors (above eps_svd of
// the largest, descending) become extra rows of the node's basis.
constexpr int kHssSvdCap = 64;     // singular vectors kept per node at most
constexpr int kJacobiSweeps = 60;
constexpr double kJacobiEps = 1e-15;
constexpr double kJacobiFloor = 1e-30;

struct SvdArgs {
    int64_t n0, nl;
    int side, kid;
    const int32_t *leaf;
    const int64_t *start_o;            // first point of a leaf on the other side
    const int32_t *count_o;
    const int32_t *m_s, *m_o;          // working-set sizes (this level, both sides)
    const int64_t *in_off_s, *in_off_o, *start_s;
    const int64_t *skel_s, *skel_o;    // skeleton slot -> sorted point, per side
    const double *pts_s, *pts_o;       // sorted coordinates, stride 4
    const int64_t *nf_ptr;
    const int32_t *nf_col;
    double eps_svd;
    int m_cap;                         // largest working set of the level (sizes the round's records)
    double *work;
    int64_t slot_doubles;
    int64_t a_doubles;                 // m_cap * n_cap: JT follows A in a slot
    double *ST;                        // per node kHssSvdCap x m_cap rows
    int64_t st_stride;
    int32_t *s_out;
    int *overflow;
};

__device__ __forceinline__ double kappa_1d(int kid, double x, double y) {
    const double t = x - y;
    if (kid == SMASH_K_CAUCHY1D) return t == 0.0 ? 0.0 : 1.0 / t;
    const double r2 = t * t;
    if (r2 == 0.0) return 0.0;
    const double r = sqrt(r2);
    if (kid == SMASH_K_LOG) return log(r);
    if (kid == SMASH_K_INVR) return 1.0 / r;
    return exp(-r) / r;  // SMASH_K_YUKAWA
}

// sorted point index of working-set position pos of node j (leaf: its points)
__device__ __forceinline__ int64_t ws_other(const SvdArgs &a, int32_t j, int pos) {
    return a.leaf[j] ? a.start_o[j] + pos : a.skel_o[a.in_off_o[j] + pos];
}

__device__ __forceinline__ int ws_other_size(const SvdArgs &a, int32_t j) {
    return a.leaf[j] ? a.count_o[j] : a.m_o[j];
}

__global__ void nf_width_kernel(SvdArgs a, int64_t *__restrict__ width) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nl) return;
    const int64_t g = a.n0 + i;
    int64_t n = 0;
    for (int64_t e = a.nf_ptr[g]; e < a.nf_ptr[g + 1]; ++e) n += ws_other_size(a, a.nf_col[e]);
    width[i] = n;
}

// cluster-wide barrier: release of this thread's writes (shared and global)
// to the other CTAs of the cluster, acquire of theirs
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// C = 1: one CTA per node, persistent over the level's nodes, every per-node
// array in shared memory.  C > 1: a cluster of C CTAs (C SMs) per node, for
// levels with fewer nodes than SMs: the dot-product chains, the rotations,
// the kernel entries and the row norms are spread over the cluster's
// threads, the shared per-node arrays (dot products, norms) live in the
// node's global slot, and cluster barriers (release/acquire) separate the
// phases; loads of data another CTA wrote bypass L1.  The same operations in
// the same order either way, so the same bits.
template <int NT, int C>
__global__ void __launch_bounds__(NT) nearfield_svd_kernel(SvdArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int np_cap = a.m_cap / 2 + 1;  // pairs of a round at most
    double *sig_s = reinterpret_cast<double *>(smraw);  // m_cap
    // the rotations of a round: (c, s) and the rows (p, q); p = -1 for none
    double *rot_c = sig_s + a.m_cap, *rot_s = rot_c + np_cap;
    double *dots_s = rot_s + np_cap;  // [3][np_cap]: alpha, beta, gamma of each pair (C = 1)
    int *rot_p = reinterpret_cast<int *>(dots_s + 3 * np_cap), *rot_q = rot_p + np_cap;
    // C > 1: the rows of this CTA's pairs of a round, 2 per pair, n_cap each
    double *rowbuf = reinterpret_cast<double *>(rot_q + np_cap);  // 8-byte aligned: 2 np_cap ints
    __shared__ int rotated;
    __shared__ int s_sel;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned rank = 0;
    if (C > 1) asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    const int gt = (int)rank * NT + tid, gw = (int)rank * (NT / 32) + warp;  // thread / warp in the node's group
    constexpr int GT = C * NT, GW = C * (NT / 32);
    const int64_t cid = blockIdx.x / C;  // the group (CTA or cluster)
    double *B = a.work + cid * a.slot_doubles;
    double *JT = B + a.a_doubles;
    // per-node arrays shared by the group: shared memory for one CTA, the
    // node's slot for a cluster
    double *dots = C == 1 ? dots_s : JT + (int64_t)a.m_cap * a.m_cap;
    double *sig = C == 1 ? sig_s : dots + 3 * np_cap;  // m_cap (sig[0] first holds ||A||_F^2)
    auto ld = [](const double *p) {
        if constexpr (C == 1) return *p;
        else return __ldcg(p);
    };
    auto node_sync = [] {
        if constexpr (C == 1) __syncthreads();
        else cluster_sync_all();
    };
    for (int64_t ni = cid; ni < a.nl; ni += (C == 1 ? (int64_t)gridDim.x : a.nl)) {
        const int64_t g = a.n0 + ni;
        const int m = a.m_s[g];
        int n = 0;
        for (int64_t e = a.nf_ptr[g]; e < a.nf_ptr[g + 1]; ++e) n += ws_other_size(a, a.nf_col[e]);
        if (m == 0 || n == 0) {
            if (gt == 0) a.s_out[g] = 0;
            continue;
        }
        // A: rows = the node's working set, columns = the working sets of N_g
        for (int col = gt; col < n; col += GT) {
            int64_t e = a.nf_ptr[g];
            int base = 0, w = ws_other_size(a, a.nf_col[e]);
            while (col >= base + w) { base += w; ++e; w = ws_other_size(a, a.nf_col[e]); }
            const double yo = a.pts_o[ws_other(a, a.nf_col[e], col - base) * 4];
            for (int r = 0; r < m; ++r) {
                const int64_t ps = a.leaf[g] ? a.start_s[g] + r : a.skel_s[a.in_off_s[g] + r];
                const double xs = a.pts_s[ps * 4];
                B[(int64_t)r * n + col] = a.side == 0 ? kappa_1d(a.kid, xs, yo) : kappa_1d(a.kid, yo, xs);
            }
        }
        for (int e = gt; e < m * m; e += GT) JT[e] = (e / m == e % m) ? 1.0 : 0.0;
        node_sync();
        if (gt == 0) {  // ||A||_F^2 in the oracle's (row-major) order: it sets the rotation floor
            double f2 = 0.0;
            for (int64_t e = 0; e < (int64_t)m * n; ++e) {
                const double b = ld(B + e);
                f2 = __fma_rn(b, b, f2);
            }
            sig[0] = f2;
        }
        node_sync();
        const double floor_ab = kJacobiFloor * ld(sig);
        node_sync();
        const int M = m + (m & 1);
        for (int sweep = 0; sweep < kJacobiSweeps && m > 1; ++sweep) {
            if (tid == 0) rotated = 0;
            __syncthreads();
            for (int rr = 0; rr < M - 1; ++rr) {
                // (1) the three dot products of every pair of the round, one
                // sequential chain per thread in the oracle's order (a pair's
                // three chains on neighbouring lanes of one warp)
                const int np = M / 2;
                if constexpr (C == 1) {
                    for (int it = tid; it < 3 * np; it += NT) {
                        const int i = it / 3, which = it - 3 * i;
                        int pa, pb;
                        if (i == 0) { pa = M - 1; pb = rr; }
                        else { pa = (rr + i) % (M - 1); pb = (rr - i + (M - 1)) % (M - 1); }
                        const int p = pa < pb ? pa : pb, q = pa < pb ? pb : pa;
                        if (q >= m) continue;
                        const double *bu = B + (int64_t)(which == 1 ? q : p) * n;
                        const double *bv = B + (int64_t)(which == 0 ? p : q) * n;
                        double acc = 0.0;
                        for (int e = 0; e < n; ++e) acc = __fma_rn(bu[e], bv[e], acc);
                        dots[which * np_cap + i] = acc;
                    }
                } else {
                    // pair i to CTA i % C; its two rows are first copied from the
                    // node's slot into shared memory by all the CTA's threads
                    // (coalesced, from L2), then each chain runs from there
                    const int npl = (np - (int)rank + C - 1) / C;  // this CTA's pairs
                    for (int idx = tid; idx < 2 * npl * n; idx += NT) {
                        const int r2 = idx / n, e = idx - r2 * n;
                        const int i = (r2 >> 1) * C + (int)rank;
                        int pa, pb;
                        if (i == 0) { pa = M - 1; pb = rr; }
                        else { pa = (rr + i) % (M - 1); pb = (rr - i + (M - 1)) % (M - 1); }
                        const int row = (r2 & 1) ? (pa < pb ? pb : pa) : (pa < pb ? pa : pb);
                        if (row < m) rowbuf[(int64_t)r2 * n + e] = __ldcg(B + (int64_t)row * n + e);
                    }
                    __syncthreads();
                    for (int it = tid; it < 3 * npl; it += NT) {
                        const int li = it / 3, which = it - 3 * li, i = li * C + (int)rank;
                        int pa, pb;
                        if (i == 0) { pa = M - 1; pb = rr; }
                        else { pa = (rr + i) % (M - 1); pb = (rr - i + (M - 1)) % (M - 1); }
                        if ((pa < pb ? pb : pa) >= m) continue;
                        const double *bu = rowbuf + (int64_t)(2 * li + (which == 1 ? 1 : 0)) * n;
                        const double *bv = rowbuf + (int64_t)(2 * li + (which == 0 ? 0 : 1)) * n;
                        double acc = 0.0;
                        for (int e = 0; e < n; ++e) acc = __fma_rn(bu[e], bv[e], acc);
                        dots[which * np_cap + i] = acc;
                    }
                }
                node_sync();
                // (1b) each pair's rotation (every CTA of a cluster decides all
                // of them, from the same dot products)
                for (int i = tid; i < np; i += NT) {
                    int pa, pb;
                    if (i == 0) { pa = M - 1; pb = rr; }
                    else { pa = (rr + i) % (M - 1); pb = (rr - i + (M - 1)) % (M - 1); }
                    const int p = pa < pb ? pa : pb, q = pa < pb ? pb : pa;
                    rot_p[i] = -1;
                    if (q >= m) continue;
                    const double al = ld(dots + i), be = ld(dots + np_cap + i), ga = ld(dots + 2 * np_cap + i);
                    const double nab = sqrt(al) * sqrt(be);
                    if (ga == 0.0 || !(fabs(ga) > kJacobiEps * nab) || !(nab > floor_ab)) continue;
                    const double zeta = (be - al) / (2.0 * ga);
                    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double c = 1.0 / sqrt(1.0 + t * t);
                    rot_c[i] = c;
                    rot_s[i] = c * t;
                    rot_p[i] = p;
                    rot_q[i] = q;
                    rotated = 1;
                }
                __syncthreads();
                // (2) the rotations, element by element over all threads (each
                // element's two products and difference as in the oracle)
                for (int i = gw; i < np; i += GW) {
                    const int p = rot_p[i];
                    if (p < 0) continue;
                    const int q = rot_q[i];
                    const double c = rot_c[i], sn = rot_s[i];
                    double *bp = B + (int64_t)p * n, *bq = B + (int64_t)q * n;
                    double *jp = JT + (int64_t)p * m, *jq = JT + (int64_t)q * m;
                    if constexpr (C == 1) {
                        for (int e = lane; e < n; e += 32) {
                            const double u = bp[e], v = bq[e];
                            bp[e] = c * u - sn * v;
                            bq[e] = sn * u + c * v;
                        }
                        for (int e = lane; e < m; e += 32) {
                            const double u = jp[e], v = jq[e];
                            jp[e] = c * u - sn * v;
                            jq[e] = sn * u + c * v;
                        }
                    } else {
                        // from L2: a batch of loads in flight before its stores
                        constexpr int kB = 8;
                        for (int e0 = lane; e0 < n; e0 += 32 * kB) {
                            double u[kB], v[kB];
#pragma unroll
                            for (int k = 0; k < kB; ++k) {
                                const int e = e0 + 32 * k;
                                u[k] = e < n ? __ldcg(bp + e) : 0.0;
                                v[k] = e < n ? __ldcg(bq + e) : 0.0;
                            }
#pragma unroll
                            for (int k = 0; k < kB; ++k) {
                                const int e = e0 + 32 * k;
                                if (e < n) {
                                    bp[e] = c * u[k] - sn * v[k];
                                    bq[e] = sn * u[k] + c * v[k];
                                }
                            }
                        }
                        for (int e0 = lane; e0 < m; e0 += 32 * kB) {
                            double u[kB], v[kB];
#pragma unroll
                            for (int k = 0; k < kB; ++k) {
                                const int e = e0 + 32 * k;
                                u[k] = e < m ? __ldcg(jp + e) : 0.0;
                                v[k] = e < m ? __ldcg(jq + e) : 0.0;
                            }
#pragma unroll
                            for (int k = 0; k < kB; ++k) {
                                const int e = e0 + 32 * k;
                                if (e < m) {
                                    jp[e] = c * u[k] - sn * v[k];
                                    jq[e] = sn * u[k] + c * v[k];
                                }
                            }
                        }
                    }
                }
                node_sync();
            }
            const bool any = rotated != 0;
            __syncthreads();
            if (!any) break;
        }
        for (int p = gt; p < m; p += GT) {
            double s2 = 0.0;
            for (int e = 0; e < n; ++e) {
                const double b = ld(B + (int64_t)p * n + e);
                s2 = __fma_rn(b, b, s2);
            }
            sig[p] = sqrt(s2);
        }
        node_sync();
        // the rest on one CTA (rank 0 of a cluster; no cluster barrier follows)
        if (rank != 0) continue;
        if (C > 1) {
            for (int p = tid; p < m; p += NT) sig_s[p] = ld(sig + p);
            __syncthreads();
        }
        // keep the singular values above eps_svd of the largest, descending
        // (ties: the lower row first); sig of a kept row is set to -1
        double *dst = a.ST + ni * a.st_stride;
        if (tid == 0) {
            double smax = 0.0;
            for (int p = 0; p < m; ++p) if (sig_s[p] > smax) smax = sig_s[p];
            int sc = 0;
            for (;;) {
                int best = -1;
                for (int p = 0; p < m; ++p)
                    if (sig_s[p] >= 0.0 && (best < 0 || sig_s[p] > sig_s[best])) best = p;
                if (best < 0 || !(sig_s[best] > a.eps_svd * smax) || !(sig_s[best] > 0.0)) break;
                if (sc == kHssSvdCap) { *a.overflow = 1; break; }
                sig_s[best] = -1.0 - (double)sc;  // kept, in this order
                ++sc;
            }
            s_sel = sc;
        }
        __syncthreads();
        const int sc = s_sel;
        for (int p = 0; p < m; ++p) {
            const double v = sig_s[p];
            if (v >= 0.0) continue;
            const int t = (int)(-v - 1.0);
            for (int e = tid; e < m; e += NT) dst[(int64_t)t * m + e] = ld(JT + (int64_t)p * m + e);
        }
        if (tid == 0) a.s_out[g] = sc;
        __syncthreads();
    }
}

namespace {

struct HssSide {
    Side *S;
    bool rows;
    std::vector<int64_t> lmax;
};

// the per-side preamble of compress_side with the rank bound r + kHssSvdCap
void hss_prepare(smash_h2 *h, Side &S, bool rows, std::vector<int64_t> &lmax, int64_t *base, Arena &scratch) {
    cudaStream_t st = h->stream;
    const int64_t nn = h->nnodes;
    const int32_t *cnt = rows ? h->rc : h->cc;
    S.m = h->mem.alloc<int32_t>(nn);
    S.k = h->mem.alloc<int32_t>(nn);
    S.in_off = h->mem.alloc<int64_t>(nn);
    S.sk_off = h->mem.alloc<int64_t>(nn);
    S.loc_off = h->mem.alloc<int64_t>(nn + 1);
    S.g_off = h->mem.alloc<int64_t>(nn + 1);
    S.nswaps = h->mem.alloc<int32_t>(nn);
    CK(cudaMemsetAsync(S.m, 0, nn * 4, st));
    CK(cudaMemsetAsync(S.k, 0, nn * 4, st));
    CK(cudaMemsetAsync(S.nswaps, 0, nn * 4, st));
    CK(cudaMemsetAsync(S.sk_off, 0, nn * 8, st));
    CK(cudaMemsetAsync(S.in_off, 0, nn * 8, st));
    int64_t *kub = scratch.alloc<int64_t>(nn), *mub = scratch.alloc<int64_t>(nn), *gub = scratch.alloc<int64_t>(nn);
    int64_t *tot = scratch.alloc<int64_t>(3);
    bounds_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(nn, h->r + kHssSvdCap, h->level, h->leaf, cnt,
                                                                 h->child0, h->nchild, kub, mub, gub);
    LAUNCHED();
    int64_t *kub_off = scratch.alloc<int64_t>(nn);
    exclusive_scan<int64_t>(kub, kub_off, nn, nullptr, tot + 0, st, scratch);
    exclusive_scan<int64_t>(mub, S.loc_off, nn, nullptr, tot + 1, st, scratch);
    exclusive_scan<int64_t>(gub, S.g_off, nn, nullptr, tot + 2, st, scratch);
    lmax.assign(h->L + 1, 0);
    int64_t *lm = scratch.alloc<int64_t>(h->L + 1);
    for (int l = 2; l <= h->L; ++l) {
        int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        reduce_max(mub + n0, nl, lm + l, st);
    }
    int64_t ht[3];
    CK(cudaMemcpyAsync(ht, tot, 3 * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(lmax.data(), lm, (h->L + 1) * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    S.skel_cap = std::max<int64_t>(ht[0], 1);
    S.total_loc = ht[1];
    S.total_g = ht[2];
    S.mub_max = lmax;
    S.loc = h->mem.alloc<int32_t>(std::max<int64_t>(S.total_loc, 1));
    S.skg_tmp = scratch.alloc<int64_t>(std::max<int64_t>(S.total_loc, 1));
    S.G = h->mem.alloc<double>(std::max<int64_t>(S.total_g, 1));
    S.skel_gidx = h->mem.alloc<int64_t>(S.skel_cap);
    S.skel_xyz = h->mem.alloc<double>(S.skel_cap * 4);
    CK(cudaMemsetAsync(base, 0, 8, st));
    scratch.free(kub); scratch.free(mub); scratch.free(gub); scratch.free(kub_off); scratch.free(lm);
    scratch.free(tot);
}

}  // namespace

void build_compression_hss(smash_h2 *h, Arena &scratch) {
    cudaStream_t st = h->stream;
    const int64_t nn = h->nnodes;
    const bool two = !h->same;
    std::vector<HssSide> sides;
    sides.push_back({&h->row, true, {}});
    if (two) sides.push_back({&h->colside, false, {}});
    h->col = two ? &h->colside : &h->row;
    int64_t *bases = scratch.alloc<int64_t>(2);
    for (size_t i = 0; i < sides.size(); ++i) hss_prepare(h, *sides[i].S, sides[i].rows, sides[i].lmax, bases + i, scratch);
    h->svd_row = h->mem.alloc<int32_t>(nn);
    h->svd_col = two ? h->mem.alloc<int32_t>(nn) : h->svd_row;
    CK(cudaMemsetAsync(h->svd_row, 0, nn * 4, st));
    if (two) CK(cudaMemsetAsync(h->svd_col, 0, nn * 4, st));
    int *overflow = scratch.alloc<int>(1);
    CK(cudaMemsetAsync(overflow, 0, sizeof(int), st));
    int64_t *wmax = scratch.alloc<int64_t>(1);
    double weights[kMaxP] = {0};
    for (int m = 0; m < h->order; ++m) {
        double den = 1.0;
        for (int n = 0; n < h->order; ++n)
            if (n != m) den = den * (h->anchors[m] - h->anchors[n]);
        weights[m] = 1.0 / den;
    }
    const int rcap = h->r + kHssSvdCap;
    for (int l = h->L; l >= 2; --l) {
        const int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        std::vector<CompressArgs> args(sides.size());
        for (size_t i = 0; i < sides.size(); ++i) {
            Side &S = *sides[i].S;
            CompressArgs &a = args[i];
            a = CompressArgs{};
            a.d = h->dim; a.p = h->order; a.r = h->r; a.level = l;
            a.tol = h->tol; a.f = h->f;
            a.geo4 = h->tree_geo; a.node_tree = h->node_tree;
            for (int t = 0; t < kMaxP; ++t) {
                a.anchors[t] = t < h->order ? h->anchors[t] : 0.0;
                a.weights[t] = t < h->order ? weights[t] : 0.0;
            }
            a.n0 = n0; a.nl = nl;
            a.leaf = h->leaf; a.cell = h->cell;
            a.start = sides[i].rows ? h->rs : h->cs;
            a.count = sides[i].rows ? h->rc : h->cc;
            a.child0 = h->child0; a.nchild = h->nchild;
            a.pts = sides[i].rows ? h->xs : h->ys;
            a.skel_gidx = S.skel_gidx;
            a.m = S.m; a.k = S.k; a.in_off = S.in_off; a.sk_off = S.sk_off; a.loc_off = S.loc_off;
            a.g_off = S.g_off; a.loc = S.loc; a.skg_tmp = S.skg_tmp; a.G = S.G; a.nswaps = S.nswaps;
            a.m_cap = (int)std::max<int64_t>(sides[i].lmax[l], 1);
            a.rcap = rcap;
            level_setup_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(a);
            LAUNCHED();
        }
        // the truncated SVDs of the level's nearfield blocks, both sides
        std::vector<double *> stbuf(sides.size(), nullptr);
        for (size_t i = 0; i < sides.size(); ++i) {
            const Side &S = *sides[i].S;
            const Side &O = *sides[sides.size() == 1 ? 0 : 1 - i].S;
            const bool rows = sides[i].rows;
            SvdArgs v{};
            v.n0 = n0; v.nl = nl; v.side = rows ? 0 : 1; v.kid = h->kernel_id;
            v.leaf = h->leaf;
            v.start_o = rows ? h->cs : h->rs;
            v.count_o = rows ? h->cc : h->rc;
            v.start_s = rows ? h->rs : h->cs;
            v.m_s = S.m; v.m_o = O.m; v.in_off_s = S.in_off; v.in_off_o = O.in_off;
            v.skel_s = S.skel_gidx; v.skel_o = O.skel_gidx;
            v.pts_s = rows ? h->xs : h->ys;
            v.pts_o = rows ? h->ys : h->xs;
            v.nf_ptr = h->nf_ptr; v.nf_col = h->nf_col;
            v.eps_svd = h->eps_svd;
            v.s_out = rows ? h->svd_row : h->svd_col;
            v.overflow = overflow;
            int64_t *width = scratch.alloc<int64_t>(nl);
            nf_width_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, st>>>(v, width);
            LAUNCHED();
            reduce_max(width, nl, wmax, st);
            int64_t n_cap = 0;
            CK(cudaMemcpyAsync(&n_cap, wmax, 8, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            scratch.free(width);
            const int64_t m_cap = std::max<int64_t>(sides[i].lmax[l], 1);
            n_cap = std::max<int64_t>(n_cap, 1);
            v.a_doubles = m_cap * n_cap;
            v.slot_doubles = v.a_doubles + m_cap * m_cap;
            v.st_stride = (int64_t)kHssSvdCap * m_cap;
            stbuf[i] = scratch.alloc<double>((size_t)nl * v.st_stride);
            v.ST = stbuf[i];
            // eight warps per node: a round's dot-product chains (three per
            // pair) fill them.  Levels of at most 64 nodes give each node a
            // cluster of 8 CTAs (8 SMs); the others run one CTA per node,
            // persistent, slots of at most 256 MiB in all and at least one CTA
            // per SM
            constexpr int NT = 256;
            v.m_cap = (int)m_cap;
            const int64_t np_cap = m_cap / 2 + 1;
            size_t smem = sizeof(double) * (size_t)m_cap + (5 * sizeof(double) + 2 * sizeof(int)) * (size_t)np_cap;
            const int64_t room = 4 * (int64_t)h->num_sms;
            // (measured: clusters pay on the top levels only; at 128 or more
            // nodes one CTA per node does better)
            int C = nl <= 64 ? 8 : 1;
            // a cluster CTA also holds the rows of its pairs (2 per pair)
            auto rows_bytes = [&](int c) { return sizeof(double) * 2 * (size_t)((np_cap + c - 1) / c) * (size_t)n_cap; };
            while (C > 1 && smem + rows_bytes(C) > (size_t)200 * 1024) C /= 2;
            if (C > 1) smem += rows_bytes(C);
            double *slots = nullptr;
            if (C == 1) {
                const int64_t fit = std::max<int64_t>(1, (int64_t)(256ll << 20) / (v.slot_doubles * 8));
                const int64_t grid = std::max<int64_t>(
                    1, std::min<int64_t>(nl, std::max<int64_t>(std::min<int64_t>(fit, room), h->num_sms)));
                slots = scratch.alloc<double>((size_t)grid * v.slot_doubles);
                v.work = slots;
                allow_max_dynamic_smem((const void *)nearfield_svd_kernel<NT, 1>);
                nearfield_svd_kernel<NT, 1><<<(unsigned)grid, NT, smem, st>>>(v);
            } else {
                // one slot per node: B, JT, then the dot products and row norms
                // that the cluster shares
                v.slot_doubles += 3 * (m_cap / 2 + 1) + m_cap;
                slots = scratch.alloc<double>((size_t)nl * v.slot_doubles);
                v.work = slots;
                void (*kern)(SvdArgs) = C == 8 ? nearfield_svd_kernel<NT, 8>
                                               : (C == 4 ? nearfield_svd_kernel<NT, 4> : nearfield_svd_kernel<NT, 2>);
                allow_max_dynamic_smem((const void *)kern);
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)(nl * C));
                cfg.blockDim = dim3(NT);
                cfg.dynamicSmemBytes = smem;
                cfg.stream = st;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = (unsigned)C;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                CK(cudaLaunchKernelEx(&cfg, kern, v));
            }
            LAUNCHED();
            scratch.free(slots);
        }
        // compr of [U^_i, S_i] (3.9)/(3.13)
        for (size_t i = 0; i < sides.size(); ++i) {
            Side &S = *sides[i].S;
            CompressArgs b = args[i];
            b.extra = stbuf[i];
            b.extra_rows = sides[i].rows ? h->svd_row : h->svd_col;
            b.extra_stride = (int64_t)kHssSvdCap * b.m_cap;
            const int NT = b.m_cap <= 64 ? 64 : (b.m_cap <= 128 ? 128 : (b.m_cap <= 256 ? 256 : 512));
            const size_t smem = sizeof(double) * ((size_t)b.m_cap + 2 * rcap + NT / 32 + 8 + NT / 32) +
                                sizeof(int) * ((size_t)2 * b.m_cap + NT) + 64;
            b.w_smem_doubles = 0;
            b.x_off = (int64_t)rcap * b.m_cap;
            b.slot_doubles = b.x_off + (int64_t)rcap * rcap;
            const bool small_p = h->order <= 16;
            void (*kern)(CompressArgs) = nullptr;
            if (NT == 64) kern = small_p ? compress_kernel<64, 16> : compress_kernel<64, kMaxP>;
            else if (NT == 128) kern = small_p ? compress_kernel<128, 16> : compress_kernel<128, kMaxP>;
            else if (NT == 256) kern = small_p ? compress_kernel<256, 16> : compress_kernel<256, kMaxP>;
            else kern = small_p ? compress_kernel<512, 16> : compress_kernel<512, kMaxP>;
            allow_max_dynamic_smem((const void *)kern);
            int per_sm = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
            if (per_sm < 1) fail(SMASH_ENOTSUP, "HSS compression kernel does not fit on an SM");
            const int64_t fit = std::max<int64_t>(1, (int64_t)(256ll << 20) / (b.slot_doubles * 8));
            const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(nl, std::min<int64_t>((int64_t)per_sm * h->num_sms,
                                                                                              std::max<int64_t>(fit, 1))));
            double *slots = scratch.alloc<double>((size_t)grid * b.slot_doubles);
            b.work = slots;
            kern<<<(unsigned)grid, NT, smem, st>>>(b);
            LAUNCHED();
            exclusive_scan<int32_t>(S.k + n0, S.sk_off + n0, nl, bases + i, bases + i, st, scratch);
            compact_skeleton_kernel<<<(unsigned)nl, 128, 0, st>>>(n0, nl, S.k, S.sk_off, S.loc_off, S.skg_tmp, b.pts,
                                                                   S.skel_gidx, S.skel_xyz);
            LAUNCHED();
            scratch.free(slots);
        }
        for (size_t i = 0; i < sides.size(); ++i) scratch.free(stbuf[i]);
    }
    int ov = 0;
    int64_t tot[2] = {0, 0};
    CK(cudaMemcpyAsync(&ov, overflow, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(tot, bases, 8 * sides.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ov) fail(SMASH_ENOTSUP, "a nearfield block needs more than %d singular vectors at eps_svd %g", kHssSvdCap,
                 h->eps_svd);
    for (size_t i = 0; i < sides.size(); ++i) {
        sides[i].S->total_skel = tot[i];
        scratch.free(sides[i].S->skg_tmp);
        sides[i].S->skg_tmp = nullptr;
    }
    scratch.free(overflow); scratch.free(wmax); scratch.free(bases);
}

}  // namespace smash
