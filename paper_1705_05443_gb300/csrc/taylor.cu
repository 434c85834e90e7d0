// taylor.cu -- the node-wise matvec of Section 3.4 for the representation
// built on the Taylor expansion (2.4)-(2.5) of kappa(x, y) = 1/(x - y) on C
// ((2.1): points are complex numbers x_0 + i x_1, kappa(x, x) = d_x).  Every
// vector, generator and kernel entry is complex FP64:
//   gather q into Morton order; near field over L^- (3.20); upward pass
//   q^_i = [I G^T] P^T q (plain transpose: A^ = U B V^T with V = U); coupling
//   over L with kernel entries on skeleton pairs (3.19); downward pass;
//   scatter back to the caller's order.
// One CTA per node; each thread owns (target, column) pairs and sums its
// sources in a fixed order, so results are deterministic.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace smash {

namespace {

struct C2 { double re, im; };

__device__ __forceinline__ C2 cmul(C2 a, C2 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ void cadd(C2 &s, C2 v) { s.re += v.re; s.im += v.im; }

// kappa of (2.1): 1/(x - y), d_x at coincident points
__device__ __forceinline__ C2 cauchy_c(const double *x, const double *y, double dxr, double dxi) {
    const double tr = x[0] - y[0], ti = x[1] - y[1];
    if (tr == 0.0 && ti == 0.0) return {dxr, dxi};
    const double den = tr * tr + ti * ti;
    return {tr / den, -ti / den};
}

constexpr int kThreads = 128;
constexpr int kTile = 128;  // sources staged per round

__global__ void gather_c_kernel(const C2 *__restrict__ X, int nrhs, const int64_t *__restrict__ perm, int64_t n,
                                C2 *__restrict__ qs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nrhs) return;
    qs[i] = X[perm[i / nrhs] * nrhs + i % nrhs];
}

__global__ void scatter_c_kernel(const C2 *__restrict__ zs, int nrhs, const int64_t *__restrict__ perm, int64_t n,
                                 C2 *__restrict__ Y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nrhs) return;
    Y[perm[i / nrhs] * nrhs + i % nrhs] = zs[i];
}

// out[t_off(g) + a] = sum over the partners j of g (CSR), over the points b of
// j: kappa(x_a, y_b) q[s_off(j) + b]; coordinates stride 4, vectors nrhs wide.
struct KsumCArgs {
    const int32_t *tnodes;
    const int64_t *t_off;
    const int32_t *t_cnt;
    const int64_t *ptr;
    const int32_t *col;
    const int64_t *s_off;
    const int32_t *s_cnt;
    const double *xt, *ys;
    const C2 *q;
    C2 *out;
    int nrhs;
    double dxr, dxi;
};

__global__ void __launch_bounds__(kThreads) ksum_c_kernel(KsumCArgs a) {
    __shared__ double sy[kTile][2];
    __shared__ int64_t sidx[kTile];
    const int64_t g = a.tnodes[blockIdx.x];
    const int T = a.t_cnt[g];
    if (T == 0) return;
    const int64_t toff = a.t_off[g];
    const int nrhs = a.nrhs;
    const int64_t e0 = a.ptr[g], e1 = a.ptr[g + 1];
    for (int base = 0; base < T * nrhs; base += kThreads) {
        const int e = base + threadIdx.x;
        const bool active = e < T * nrhs;
        const int t = active ? e / nrhs : 0, c = active ? e % nrhs : 0;
        double xt[2] = {0.0, 0.0};
        if (active) { xt[0] = a.xt[(toff + t) * 4]; xt[1] = a.xt[(toff + t) * 4 + 1]; }
        C2 acc = {0.0, 0.0};
        for (int64_t p = e0; p < e1; ++p) {
            const int32_t j = a.col[p];
            const int64_t so = a.s_off[j];
            const int S = a.s_cnt[j];
            for (int b0 = 0; b0 < S; b0 += kTile) {
                const int fill = min(kTile, S - b0);
                __syncthreads();
                for (int b = threadIdx.x; b < fill; b += kThreads) {
                    sidx[b] = so + b0 + b;
                    sy[b][0] = a.ys[(so + b0 + b) * 4];
                    sy[b][1] = a.ys[(so + b0 + b) * 4 + 1];
                }
                __syncthreads();
                if (active)
                    for (int b = 0; b < fill; ++b) {
                        const C2 kv = cauchy_c(xt, sy[b], a.dxr, a.dxi);
                        cadd(acc, cmul(kv, a.q[sidx[b] * nrhs + c]));
                    }
            }
        }
        if (active) a.out[(toff + t) * nrhs + c] = acc;
    }
}

struct PassCArgs {
    int64_t n0;
    const int32_t *leaf, *m, *k;
    const int64_t *in_off, *sk_off, *loc_off, *g_off;
    const int32_t *loc;
    const C2 *G;
    const C2 *pts_vec;
    C2 *skel_in, *skel_out, *pts_out;
    int nrhs;
};

// q^_i[t] = x[skel_t] + sum_u G[u][t] x[rest_u]
__global__ void __launch_bounds__(256) upward_c_kernel(PassCArgs a) {
    const int64_t g = a.n0 + blockIdx.x;
    const int m = a.m[g], k = a.k[g];
    if (k == 0) return;
    const int n = a.nrhs;
    const C2 *in = a.leaf[g] ? a.pts_vec + a.in_off[g] * n : a.skel_in + a.in_off[g] * n;
    const int32_t *loc = a.loc + a.loc_off[g];
    const C2 *G = a.G + a.g_off[g];
    C2 *out = a.skel_out + a.sk_off[g] * n;
    const int mk = m - k;
    for (int e = threadIdx.x; e < k * n; e += blockDim.x) {
        const int t = e / n, c = e % n;
        C2 s = in[(int64_t)loc[t] * n + c];
        for (int u = 0; u < mk; ++u) cadd(s, cmul(G[(int64_t)u * k + t], in[(int64_t)loc[k + u] * n + c]));
        out[(int64_t)t * n + c] = s;
    }
}

// out[skel_t] += z^_i[t];  out[rest_u] += sum_t G[u][t] z^_i[t]
__global__ void __launch_bounds__(256) downward_c_kernel(PassCArgs a) {
    const int64_t g = a.n0 + blockIdx.x;
    const int m = a.m[g], k = a.k[g];
    if (k == 0) return;
    const int n = a.nrhs;
    const C2 *zin = a.skel_in + a.sk_off[g] * n;
    C2 *out = a.leaf[g] ? a.pts_out + a.in_off[g] * n : a.skel_out + a.in_off[g] * n;
    const int32_t *loc = a.loc + a.loc_off[g];
    const C2 *G = a.G + a.g_off[g];
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
        const int row = e / n, c = e % n;
        C2 s;
        if (row < k) {
            s = zin[(int64_t)row * n + c];
        } else {
            const C2 *gr = G + (int64_t)(row - k) * k;
            s = {0.0, 0.0};
            for (int t = 0; t < k; ++t) cadd(s, cmul(gr[t], zin[(int64_t)t * n + c]));
        }
        cadd(out[(int64_t)loc[row] * n + c], s);
    }
}

}  // namespace

void matvec_taylor(const smash_h2 *h, const double *X, double *Y, int nrhs, cudaStream_t s, Profile *prof) {
    const Side &R = h->row;
    Arena tmp(s);
    C2 *qs = tmp.alloc<C2>((size_t)h->nx * nrhs);
    C2 *zs = tmp.alloc<C2>((size_t)h->nx * nrhs);
    C2 *qhat = tmp.alloc<C2>((size_t)std::max<int64_t>(R.total_skel, 1) * nrhs);
    C2 *zhat = tmp.alloc<C2>((size_t)std::max<int64_t>(R.total_skel, 1) * nrhs);
    const C2 *G = reinterpret_cast<const C2 *>(R.G);
    PhaseTimer tm(s, prof);
    tm.mark();
    const int64_t tot = h->nx * nrhs;
    gather_c_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(reinterpret_cast<const C2 *>(X), nrhs, h->permx,
                                                                  h->nx, qs);
    LAUNCHED();
    tm.mark();
    {
        KsumCArgs a{};
        a.tnodes = h->leaf_list; a.t_off = h->rs; a.t_cnt = h->rc;
        a.ptr = h->near_ptr; a.col = h->near_col; a.s_off = h->cs; a.s_cnt = h->cc;
        a.xt = h->xs; a.ys = h->ys; a.q = qs; a.out = zs; a.nrhs = nrhs; a.dxr = h->dx_re; a.dxi = h->dx_im;
        if (h->nleaves > 0) {
            ksum_c_kernel<<<(unsigned)h->nleaves, kThreads, 0, s>>>(a);
            LAUNCHED();
        }
    }
    tm.mark();
    for (int l = h->L; l >= 2; --l) {
        const int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        PassCArgs p{n0, h->leaf, R.m, R.k, R.in_off, R.sk_off, R.loc_off, R.g_off, R.loc, G, qs, qhat, qhat, nullptr,
                    nrhs};
        upward_c_kernel<<<(unsigned)nl, 256, 0, s>>>(p);
        LAUNCHED();
    }
    tm.mark();
    if (h->nnodes > h->nroots) {
        KsumCArgs a{};
        a.tnodes = h->nonroot_list; a.t_off = R.sk_off; a.t_cnt = R.k;
        a.ptr = h->adm_ptr; a.col = h->adm_col; a.s_off = R.sk_off; a.s_cnt = R.k;
        a.xt = R.skel_xyz; a.ys = R.skel_xyz; a.q = qhat; a.out = zhat; a.nrhs = nrhs;
        a.dxr = h->dx_re; a.dxi = h->dx_im;
        ksum_c_kernel<<<(unsigned)(h->nnodes - h->nroots), kThreads, 0, s>>>(a);
        LAUNCHED();
    }
    tm.mark();
    for (int l = 2; l <= h->L; ++l) {
        const int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        PassCArgs p{n0, h->leaf, R.m, R.k, R.in_off, R.sk_off, R.loc_off, R.g_off, R.loc, G, nullptr, zhat, zhat, zs,
                    nrhs};
        downward_c_kernel<<<(unsigned)nl, 256, 0, s>>>(p);
        LAUNCHED();
    }
    tm.mark();
    scatter_c_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(zs, nrhs, h->permx, h->nx,
                                                                   reinterpret_cast<C2 *>(Y));
    LAUNCHED();
    tm.mark();
    tm.finish(4);
    tmp.release();
}

}  // namespace smash
