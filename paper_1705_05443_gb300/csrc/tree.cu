// tree.cu -- Section 3.1 partition and the (3.3)/(3.4) interaction lists.
//
// Compiled with --fmad=false: the cube, the Morton quantisation and the
// admissibility test use separately rounded IEEE operations so that every
// integer decision (cell of a point, admissible or not) is reproducible.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace smash {

// ------------------------------------------------------------------ cube
struct Geo {
    double lo[3];
    double hi[3];
    double s;
    int bad;
};

__global__ void bbox_partial_kernel(const double *__restrict__ p, int64_t n, int d, double *__restrict__ part,
                                    int *__restrict__ bad) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int nonfinite = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < d; ++a) {
            double v = p[i * d + a];
            if (!isfinite(v)) nonfinite = 1;
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    for (int a = 0; a < d; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    __shared__ double slo[32][3], shi[32][3];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) { slo[w][a] = lo[a]; shi[w][a] = hi[a]; }
    if (nonfinite) atomicOr(bad, 1);
    __syncthreads();
    if (threadIdx.x < 3) {
        int a = threadIdx.x;
        double l = INFINITY, h = -INFINITY;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) { l = fmin(l, slo[ww][a]); h = fmax(h, shi[ww][a]); }
        part[blockIdx.x * 6 + a] = l;
        part[blockIdx.x * 6 + 3 + a] = h;
    }
}

__global__ void bbox_final_kernel(const double *__restrict__ part, int nparts, int d, Geo *g) {
    if (threadIdx.x != 0) return;
    for (int a = 0; a < 3; ++a) { g->lo[a] = INFINITY; g->hi[a] = -INFINITY; }
    for (int i = 0; i < nparts; ++i)
        for (int a = 0; a < 3; ++a) {
            g->lo[a] = fmin(g->lo[a], part[i * 6 + a]);
            g->hi[a] = fmax(g->hi[a], part[i * 6 + 3 + a]);
        }
    double ext = 0.0;
    for (int a = 0; a < d; ++a)
        if (g->hi[a] - g->lo[a] > ext) ext = g->hi[a] - g->lo[a];
    // largest extent times (1 + 2^-40); 1 when all points coincide
    g->s = ext > 0.0 ? ext * (1.0 + 0x1p-40) : 1.0;
    for (int a = d; a < 3; ++a) g->lo[a] = 0.0;
}

// ------------------------------------------------------------------ Morton keys
__device__ __forceinline__ uint64_t quantize(double v, double lo, double s, int b) {
    double t = (v - lo) / s;
    double two_b = ldexp(1.0, b);
    double f = floor(t * two_b);
    uint64_t top = (((uint64_t)1) << b) - 1;
    if (!(f > 0.0)) return 0;
    if (f >= two_b) return top;
    uint64_t q = (uint64_t)f;
    return q > top ? top : q;
}

// key: b digits of d bits, most significant digit first, dimension 0 the
// most significant bit within a digit.
__global__ void morton_kernel(const double *__restrict__ p, int64_t n, int d, int b, const Geo *__restrict__ g,
                              uint64_t *__restrict__ keys, int32_t *__restrict__ idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t q[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) q[a] = quantize(p[i * d + a], g->lo[a], g->s, b);
    uint64_t key = 0;
    for (int l = 0; l < b; ++l)
        for (int a = 0; a < d; ++a) key = (key << 1) | ((q[a] >> (b - 1 - l)) & 1u);
    keys[i] = key;
    idx[i] = (int32_t)i;
}

__global__ void gather_points_kernel(const double *__restrict__ p, int64_t n, int d, const int32_t *__restrict__ idx,
                                     int64_t *__restrict__ perm, double *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t src = idx[i];
    perm[i] = src;
    P4 v{0.0, 0.0, 0.0, 0.0};
    v.x = p[src * d];
    if (d > 1) v.y = p[src * d + 1];
    if (d > 2) v.z = p[src * d + 2];
    reinterpret_cast<P4 *>(out)[i] = v;
}

static void sort_side(smash_h2 *h, const double *p, int64_t n, const Geo *g, uint64_t *&keys, int64_t *&perm,
                      double *&pts, Arena &scratch) {
    cudaStream_t s = h->stream;
    keys = h->mem.alloc<uint64_t>(n);
    perm = h->mem.alloc<int64_t>(n);
    pts = h->mem.alloc<double>((size_t)n * 4);
    int32_t *idx = scratch.alloc<int32_t>(n);
    unsigned blocks = (unsigned)((n + 255) / 256);
    morton_kernel<<<blocks, 256, 0, s>>>(p, n, h->dim, h->bits, g, keys, idx);
    LAUNCHED();
    radix_sort(keys, idx, n, h->dim * h->bits, s, scratch);
    gather_points_kernel<<<blocks, 256, 0, s>>>(p, n, h->dim, idx, perm, pts);
    LAUNCHED();
    scratch.free(idx);
}

void build_geometry(smash_h2 *h, const double *x_dev, const double *y_dev, Arena &scratch) {
    cudaStream_t s = h->stream;
    int nparts = 256;
    double *part = scratch.alloc<double>((size_t)nparts * 6 * 2);
    Geo *g = scratch.alloc<Geo>(1);
    int *bad = scratch.alloc<int>(1);
    CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
    bbox_partial_kernel<<<nparts, 256, 0, s>>>(x_dev, h->nx, h->dim, part, bad);
    LAUNCHED();
    int np = nparts;
    if (!h->same) {
        bbox_partial_kernel<<<nparts, 256, 0, s>>>(y_dev, h->ny, h->dim, part + nparts * 6, bad);
        LAUNCHED();
        np = 2 * nparts;
    }
    bbox_final_kernel<<<1, 32, 0, s>>>(part, np, h->dim, g);
    LAUNCHED();
    Geo hg;
    int hbad = 0;
    CK(cudaMemcpyAsync(&hg, g, sizeof(Geo), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hbad) fail(SMASH_EINVAL, "non-finite point coordinate");
    for (int a = 0; a < 3; ++a) h->lo[a] = hg.lo[a];
    h->s = hg.s;
    h->tree_geo_host = {hg.lo[0], hg.lo[1], hg.lo[2], hg.s};
    h->tree_geo = h->mem.alloc<double>(4);
    CK(cudaMemcpyAsync(h->tree_geo, h->tree_geo_host.data(), 4 * sizeof(double), cudaMemcpyHostToDevice, s));
    sort_side(h, x_dev, h->nx, g, h->keyx, h->permx, h->xs, scratch);
    if (h->same) {
        h->keyy = h->keyx;
        h->permy = h->permx;
        h->ys = h->xs;
    } else {
        sort_side(h, y_dev, h->ny, g, h->keyy, h->permy, h->ys, scratch);
    }
    scratch.free(part);
    scratch.free(g);
    scratch.free(bad);
}

// ------------------------------------------------------------------ batch of problems
// One CTA per problem: its bounding cube exactly as for a single problem
// (componentwise min and max, largest extent times (1 + 2^-40)).
__global__ void bbox_segment_kernel(const double *__restrict__ p, const int64_t *__restrict__ off, int d,
                                    double *__restrict__ geo7, int *__restrict__ bad) {
    const int64_t t = blockIdx.x;
    const int64_t i0 = off[t], i1 = off[t + 1];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int nonfinite = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
        for (int a = 0; a < d; ++a) {
            double v = p[i * d + a];
            if (!isfinite(v)) nonfinite = 1;
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    for (int a = 0; a < d; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    __shared__ double slo[32][3], shi[32][3];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) { slo[w][a] = lo[a]; shi[w][a] = hi[a]; }
    if (nonfinite) atomicOr(bad, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        double L[3], H[3];
        for (int a = 0; a < 3; ++a) {
            L[a] = INFINITY; H[a] = -INFINITY;
            for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) { L[a] = fmin(L[a], slo[ww][a]); H[a] = fmax(H[a], shi[ww][a]); }
        }
        double ext = 0.0;
        for (int a = 0; a < d; ++a)
            if (H[a] - L[a] > ext) ext = H[a] - L[a];
        for (int a = d; a < 3; ++a) { L[a] = 0.0; H[a] = 0.0; }
        double *o = geo7 + t * 7;
        for (int a = 0; a < 3; ++a) { o[a] = L[a]; o[3 + a] = H[a]; }
        o[6] = ext > 0.0 ? ext * (1.0 + 0x1p-40) : 1.0;
    }
}

// Morton key of every point in the cube of its own problem; tkey = problem.
__global__ void morton_batch_kernel(const double *__restrict__ p, int64_t n, int d, int b,
                                    const int64_t *__restrict__ off, int ntrees, const double *__restrict__ geo4,
                                    uint64_t *__restrict__ keys, uint64_t *__restrict__ tkeys,
                                    int32_t *__restrict__ idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = ntrees - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    const double *g = geo4 + (int64_t)lo * 4;
    uint64_t q[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) q[a] = quantize(p[i * d + a], g[a], g[3], b);
    uint64_t key = 0;
    for (int l = 0; l < b; ++l)
        for (int a = 0; a < d; ++a) key = (key << 1) | ((q[a] >> (b - 1 - l)) & 1u);
    keys[i] = key;
    tkeys[i] = (uint64_t)lo;
    idx[i] = (int32_t)i;
}

__global__ void gather_u64_kernel(const uint64_t *__restrict__ src, const int32_t *__restrict__ idx, int64_t n,
                                  uint64_t *__restrict__ dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

// Points of all problems sorted by (problem, Morton key): a stable sort by
// key, then a stable sort by problem.
void build_geometry_batch(smash_h2 *h, const double *x_dev, Arena &scratch) {
    cudaStream_t s = h->stream;
    const int64_t T = h->nroots, n = h->nx;
    const int d = h->dim;
    int64_t *off = scratch.alloc<int64_t>(T + 1);
    CK(cudaMemcpyAsync(off, h->tree_off.data(), (T + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    double *geo7 = scratch.alloc<double>(T * 7);
    int *bad = scratch.alloc<int>(1);
    CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
    bbox_segment_kernel<<<(unsigned)T, 256, 0, s>>>(x_dev, off, d, geo7, bad);
    LAUNCHED();
    std::vector<double> g7((size_t)T * 7);
    int hbad = 0;
    CK(cudaMemcpyAsync(g7.data(), geo7, T * 7 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hbad) fail(SMASH_EINVAL, "non-finite point coordinate");
    h->tree_geo_host.assign((size_t)T * 4, 0.0);
    double flo[3] = {INFINITY, INFINITY, INFINITY}, fhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t t = 0; t < T; ++t) {
        for (int a = 0; a < 3; ++a) {
            h->tree_geo_host[t * 4 + a] = g7[t * 7 + a];
            flo[a] = std::min(flo[a], g7[t * 7 + a]);
            fhi[a] = std::max(fhi[a], g7[t * 7 + 3 + a]);
        }
        h->tree_geo_host[t * 4 + 3] = g7[t * 7 + 6];
    }
    // the matvec frame: the cube of all problems
    double ext = 0.0;
    for (int a = 0; a < d; ++a) ext = std::max(ext, fhi[a] - flo[a]);
    for (int a = 0; a < 3; ++a) h->lo[a] = a < d ? flo[a] : 0.0;
    h->s = ext > 0.0 ? ext * (1.0 + 0x1p-40) : 1.0;
    h->tree_geo = h->mem.alloc<double>(T * 4);
    CK(cudaMemcpyAsync(h->tree_geo, h->tree_geo_host.data(), T * 4 * sizeof(double), cudaMemcpyHostToDevice, s));

    uint64_t *kraw = scratch.alloc<uint64_t>(n), *tk = scratch.alloc<uint64_t>(n), *tk2 = scratch.alloc<uint64_t>(n);
    int32_t *idx = scratch.alloc<int32_t>(n);
    h->keyx = h->mem.alloc<uint64_t>(n);
    h->permx = h->mem.alloc<int64_t>(n);
    h->xs = h->mem.alloc<double>((size_t)n * 4);
    unsigned blocks = (unsigned)((n + 255) / 256);
    morton_batch_kernel<<<blocks, 256, 0, s>>>(x_dev, n, d, h->bits, off, (int)T, h->tree_geo, kraw, tk, idx);
    LAUNCHED();
    CK(cudaMemcpyAsync(h->keyx, kraw, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    radix_sort(h->keyx, idx, n, d * h->bits, s, scratch);
    gather_u64_kernel<<<blocks, 256, 0, s>>>(tk, idx, n, tk2);
    LAUNCHED();
    int tbits = 1;
    while ((1ll << tbits) < T) ++tbits;
    radix_sort(tk2, idx, n, tbits, s, scratch);
    gather_u64_kernel<<<blocks, 256, 0, s>>>(kraw, idx, n, h->keyx);
    LAUNCHED();
    gather_points_kernel<<<blocks, 256, 0, s>>>(x_dev, n, d, idx, h->permx, h->xs);
    LAUNCHED();
    h->keyy = h->keyx;
    h->permy = h->permx;
    h->ys = h->xs;
    scratch.free(kraw); scratch.free(tk); scratch.free(tk2); scratch.free(idx);
    scratch.free(off); scratch.free(geo7); scratch.free(bad);
}

// ------------------------------------------------------------------ tree
struct NodeArrays {
    int32_t *level, *leaf, *parent, *child0, *nchild, *rc, *cc;
    int64_t *rs, *cs;
    uint64_t *cell;
    int32_t *tree;
};

// first position in [lo, hi) whose digit (key >> shift) & mask is >= c
__device__ __forceinline__ int64_t digit_lower_bound(const uint64_t *__restrict__ keys, int64_t lo, int64_t hi,
                                                     int shift, uint64_t mask, uint64_t c) {
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (((keys[mid] >> shift) & mask) < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// one thread per (node of the level, digit): child ranges of splitting nodes
__global__ void split_ranges_kernel(NodeArrays A, int64_t n0, int64_t nl, int d, int b, int l,
                                    const uint64_t *__restrict__ keyx, const uint64_t *__restrict__ keyy,
                                    int64_t *__restrict__ crs, int32_t *__restrict__ crc,
                                    int64_t *__restrict__ ccs, int32_t *__restrict__ ccc) {
    int nd = 1 << d;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nl * nd) return;
    int64_t g = n0 + t / nd;
    uint64_t c = (uint64_t)(t % nd);
    if (A.leaf[g]) { crc[t] = 0; ccc[t] = 0; crs[t] = 0; ccs[t] = 0; return; }
    int shift = d * (b - l);
    uint64_t mask = (uint64_t)nd - 1;
    int64_t r0 = A.rs[g], r1 = r0 + A.rc[g];
    int64_t a0 = digit_lower_bound(keyx, r0, r1, shift, mask, c);
    int64_t a1 = digit_lower_bound(keyx, a0, r1, shift, mask, c + 1);
    int64_t c0 = A.cs[g], c1 = c0 + A.cc[g];
    int64_t b0 = digit_lower_bound(keyy, c0, c1, shift, mask, c);
    int64_t b1 = digit_lower_bound(keyy, b0, c1, shift, mask, c + 1);
    crs[t] = a0; crc[t] = (int32_t)(a1 - a0);
    ccs[t] = b0; ccc[t] = (int32_t)(b1 - b0);
}

__global__ void count_children_kernel(int64_t nl, int d, const int32_t *__restrict__ crc,
                                      const int32_t *__restrict__ ccc, int32_t *__restrict__ nch) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl) return;
    int nd = 1 << d, c = 0;
    for (int j = 0; j < nd; ++j) c += (crc[i * nd + j] + ccc[i * nd + j]) > 0;
    nch[i] = c;
}

__global__ void emit_children_kernel(NodeArrays A, int64_t n0, int64_t nl, int d, int b, int l, int leaf_size,
                                     int64_t nnext0, const int64_t *__restrict__ choff,
                                     const int64_t *__restrict__ crs, const int32_t *__restrict__ crc,
                                     const int64_t *__restrict__ ccs, const int32_t *__restrict__ ccc) {
    int nd = 1 << d;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nl * nd) return;
    int64_t i = t / nd;
    int dig = (int)(t % nd);
    int64_t g = n0 + i;
    if ((crc[t] + ccc[t]) == 0) return;
    int before = 0;
    for (int j = 0; j < dig; ++j) before += (crc[i * nd + j] + ccc[i * nd + j]) > 0;
    int64_t c = nnext0 + choff[i] + before;
    A.level[c] = l + 1;
    A.parent[c] = (int32_t)g;
    A.tree[c] = A.tree[g];
    A.child0[c] = -1;
    A.nchild[c] = 0;
    A.rs[c] = crs[t];
    A.rc[c] = crc[t];
    A.cs[c] = ccs[t];
    A.cc[c] = ccc[t];
    for (int a = 0; a < 3; ++a)
        A.cell[c * 3 + a] = a < d ? 2 * A.cell[g * 3 + a] + (uint64_t)((dig >> (d - 1 - a)) & 1) : 0;
    int big = max(crc[t], ccc[t]);
    A.leaf[c] = !(big > leaf_size && (l + 1) <= b);
    if (before == 0) A.child0[g] = (int32_t)c;
    atomicAdd(&A.nchild[g], 1);
}

template <class T>
static void grow(T *&p, int64_t used, int64_t cap_new, Arena &mem, cudaStream_t s) {
    T *q = mem.alloc<T>(cap_new);
    if (p && used) CK(cudaMemcpyAsync(q, p, used * sizeof(T), cudaMemcpyDeviceToDevice, s));
    mem.free(p);
    p = q;
}

static void grow_nodes(NodeArrays &A, int64_t used, int64_t cap, Arena &mem, cudaStream_t s) {
    grow(A.level, used, cap, mem, s);
    grow(A.leaf, used, cap, mem, s);
    grow(A.parent, used, cap, mem, s);
    grow(A.child0, used, cap, mem, s);
    grow(A.nchild, used, cap, mem, s);
    grow(A.rc, used, cap, mem, s);
    grow(A.cc, used, cap, mem, s);
    grow(A.rs, used, cap, mem, s);
    grow(A.cs, used, cap, mem, s);
    grow(A.cell, used * 3, cap * 3, mem, s);
    grow(A.tree, used, cap, mem, s);
}

__global__ void leaf_list_kernel(const int32_t *__restrict__ leaf, int64_t n, const int64_t *__restrict__ pos,
                                 int32_t *__restrict__ out) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n && leaf[g]) out[pos[g]] = (int32_t)g;
}

__global__ void iota_kernel(int32_t *out, int64_t n, int32_t first) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = first + (int32_t)i;
}

void build_tree(smash_h2 *h, Arena &scratch) {
    cudaStream_t s = h->stream;
    int d = h->dim, b = h->bits, nd = 1 << d;
    NodeArrays A{};
    // level 1: one root per problem
    const int64_t R = h->nroots;
    int64_t cap = std::max<int64_t>(1024, 2 * R);
    grow_nodes(A, 0, cap, h->mem, s);
    {
        std::vector<int32_t> lv(R, 1), pa(R, -1), c0(R, -1), nc(R, 0), rc(R), cc(R), lf(R), tr(R);
        std::vector<int64_t> rs(R), cs(R);
        std::vector<uint64_t> cell0((size_t)R * 3, 0);
        for (int64_t t = 0; t < R; ++t) {
            if (R == 1) {
                rs[t] = cs[t] = 0;
                rc[t] = (int32_t)h->nx;
                cc[t] = (int32_t)h->ny;
            } else {
                rs[t] = cs[t] = h->tree_off[t];
                rc[t] = cc[t] = (int32_t)(h->tree_off[t + 1] - h->tree_off[t]);
            }
            int64_t big = std::max(rc[t], cc[t]);
            lf[t] = !(big > h->leaf_size && 1 <= b);
            tr[t] = (int32_t)t;
        }
        CK(cudaMemcpyAsync(A.level, lv.data(), R * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(A.parent, pa.data(), R * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(A.child0, c0.data(), R * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(A.nchild, nc.data(), R * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(A.rc, rc.data(), R * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(A.cc, cc.data(), R * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(A.rs, rs.data(), R * 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(A.cs, cs.data(), R * 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(A.leaf, lf.data(), R * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(A.cell, cell0.data(), R * 24, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(A.tree, tr.data(), R * 4, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    h->lvl_off.assign(1, 0);
    h->lvl_off.push_back(R);
    int64_t total = R;
    int l = 1;
    int64_t *next_total = scratch.alloc<int64_t>(1);
    for (;;) {
        int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        int64_t *crs = scratch.alloc<int64_t>(nl * nd), *ccs = scratch.alloc<int64_t>(nl * nd);
        int32_t *crc = scratch.alloc<int32_t>(nl * nd), *ccc = scratch.alloc<int32_t>(nl * nd);
        int32_t *nch = scratch.alloc<int32_t>(nl);
        int64_t *choff = scratch.alloc<int64_t>(nl);
        unsigned blocks = (unsigned)((nl * nd + 255) / 256);
        split_ranges_kernel<<<blocks, 256, 0, s>>>(A, n0, nl, d, b, l, h->keyx, h->keyy, crs, crc, ccs, ccc);
        LAUNCHED();
        count_children_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, s>>>(nl, d, crc, ccc, nch);
        LAUNCHED();
        exclusive_scan<int32_t>(nch, choff, nl, nullptr, next_total, s, scratch);
        int64_t nnext = 0;
        CK(cudaMemcpyAsync(&nnext, next_total, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (nnext > 0) {
            if (total + nnext > cap) {
                int64_t nc = std::max(cap * 2, total + nnext);
                grow_nodes(A, total, nc, h->mem, s);
                cap = nc;
            }
            emit_children_kernel<<<blocks, 256, 0, s>>>(A, n0, nl, d, b, l, h->leaf_size, total, choff, crs, crc,
                                                        ccs, ccc);
            LAUNCHED();
        }
        scratch.free(crs); scratch.free(ccs); scratch.free(crc); scratch.free(ccc);
        scratch.free(nch); scratch.free(choff);
        if (nnext == 0) break;
        total += nnext;
        ++l;
        h->lvl_off.push_back(total);
        if (l > b + 1) fail(SMASH_EDEPTH, "tree deeper than %d levels", b + 1);
    }
    h->L = l;
    h->nnodes = total;
    h->level = A.level; h->leaf = A.leaf; h->parent = A.parent; h->child0 = A.child0; h->nchild = A.nchild;
    h->rs = A.rs; h->cs = A.cs; h->rc = A.rc; h->cc = A.cc; h->cell = A.cell; h->node_tree = A.tree;
    // leaf list
    int64_t *pos = scratch.alloc<int64_t>(total);
    exclusive_scan<int32_t>(h->leaf, pos, total, nullptr, next_total, s, scratch);
    CK(cudaMemcpyAsync(&h->nleaves, next_total, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->leaf_list = h->mem.alloc<int32_t>(std::max<int64_t>(h->nleaves, 1));
    leaf_list_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(h->leaf, total, pos, h->leaf_list);
    LAUNCHED();
    h->nonroot_list = h->mem.alloc<int32_t>(std::max<int64_t>(total - R, 1));
    if (total > R) {
        iota_kernel<<<(unsigned)((total - R + 255) / 256), 256, 0, s>>>(h->nonroot_list, total - R, (int32_t)R);
        LAUNCHED();
    }
    scratch.free(pos);
    scratch.free(next_total);
}

// ------------------------------------------------------------------ lists
// Definition 2.1 on cells, in units of half the finer cell: centres are the
// integers (2c+1) 2^(m-l), radii sqrt(d) 2^(m-l); (2.3) squared reads
// d (2^(m-li) + 2^(m-lj))^2 <= tau^2 sum_a D_a^2.
__device__ __forceinline__ bool admissible(int d, int li, const uint64_t *ci, int lj, const uint64_t *cj,
                                           double tau) {
    int m = li > lj ? li : lj;
    double e = ldexp(1.0, m - li) + ldexp(1.0, m - lj);
    double lhs = (double)d * (e * e);
    double sum = 0.0;
    for (int a = 0; a < d; ++a) {
        uint64_t Ci = (2 * ci[a] + 1) << (m - li);
        uint64_t Cj = (2 * cj[a] + 1) << (m - lj);
        uint64_t D = Ci >= Cj ? Ci - Cj : Cj - Ci;
        double Dd = (double)D;
        sum = sum + Dd * Dd;
    }
    double tau2 = tau * tau;
    return lhs <= tau2 * sum;
}

enum : int8_t { P_DROP = 0, P_ADM = 1, P_NEAR = 2, P_SPLIT = 3 };

__global__ void classify_kernel(const uint64_t *__restrict__ fr, int64_t nf, NodeArrays A, int d, double tau,
                                int nb, int32_t *__restrict__ ca, int32_t *__restrict__ cn,
                                int32_t *__restrict__ cs_) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nf) return;
    uint64_t pr = fr[t];
    int64_t i = (int64_t)(pr >> nb), j = (int64_t)(pr & ((1ull << nb) - 1));
    int a = 0, n = 0, sp = 0;
    if (A.rc[i] > 0 && A.cc[j] > 0) {
        if (admissible(d, A.level[i], A.cell + i * 3, A.level[j], A.cell + j * 3, tau)) a = 1;
        else if (A.leaf[i] && A.leaf[j]) n = 1;
        else sp = (A.leaf[i] ? 1 : A.nchild[i]) * (A.leaf[j] ? 1 : A.nchild[j]);
    }
    ca[t] = a;
    cn[t] = n;
    cs_[t] = sp;
}

__global__ void emit_pairs_kernel(const uint64_t *__restrict__ fr, int64_t nf, NodeArrays A, int nb,
                                  const int32_t *__restrict__ ca, const int32_t *__restrict__ cn,
                                  const int64_t *__restrict__ oa, const int64_t *__restrict__ on,
                                  const int64_t *__restrict__ os, const int64_t *__restrict__ base_a,
                                  const int64_t *__restrict__ base_n, uint64_t *__restrict__ adm,
                                  uint64_t *__restrict__ near, uint64_t *__restrict__ next) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nf) return;
    uint64_t pr = fr[t];
    if (ca[t]) { adm[*base_a + oa[t]] = pr; return; }
    if (cn[t]) { near[*base_n + on[t]] = pr; return; }
    int64_t i = (int64_t)(pr >> nb), j = (int64_t)(pr & ((1ull << nb) - 1));
    if (!(A.rc[i] > 0 && A.cc[j] > 0)) return;
    int64_t o = os[t];
    int ni = A.leaf[i] ? 1 : A.nchild[i], nj = A.leaf[j] ? 1 : A.nchild[j];
    int64_t i0 = A.leaf[i] ? i : A.child0[i], j0 = A.leaf[j] ? j : A.child0[j];
    for (int x = 0; x < ni; ++x)
        for (int y = 0; y < nj; ++y) next[o++] = ((uint64_t)(i0 + x) << nb) | (uint64_t)(j0 + y);
}

__global__ void csr_count_kernel(const uint64_t *__restrict__ pairs, int64_t n, int nb, int32_t *__restrict__ cnt,
                                 int32_t *__restrict__ col) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint64_t pr = pairs[t];
    atomicAdd(&cnt[pr >> nb], 1);
    col[t] = (int32_t)(pr & ((1ull << nb) - 1));
}

static void to_csr(smash_h2 *h, uint64_t *pairs, int64_t n, int nb, int64_t *&ptr, int32_t *&col, Arena &scratch) {
    cudaStream_t s = h->stream;
    radix_sort(pairs, nullptr, n, 2 * nb, s, scratch);
    int32_t *cnt = scratch.alloc<int32_t>(h->nnodes);
    CK(cudaMemsetAsync(cnt, 0, h->nnodes * sizeof(int32_t), s));
    ptr = h->mem.alloc<int64_t>(h->nnodes + 1);
    col = h->mem.alloc<int32_t>(std::max<int64_t>(n, 1));
    if (n > 0) {
        csr_count_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pairs, n, nb, cnt, col);
        LAUNCHED();
    }
    exclusive_scan<int32_t>(cnt, ptr, h->nnodes, nullptr, ptr + h->nnodes, s, scratch);
    scratch.free(cnt);
}

void build_lists(smash_h2 *h, Arena &scratch) {
    cudaStream_t s = h->stream;
    NodeArrays A{h->level, h->leaf, h->parent, h->child0, h->nchild, h->rc, h->cc, h->rs, h->cs, h->cell,
                 h->node_tree};
    int nb = 1;
    while ((1ll << nb) < h->nnodes) ++nb;
    int64_t cap_a = 1 << 16, cap_n = 1 << 16;
    uint64_t *adm = scratch.alloc<uint64_t>(cap_a), *near = scratch.alloc<uint64_t>(cap_n);
    int64_t na = 0, nn = 0;
    // traversal from (root, root) of every problem
    int64_t nf = h->nroots;
    uint64_t *fr = scratch.alloc<uint64_t>(nf);
    {
        std::vector<uint64_t> f0((size_t)nf);
        for (int64_t t = 0; t < nf; ++t) f0[t] = ((uint64_t)t << nb) | (uint64_t)t;
        CK(cudaMemcpyAsync(fr, f0.data(), nf * 8, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    int64_t *tot = scratch.alloc<int64_t>(5);  // [0] adm base, [1] near base, [2..4] totals
    CK(cudaMemsetAsync(tot, 0, 5 * sizeof(int64_t), s));
    while (nf > 0) {
        int32_t *ca = scratch.alloc<int32_t>(nf), *cn = scratch.alloc<int32_t>(nf), *csp = scratch.alloc<int32_t>(nf);
        int64_t *oa = scratch.alloc<int64_t>(nf), *on = scratch.alloc<int64_t>(nf), *os = scratch.alloc<int64_t>(nf);
        unsigned blocks = (unsigned)((nf + 255) / 256);
        classify_kernel<<<blocks, 256, 0, s>>>(fr, nf, A, h->dim, h->tau, nb, ca, cn, csp);
        LAUNCHED();
        exclusive_scan<int32_t>(ca, oa, nf, nullptr, tot + 2, s, scratch);
        exclusive_scan<int32_t>(cn, on, nf, nullptr, tot + 3, s, scratch);
        exclusive_scan<int32_t>(csp, os, nf, nullptr, tot + 4, s, scratch);
        int64_t ht[3];
        CK(cudaMemcpyAsync(ht, tot + 2, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (na + ht[0] > cap_a) {
            int64_t c = std::max(cap_a * 2, na + ht[0]);
            grow(adm, na, c, scratch, s);
            cap_a = c;
        }
        if (nn + ht[1] > cap_n) {
            int64_t c = std::max(cap_n * 2, nn + ht[1]);
            grow(near, nn, c, scratch, s);
            cap_n = c;
        }
        uint64_t *next = scratch.alloc<uint64_t>(std::max<int64_t>(ht[2], 1));
        emit_pairs_kernel<<<blocks, 256, 0, s>>>(fr, nf, A, nb, ca, cn, oa, on, os, tot + 0, tot + 1, adm, near,
                                                 next);
        LAUNCHED();
        na += ht[0];
        nn += ht[1];
        CK(cudaMemcpyAsync(tot + 0, &na, 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(tot + 1, &nn, 8, cudaMemcpyHostToDevice, s));
        scratch.free(ca); scratch.free(cn); scratch.free(csp);
        scratch.free(oa); scratch.free(on); scratch.free(os);
        scratch.free(fr);
        fr = next;
        nf = ht[2];
        CK(cudaStreamSynchronize(s));  // the host values na/nn above must be consumed before reuse
    }
    scratch.free(fr);
    scratch.free(tot);
    h->nadm = na;
    h->nnear = nn;
    to_csr(h, adm, na, nb, h->adm_ptr, h->adm_col, scratch);
    to_csr(h, near, nn, nb, h->near_ptr, h->near_col, scratch);
    scratch.free(adm);
    scratch.free(near);
}

// ------------------------------------------------------------------ HSS lists
// (3.5): L = the siblings of every node, L^- = every leaf with itself.
__global__ void hss_count_kernel(int64_t nn, const int32_t *__restrict__ parent, const int32_t *__restrict__ nchild,
                                 const int32_t *__restrict__ leaf, int32_t *__restrict__ ca,
                                 int32_t *__restrict__ cn) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nn) return;
    ca[g] = parent[g] >= 0 ? nchild[parent[g]] - 1 : 0;
    cn[g] = leaf[g] ? 1 : 0;
}

__global__ void hss_fill_kernel(int64_t nn, const int32_t *__restrict__ parent, const int32_t *__restrict__ child0,
                                const int32_t *__restrict__ nchild, const int32_t *__restrict__ leaf,
                                const int64_t *__restrict__ adm_ptr, int32_t *__restrict__ adm_col,
                                const int64_t *__restrict__ near_ptr, int32_t *__restrict__ near_col) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nn) return;
    const int32_t p = parent[g];
    if (p >= 0) {
        int64_t o = adm_ptr[g];
        for (int c = 0; c < nchild[p]; ++c)
            if (child0[p] + c != g) adm_col[o++] = child0[p] + c;
    }
    if (leaf[g]) near_col[near_ptr[g]] = (int32_t)g;
}

// (A.1) for the nodes of one level: N_i = the siblings of i, the children k of
// the non-leaf nodes of N_{p_i} with (i, k) not well separated, and the leaves
// of N_{p_i} not well separated from i; ascending node id.  Two passes: count,
// then fill and sort.
__device__ __forceinline__ int nf_visit(NodeArrays A, int d, double tau, int64_t g, const int64_t *__restrict__ nf_ptr,
                                        const int32_t *__restrict__ nf_col, int32_t *out) {
    const int32_t p = A.parent[g];
    int cnt = 0;
    for (int c = 0; c < A.nchild[p]; ++c) {
        const int32_t k = A.child0[p] + c;
        if (k == g) continue;
        if (out) out[cnt] = k;
        ++cnt;
    }
    for (int64_t e = nf_ptr[p]; e < nf_ptr[p + 1]; ++e) {
        const int32_t kq = nf_col[e];
        if (A.leaf[kq]) {
            if (!admissible(d, A.level[g], A.cell + 3 * g, A.level[kq], A.cell + 3 * (int64_t)kq, tau)) {
                if (out) out[cnt] = kq;
                ++cnt;
            }
        } else {
            for (int c = 0; c < A.nchild[kq]; ++c) {
                const int32_t k = A.child0[kq] + c;
                if (!admissible(d, A.level[g], A.cell + 3 * g, A.level[k], A.cell + 3 * (int64_t)k, tau)) {
                    if (out) out[cnt] = k;
                    ++cnt;
                }
            }
        }
    }
    return cnt;
}

__global__ void nf_count_kernel(NodeArrays A, int d, double tau, int64_t n0, int64_t nl,
                                const int64_t *__restrict__ nf_ptr, const int32_t *__restrict__ nf_col,
                                int32_t *__restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl) return;
    cnt[i] = nf_visit(A, d, tau, n0 + i, nf_ptr, nf_col, nullptr);
}

__global__ void nf_fill_kernel(NodeArrays A, int d, double tau, int64_t n0, int64_t nl, const int64_t *__restrict__ nf_ptr,
                               int32_t *__restrict__ nf_col) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl) return;
    const int64_t g = n0 + i;
    int32_t *out = nf_col + nf_ptr[g];
    const int cnt = nf_visit(A, d, tau, g, nf_ptr, nf_col, out);
    for (int a = 1; a < cnt; ++a) {  // insertion sort: the lists hold a handful of nodes
        int32_t v = out[a];
        int b = a - 1;
        while (b >= 0 && out[b] > v) { out[b + 1] = out[b]; --b; }
        out[b + 1] = v;
    }
}

void build_lists_hss(smash_h2 *h, Arena &scratch) {
    cudaStream_t s = h->stream;
    const int64_t nn = h->nnodes;
    const unsigned blocks = (unsigned)((nn + 255) / 256);
    int32_t *ca = scratch.alloc<int32_t>(nn), *cn = scratch.alloc<int32_t>(nn);
    int64_t *tot = scratch.alloc<int64_t>(3);
    hss_count_kernel<<<blocks, 256, 0, s>>>(nn, h->parent, h->nchild, h->leaf, ca, cn);
    LAUNCHED();
    h->adm_ptr = h->mem.alloc<int64_t>(nn + 1);
    h->near_ptr = h->mem.alloc<int64_t>(nn + 1);
    exclusive_scan<int32_t>(ca, h->adm_ptr, nn, nullptr, h->adm_ptr + nn, s, scratch);
    exclusive_scan<int32_t>(cn, h->near_ptr, nn, nullptr, h->near_ptr + nn, s, scratch);
    int64_t ht[2];
    CK(cudaMemcpyAsync(&ht[0], h->adm_ptr + nn, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&ht[1], h->near_ptr + nn, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->nadm = ht[0];
    h->nnear = ht[1];
    h->adm_col = h->mem.alloc<int32_t>(std::max<int64_t>(h->nadm, 1));
    h->near_col = h->mem.alloc<int32_t>(std::max<int64_t>(h->nnear, 1));
    hss_fill_kernel<<<blocks, 256, 0, s>>>(nn, h->parent, h->child0, h->nchild, h->leaf, h->adm_ptr, h->adm_col,
                                           h->near_ptr, h->near_col);
    LAUNCHED();
    // the nearfield sets, level by level from the top
    NodeArrays A{h->level, h->leaf, h->parent, h->child0, h->nchild, h->rc, h->cc, h->rs, h->cs, h->cell,
                 h->node_tree};
    h->nf_ptr = h->mem.alloc<int64_t>(nn + 1);
    CK(cudaMemsetAsync(h->nf_ptr, 0, sizeof(int64_t) * (nn + 1), s));
    int64_t cap = std::max<int64_t>(nn, 16), used = 0;
    h->nf_col = h->mem.alloc<int32_t>(cap);
    CK(cudaMemsetAsync(tot, 0, 8, s));
    for (int l = 2; l <= h->L; ++l) {
        const int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        const unsigned lb = (unsigned)((nl + 255) / 256);
        nf_count_kernel<<<lb, 256, 0, s>>>(A, h->dim, h->tau, n0, nl, h->nf_ptr, h->nf_col, ca);
        LAUNCHED();
        exclusive_scan<int32_t>(ca, h->nf_ptr + n0, nl, tot, tot, s, scratch);
        // the end of the level's last list (the next level's scan writes the same value)
        CK(cudaMemcpyAsync(h->nf_ptr + n0 + nl, tot, 8, cudaMemcpyDeviceToDevice, s));
        int64_t total = 0;
        CK(cudaMemcpyAsync(&total, tot, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (total > cap) {
            const int64_t c2 = std::max(2 * cap, total);
            grow(h->nf_col, used, c2, h->mem, s);
            cap = c2;
        }
        nf_fill_kernel<<<lb, 256, 0, s>>>(A, h->dim, h->tau, n0, nl, h->nf_ptr, h->nf_col);
        LAUNCHED();
        used = total;
    }
    h->nnf = used;
    CK(cudaStreamSynchronize(s));
    scratch.free(ca); scratch.free(cn); scratch.free(tot);
}

}  // namespace smash
