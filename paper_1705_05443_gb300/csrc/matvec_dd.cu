// matvec_dd.cu -- the Section 3.4 matvec with the coupling (3.19) and the
// near field (3.20) in double-float arithmetic on the FP32 pipe.
//
// GB300 executes FP32 FMA ~61x faster than FP64 FMA, and the FP64 kernel-sum
// kernel saturates the FP64 pipe.  Here every value of the kernel sums is an
// unevaluated sum of two floats (hi + lo, ~48-bit significand) and every
// operation is an error-free transformation (Knuth's TwoSum, Dekker's
// product via FMA), so the result keeps FP64-class accuracy (~1e-12 relative
// against the FP64 oracle) while running on the FP32 pipe.
//
//  * Coordinates, two representations:
//    - normalised: x'' = 1 + (x - lo)/s in [1, 2) split into (hi, lo) floats.
//      Two hi parts in [1, 2] differ by an exactly representable float
//      (Sterbenz), so a difference is hi_a - hi_b (exact) plus lo_a - lo_b,
//      with an absolute error ~2^-48.  Used for the coupling of trees with at
//      most 10 levels, where admissible pairs are at least ~0.4 cell widths
//      apart and the relative error stays below ~5e-12.
//    - exact: x~ = x 2^-e (a power-of-two scaling, exact) split into three
//      floats hi + mid + lo that represent the FP64 value exactly; differences
//      by TwoDiff on hi and mid parts carry ~2^-48 relative precision however
//      close the points are (FP64 subtracts close points exactly too).  Used
//      for the near field and for the coupling of deeper trees.
//    The kernel is evaluated in these units and the sums are scaled at the
//    end: 1/|x - y| = (1/s) / |x'' - y''| = 2^-e / |x~ - y~|, and likewise
//    1/(x - y) in 1D.
//  * 1/sqrt(r2): hardware reciprocal square root of hi(r2) as the seed, then
//    one Newton step y1 = y0 + y0 (1 - r2 y0^2) / 2 in double-float
//    (relative error ~3 eps_f^2 / 8 ~ 2e-14).  1/d in 1D: reciprocal seed and
//    one Newton step y1 = y0 + y0 (1 - d y0).
//  * q vectors are split into (hi, lo) floats by a conversion pass; the
//    accumulators are double-float pairs renormalised after every source
//    tile, and written out in FP64.
// Compiled with --fmad=false: every fused operation below is an explicit fmaf.
#include <algorithm>
#include <cstdio>
#include <cmath>

#include "dd_arith.cuh"
#include "internal.cuh"
#include "ksum_tiles.cuh"

namespace smash {

// ------------------------------------------------------------------ conversions
// per point: (hi x, hi y, hi z, 0, lo x, lo y, lo z, 0) of x'' = 1 + (x - lo)/s
__global__ void dd_coords_kernel(const double *__restrict__ pts, int64_t n, double lo0, double lo1, double lo2,
                                 double s, float *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double lo[3] = {lo0, lo1, lo2};
    float hi[4] = {0, 0, 0, 0}, lw[4] = {0, 0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        double v = 1.0 + (pts[i * 4 + a] - lo[a]) / s;
        float h = __double2float_rn(v);
        hi[a] = h;
        lw[a] = __double2float_rn(v - (double)h);
    }
    float4 *o = reinterpret_cast<float4 *>(out + i * 8);
    o[0] = make_float4(hi[0], hi[1], hi[2], 0.f);
    o[1] = make_float4(lw[0], lw[1], lw[2], 0.f);
}

// per point: three float4 (hi, mid, lo) of x~ = x 2^-e; hi + mid + lo == x~ exactly
__global__ void dd_coords3_kernel(const double *__restrict__ pts, int64_t n, int e, float *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h[3] = {0, 0, 0}, m[3] = {0, 0, 0}, l[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        double v = ldexp(pts[i * 4 + a], -e);
        h[a] = __double2float_rn(v);
        double r = v - (double)h[a];
        m[a] = __double2float_rn(r);
        l[a] = __double2float_rn(r - (double)m[a]);
    }
    float4 *o = reinterpret_cast<float4 *>(out + i * 12);
    o[0] = make_float4(h[0], h[1], h[2], 0.f);
    o[1] = make_float4(m[0], m[1], m[2], 0.f);
    o[2] = make_float4(l[0], l[1], l[2], 0.f);
}

// (hi, lo) float pairs of FP64 values
__global__ void dd_split_kernel(const double *__restrict__ in, int64_t n, float2 *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = in[i];
    float h = __double2float_rn(v);
    out[i] = make_float2(h, __double2float_rn(v - (double)h));
}

bool dd_supported(int kernel_id) { return kernel_id == SMASH_K_INVR || kernel_id == SMASH_K_CAUCHY1D; }

void dd_coords(const double *pts, int64_t n, const double *lo, double s, float *out, cudaStream_t st) {
    if (n <= 0) return;
    dd_coords_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pts, n, lo[0], lo[1], lo[2], s, out);
    LAUNCHED();
}

void dd_coords3(const double *pts, int64_t n, int e, float *out, cudaStream_t st) {
    if (n <= 0) return;
    dd_coords3_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pts, n, e, out);
    LAUNCHED();
}

int dd_exact_exponent(double s) { return ilogb(s); }

static void dd_split(const double *in, int64_t n, float2 *out, cudaStream_t st) {
    if (n <= 0) return;
    dd_split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, n, out);
    LAUNCHED();
}

// ------------------------------------------------------------------ kernel sums
struct KsumDDArgs {
    const int32_t *tnodes;
    const int64_t *t_off;
    const int32_t *t_cnt;
    const int64_t *ptr;
    const int32_t *col;
    const int64_t *s_off;
    const int32_t *s_cnt;
    const float *xt;   // target coordinates, 8 floats per point
    const float *ys;   // source coordinates, 8 floats per point
    const float2 *qv;  // source vectors as (hi, lo), ldq per point
    double *out;       // target vectors (FP64), ldq
    double scale;      // 1/s
    int ldq, nchunks, tbp, groups;
    int tile;          // source points staged per round (at least; <= tile_cap)
    int tile_cap;      // shared-memory capacity in sources (the layout's stride)
    const int *only;   // if set, CTA i runs only when only[i] != 0
};

constexpr int kDdThreads = 256;
constexpr int kDdTile = 128;
constexpr int kDdTileMax = 256;

// Up to 16 RHS per chunk the kernel fits 80 registers, so three CTAs share an
// SM and hide the latencies of the dependent double-float chains; 32 RHS
// need about twice the accumulators and run at one CTA per SM.
template <int KID, int D, int RC, bool EXACT>
__global__ void __launch_bounds__(kDdThreads, RC <= 16 ? 3 : 1) ksum_dd_kernel(KsumDDArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ PartnerChunk pc;
    constexpr int NC = EXACT ? 3 : 2;                                 // float4 per point
    const int cap = a.tile_cap;
    float4 *sy = reinterpret_cast<float4 *>(smraw);                  // cap * NC
    float2 *sq = reinterpret_cast<float2 *>(sy + NC * cap);          // cap * ldq
    double *red = reinterpret_cast<double *>(sq + (size_t)cap * a.ldq);  // tbp * ldq
    int64_t *sidx = reinterpret_cast<int64_t *>(red + (size_t)a.tbp * a.ldq);  // cap

    if (a.only && !a.only[blockIdx.x]) return;
    const int64_t g = a.tnodes[blockIdx.x];
    const int T = a.t_cnt[g];
    if (T == 0) return;
    const int64_t toff = a.t_off[g];
    const int64_t e0 = a.ptr[g], e1 = a.ptr[g + 1];
    const int ldq = a.ldq;
    const int tid = threadIdx.x;
    // targets per thread block row: T itself (at most a.tbp), so that no lane
    // of a group idles, but at least 16 lanes per group (at most 16 groups to
    // reduce); the remaining threads split the sources into groups
    const int tbp = min(max(T, (16 + a.nchunks - 1) / a.nchunks), a.tbp);
    const int groups = kDdThreads / (tbp * a.nchunks);
    const int per_group = tbp * a.nchunks;
    const int grp = tid / per_group;
    const int lt = tid % per_group;
    const int ta = lt % tbp;
    const int ch = lt / tbp;
    const bool active = grp < groups;
    // sources per round: at least a.tile, and enough that each source group
    // takes 32 of them between two barriers (small target blocks have many groups)
    const int tile = max(a.tile, min(cap, 32 * groups));

    for (int tb = 0; tb < T; tb += tbp) {
        const int tcount = min(tbp, T - tb);
        const bool have = active && ta < tcount;
        float4 xc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) xc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (have) {
            const float4 *xp = reinterpret_cast<const float4 *>(a.xt + (toff + tb + ta) * (4 * NC));
#pragma unroll
            for (int c = 0; c < NC; ++c) xc[c] = xp[c];
        }
        float ah[RC], al[RC];
#pragma unroll
        for (int r = 0; r < RC; ++r) { ah[r] = 0.f; al[r] = 0.f; }
        for (int64_t e = e0; e < e1;) {
            load_partner_chunk<kDdThreads>(pc, e, e1, a.col, a.s_off, a.s_cnt);
            const int nchunk = pc.n, total = pc.pre[pc.n];
            e += nchunk;
            for (int pos = 0; pos < total; pos += tile) {
            const int fill = min(tile, total - pos);
            for (int q = tid; q < fill; q += kDdThreads) sidx[q] = chunk_source(pc, pos + q);
            __syncthreads();
            for (int q = tid; q < fill * NC; q += kDdThreads) {
                int b = q / NC, c = q % NC;
                sy[c * tile + b] = reinterpret_cast<const float4 *>(a.ys + sidx[b] * (4 * NC))[c];
            }
            for (int q = tid; q < fill * ldq; q += kDdThreads) {
                int b = q / ldq, c = q % ldq;
                sq[q] = a.qv[sidx[b] * ldq + c];
            }
            __syncthreads();
            if (have) {
                for (int b = grp; b < fill; b += groups) {
                    float dh[3], dl[3];
                    if (EXACT) {
                        float4 yh = sy[b], ym = sy[tile + b], yl = sy[2 * tile + b];
                        diff3(xc[0].x, xc[1].x, xc[2 % NC].x, yh.x, ym.x, yl.x, dh[0], dl[0]);
                        diff3(xc[0].y, xc[1].y, xc[2 % NC].y, yh.y, ym.y, yl.y, dh[1], dl[1]);
                        diff3(xc[0].z, xc[1].z, xc[2 % NC].z, yh.z, ym.z, yl.z, dh[2], dl[2]);
                    } else {
                        float4 yh = sy[b], yl = sy[tile + b];
                        dh[0] = xc[0].x - yh.x; dh[1] = xc[0].y - yh.y; dh[2] = xc[0].z - yh.z;
                        dl[0] = xc[1].x - yl.x; dl[1] = xc[1].y - yl.y; dl[2] = xc[1].z - yl.z;
                    }
                    float kh, kl;
                    kappa_dd<KID, D>(dh, dl, kh, kl);
                    const float2 *qb = sq + (size_t)b * ldq + ch * RC;
                    float2 qv[RC];
                    if (RC >= 2) {
#pragma unroll
                        for (int r = 0; r < RC; r += 2) {
                            float4 v = *reinterpret_cast<const float4 *>(qb + r);
                            qv[r] = make_float2(v.x, v.y);
                            qv[r + 1] = make_float2(v.z, v.w);
                        }
                    } else {
                        qv[0] = qb[0];
                    }
#pragma unroll
                    for (int r = 0; r < RC; ++r) {
                        float2 qq = qv[r];
                        float p = kh * qq.x;
                        float pe = fmaf(kh, qq.x, -p);
                        pe = fmaf(kh, qq.y, pe);
                        pe = fmaf(kl, qq.x, pe);
                        float s, t;
                        two_sum_ordered(ah[r], p, s, t);
                        ah[r] = s;
                        al[r] = al[r] + (t + pe);
                    }
                }
#pragma unroll
                for (int r = 0; r < RC; ++r) fast_two_sum(ah[r], al[r], ah[r], al[r]);
            }
            __syncthreads();
            }
        }
        for (int gg = 0; gg < groups; ++gg) {
            if (have && grp == gg) {
#pragma unroll
                for (int r = 0; r < RC; ++r) {
                    double v = (double)ah[r] + (double)al[r];
                    double *dst = red + (size_t)ta * ldq + ch * RC + r;
                    *dst = gg == 0 ? v : *dst + v;
                }
            }
            __syncthreads();
        }
        for (int q = tid; q < tcount * ldq; q += kDdThreads) a.out[(toff + tb) * ldq + q] = red[q] * a.scale;
        __syncthreads();
    }
}

template <int KID, int D, bool EXACT>
static void launch_dd(KsumDDArgs a, int64_t ntn, int RC, cudaStream_t s) {
    if (ntn <= 0) return;
    constexpr int NC = EXACT ? 3 : 2;
    auto bytes = [&](int cap) {
        return sizeof(float4) * NC * cap + sizeof(float2) * (size_t)cap * a.ldq + sizeof(double) * (size_t)a.tbp * a.ldq +
               sizeof(int64_t) * cap;
    };
    // room for the larger rounds of small target blocks while two CTAs fit per SM
    a.tile_cap = bytes(kDdTileMax) <= 96 * 1024 ? std::max(a.tile, kDdTileMax) : a.tile;
    size_t smem = bytes(a.tile_cap);
    void (*kern)(KsumDDArgs) = nullptr;
    switch (RC) {
    case 1: kern = ksum_dd_kernel<KID, D, 1, EXACT>; break;
    case 2: kern = ksum_dd_kernel<KID, D, 2, EXACT>; break;
    case 4: kern = ksum_dd_kernel<KID, D, 4, EXACT>; break;
    case 8: kern = ksum_dd_kernel<KID, D, 8, EXACT>; break;
    case 16: kern = ksum_dd_kernel<KID, D, 16, EXACT>; break;
    default: kern = ksum_dd_kernel<KID, D, 32, EXACT>; break;
    }
    allow_max_dynamic_smem((const void *)kern);
    kern<<<(unsigned)ntn, kDdThreads, smem, s>>>(a);
    LAUNCHED();
}

template <bool EXACT>
static void ksum_dd_dispatch(int kid, int dim, KsumDDArgs a, int64_t ntn, int RC, cudaStream_t s) {
    if (kid == SMASH_K_CAUCHY1D) {
        launch_dd<SMASH_K_CAUCHY1D, 1, EXACT>(a, ntn, RC, s);
    } else if (dim == 3) {
        launch_dd<SMASH_K_INVR, 3, EXACT>(a, ntn, RC, s);
    } else if (dim == 2) {
        launch_dd<SMASH_K_INVR, 2, EXACT>(a, ntn, RC, s);
    } else {
        launch_dd<SMASH_K_INVR, 1, EXACT>(a, ntn, RC, s);
    }
}

// Tuned shape: bit 0 halves the source tile, bit 1 halves the cap of the
// target block (more source groups per target).  `untuned` launches the
// default shape (a launch filtered by `only` would time unrepresentatively).
static void ksum_dd(const smash_h2 *h, int kid, bool exact, KsumDDArgs a, int64_t ntn, int max_targets, int RC,
                    cudaStream_t s, bool untuned = false) {
    const int dim = h->dim;
    a.nchunks = a.ldq / RC;
    int tbp = 32;
    while (tbp < max_targets && tbp * 2 * a.nchunks <= kDdThreads) tbp *= 2;
    if (tbp * a.nchunks > kDdThreads) tbp = std::max(1, kDdThreads / a.nchunks);
    std::vector<int> cands = {0, 1};
    if (tbp >= 64) { cands.push_back(2); cands.push_back(3); }
    auto run = [&](int c) {
        KsumDDArgs b = a;
        b.tile = (c & 1) ? kDdTile / 2 : kDdTile;
        b.tbp = (c & 2) ? tbp / 2 : tbp;
        b.groups = std::max(1, kDdThreads / (b.tbp * b.nchunks));
        if (exact)
            ksum_dd_dispatch<true>(kid, dim, b, ntn, RC, s);
        else
            ksum_dd_dispatch<false>(kid, dim, b, ntn, RC, s);
    };
    if (untuned) {
        run(0);
        return;
    }
    char key[160];
    std::snprintf(key, sizeof(key), "ksum_dd/sm%d/k%d/d%d/x%d/rc%d/ld%d/t%lld/n%lld", h->num_sms, kid, dim,
                  exact ? 1 : 0, RC, a.ldq, pow2_at_least(max_targets), pow2_at_least(ntn));
    tune_choose(key, cands, 0, s, run);
}

// ------------------------------------------------------------------ transfers (double-float)
// The upward and downward passes of Section 3.4 with the products of G in
// double-float on the FP32 pipe: 2 nrhs FP64 flops per 8-byte G entry would
// keep them on the FP64 pipe.  One CTA per node; rows of G are split into
// (hi, lo) pairs once per CTA in shared memory, kTrRows at a time.
constexpr int kTrThreads = 256;
constexpr int kTrRows = 32;

struct PassDDArgs {
    int64_t n0;
    const int32_t *leaf, *m, *k;
    const int64_t *in_off, *sk_off, *loc_off, *g_off;
    const int32_t *loc;
    const double *G;
    const float2 *pts2;  // upward: leaf inputs (sorted points, ldq)
    float2 *skel2;       // upward: q^ as (hi, lo) (children read, the node written)
    double *skel64;      // upward: q^ in FP64 (written); downward: z^ (the node read, children +=)
    double *pts_out;     // downward: zs of the leaves (+=)
    int ldq;
};

__device__ __forceinline__ float2 split_f64(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}

// (sh, sl) += (gh + gl)(x.x + x.y): the product hi * hi exact by FMA, cross
// terms rounded into the error term, the running sum by error-free Fast2Sum
__device__ __forceinline__ void dd_mac(float gh, float gl, float2 x, float &sh, float &sl) {
    const float p = gh * x.x;
    float pe = fmaf(gh, x.x, -p);
    pe = fmaf(gh, x.y, pe);
    pe = fmaf(gl, x.x, pe);
    float s, t;
    two_sum_ordered(sh, p, s, t);
    sh = s;
    sl = sl + (t + pe);
}

// q^_i[t] = x[skel_t] + sum_u G[u][t] x[rest_u],  x = q|_i (leaf) or [q^_c] (parent)
__global__ void __launch_bounds__(kTrThreads) upward_dd_kernel(PassDDArgs a) {
    extern __shared__ float2 sG[];  // kTrRows x k
    const int64_t g = a.n0 + blockIdx.x;
    const int m = a.m[g], k = a.k[g];
    if (k == 0) return;
    const int ldq = a.ldq, mk = m - k;
    const float2 *in = a.leaf[g] ? a.pts2 + a.in_off[g] * ldq : a.skel2 + a.in_off[g] * ldq;
    const int32_t *loc = a.loc + a.loc_off[g];
    const double *G = a.G + a.g_off[g];
    float2 *out2 = a.skel2 + a.sk_off[g] * ldq;
    double *out64 = a.skel64 + a.sk_off[g] * ldq;
    const int nout = k * ldq;
    const int tid = threadIdx.x;
    for (int b0 = 0; b0 < nout; b0 += 4 * kTrThreads) {
        float sh[4], sl[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = b0 + j * kTrThreads + tid;
            sh[j] = 0.f;
            sl[j] = 0.f;
            if (e < nout) {
                const float2 x = in[(int64_t)loc[e / ldq] * ldq + e % ldq];
                sh[j] = x.x;
                sl[j] = x.y;
            }
        }
        for (int u0 = 0; u0 < mk; u0 += kTrRows) {
            const int rows = min(kTrRows, mk - u0);
            __syncthreads();  // the previous rows are consumed
            for (int q = tid; q < rows * k; q += kTrThreads) sG[q] = split_f64(G[(int64_t)u0 * k + q]);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int e = b0 + j * kTrThreads + tid;
                if (e < nout) {
                    const int t = e / ldq, c = e % ldq;
                    for (int u = 0; u < rows; ++u) {
                        const float2 gg = sG[u * k + t];
                        dd_mac(gg.x, gg.y, in[(int64_t)loc[k + u0 + u] * ldq + c], sh[j], sl[j]);
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = b0 + j * kTrThreads + tid;
            if (e < nout) {
                float h, l;
                fast_two_sum(sh[j], sl[j], h, l);
                out2[e] = make_float2(h, l);
                out64[e] = (double)h + (double)l;
            }
        }
    }
}

// out[skel_t] += z^_i[t];  out[rest_u] += sum_t G[u][t] z^_i[t] (the sum in double-float)
__global__ void __launch_bounds__(kTrThreads) downward_dd_kernel(PassDDArgs a) {
    extern __shared__ float2 smem2[];
    const int64_t g = a.n0 + blockIdx.x;
    const int m = a.m[g], k = a.k[g];
    if (k == 0) return;
    const int ldq = a.ldq, mk = m - k;
    const double *zin = a.skel64 + a.sk_off[g] * ldq;
    double *out = a.leaf[g] ? a.pts_out + a.in_off[g] * ldq : a.skel64 + a.in_off[g] * ldq;
    const int32_t *loc = a.loc + a.loc_off[g];
    const double *G = a.G + a.g_off[g];
    float2 *sz = smem2;            // k x ldq
    float2 *sG = smem2 + k * ldq;  // kTrRows x k
    const int tid = threadIdx.x;
    for (int e = tid; e < k * ldq; e += kTrThreads) {
        const double v = zin[e];
        sz[e] = split_f64(v);
        out[(int64_t)loc[e / ldq] * ldq + e % ldq] += v;
    }
    for (int r0 = 0; r0 < mk; r0 += kTrRows) {
        const int rows = min(kTrRows, mk - r0);
        __syncthreads();  // sz is staged; the previous rows are consumed
        for (int q = tid; q < rows * k; q += kTrThreads) sG[q] = split_f64(G[(int64_t)r0 * k + q]);
        __syncthreads();
        for (int e = tid; e < rows * ldq; e += kTrThreads) {
            const int rr = e / ldq, c = e % ldq;
            float sh = 0.f, sl = 0.f;
            for (int t = 0; t < k; ++t) {
                const float2 gg = sG[rr * k + t];
                dd_mac(gg.x, gg.y, sz[t * ldq + c], sh, sl);
            }
            out[(int64_t)loc[k + r0 + rr] * ldq + c] += (double)sh + (double)sl;
        }
    }
}

static void matvec_upward_dd(const smash_h2 *h, const float2 *qs2, float2 *qhat2, double *qhat, int ldq,
                             cudaStream_t s) {
    const Side &Cs = *h->col;
    const size_t smem = sizeof(float2) * kTrRows * (size_t)std::max(h->r, 1);
    allow_max_dynamic_smem((const void *)upward_dd_kernel);
    for (int l = h->L; l >= 2; --l) {
        const int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        PassDDArgs p{n0, h->leaf, Cs.m, Cs.k, Cs.in_off, Cs.sk_off, Cs.loc_off, Cs.g_off, Cs.loc, Cs.G,
                     qs2, qhat2, qhat, nullptr, ldq};
        upward_dd_kernel<<<(unsigned)nl, kTrThreads, smem, s>>>(p);
        LAUNCHED();
    }
}

static void matvec_downward_dd(const smash_h2 *h, double *zhat, double *zs, int ldq, cudaStream_t s) {
    const Side &R = h->row;
    const size_t kmax = (size_t)std::max(h->r, 1);
    const size_t smem = sizeof(float2) * (kmax * ldq + kTrRows * kmax);
    allow_max_dynamic_smem((const void *)downward_dd_kernel);
    for (int l = 2; l <= h->L; ++l) {
        const int64_t n0 = h->lvl_off[l - 1], nl = h->lvl_off[l] - n0;
        PassDDArgs p{n0, h->leaf, R.m, R.k, R.in_off, R.sk_off, R.loc_off, R.g_off, R.loc, R.G,
                     nullptr, nullptr, zhat, zs, ldq};
        downward_dd_kernel<<<(unsigned)nl, kTrThreads, smem, s>>>(p);
        LAUNCHED();
    }
}

void matvec_dd(const smash_h2 *h, const double *X, double *Y, int nrhs, cudaStream_t s, Profile *prof, int kid) {
    const Side &R = h->row;
    const Side &Cs = *h->col;
    int ldq, RC;
    if (nrhs <= 32) {
        RC = 1;
        while (RC < nrhs) RC *= 2;
        ldq = RC;
    } else {
        RC = 32;
        ldq = (nrhs + 31) / 32 * 32;
    }
    Arena tmp(s);
    double *qs = tmp.alloc<double>((size_t)h->ny * ldq);
    double *zs = tmp.alloc<double>((size_t)h->nx * ldq);
    double *qhat = tmp.alloc<double>((size_t)std::max<int64_t>(Cs.total_skel, 1) * ldq);
    double *zhat = tmp.alloc<double>((size_t)std::max<int64_t>(R.total_skel, 1) * ldq);
    float2 *qs2 = tmp.alloc<float2>((size_t)h->ny * ldq);
    float2 *qhat2 = tmp.alloc<float2>((size_t)std::max<int64_t>(Cs.total_skel, 1) * ldq);
    const double scale = 1.0 / h->s;
    PhaseTimer tm(s, prof);
    tm.mark();
    matvec_gather(h, X, nrhs, ldq, qs, s);
    dd_split(qs, h->ny * ldq, qs2, s);
    tm.mark();
    {
        // the near field: digit-split products on the tensor cores where the
        // node allows it (the rest by the double-float kernel), else all in
        // double-float on the FP32 pipe; the tuner may take either
        KsumDDArgs a{};
        a.tnodes = h->leaf_list; a.t_off = h->rs; a.t_cnt = h->rc;
        a.ptr = h->near_ptr; a.col = h->near_col; a.s_off = h->cs; a.s_cnt = h->cc;
        a.xt = h->xs_x3; a.ys = h->ys_x3; a.qv = qs2; a.out = zs; a.scale = ldexp(1.0, -h->dd_e); a.ldq = ldq;
        const int max_t = (int)std::min<int64_t>(h->leaf_size, 256);
        if (near_oz_supported(h, kid, ldq)) {
            int *fallback = tmp.alloc<int>((size_t)std::max<int64_t>(h->nleaves, 1));
            char key[128];
            std::snprintf(key, sizeof(key), "near_dd/sm%d/k%d/d%d/ld%d/n%lld", h->num_sms, kid, h->dim, ldq,
                          pow2_at_least(h->nleaves));
            tune_choose(key, {0, 1}, ldq >= 8 ? 0 : 1, s, [&](int c) {
                if (c == 0) {
                    near_oz(h, kid, qs, zs, ldq, fallback, s);
                    KsumDDArgs b = a;
                    b.only = fallback;
                    ksum_dd(h, kid, true, b, h->nleaves, max_t, RC, s, true);
                } else {
                    ksum_dd(h, kid, true, a, h->nleaves, max_t, RC, s);
                }
            });
        } else {
            ksum_dd(h, kid, true, a, h->nleaves, max_t, RC, s);
        }
    }
    tm.mark();
    matvec_upward_dd(h, qs2, qhat2, qhat, ldq, s);
    tm.mark();
    // the coupling: products on the tensor cores (exact digit splits) where
    // the tree allows it, else every operation in double-float on the FP32
    // pipe; the tuner may take either.  Untuned, the digit split is the
    // default from 8 columns per pass: its entry and digit work (~90
    // instructions per entry) is fixed, while the FP32-pipe products cost 12
    // instructions per column.
    auto dd_coupling = [&] {
        KsumDDArgs a{};
        a.tnodes = h->nonroot_list; a.t_off = R.sk_off; a.t_cnt = R.k;
        a.ptr = h->adm_ptr; a.col = h->adm_col; a.s_off = Cs.sk_off; a.s_cnt = Cs.k;
        const bool exact = dd_exact_coupling(h);
        a.xt = exact ? R.skel_x3 : R.skel_dd;
        a.ys = exact ? Cs.skel_x3 : Cs.skel_dd;
        a.qv = qhat2; a.out = zhat; a.scale = exact ? ldexp(1.0, -h->dd_e) : scale; a.ldq = ldq;
        ksum_dd(h, kid, exact, a, h->nnodes - h->nroots, h->r, RC, s);
    };
    if (h->nnodes > h->nroots) {
        if (coupling_oz_supported(h, kid, ldq)) {
            char key[128];
            std::snprintf(key, sizeof(key), "coupling_dd/sm%d/k%d/d%d/ld%d/n%lld", h->num_sms, kid, h->dim, ldq,
                          pow2_at_least(h->nnodes));
            tune_choose(key, {0, 1, 2}, ldq >= 8 ? 0 : 1, s, [&](int c) {
                if (c == 0) coupling_oz(h, kid, qhat, zhat, ldq, s);
                else if (c == 2) coupling_oz(h, kid, qhat, zhat, ldq, s, true);
                else dd_coupling();
            });
        } else {
            dd_coupling();
        }
    }
    tm.mark();
    matvec_downward_dd(h, zhat, zs, ldq, s);
    tm.mark();
    matvec_scatter(h, zs, ldq, nrhs, Y, s);
    tm.mark();
    tm.finish(4);
    tmp.release();
}

}  // namespace smash
