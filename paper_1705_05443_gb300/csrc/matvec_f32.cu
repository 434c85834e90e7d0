// matvec_f32.cu -- the Section 3.4 matvec with the coupling (3.19) and the
// near field (3.20) in FP32 (SMASH_PREC_F32, the mixed-precision mode).
//
//  * Differences come from the normalised two-float coordinates
//    x'' = 1 + (x - lo)/s in [1, 2): (hi_a - hi_b) is exact (Sterbenz) and
//    (lo_a - lo_b) restores the low bits, so a difference is accurate to
//    ~2^-47 in absolute terms before it is rounded to FP32.  That is below
//    half an FP32 ulp of the difference for pairs at least 2^-22 apart (in
//    units of the cube side).  The near field meets closer pairs too (the
//    interlaced points of Section 6.3 lie 1e-7 U(0,1) apart): for a pair
//    closer than 2^-22 it recomputes the difference from the exact
//    three-float coordinates with an error-free sum, so every entry keeps
//    FP32 accuracy.
//  * The kernel entry, the products and the sums are FP32 (relative error of
//    an entry ~1e-7).  The coupling accumulates in FP32; the near field, whose
//    closest pairs dominate their rows, accumulates with Kahan's compensated
//    summation.  Sums are written out in FP64; the upward and downward
//    passes stay FP64.
//  * Kernels in the normalised frame: 1/|x-y| = (1/s) / |d''|, 1/(x-y) =
//    (1/s) / d'', log|x-y| = log s + log|d''|, exp(-|x-y|)/|x-y| with
//    |x-y| = s |d''|.
#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "kappa_f32.cuh"
#include "ksum_tiles.cuh"

namespace smash {

struct KsumF32Args {
    const int32_t *tnodes;
    const int64_t *t_off;
    const int32_t *t_cnt;
    const int64_t *ptr;
    const int32_t *col;
    const int64_t *s_off;
    const int32_t *s_cnt;
    const float *xt;   // normalised two-float coordinates, 8 floats per point
    const float *ys;
    const float *xt3;  // exact three-float coordinates x 2^-e, 12 floats per point (near field)
    const float *ys3;
    float x3_norm;     // 2^e / s: a difference in the three-float frame times this is normalised
    const float *qv;   // source vectors, FP32, ldq per point
    double *out;       // target vectors (FP64), ldq
    double scale;      // multiplies the sums (1/s for 1/r and 1/(x-y), else 1)
    float s_f;         // s, for the Yukawa kernel
    float inv_s;       // 1/s, for the Yukawa kernel
    float log_s;       // log s, for the log kernel
    int ldq, nchunks, tbp;
    int tile;          // source points staged per round (<= kF32Tile)
};

constexpr int kF32Threads = 256;
constexpr int kF32Tile = 256;

// x - y, normalised, from the exact three-float coordinates of a close pair:
// the hi parts differ exactly (Sterbenz), the mid parts by an error-free
// TwoSum, the lo parts (below 2^-48 of the coordinate) by a rounded
// difference; the parts are then added from the smallest up and rounded once
// more by the normalisation.
template <int D>
__device__ __forceinline__ void exact_diff3(const float *x3, const float *y3, float norm, float *d) {
    const float4 xh = reinterpret_cast<const float4 *>(x3)[0], xm = reinterpret_cast<const float4 *>(x3)[1],
                 xl = reinterpret_cast<const float4 *>(x3)[2];
    const float4 yh = reinterpret_cast<const float4 *>(y3)[0], ym = reinterpret_cast<const float4 *>(y3)[1],
                 yl = reinterpret_cast<const float4 *>(y3)[2];
    const float h[3] = {xh.x - yh.x, xh.y - yh.y, xh.z - yh.z};
    const float am[3] = {xm.x, xm.y, xm.z}, bm[3] = {-ym.x, -ym.y, -ym.z};
    const float l[3] = {xl.x - yl.x, xl.y - yl.y, xl.z - yl.z};
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const float sm = am[c] + bm[c];
        const float bb = sm - am[c];
        const float err = (am[c] - (sm - bb)) + (bm[c] - bb);
        d[c] = ((h[c] + sm) + (err + l[c])) * norm;
    }
}

// One thread: TA targets x RC right-hand sides; the right-hand sides of a
// source are read from shared memory as float4 (RC >= 4) and reused by the
// TA targets.
template <int KID, int D, int RC, bool KAHAN, int TA>
__global__ void __launch_bounds__(kF32Threads, (KAHAN && RC >= 32) || (!KAHAN && RC == 16) ? 2 : 3) ksum_f32_kernel(KsumF32Args a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ PartnerChunk pc;
    const int tile = a.tile;                                      // <= kF32Tile
    float4 *syh = reinterpret_cast<float4 *>(smraw);             // tile
    float4 *syl = syh + tile;                                     // tile
    float *sq = reinterpret_cast<float *>(syl + tile);            // tile * ldq
    double *red = reinterpret_cast<double *>(sq + (size_t)tile * a.ldq);  // TA * tbp * ldq
    int64_t *sidx = reinterpret_cast<int64_t *>(red + (size_t)TA * a.tbp * a.ldq);

    const int64_t g = a.tnodes[blockIdx.x];
    const int T = a.t_cnt[g];
    if (T == 0) return;
    const int64_t toff = a.t_off[g];
    const int64_t e0 = a.ptr[g], e1 = a.ptr[g + 1];
    const int ldq = a.ldq;
    const int tid = threadIdx.x;
    // thread rows, each covering TA targets: as many as T needs (at most a.tbp,
    // at least 16 lanes per group)
    const int tbp = min(max((T + TA - 1) / TA, (16 + a.nchunks - 1) / a.nchunks), a.tbp);
    const int groups = kF32Threads / (tbp * a.nchunks);
    const int per_group = tbp * a.nchunks;
    const int grp = tid / per_group;
    const int lt = tid % per_group;
    const int ta = lt % tbp;
    const int ch = lt / tbp;
    const bool active = grp < groups;
    const int span = TA * tbp;

    for (int tb = 0; tb < T; tb += span) {
        const int tcount = min(span, T - tb);
        bool have[TA];
        float4 xh[TA], xl[TA];
#pragma unroll
        for (int u = 0; u < TA; ++u) {
            have[u] = active && ta + u * tbp < tcount;
            xh[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            xl[u] = xh[u];
            if (have[u]) {
                const float4 *xp = reinterpret_cast<const float4 *>(a.xt + (toff + tb + ta + u * tbp) * 8);
                xh[u] = xp[0];
                xl[u] = xp[1];
            }
        }
        const bool any = have[0];
        float acc[TA][RC], cmp[TA][RC];
#pragma unroll
        for (int u = 0; u < TA; ++u)
#pragma unroll
            for (int r = 0; r < RC; ++r) { acc[u][r] = 0.f; cmp[u][r] = 0.f; }
        for (int64_t e = e0; e < e1;) {
            load_partner_chunk<kF32Threads>(pc, e, e1, a.col, a.s_off, a.s_cnt);
            const int nchunk = pc.n, total = pc.pre[pc.n];
            e += nchunk;
            for (int pos = 0; pos < total; pos += tile) {
            const int fill = min(tile, total - pos);
            for (int q = tid; q < fill; q += kF32Threads) sidx[q] = chunk_source(pc, pos + q);
            __syncthreads();
            for (int q = tid; q < fill; q += kF32Threads) {
                const float4 *yp = reinterpret_cast<const float4 *>(a.ys + sidx[q] * 8);
                syh[q] = yp[0];
                syl[q] = yp[1];
            }
            for (int q = tid; q < fill * ldq; q += kF32Threads) {
                int b = q / ldq, c = q % ldq;
                sq[q] = a.qv[sidx[b] * ldq + c];
            }
            __syncthreads();
            if (any) {
                for (int b = grp; b < fill; b += groups) {
                    float4 yh = syh[b], yl = syl[b];
                    float kv[TA];
#pragma unroll
                    for (int u = 0; u < TA; ++u) {
                        float d[3] = {(xh[u].x - yh.x) + (xl[u].x - yl.x), (xh[u].y - yh.y) + (xl[u].y - yl.y),
                                      (xh[u].z - yh.z) + (xl[u].z - yl.z)};
                        if (KAHAN && have[u]) {
                            float r2 = d[0] * d[0];
                            if (D > 1) r2 = fmaf(d[1], d[1], r2);
                            if (D > 2) r2 = fmaf(d[2], d[2], r2);
                            if (r2 < 0x1p-44f)
                                exact_diff3<D>(a.xt3 + (toff + tb + ta + u * tbp) * 12, a.ys3 + sidx[b] * 12,
                                               a.x3_norm, d);
                        }
                        kv[u] = have[u] ? kappa_f32<KID, D>(d, a.s_f, a.inv_s, a.log_s) : 0.f;
                    }
                    const float *qb = sq + (size_t)b * ldq + ch * RC;
                    constexpr int VW = RC >= 4 ? 4 : 1;  // vector width of the loads
#pragma unroll
                    for (int r0 = 0; r0 < RC; r0 += VW) {
                        float qv[VW];
                        if (VW == 4) {
                            float4 v = *reinterpret_cast<const float4 *>(qb + r0);
                            qv[0] = v.x; qv[VW > 1 ? 1 : 0] = v.y; qv[VW > 2 ? 2 : 0] = v.z; qv[VW > 3 ? 3 : 0] = v.w;
                        } else {
                            qv[0] = qb[r0];
                        }
#pragma unroll
                        for (int u = 0; u < TA; ++u)
#pragma unroll
                            for (int i = 0; i < VW; ++i) {
                                const int r = r0 + i;
                                if (KAHAN) {
                                    float y = fmaf(kv[u], qv[i], -cmp[u][r]);
                                    float t = acc[u][r] + y;
                                    cmp[u][r] = (t - acc[u][r]) - y;
                                    acc[u][r] = t;
                                } else {
                                    acc[u][r] = fmaf(kv[u], qv[i], acc[u][r]);
                                }
                            }
                    }
                }
            }
            __syncthreads();
            }
        }
        for (int gg = 0; gg < groups; ++gg) {
            if (grp == gg) {
#pragma unroll
                for (int u = 0; u < TA; ++u) {
                    if (!have[u]) continue;
#pragma unroll
                    for (int r = 0; r < RC; ++r) {
                        double v = KAHAN ? (double)acc[u][r] - (double)cmp[u][r] : (double)acc[u][r];
                        double *dst = red + (size_t)(ta + u * tbp) * ldq + ch * RC + r;
                        *dst = gg == 0 ? v : *dst + v;
                    }
                }
            }
            __syncthreads();
        }
        for (int q = tid; q < tcount * ldq; q += kF32Threads) a.out[(toff + tb) * ldq + q] = red[q] * a.scale;
        __syncthreads();
    }
}

template <int KID, int D, bool KAHAN>
static void launch_f32(KsumF32Args a, int64_t ntn, int RC, cudaStream_t s) {
    if (ntn <= 0) return;
    // two targets per thread where the registers allow it (RC <= 16, no compensation)
    const int TA = (KAHAN || RC > 16) ? 1 : 2;
    size_t smem = sizeof(float4) * 2 * a.tile + sizeof(float) * (size_t)a.tile * a.ldq +
                  sizeof(double) * (size_t)TA * a.tbp * a.ldq + sizeof(int64_t) * a.tile;
    void (*kern)(KsumF32Args) = nullptr;
    constexpr int T2 = KAHAN ? 1 : 2;
    switch (RC) {
    case 1: kern = ksum_f32_kernel<KID, D, 1, KAHAN, T2>; break;
    case 2: kern = ksum_f32_kernel<KID, D, 2, KAHAN, T2>; break;
    case 4: kern = ksum_f32_kernel<KID, D, 4, KAHAN, T2>; break;
    case 8: kern = ksum_f32_kernel<KID, D, 8, KAHAN, T2>; break;
    case 16: kern = ksum_f32_kernel<KID, D, 16, KAHAN, T2>; break;
    default: kern = ksum_f32_kernel<KID, D, 32, KAHAN, 1>; break;
    }
    allow_max_dynamic_smem((const void *)kern);
    kern<<<(unsigned)ntn, kF32Threads, smem, s>>>(a);
    LAUNCHED();
}

template <bool KAHAN>
static void dispatch_f32(int kid, int dim, KsumF32Args a, int64_t ntn, int RC, cudaStream_t s) {
    switch (kid) {
    case SMASH_K_CAUCHY1D: launch_f32<SMASH_K_CAUCHY1D, 1, KAHAN>(a, ntn, RC, s); return;
    case SMASH_K_DLP1: launch_f32<SMASH_K_DLP1, 2, KAHAN>(a, ntn, RC, s); return;  // dim == 2
    case SMASH_K_DLP2: launch_f32<SMASH_K_DLP2, 2, KAHAN>(a, ntn, RC, s); return;
    case SMASH_K_LOG:
        if (dim == 3) launch_f32<SMASH_K_LOG, 3, KAHAN>(a, ntn, RC, s);
        else if (dim == 2) launch_f32<SMASH_K_LOG, 2, KAHAN>(a, ntn, RC, s);
        else launch_f32<SMASH_K_LOG, 1, KAHAN>(a, ntn, RC, s);
        return;
    case SMASH_K_INVR:
        if (dim == 3) launch_f32<SMASH_K_INVR, 3, KAHAN>(a, ntn, RC, s);
        else if (dim == 2) launch_f32<SMASH_K_INVR, 2, KAHAN>(a, ntn, RC, s);
        else launch_f32<SMASH_K_INVR, 1, KAHAN>(a, ntn, RC, s);
        return;
    default:
        if (dim == 3) launch_f32<SMASH_K_YUKAWA, 3, KAHAN>(a, ntn, RC, s);
        else if (dim == 2) launch_f32<SMASH_K_YUKAWA, 2, KAHAN>(a, ntn, RC, s);
        else launch_f32<SMASH_K_YUKAWA, 1, KAHAN>(a, ntn, RC, s);
        return;
    }
}

static void ksum_f32(const smash_h2 *h, int kid, bool kahan, KsumF32Args a, int64_t ntn, int max_targets, int RC,
                     cudaStream_t s) {
    a.nchunks = a.ldq / RC;
    int tbp = 32;
    while (tbp < max_targets && tbp * 2 * a.nchunks <= kF32Threads) tbp *= 2;
    if (tbp * a.nchunks > kF32Threads) tbp = std::max(1, kF32Threads / a.nchunks);
    const bool mult = kid == SMASH_K_INVR || kid == SMASH_K_CAUCHY1D || kid == SMASH_K_DLP1 || kid == SMASH_K_DLP2;
    a.scale = mult ? 1.0 / h->s : 1.0;
    a.s_f = (float)h->s;
    a.inv_s = (float)(1.0 / h->s);
    a.log_s = (float)log(h->s);
    // tuned shape: bit 0 halves the source tile, bit 1 halves the target block cap
    std::vector<int> cands = {0, 1};
    if (tbp >= 64) { cands.push_back(2); cands.push_back(3); }
    auto run = [&](int c) {
        KsumF32Args b = a;
        b.tile = (c & 1) ? kF32Tile / 2 : kF32Tile;
        b.tbp = (c & 2) ? tbp / 2 : tbp;
        if (kahan)
            dispatch_f32<true>(kid, h->dim, b, ntn, RC, s);
        else
            dispatch_f32<false>(kid, h->dim, b, ntn, RC, s);
    };
    char key[160];
    std::snprintf(key, sizeof(key), "ksum_f32/sm%d/k%d/d%d/c%d/rc%d/ld%d/t%lld/n%lld", h->num_sms, kid,
                  h->dim, kahan ? 1 : 0, RC, a.ldq, pow2_at_least(max_targets), pow2_at_least(ntn));
    tune_choose(key, cands, 0, s, run);
}

__global__ void to_f32_kernel(const double *__restrict__ in, int64_t n, float *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __double2float_rn(in[i]);
}

static void to_f32(const double *in, int64_t n, float *out, cudaStream_t s) {
    if (n <= 0) return;
    to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, n, out);
    LAUNCHED();
}

void matvec_f32(const smash_h2 *h, const double *X, double *Y, int nrhs, cudaStream_t s, Profile *prof,
                int precision, int kid) {
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
    float *qs1 = tmp.alloc<float>((size_t)h->ny * ldq);
    float *qhat1 = tmp.alloc<float>((size_t)std::max<int64_t>(Cs.total_skel, 1) * ldq);
    PhaseTimer tm(s, prof);
    tm.mark();
    matvec_gather(h, X, nrhs, ldq, qs, s);
    to_f32(qs, h->ny * ldq, qs1, s);
    tm.mark();
    {
        KsumF32Args a{};
        a.tnodes = h->leaf_list; a.t_off = h->rs; a.t_cnt = h->rc;
        a.ptr = h->near_ptr; a.col = h->near_col; a.s_off = h->cs; a.s_cnt = h->cc;
        a.xt = h->xs_dd; a.ys = h->ys_dd; a.qv = qs1; a.out = zs; a.ldq = ldq;
        a.xt3 = h->xs_x3; a.ys3 = h->ys_x3; a.x3_norm = (float)(ldexp(1.0, h->dd_e) / h->s);
        ksum_f32(h, kid, true, a, h->nleaves, std::min<int64_t>(h->leaf_size, 256), RC, s);
    }
    tm.mark();
    matvec_upward(h, qs, qhat, ldq, s);
    to_f32(qhat, Cs.total_skel * ldq, qhat1, s);
    tm.mark();
    if (h->nnodes > h->nroots && precision != SMASH_PREC_F32) {
        coupling_tc(h, precision, qhat1, zhat, ldq, s, kid);
    } else if (h->nnodes > h->nroots) {
        KsumF32Args a{};
        a.tnodes = h->nonroot_list; a.t_off = R.sk_off; a.t_cnt = R.k;
        a.ptr = h->adm_ptr; a.col = h->adm_col; a.s_off = Cs.sk_off; a.s_cnt = Cs.k;
        a.xt = R.skel_dd; a.ys = Cs.skel_dd; a.qv = qhat1; a.out = zhat; a.ldq = ldq;
        ksum_f32(h, kid, false, a, h->nnodes - h->nroots, h->r, RC, s);
    }
    tm.mark();
    matvec_downward(h, zhat, zs, ldq, s);
    tm.mark();
    matvec_scatter(h, zs, ldq, nrhs, Y, s);
    tm.mark();
    tm.finish(4);
    tmp.release();
}

}  // namespace smash
