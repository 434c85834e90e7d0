// matvec_tc.cu -- the coupling (3.19) of the mixed-precision matvec with its
// products on the tensor cores (SMASH_PREC_TF32, SMASH_PREC_BF16,
// SMASH_PREC_TF32X3).
//
// For a target node i, z^_i = sum over partners j of K(x_i^, y_j^) q^_j is one
// product of a k_i x S block (S = all partner skeletons of i, as one source
// stream) with the S x nrhs block of q^.  The block is never stored: a warp
// owns 16 targets and, for every MMA step of 8 (TF32) or 16 (BF16) sources,
// each lane evaluates the kernel entries at exactly the (target, source)
// positions that the A-fragment layout of mma.m16n8k8 / m16n8k16 assigns to
// it, in FP32 from the normalised two-float coordinates, and rounds them into
// the operand registers.  q^ slabs are staged in shared memory, already
// rounded (TF32: hi and, for the split mode, lo parts; BF16: pairs along the
// source index).  Each staged tile is accumulated by the MMAs from zero and
// then added to FP32 register sums (so the tensor cores' own accumulation
// spans one tile, not the whole stream); the sums are written out in FP64
// times the frame factor.  Warps not needed for the
// targets of a node split its source stream and are reduced in a fixed order.
#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "kappa_f32.cuh"
#include "ksum_tiles.cuh"

namespace smash {

namespace {

enum { TC_TF32 = 0, TC_BF16 = 1, TC_TF32X3 = 2 };
constexpr int kTcThreads = 256;  // 8 warps
constexpr int kTcMaxTile = 256;  // sources staged per round: 64, 128 or 256 (a multiple of 16)
constexpr int kTcRows = 128;     // targets per pass: 8 warps x 16
constexpr int kTcMaxNt = 8;      // up to 64 right-hand sides (8 n-tiles of 8)
constexpr int kTcUseTcgen05 = 1; // tuning choice: the tcgen05 kernel instead of a warp-MMA tile

struct TcArgs {
    const int32_t *tnodes;
    const int64_t *t_off;
    const int32_t *t_cnt;
    const int64_t *ptr;
    const int32_t *col;
    const int64_t *s_off;
    const int32_t *s_cnt;
    const float *xt;   // normalised two-float coordinates, 8 floats per slot
    const float *ys;
    const float *qv;   // q^ in FP32, ldq per slot
    double *out;       // z^ (FP64), ldq per slot
    double scale;
    float s_f, log_s;
    float inv_s;
    int ldq;           // columns of qv / out: a power of two, or a multiple of 32 up to 64
    int ldq_log2;
    int nt;            // n-tiles of 8: ldq rounded up to 8, / 8 (1, 2, 4 or 8)
    int tile;          // sources staged per round
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// two floats as bf16x2: `first` (lower source index) in the low half
__device__ __forceinline__ uint32_t pack_bf16(float first, float second) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(second), "f"(first));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// kernel entry between a target (hi, lo) and staged source b (hi, lo float4
// at sy[2b], sy[2b + 1]); 0 when masked (a select: stale rows cannot leak)
template <int KID, int D>
__device__ __forceinline__ float entry(const float4 &xh, const float4 &xl, const float4 *sy, int b, bool ok,
                                       const TcArgs &a) {
    const float4 yh = sy[2 * b], yl = sy[2 * b + 1];
    float d[3] = {(xh.x - yh.x) + (xl.x - yl.x), (xh.y - yh.y) + (xl.y - yl.y), (xh.z - yh.z) + (xl.z - yl.z)};
    float v = kappa_f32<KID, D>(d, a.s_f, a.inv_s, a.log_s);
    return ok ? v : 0.f;
}

// shared-memory row stride (words) of the staged q^: a multiple of 4 (16-byte
// rows for cp.async) chosen so that the rows one B-fragment load touches
// (TF32: four consecutive rows; BF16: every other row) fall in distinct banks
__host__ __device__ constexpr int qstride(int nt, int mode) {
    return nt * 8 + (((mode == TC_BF16 ? 4 : 8) - (nt * 8) % 32) + 32) % 32;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Shared memory (dynamic): two staging buffers of {coordinates (two float4
// per source), raw FP32 q^ rows}, the group reduction rows and the source
// indices of the next tile.
struct TcSmem {
    float4 *sy[2];
    float *qraw[2];
    float *red;      // kTcRows x ldq8
    int64_t *sidx;   // tile
};

__host__ __device__ inline size_t tc_layout(int mode, int nt, int tile, unsigned char *base, TcSmem *L) {
    const size_t QS = (size_t)qstride(nt, mode);
    size_t off = 0;
    for (int b = 0; b < 2; ++b) {
        if (L) L->sy[b] = reinterpret_cast<float4 *>(base + off);
        off += sizeof(float4) * 2 * tile;
        if (L) L->qraw[b] = reinterpret_cast<float *>(base + off);
        off += sizeof(float) * tile * QS;
    }
    if (L) L->red = reinterpret_cast<float *>(base + off);
    off += sizeof(float) * kTcRows * nt * 8;
    if (L) L->sidx = reinterpret_cast<int64_t *>(base + off);
    off += sizeof(int64_t) * tile;
    return off;
}

// source indices of stream positions [pos, pos + fill) of the partner chunk
__device__ __forceinline__ void tc_stage_indices(const PartnerChunk &pc, int pos, int fill, int64_t *sidx) {
    for (int q = threadIdx.x; q < fill; q += kTcThreads) sidx[q] = chunk_source(pc, pos + q);
}

// gathers `fill` sources into a staging buffer by cp.async: coordinates (two
// float4 per source) and q^ rows (16-byte pieces when ldq % 4 == 0)
__device__ __forceinline__ void tc_issue(const TcArgs &a, const int64_t *sidx, int fill, int QS, float4 *sy,
                                         float *qraw) {
    for (int q = threadIdx.x; q < 2 * fill; q += kTcThreads) {
        const int sq = q >> 1, h = q & 1;
        cp_async16(sy + 2 * sq + h, a.ys + sidx[sq] * 8 + 4 * h);
    }
    if ((a.ldq & 3) == 0) {
        const int sh = a.ldq_log2 - 2;  // pieces per row = ldq / 4, a power of two
        for (int q = threadIdx.x; q < (fill << sh); q += kTcThreads) {
            const int sq = q >> sh, p4 = q & ((1 << sh) - 1);
            cp_async16(qraw + sq * QS + 4 * p4, a.qv + sidx[sq] * a.ldq + 4 * p4);
        }
    } else {
        for (int q = threadIdx.x; q < (fill << a.ldq_log2); q += kTcThreads) {
            const int sq = q >> a.ldq_log2, n = q & (a.ldq - 1);
            cp_async4(qraw + sq * QS + n, a.qv + sidx[sq] * a.ldq + n);
        }
    }
}

template <int KID, int D, int MODE, int NT>
__global__ void __launch_bounds__(kTcThreads) ksum_tc_kernel(TcArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ PartnerChunk pc;
    constexpr int KSTEP = MODE == TC_BF16 ? 16 : 8;
    constexpr int QS = qstride(NT, MODE);
    constexpr int LDQ8 = NT * 8;
    const int tile = a.tile;
    TcSmem L;
    tc_layout(MODE, NT, tile, smraw, &L);
    float4 *const sy0 = L.sy[0], *const sy1 = L.sy[1];
    float *const qr0 = L.qraw[0], *const qr1 = L.qraw[1];

    const int64_t node = a.tnodes[blockIdx.x];
    const int T = a.t_cnt[node];
    if (T == 0) return;
    const int64_t toff = a.t_off[node];
    const int64_t e0 = a.ptr[node], e1 = a.ptr[node + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t4 = lane & 3;

    for (int tb = 0; tb < T; tb += kTcRows) {
        const int tcount = min(kTcRows, T - tb);
        const int wr = (tcount + 15) / 16;  // warps along the targets
        const int groups = 8 / wr;          // warps along the sources
        const int grp = warp / wr, rt = warp % wr;
        const bool active = grp < groups;
        const int r0 = rt * 16 + g, r1 = r0 + 8;
        const bool ok0 = active && r0 < tcount, ok1 = active && r1 < tcount;
        float4 x0h = make_float4(0.f, 0.f, 0.f, 0.f), x0l = x0h, x1h = x0h, x1l = x0h;
        if (ok0) {
            const float4 *p = reinterpret_cast<const float4 *>(a.xt + (toff + tb + r0) * 8);
            x0h = p[0];
            x0l = p[1];
        }
        if (ok1) {
            const float4 *p = reinterpret_cast<const float4 *>(a.xt + (toff + tb + r1) * 8);
            x1h = p[0];
            x1l = p[1];
        }
        float acc[NT][4];
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[n][c] = 0.f;

        for (int64_t e = e0; e < e1;) {
            load_partner_chunk<kTcThreads>(pc, e, e1, a.col, a.s_off, a.s_cnt);
            const int nchunk = pc.n, total = pc.pre[pc.n];
            e += nchunk;
            const int ntiles = (total + tile - 1) / tile;
            // pipeline: the gathers of tile it + 1 run while tile it computes
            tc_stage_indices(pc, 0, min(tile, total), L.sidx);
            __syncthreads();
            tc_issue(a, L.sidx, min(tile, total), QS, sy0, qr0);
            cp_async_commit();
            __syncthreads();  // every thread has read sidx(0)
            if (ntiles > 1) tc_stage_indices(pc, tile, min(tile, total - tile), L.sidx);
            __syncthreads();
            for (int it = 0; it < ntiles; ++it) {
                const int b = it & 1;
                const int fill = min(tile, total - it * tile);
                const int fillk = (fill + KSTEP - 1) / KSTEP * KSTEP;
                if (it + 1 < ntiles)
                    tc_issue(a, L.sidx, min(tile, total - (it + 1) * tile), QS, b ? sy0 : sy1, b ? qr0 : qr1);
                cp_async_commit();
                cp_async_wait_one();  // this thread's copies of tile it have landed
                __syncthreads();      // (A) everyone's; sidx(it + 1) consumed
                if (it + 2 < ntiles) tc_stage_indices(pc, (it + 2) * tile, min(tile, total - (it + 2) * tile), L.sidx);
                const float4 *sy = b ? sy1 : sy0;
                const float *qr = b ? qr1 : qr0;
                if (active) {
                    float part[NT][4];
#pragma unroll
                    for (int n = 0; n < NT; ++n)
#pragma unroll
                        for (int c = 0; c < 4; ++c) part[n][c] = 0.f;
                    for (int ks = grp * KSTEP; ks < fillk; ks += groups * KSTEP) {
                        if (MODE == TC_BF16) {
                            const int c0 = ks + 2 * t4, c2 = c0 + 8;
                            float ev[8];
                            const int cs[4] = {c0, c0 + 1, c2, c2 + 1};
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                ev[u] = entry<KID, D>(x0h, x0l, sy, cs[u], ok0 && cs[u] < fill, a);
                                ev[4 + u] = entry<KID, D>(x1h, x1l, sy, cs[u], ok1 && cs[u] < fill, a);
                            }
                            const uint32_t a0 = pack_bf16(ev[0], ev[1]), a1 = pack_bf16(ev[4], ev[5]);
                            const uint32_t a2 = pack_bf16(ev[2], ev[3]), a3 = pack_bf16(ev[6], ev[7]);
                            bool okc[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) okc[u] = cs[u] < fill;
#pragma unroll
                            for (int n = 0; n < NT; ++n) {
                                const int col = n * 8 + g;
                                float qv[4];
#pragma unroll
                                for (int u = 0; u < 4; ++u) qv[u] = okc[u] ? qr[cs[u] * QS + col] : 0.f;
                                mma_bf16(part[n], a0, a1, a2, a3, pack_bf16(qv[0], qv[1]), pack_bf16(qv[2], qv[3]));
                            }
                        } else {
                            const int c0 = ks + t4, c1 = c0 + 4;
                            float v[4];
                            v[0] = entry<KID, D>(x0h, x0l, sy, c0, ok0 && c0 < fill, a);
                            v[1] = entry<KID, D>(x1h, x1l, sy, c0, ok1 && c0 < fill, a);
                            v[2] = entry<KID, D>(x0h, x0l, sy, c1, ok0 && c1 < fill, a);
                            v[3] = entry<KID, D>(x1h, x1l, sy, c1, ok1 && c1 < fill, a);
                            uint32_t ah[4], al[4];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                ah[c] = to_tf32(v[c]);
                                al[c] = MODE == TC_TF32X3 ? to_tf32(v[c] - __uint_as_float(ah[c])) : 0u;
                            }
                            const bool ok_c0 = c0 < fill, ok_c1 = c1 < fill;
#pragma unroll
                            for (int n = 0; n < NT; ++n) {
                                const int col = n * 8 + g;
                                const float q0 = ok_c0 ? qr[c0 * QS + col] : 0.f;
                                const float q1 = ok_c1 ? qr[c1 * QS + col] : 0.f;
                                const uint32_t b0 = to_tf32(q0), b1 = to_tf32(q1);
                                mma_tf32(part[n], ah[0], ah[1], ah[2], ah[3], b0, b1);
                                if (MODE == TC_TF32X3) {
                                    const uint32_t l0 = to_tf32(q0 - __uint_as_float(b0));
                                    const uint32_t l1 = to_tf32(q1 - __uint_as_float(b1));
                                    mma_tf32(part[n], ah[0], ah[1], ah[2], ah[3], l0, l1);
                                    mma_tf32(part[n], al[0], al[1], al[2], al[3], b0, b1);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int n = 0; n < NT; ++n)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[n][c] += part[n][c];
                }
                __syncthreads();  // (C) tile it consumed; sidx(it + 2) visible
            }
        }
        // fixed-order reduction over the source groups: C rows g, g + 8, columns 2 t4, 2 t4 + 1
        float *red = L.red;
        for (int gg = 0; gg < groups; ++gg) {
            if (active && grp == gg) {
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    const int cc = n * 8 + 2 * t4;
                    if (ok0) {
                        float *d0 = red + (size_t)r0 * LDQ8 + cc;
                        d0[0] = gg == 0 ? acc[n][0] : d0[0] + acc[n][0];
                        d0[1] = gg == 0 ? acc[n][1] : d0[1] + acc[n][1];
                    }
                    if (ok1) {
                        float *d1 = red + (size_t)r1 * LDQ8 + cc;
                        d1[0] = gg == 0 ? acc[n][2] : d1[0] + acc[n][2];
                        d1[1] = gg == 0 ? acc[n][3] : d1[1] + acc[n][3];
                    }
                }
            }
            __syncthreads();
        }
        for (int q = tid; q < tcount * a.ldq; q += kTcThreads) {
            const int row = q >> a.ldq_log2, n = q & (a.ldq - 1);
            a.out[(toff + tb + row) * a.ldq + n] = (double)red[row * LDQ8 + n] * a.scale;
        }
        __syncthreads();
    }
}

size_t tc_smem(int mode, int nt, int tile) { return tc_layout(mode, nt, tile, nullptr, nullptr); }

// n-tiles a kernel is compiled for: 2, 4 or 8 (one n-tile runs as two; the
// extra columns are never written out)
inline int tc_nt(int nt) { return nt <= 2 ? 2 : (nt <= 4 ? 4 : 8); }

template <int KID, int D, int MODE>
void (*pick_tc(int nt))(TcArgs) {
    switch (tc_nt(nt)) {
    case 2: return ksum_tc_kernel<KID, D, MODE, 2>;
    case 4: return ksum_tc_kernel<KID, D, MODE, 4>;
    default: return ksum_tc_kernel<KID, D, MODE, 8>;
    }
}

template <int KID, int D>
void launch_tc(int mode, const TcArgs &a, int64_t ntn, cudaStream_t s) {
    void (*kern)(TcArgs) = nullptr;
    if (mode == TC_BF16) kern = pick_tc<KID, D, TC_BF16>(a.nt);
    else if (mode == TC_TF32X3) kern = pick_tc<KID, D, TC_TF32X3>(a.nt);
    else kern = pick_tc<KID, D, TC_TF32>(a.nt);
    allow_max_dynamic_smem((const void *)kern);
    kern<<<(unsigned)ntn, kTcThreads, tc_smem(mode, tc_nt(a.nt), a.tile), s>>>(a);
    LAUNCHED();
}

}  // namespace

void coupling_tc(const smash_h2 *h, int precision, const float *qhat, double *zhat, int ldq, cudaStream_t s,
                 int kid) {
    const Side &R = h->row;
    const Side &Cs = *h->col;
    const int64_t ntn = h->nnodes - h->nroots;
    if (ntn <= 0) return;
    if (ldq > kTcMaxNt * 8) fail(SMASH_EINVAL, "tensor-core coupling supports at most %d right-hand sides", kTcMaxNt * 8);
    TcArgs a{};
    a.tnodes = h->nonroot_list; a.t_off = R.sk_off; a.t_cnt = R.k;
    a.ptr = h->adm_ptr; a.col = h->adm_col; a.s_off = Cs.sk_off; a.s_cnt = Cs.k;
    a.xt = R.skel_dd; a.ys = Cs.skel_dd; a.qv = qhat; a.out = zhat;
    a.ldq = ldq;
    a.ldq_log2 = 0;
    while ((1 << a.ldq_log2) < ldq) ++a.ldq_log2;
    if ((1 << a.ldq_log2) != ldq) fail(SMASH_EINVAL, "tensor-core coupling needs a power-of-two RHS stride");
    a.nt = (ldq + 7) / 8;
    const bool mult = kid == SMASH_K_INVR || kid == SMASH_K_CAUCHY1D || kid == SMASH_K_DLP1 || kid == SMASH_K_DLP2;
    a.scale = mult ? 1.0 / h->s : 1.0;
    a.s_f = (float)h->s;
    a.inv_s = (float)(1.0 / h->s);
    a.log_s = (float)log(h->s);
    const int mode = precision == SMASH_PREC_BF16 ? TC_BF16 : (precision == SMASH_PREC_TF32X3 ? TC_TF32X3 : TC_TF32);
    auto run = [&](int tile) {
        if (tile == kTcUseTcgen05) {
            coupling_tc05(h, qhat, zhat, ldq, s, kid);
            return;
        }
        TcArgs b = a;
        b.tile = tile;
        // unused axes hold 0 in every coordinate copy, so the 3D entry serves
        // 1D and 2D points as well
        switch (kid) {
        case SMASH_K_CAUCHY1D: launch_tc<SMASH_K_CAUCHY1D, 1>(mode, b, ntn, s); return;
        case SMASH_K_DLP1: launch_tc<SMASH_K_DLP1, 3>(mode, b, ntn, s); return;
        case SMASH_K_DLP2: launch_tc<SMASH_K_DLP2, 3>(mode, b, ntn, s); return;
        case SMASH_K_LOG: launch_tc<SMASH_K_LOG, 3>(mode, b, ntn, s); return;
        case SMASH_K_INVR: launch_tc<SMASH_K_INVR, 3>(mode, b, ntn, s); return;
        default: launch_tc<SMASH_K_YUKAWA, 3>(mode, b, ntn, s); return;
        }
    };
    // the staged tile (64, 128 or 256 sources) is tuned; the default is the
    // largest whose shared memory leaves room for two CTAs per SM
    std::vector<int> cands;
    int dflt = 64;
    for (int tile = 64; tile <= kTcMaxTile; tile *= 2) {
        const size_t sm = tc_smem(mode, tc_nt(a.nt), tile);
        if (sm <= 200 * 1024) cands.push_back(tile);
        if (sm <= 100 * 1024) dflt = tile;
    }
    // TF32 products also have the tcgen05 kernel (tensor-memory accumulator)
    if (mode == TC_TF32) cands.push_back(kTcUseTcgen05);
    char key[160];
    std::snprintf(key, sizeof(key), "ksum_tc/sm%d/k%d/d%d/m%d/nt%d/t%lld/n%lld", h->num_sms, kid, h->dim,
                  mode, a.nt, pow2_at_least(h->r), pow2_at_least(ntn));
    tune_choose(key, cands, dflt, s, run);
}

}  // namespace smash
