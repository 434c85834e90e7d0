// matvec_tc05.cu -- the coupling (3.19) of SMASH_PREC_TF32 on the 5th-generation
// tensor cores: tcgen05.mma with the accumulator in tensor memory.
//
// For a target node i with k_i <= 128 targets per pass, z^_i = sum_j K(x_i^, y_j^) q^_j
// is the product of the 128 x S block of kernel entries (rows >= k_i are 0) with the
// S x nrhs block of q^, S the concatenated partner skeletons.  The source stream
// is consumed in stages of kStage sources:
//   * every thread evaluates kernel entries in FP32 (from the normalised two-float
//     coordinates), rounds them to TF32 and stores them as 16-byte rows of the
//     K-major operand tile A (128 x kStage) in shared memory; q^ of the stage is
//     staged transposed into the K-major tile B (NP x kStage), also TF32;
//   * one thread issues kStage / 8 tcgen05.mma (M = 128, N = NP, K = 8) that
//     accumulate D = A B^T in tensor memory, and commits them to an mbarrier;
//   * two stage buffers alternate, so the entries of stage s + 1 are evaluated
//     while the tensor cores multiply stage s; a buffer is rewritten only after
//     the mbarrier shows that its MMAs have completed (bounded wait).
// At the end of a pass four warps read D from tensor memory (tcgen05.ld, one lane
// per target row) and write z^ in FP64 times the frame factor.
//
// Operand tiles use the canonical K-major layout without swizzle: 8-row x 16-byte
// core matrices, consecutive along K at 128 bytes, 8-row groups at kStage/4 * 128
// bytes; smem descriptors carry (address, LBO = 128, SBO) in 16-byte units.
#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "kappa_f32.cuh"
#include "ksum_tiles.cuh"

namespace smash {

namespace {

constexpr int kT5Threads = 256;
constexpr int kT5Rows = 128;   // M of the MMA: targets per pass
constexpr int kStage = 64;     // sources per stage (K extent of the operand tiles)
constexpr long kT5MaxSpin = 1L << 26;

__device__ int g_tc05_timeouts;

struct T5Args {
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
    float s_f, inv_s, log_s;
    int ldq;
};

// byte offset of element (row, k) in a K-major tile of kStage columns
__device__ __forceinline__ uint32_t kmaj(int row, int k) {
    return (uint32_t)((row >> 3) * (kStage / 4) * 128 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;                      // LBO: next core matrix along K
    d |= (uint64_t)(((kStage / 4) * 128) >> 4) << 32;     // SBO: next 8-row group
    d |= (uint64_t)1 << 46;                               // descriptor version
    return d;                                             // no swizzle
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// bounded wait for phase `parity` of an mbarrier; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long it = 0; it < kT5MaxSpin; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <int NP>
struct T5Smem {
    static constexpr int kA = kT5Rows * kStage * 4;  // bytes of A per buffer
    static constexpr int kB = NP * kStage * 4;       // bytes of B per buffer
    static constexpr int kY = kStage * 32;           // source coordinates per buffer (cp.async)
    static constexpr int kQ = kStage * NP * 4;       // raw FP32 q^ rows per buffer (cp.async)
    static constexpr int kT = kT5Rows * 32;          // target coordinates
    static constexpr int bytes = 2 * (kA + kB + kY + kQ) + kT + kStage * 8 + 64;
};

__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp4(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)), "l"(gmem));
}

// gathers the sources of one stage (coordinates, raw q^ rows of stride NP floats)
template <int NP>
__device__ __forceinline__ void t5_issue(const T5Args &a, const int64_t *sidx, int fill, float4 *cy, float *qr) {
    for (int q = threadIdx.x; q < 2 * fill; q += kT5Threads)
        cp16(cy + q, a.ys + sidx[q >> 1] * 8 + 4 * (q & 1));
    if ((a.ldq & 3) == 0) {
        const int pieces = a.ldq >> 2;
        for (int q = threadIdx.x; q < fill * pieces; q += kT5Threads) {
            const int k = q / pieces, p4 = q - k * pieces;
            cp16(qr + k * NP + 4 * p4, a.qv + sidx[k] * a.ldq + 4 * p4);
        }
    } else {
        for (int q = threadIdx.x; q < fill * a.ldq; q += kT5Threads) {
            const int k = q / a.ldq, n = q - k * a.ldq;
            cp4(qr + k * NP + n, a.qv + sidx[k] * a.ldq + n);
        }
    }
    asm volatile("cp.async.commit_group;");
}

template <int KID, int D, int NP>
__global__ void __launch_bounds__(kT5Threads) ksum_tc05_kernel(T5Args a) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ PartnerChunk pc;
    using S = T5Smem<NP>;
    // buffer b: A, B, gathered coordinates and raw q^ rows of one stage
    auto sA = [&](int b) { return smraw + b * S::kA; };
    auto sB = [&](int b) { return smraw + 2 * S::kA + b * S::kB; };
    auto sy = [&](int b) { return reinterpret_cast<float4 *>(smraw + 2 * (S::kA + S::kB) + b * S::kY); };
    auto sq = [&](int b) { return reinterpret_cast<float *>(smraw + 2 * (S::kA + S::kB + S::kY) + b * S::kQ); };
    float4 *tco = reinterpret_cast<float4 *>(smraw + 2 * (S::kA + S::kB + S::kY + S::kQ));  // 2 per target row
    int64_t *sidx = reinterpret_cast<int64_t *>(smraw + 2 * (S::kA + S::kB + S::kY + S::kQ) + S::kT);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sidx + kStage);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);

    const int64_t node = a.tnodes[blockIdx.x];
    const int T = a.t_cnt[node];
    if (T == 0) return;
    const int64_t toff = a.t_off[node];
    const int64_t e0 = a.ptr[node], e1 = a.ptr[node + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr uint32_t kCols = NP < 32 ? 32 : NP;
    constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NP >> 3) << 17) |
                                ((uint32_t)(kT5Rows >> 4) << 24);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    bool timed_out = false;
    int sc = 0;  // stages issued by this CTA (all threads keep the same count)

    for (int tb = 0; tb < T; tb += kT5Rows) {
        const int tcount = min(kT5Rows, T - tb);
        // target coordinates of the pass; rows >= tcount of A stay 0 in both buffers
        for (int q = tid; q < 2 * tcount; q += kT5Threads)
            tco[q] = reinterpret_cast<const float4 *>(a.xt + (toff + tb + (q >> 1)) * 8)[q & 1];
        for (int q = tid; q < 2 * (kT5Rows - tcount) * (kStage / 4); q += kT5Threads) {
            const int b = q & 1, e = q >> 1;
            const int m = tcount + e / (kStage / 4), kq = e % (kStage / 4);
            *reinterpret_cast<uint4 *>(sA(b) + kmaj(m, 4 * kq)) = make_uint4(0u, 0u, 0u, 0u);
        }
        // this thread's rows and quads of the entry tile: row m, quads g, g + G, ...
        const int RP = (tcount + 7) & ~7;
        const int G = kT5Threads / RP;
        const int my_m = tid % RP, my_g = tid / RP;
        const bool has_row = my_g < G && my_m < tcount;
        bool first = true;  // the next MMA starts the accumulation of this pass

        for (int64_t e = e0; e < e1;) {
            load_partner_chunk<kT5Threads>(pc, e, e1, a.col, a.s_off, a.s_cnt);
            const int nchunk = pc.n, total = pc.pre[pc.n];
            e += nchunk;
            const int nst = (total + kStage - 1) / kStage;
            // prologue: gather stage 0 of the chunk
            for (int q = tid; q < min(kStage, total); q += kT5Threads) sidx[q] = chunk_source(pc, q);
            __syncthreads();
            t5_issue<NP>(a, sidx, min(kStage, total), sy(sc & 1), sq(sc & 1));
            __syncthreads();  // sidx is rewritten below
            for (int i = 0; i < nst; ++i, ++sc) {
                const int b = sc & 1;
                const int fill = min(kStage, total - i * kStage);
                const int nfill = i + 1 < nst ? min(kStage, total - (i + 1) * kStage) : 0;
                for (int q = tid; q < nfill; q += kT5Threads) sidx[q] = chunk_source(pc, (i + 1) * kStage + q);
                __syncthreads();
                // gather stage i + 1 while stage i is evaluated (an empty group at the end)
                if (nfill > 0) t5_issue<NP>(a, sidx, nfill, sy(b ^ 1), sq(b ^ 1));
                else asm volatile("cp.async.commit_group;");
                asm volatile("cp.async.wait_group 1;" ::: "memory");  // stage i has landed (own copies)
                // the buffer's previous MMAs must have completed
                if (sc >= 2 && !mbar_wait(smem_u32(&mbar[b]), (uint32_t)(((sc - 2) >> 1) & 1))) timed_out = true;
                __syncthreads();  // stage i visible to all; A and B of buffer b free
                // B = q^ of the stage, transposed to K-major NP x kStage, TF32 (0 past fill / ldq)
                const float *qr = sq(b);
                for (int q = tid; q < NP * (kStage / 4); q += kT5Threads) {
                    const int n = q % NP, kq = q / NP;
                    uint32_t w[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int k = 4 * kq + j;
                        w[j] = tf32_bits((k < fill && n < a.ldq) ? qr[k * NP + n] : 0.f);
                    }
                    *reinterpret_cast<uint4 *>(sB(b) + kmaj(n, 4 * kq)) = make_uint4(w[0], w[1], w[2], w[3]);
                }
                // A = kernel entries of rows < tcount, TF32, 16 bytes per (row, quad);
                // sources past fill hold stale coordinates and are masked by a select
                if (has_row) {
                    const float4 xh = tco[2 * my_m], xl = tco[2 * my_m + 1];
                    const float4 *cy = sy(b);
                    for (int kq = my_g; kq < kStage / 4; kq += G) {
                        uint32_t w[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int k = 4 * kq + j;
                            const float4 yh = cy[2 * k], yl = cy[2 * k + 1];
                            float d[3] = {(xh.x - yh.x) + (xl.x - yl.x), (xh.y - yh.y) + (xl.y - yl.y),
                                          (xh.z - yh.z) + (xl.z - yl.z)};
                            const float v = kappa_f32<KID, D>(d, a.s_f, a.inv_s, a.log_s);
                            w[j] = tf32_bits(k < fill ? v : 0.f);
                        }
                        *reinterpret_cast<uint4 *>(sA(b) + kmaj(my_m, 4 * kq)) = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(sA(b)), b0 = smem_u32(sB(b));
#pragma unroll
                    for (int s = 0; s < kStage / 8; ++s) {
                        const uint64_t ad = smem_desc(a0 + s * 256), bd = smem_desc(b0 + s * 256);
                        const uint32_t en = (first && s == 0) ? 0u : 1u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                                     "l"(ad), "l"(bd), "r"(kIdesc), "r"(en));
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&mbar[b]))
                                 : "memory");
                }
                first = false;
            }
        }
        // read the accumulator: warps 0..3 own TMEM lanes 32 w .. 32 w + 31 (target rows)
        const bool any = !first;
        if (any && !mbar_wait(smem_u32(&mbar[(sc - 1) & 1]), (uint32_t)(((sc - 1) >> 1) & 1))) timed_out = true;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp < 4) {
            const int row = warp * 32 + lane;
#pragma unroll
            for (int c0 = 0; c0 < NP; c0 += 8) {
                uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                if (any) {
                    const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                                   "=r"(r[7])
                                 : "r"(addr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                }
                if (row < tcount)
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (c0 + j < a.ldq)
                            a.out[(toff + tb + row) * a.ldq + c0 + j] = (double)__uint_as_float(r[j]) * a.scale;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (timed_out) atomicAdd(&g_tc05_timeouts, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

template <int KID, int D>
void launch_tc05(const T5Args &a, int np, int64_t ntn, cudaStream_t s) {
    void (*kern)(T5Args) = nullptr;
    size_t smem = 0;
    if (np <= 16) { kern = ksum_tc05_kernel<KID, D, 16>; smem = T5Smem<16>::bytes; }
    else if (np <= 32) { kern = ksum_tc05_kernel<KID, D, 32>; smem = T5Smem<32>::bytes; }
    else { kern = ksum_tc05_kernel<KID, D, 64>; smem = T5Smem<64>::bytes; }
    allow_max_dynamic_smem((const void *)kern);
    kern<<<(unsigned)ntn, kT5Threads, smem, s>>>(a);
    LAUNCHED();
}

}  // namespace

int tc05_take_timeouts() {
    int v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc05_timeouts, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (v) cudaMemcpyToSymbol(g_tc05_timeouts, &z, sizeof(int));
    return v;
}

void coupling_tc05(const smash_h2 *h, const float *qhat, double *zhat, int ldq, cudaStream_t s, int kid) {
    const Side &R = h->row;
    const Side &Cs = *h->col;
    const int64_t ntn = h->nnodes - h->nroots;
    if (ntn <= 0) return;
    if (ldq > 64) fail(SMASH_EINVAL, "tensor-core coupling supports at most 64 right-hand sides");
    T5Args a{};
    a.tnodes = h->nonroot_list; a.t_off = R.sk_off; a.t_cnt = R.k;
    a.ptr = h->adm_ptr; a.col = h->adm_col; a.s_off = Cs.sk_off; a.s_cnt = Cs.k;
    a.xt = R.skel_dd; a.ys = Cs.skel_dd; a.qv = qhat; a.out = zhat;
    a.ldq = ldq;
    const bool mult = kid == SMASH_K_INVR || kid == SMASH_K_CAUCHY1D || kid == SMASH_K_DLP1 || kid == SMASH_K_DLP2;
    a.scale = mult ? 1.0 / h->s : 1.0;
    a.s_f = (float)h->s;
    a.inv_s = (float)(1.0 / h->s);
    a.log_s = (float)log(h->s);
    const int np = ldq <= 16 ? 16 : (ldq <= 32 ? 32 : 64);
    // unused axes hold 0 in every coordinate copy, so the 3D entry serves 1D and 2D points
    switch (kid) {
    case SMASH_K_CAUCHY1D: launch_tc05<SMASH_K_CAUCHY1D, 1>(a, np, ntn, s); return;
    case SMASH_K_LOG: launch_tc05<SMASH_K_LOG, 3>(a, np, ntn, s); return;
    case SMASH_K_INVR: launch_tc05<SMASH_K_INVR, 3>(a, np, ntn, s); return;
    case SMASH_K_DLP1: launch_tc05<SMASH_K_DLP1, 3>(a, np, ntn, s); return;
    case SMASH_K_DLP2: launch_tc05<SMASH_K_DLP2, 3>(a, np, ntn, s); return;
    default: launch_tc05<SMASH_K_YUKAWA, 3>(a, np, ntn, s); return;
    }
}

}  // namespace smash
