// matvec_oz.cu -- the coupling (3.19) of the double-float matvec with its
// multiply-accumulate on the tensor cores, split exactly into 8-bit digits.
//
// The coupling z^_i += sum_{j in L(i)} K(X^_i, Y^_j) q^_j is a dense
// contraction per target node: kernel entries (generated, ~2^-46 relative
// precision, double-float) times the skeleton vectors q^ (FP64).  Here both
// operands are written as short sums of 8-bit integer digits, every product
// of two digits is formed and summed on the tensor cores without rounding,
// and only the combination of the digit levels is done in double-float:
//
//  * Entries.  For a target node i, every entry of its row block is bounded by
//    the admissibility geometry (Def. 2.1, (2.3)): points lie in their cells,
//    so |x - y| >= |c_i - c_j| - r_i - r_j >= (1 - tau) |c_i - c_j| > 0 for the
//    cell centres c and half-diagonals r (tau < 1), and |x - y| is at least the
//    distance from the target point x to the partner's cell.  With 2^E_x above
//    twice the smaller of the two bounds over the row of x, K' = K 2^-E_x lies
//    in (-1/2, 1/2) and is split as K' = sum_{s<6} a_s 2^{-8(s+1)} into
//    round-to-nearest integer digits: the first three from hi(K), the last
//    three from the rest.  |a_s| <= 128, except the fourth, which also takes
//    lo(K) (|lo| <= ulp(hi)/2) and stays within 256.
//  * Vectors.  Per tree level l and column c, 2^F_lc above twice the largest
//    |q^_jc| of the level's skeletons scales q^ into (-1/2, 1/2);
//    q' = sum_{t<6} b_t 2^{-8(t+1)}, |b_t| <= 128, in FP64 once.  A row of L
//    lists its partners by level, so a tile never mixes two levels.
//  * Products.  K' q' = sum_L 2^{-8L-16} sum_{s+t=L} a_s b_t, truncated at
//    L <= 5 (dropped terms below 2^-47 relative).  A level holds at most 6
//    digit products per source, at most one of them with the fourth entry
//    digit: at most 7 * 2^14 per source, so 128 sources sum to less than
//    2^24, and every digit (<= 256) is exact in bf16: the FP32 accumulation
//    of bf16 x bf16 products
//    (mma.sync m16n8k16) is exact for every level.  After each tile (at most
//    128 sources per warp) the six level sums are folded into a double-float
//    accumulator per output: levels 0-2 by exact TwoSums, levels 3-5 as a
//    float32 tail at weight 2^-24, off by at most 2^-22 level-0 units (2^-46
//    of a full-scale level sum); the level's scale 2^(F_lc - max_l F_lc) is
//    exact.
//
// The result keeps the double-float coupling's precision (~2^-46 per entry)
// while the FP32 pipe evaluates only the entries and their digits; the
// products move to the tensor cores.  Used for the normalised two-float
// coordinates (trees of at most 10 levels, one problem) with at most 16
// right-hand sides per pass.
// Compiled with --fmad=false: every fused operation below is an explicit fmaf.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include <cuda_bf16.h>

#include "dd_arith.cuh"
#include <vector>

#include "internal.cuh"
#include "ksum_tiles.cuh"

namespace smash {

constexpr int kOzDigits = 6;
constexpr int kOzThreads = 256;
constexpr int kOzTileCap = 224;  // sources per tile when two or more warps share a target tile
constexpr int kOzRows = 64;      // targets per pass (8 target tiles of 8)

// ------------------------------------------------------------------ q^ digits
constexpr int kOzLevels = 16;  // rows of the per-level tables (levels 0..10 on this path)

// max |q^_jc| per (level, column), one warp per node; non-negative doubles
// order as their bit patterns
__global__ void oz_colmax_kernel(const double *__restrict__ q, int ldq, int64_t nnodes,
                                 const int32_t *__restrict__ level, const int32_t *__restrict__ k,
                                 const int64_t *__restrict__ sk_off, unsigned long long *__restrict__ cmax) {
    __shared__ unsigned long long sm[kOzLevels * 16];
    for (int i = threadIdx.x; i < kOzLevels * 16; i += blockDim.x) sm[i] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int64_t g = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); g < nnodes; g += (int64_t)gridDim.x * wpb) {
        const int kk = k[g];
        const double *qg = q + sk_off[g] * ldq;
        unsigned long long m = 0ull;
        for (int e = lane; e < kk * ldq; e += 32) {  // lane keeps column lane % ldq
            const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(qg[e]));
            m = b > m ? b : m;
        }
        for (int o = 16; o >= ldq; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
            m = y > m ? y : m;
        }
        if (lane < ldq && m) atomicMax(&sm[level[g] * 16 + lane], m);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kOzLevels * 16; i += blockDim.x)
        if (sm[i]) atomicMax(&cmax[i], sm[i]);
}

// F_lc = ilogb(max) + 2 puts the level's values in (-1/2, 1/2); fref_c is the
// largest over the levels, fd[l][c] = F_lc - fref_c (levels without values:
// 0; at most 60 below fref_c, which only loses digits of values that small)
__global__ void oz_scales_kernel(const unsigned long long *__restrict__ cmax, int *__restrict__ fd,
                                 int *__restrict__ fref, double *__restrict__ colscale) {
    const int c = threadIdx.x;
    if (c >= 16) return;
    int fr = 0;
    bool any = false;
    for (int l = 0; l < kOzLevels; ++l) {
        const unsigned long long m = cmax[l * 16 + c];
        if (!m) continue;
        const int f = ilogb(__longlong_as_double((long long)m)) + 2;
        fr = any ? max(fr, f) : f;
        any = true;
    }
    for (int l = 0; l < kOzLevels; ++l) {
        const unsigned long long m = cmax[l * 16 + c];
        const int f = m ? max(ilogb(__longlong_as_double((long long)m)) + 2, fr - 60) : fr;
        fd[l * 16 + c] = f - fr;
    }
    fref[c] = fr;
    colscale[c] = ldexp(1.0, fr);
}

// dig[(slot * 6 + t) * NC + c] = b_t of q^_slot,c 2^-F_lc (zero for c >= ldq),
// one warp per node
__global__ void oz_digits_kernel(const double *__restrict__ q, int ldq, int NC, int64_t nnodes,
                                 const int32_t *__restrict__ level, const int32_t *__restrict__ k,
                                 const int64_t *__restrict__ sk_off, const int *__restrict__ fd,
                                 const int *__restrict__ fref, __nv_bfloat16 *__restrict__ dig) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int64_t g = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); g < nnodes; g += (int64_t)gridDim.x * wpb) {
        const int kk = k[g], lv = level[g];
        const int64_t base = sk_off[g];
        for (int e = lane; e < kk * NC; e += 32) {
            const int t = e / NC, c = e - t * NC;
            const int64_t slot = base + t;
            double x = 0.0;
            if (c < ldq) x = ldexp(q[slot * ldq + c], -(fref[c] + fd[lv * 16 + c]));
#pragma unroll
            for (int u = 0; u < kOzDigits; ++u) {
                x *= 256.0;
                const double d = rint(x);
                x -= d;  // exact: |x - d| <= 1/2 carries the low bits of x
                dig[(slot * kOzDigits + u) * NC + c] = __float2bfloat16_rn((float)d);
            }
        }
    }
}

// ------------------------------------------------------------------ tensor-core helpers
__device__ __forceinline__ uint32_t oz_pack(float first, float second) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(second), "f"(first));
    return r;
}

__device__ __forceinline__ void oz_mma(float *c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                       uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void oz_ldsm_x4_trans(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                                 uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void oz_ldsm_x2_trans(uint32_t addr, uint32_t &r0, uint32_t &r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

__device__ __forceinline__ void oz_cp16(void *smem, const void *gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}

__device__ __forceinline__ void oz_cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// round to the nearest integer (|x| < 2^22) by the 1.5 * 2^23 shift
constexpr float kOzShift = 12582912.0f;

// digit s of an entry kh + kl in its row's frame (sc0 = 2^(8 - E)): the first
// three from kh, the fourth from the remainder r and kl (at 2^24 times the
// first digit's weight), the last two from r; r carries the remainder, exact
__device__ __forceinline__ float oz_digit(int s, float kh, float kl, float sc0, float &r) {
    float dg;
    if (s == 0) {
        dg = fmaf(kh, sc0, kOzShift) - kOzShift;
        r = fmaf(kh, sc0, -dg);
    } else if (s == 3) {
        const float x = fmaf(r, 256.0f, kl * (sc0 * 16777216.0f));
        dg = (x + kOzShift) - kOzShift;
        r = x - dg;
    } else {
        dg = fmaf(r, 256.0f, kOzShift) - kOzShift;
        r = fmaf(r, 256.0f, -dg);
    }
    return dg;
}

// ------------------------------------------------------------------ coupling kernel
struct KsumOzArgs {
    const int32_t *tnodes;
    const int64_t *t_off;
    const int32_t *t_cnt;
    const int64_t *ptr;
    const int32_t *col;
    const int64_t *s_off;
    const int32_t *s_cnt;
    const float *xt;           // target normalised coordinates, 8 floats per slot
    const float *ys;           // source normalised coordinates, 8 floats per slot
    const __nv_bfloat16 *dig;  // source digits, 6 * NC per slot
    const int *fd;             // F_lc - fref_c, kOzLevels x 16
    const double *colscale;    // 2^fref_c
    const int32_t *level;
    const uint64_t *cell;
    double *out;               // target vectors (FP64), ldq
    double scale;              // 1/s: entries are taken in the normalised frame
    int ldq, dim;
    // near field only
    const float *xt3, *ys3;    // exact three-float coordinates, 12 floats per point
    float n3h, n3l;            // 2^e / s as a two-float: exact-frame differences times it are normalised
    int *fallback;             // per CTA: 1 when the node is left to the double-float kernel
    int same;                  // X = Y: a target meets its own point (entry 0)
    int boxes;                 // one tree: cell boxes bound the normalised coordinates
};

// digit bytes per source in shared memory: 6 * NC bf16 plus 16 bytes of pad,
// which puts the 8 rows of an ldmatrix on distinct banks.  The group
// reduction at the end of a pass reuses the digit region.
template <int NC, bool NEAR>
struct OzLayout {
    static constexpr int kCap = NEAR ? 192 : kOzTileCap;  // sources per tile (three CTAs per SM)
    static constexpr int kCoordF4 = 2;                      // float4 per source: normalised (hi, lo)
    static constexpr int kDigitBytes = kOzDigits * NC * 2;
    static constexpr int kStride = kDigitBytes + 16;
    static constexpr size_t kCoords = sizeof(float4) * kCoordF4 * kCap;
    static constexpr size_t kDigits = (size_t)kStride * kCap;
    static constexpr size_t kRed = sizeof(double) * kOzRows * NC;
    static constexpr size_t kAcc = sizeof(float) * 2 * 4 * kOzThreads;  // (hi, lo) of 4 outputs per thread
    static constexpr size_t kIdx = sizeof(int64_t) * kCap;
    static constexpr size_t kBytes = kCoords + kDigits + kIdx + kAcc;
    static_assert(kRed <= kDigits, "the group reduction fits the digit region");
};

// bound of target node g's row from the cells alone: max over partners j of
// 1 / (|c_g - c_j| - r_g - r_j) in the unit frame of the normalised coordinates
// (the root, level 1, is the unit cube; a level-l cell has width 2^(1-l))
__device__ double oz_node_bound(const KsumOzArgs &a, int64_t g, int64_t e0, int64_t e1, unsigned long long *slot) {
    const int d = a.dim;
    const int li = a.level[g];
    const uint64_t *ci = a.cell + g * 3;
    unsigned long long best = 0ull;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kOzThreads) {
        const int64_t j = a.col[e];
        const int lj = a.level[j];
        const uint64_t *cj = a.cell + j * 3;
        const int m = li > lj ? li : lj;
        // centres (2c + 1) 2^(m - l) and radii sqrt(d) 2^(m - l) in units of 2^-m,
        // half the width of a level-m cell
        double sum = 0.0;
        for (int ax = 0; ax < d; ++ax) {
            const uint64_t Ci = (2 * ci[ax] + 1) << (m - li);
            const uint64_t Cj = (2 * cj[ax] + 1) << (m - lj);
            const double D = (double)(Ci >= Cj ? Ci - Cj : Cj - Ci);
            sum += D * D;
        }
        const double rad = sqrt((double)d) * (ldexp(1.0, m - li) + ldexp(1.0, m - lj));
        const double gap = sqrt(sum) - rad;
        const double kb = gap > 0.0 ? ldexp(1.0, m) / gap : INFINITY;
        const unsigned long long b = (unsigned long long)__double_as_longlong(kb);
        best = b > best ? b : best;
    }
    if (threadIdx.x == 0) *slot = 0ull;
    __syncthreads();
    atomicMax(slot, best);
    __syncthreads();
    return __longlong_as_double((long long)*slot);
}

// smallest squared distance from the point x (hi parts) to the cells of the
// row's partners; each gap is reduced by 2^-22 to cover the lo part (< 2^-23)
// and the roundings, so the result is a lower bound.  The four lanes of a
// quad split the partners.
template <int D>
__device__ __forceinline__ float oz_point_gap2(const float4 &x, const KsumOzArgs &a, int64_t e0, int64_t e1, int t4) {
    float best = INFINITY;
    for (int64_t e = e0 + t4; e < e1; e += 4) {
        const int64_t j = a.col[e];
        const float w = ldexpf(1.0f, 1 - a.level[j]);  // cell width (the root is level 1)
        const uint64_t *cj = a.cell + j * 3;
        const float xv[3] = {x.x, x.y, x.z};
        float s2 = 0.f;
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
            const float lo = fmaf((float)cj[ax], w, 1.0f);  // exact: c < 2^9, w a power of two
            const float gap = fmaxf(fmaxf(lo - xv[ax], xv[ax] - (lo + w)) - 0x1p-22f, 0.f);
            s2 = fmaf(gap, gap, s2);
        }
        best = fminf(best, s2);
    }
    best = fminf(best, __shfl_xor_sync(0xffffffffu, best, 1));
    best = fminf(best, __shfl_xor_sync(0xffffffffu, best, 2));
    return best;
}

// Near field: the nearest source of target point x (hi parts; the target's
// own point excluded) and an upper bound of the farthest, over the partners
// of its leaf g.  The leaf's own points are scanned first (the four lanes of
// a quad split them); for one tree (a batch of trees scans every partner) a
// partner leaf is scanned (by one lane) only if the
// lower bound of r^2 from its cell box does not exceed the nearest found so
// far, so the minimum is the same as over all sources: every value the FP32
// r^2 of a skipped point could take lies above the bound (gaps reduced by
// 2^-22 for the hi parts' rounding, the sum by 2^-20 relative).  The
// farthest is bounded from the boxes (gaps grown by 2^-22, 2^-20 relative).
template <int D>
__device__ __forceinline__ void oz_near_extremes(const float4 &x, const KsumOzArgs &a, int64_t g, int64_t e0,
                                                 int64_t e1, int t4, int64_t self, float &dmin2, float &dmax2) {
    const float xv[3] = {x.x, x.y, x.z};
    auto r2_of = [&](int64_t src) {
        const float4 y = __ldg(reinterpret_cast<const float4 *>(a.ys + src * 8));
        const float dx = x.x - y.x, dy = D > 1 ? x.y - y.y : 0.f, dz = D > 2 ? x.z - y.z : 0.f;
        return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    };
    float best = INFINITY, far = 0.f;
    {
        const int64_t so = a.s_off[g];
        const int cnt = a.s_cnt[g];
        for (int b = t4; b < cnt; b += 4) {
            if (so + b == self) continue;
            const float r2 = r2_of(so + b);
            best = fminf(best, r2);
            far = fmaxf(far, r2);
        }
    }
    best = fminf(best, __shfl_xor_sync(0xffffffffu, best, 1));
    best = fminf(best, __shfl_xor_sync(0xffffffffu, best, 2));
    for (int64_t e = e0 + t4; e < e1; e += 4) {
        const int64_t j = a.col[e];
        if (j == g) continue;
        const int64_t so = a.s_off[j];
        const int cnt = a.s_cnt[j];
        if (!a.boxes) {  // a batch of trees: cells are not in the normalised frame, scan all
            for (int b = 0; b < cnt; ++b) {
                if (so + b == self) continue;
                const float r2 = r2_of(so + b);
                best = fminf(best, r2);
                far = fmaxf(far, r2);
            }
            continue;
        }
        const float w = ldexpf(1.0f, 1 - a.level[j]);  // cell width (the root is level 1)
        const uint64_t *cj = a.cell + j * 3;
        float lb = 0.f, ub = 0.f;
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
            const float lo = fmaf((float)cj[ax], w, 1.0f);  // exact: c < 2^9, w a power of two
            const float below = lo - xv[ax], above = xv[ax] - (lo + w);
            const float gap = fmaxf(fmaxf(below, above) - 0x1p-22f, 0.f);
            const float span = fmaxf(-below, -above) + 0x1p-22f;  // to the far face
            lb = fmaf(gap, gap, lb);
            ub = fmaf(span, span, ub);
        }
        far = fmaxf(far, ub * (1.0f + 0x1p-20f));
        if (lb * (1.0f - 0x1p-20f) > best) continue;
        for (int b = 0; b < cnt; ++b) {
            if (so + b == self) continue;
            best = fminf(best, r2_of(so + b));
        }
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
        far = fmaxf(far, __shfl_xor_sync(0xffffffffu, far, o));
    }
    dmin2 = best;
    dmax2 = far;
}

// exponent E with K' = K 2^-E in (-1/2, 1/2) for every entry of the row of x
__device__ __forceinline__ int oz_row_exponent(float gap2, double node_kb) {
    float kb = (float)(node_kb * (1.0 + 1e-6));
    if (gap2 > 0.f) kb = fminf(kb, rsqrtf(gap2) * (1.0f + 0x1p-18f));
    return ilogbf(kb) + 2;
}

// 1/|d| in double-float for d = dh + dl, d != 0 (admissible pairs): the
// squares exactly by FMA, their sum by magnitude-ordered Fast2Sum (the squares
// are non-negative, so max/min order them), then one Newton step on the
// hardware reciprocal square root with the residual 1 - r y0^2 formed by FMA
// and the result renormalised.  The pair (dh, dl) from normalised coordinates
// is not normalised (|dl| reaches 2^-23 against |dh| >= 2^-8 or so), so r^2's
// low part rl can be ~2^-15 of rh: the seed is taken at rh + rl, which keeps
// the residual at the seed's own ~2^-22 and the Newton step's neglected
// square term below 2^-43.
template <int D, bool ZERO>
__device__ __forceinline__ void oz_invr(const float *dh, const float *dl, float &kh, float &kl) {
    float p[3], e[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < D) {
            p[a] = dh[a] * dh[a];
            const float t = fmaf(dh[a], dh[a], -p[a]);
            e[a] = fmaf(dl[a], fmaf(2.0f, dh[a], dl[a]), t);  // 2 dh dl + dl^2
        } else {
            p[a] = 0.f;
            e[a] = 0.f;
        }
    }
    const float s1 = p[0] + p[1];
    const float t1 = fminf(p[0], p[1]) - (s1 - fmaxf(p[0], p[1]));
    const float rh = s1 + p[2];
    const float t2 = fminf(s1, p[2]) - (rh - fmaxf(s1, p[2]));
    const float rl = ((e[0] + e[1]) + (e[2] + t1)) + t2;
    if (ZERO && rh == 0.f) {  // coincident points (near field): the entry is 0
        kh = 0.f;
        kl = 0.f;
        return;
    }
    const float y0 = rsqrtf(rh + rl);
    const float th = y0 * y0;
    const float tl = fmaf(y0, y0, -th);
    float ee = fmaf(-rh, th, 1.0f);
    ee = fmaf(-rh, tl, ee);
    ee = fmaf(-rl, th, ee);
    // renormalised, |kl| <= ulp(kh) / 2: the digit split takes kh whole into
    // the first three digits and kl, scaled by 2^24, into the fourth
    fast_two_sum(y0, (0.5f * y0) * ee, kh, kl);
}

template <int KID, int D>
__device__ __forceinline__ void oz_entry(const float4 &xh, const float4 &xl, const float4 &yh, const float4 &yl,
                                         float &kh, float &kl) {
    float dh[3], dl[3];
    dh[0] = xh.x - yh.x; dh[1] = xh.y - yh.y; dh[2] = xh.z - yh.z;
    dl[0] = xl.x - yl.x; dl[1] = xl.y - yl.y; dl[2] = xl.z - yl.z;
    if (KID == SMASH_K_CAUCHY1D)
        kappa_dd<KID, D>(dh, dl, kh, kl);
    else
        oz_invr<D, false>(dh, dl, kh, kl);
}

// Near-field entries (3.20).  The normalised two-float coordinates give a
// difference to ~2^-46.5 absolute (both coordinates within 2^-48 of x'', the
// lo parts' difference rounded), i.e. ~2^-38.5 relative at the threshold
// |d''| = 2^-8, as for the closest admissible pairs of the coupling.  A pair
// closer than that (rare: a ball of radius 2^-8 of the cube around the
// target) takes its difference from the exact three-float coordinates
// instead, converted to the normalised frame by the two-float 2^e / s.  A
// target's own point and coincident points give the entry 0.
constexpr float kNearExact2 = 0x1p-16f;  // (2^-8)^2

template <int KID, int D>
__device__ __forceinline__ void oz_entry_near(const float4 &xh, const float4 &xl, const float *x3p,
                                              const float4 &yh, const float4 &yl, const float *y3p, float n3h,
                                              float n3l, float &kh, float &kl) {
    float dh[3], dl[3];
    dh[0] = xh.x - yh.x; dh[1] = xh.y - yh.y; dh[2] = xh.z - yh.z;
    dl[0] = xl.x - yl.x; dl[1] = xl.y - yl.y; dl[2] = xl.z - yl.z;
    float d2 = dh[0] * dh[0];
    if (D > 1) d2 = fmaf(dh[1], dh[1], d2);
    if (D > 2) d2 = fmaf(dh[2], dh[2], d2);
    if (d2 < kNearExact2) {
        const float4 *y3 = reinterpret_cast<const float4 *>(y3p);
        const float4 yh3 = y3[0], ym3 = y3[1], yl3 = y3[2];
        const float4 *x3 = reinterpret_cast<const float4 *>(x3p);
        float eh[3], el[3];
        diff3(x3[0].x, x3[1].x, x3[2].x, yh3.x, ym3.x, yl3.x, eh[0], el[0]);
        diff3(x3[0].y, x3[1].y, x3[2].y, yh3.y, ym3.y, yl3.y, eh[1], el[1]);
        diff3(x3[0].z, x3[1].z, x3[2].z, yh3.z, ym3.z, yl3.z, eh[2], el[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {  // (eh + el)(n3h + n3l), renormalised
            const float p = eh[a] * n3h;
            const float e = fmaf(eh[a], n3h, -p);
            fast_two_sum(p, fmaf(el[a], n3h, fmaf(eh[a], n3l, e)), dh[a], dl[a]);
        }
    }
    if (KID == SMASH_K_CAUCHY1D)
        kappa_dd<KID, D>(dh, dl, kh, kl);
    else
        oz_invr<D, true>(dh, dl, kh, kl);
}


// One CTA per target node.  mma.sync m16n8k16 with the roles
//   M = 16 right-hand sides (q^ digits, A operand, ldmatrix from the staged tile),
//   N = 8 targets (entry digits, B operand, evaluated in registers),
//   K = 16 sources,
// so a warp owns 8 targets, each lane evaluates the 4 entries of its target
// and 4 sources of a k-block, and the six level sums take 24 registers.
template <int KID, int D, int NT, bool NEAR>
__global__ void __launch_bounds__(kOzThreads, 3) ksum_oz_kernel(KsumOzArgs a) {
    constexpr int NC = 8 * NT;
    using Lay = OzLayout<NC, NEAR>;
    constexpr int CAP = Lay::kCap;
    constexpr int NF = Lay::kCoordF4;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ PartnerChunk pc;
    __shared__ unsigned long long bound_slot;
    __shared__ int runend[kPartnerChunk];  // per partner: one past the last partner of its level run
    __shared__ int plev[kPartnerChunk];
    __shared__ int sfd[kOzLevels * 16];
    __shared__ int rowE[kOzRows];
    __shared__ unsigned int s_dmin[kOzRows], s_dmax[kOzRows];  // near field: squared distances as bits
    float4 *sy = reinterpret_cast<float4 *>(smraw);                  // [NF][cap]: hi, (mid,) lo
    unsigned char *sd = smraw + Lay::kCoords;                        // [cap][stride]
    int64_t *sidx = reinterpret_cast<int64_t *>(sd + Lay::kDigits);  // [cap]
    // running double-float sums, touched once per tile: [2 * output + (0 hi, 1 lo)][thread]
    float *acc = reinterpret_cast<float *>(smraw + Lay::kCoords + Lay::kDigits + Lay::kIdx);
    double *red = reinterpret_cast<double *>(sd);  // [rows][NC], after the last tile of a pass

    const int64_t g = a.tnodes[blockIdx.x];
    const int T = a.t_cnt[g];
    if (T == 0) return;
    const int64_t toff = a.t_off[g];
    const int64_t e0 = a.ptr[g], e1 = a.ptr[g + 1];
    const int ldq = a.ldq;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gq = lane >> 2, t4 = lane & 3;
    for (int i = tid; i < kOzLevels * 16; i += kOzThreads) sfd[i] = NEAR ? 0 : a.fd[i];

    const double kb_node = NEAR ? 0.0 : oz_node_bound(a, g, e0, e1, &bound_slot);
    if (!NEAR && !(kb_node < INFINITY)) {
        // no finite bound: cannot happen for tau < 1 (the build rejects
        // others); write NaN rather than a wrong sum
        for (int q = tid; q < T * ldq; q += kOzThreads) a.out[toff * ldq + q] = NAN;
        return;
    }
    // ldmatrix rows of the q^ digits: lane l addresses source
    // kb*16 + (l & 7) + 8 (source half), columns 8 (right-hand-side half)
    const int lsrc = (lane & 7) + 8 * (NT == 2 ? (lane >> 4) : ((lane >> 3) & 1));
    const int lrhs = NT == 2 ? 8 * ((lane >> 3) & 1) : 0;

    for (int tb = 0; tb < T; tb += kOzRows) {
        const int tcount = min(kOzRows, T - tb);
        const int wr = (tcount + 7) / 8;  // target tiles
        const int groups = 8 / wr;        // warps along the sources per target tile
        const int grp = warp / wr, rt = warp % wr;
        const bool active = grp < groups;
        const int tile = groups == 1 ? 128 : CAP;  // <= 128 sources per warp per flush
        // the lane's target; targets past the block take target 0's point (finite entries, discarded)
        const int tr = rt * 8 + gq;
        const int64_t tpt = toff + tb + (tr < tcount ? tr : 0);
        const float4 *px = reinterpret_cast<const float4 *>(a.xt + tpt * 8);
        const float4 xh = px[0], xl = px[1];
        const float *x3p = NEAR ? a.xt3 + tpt * 12 : nullptr;  // exact coordinates, for close pairs
        // first digit: K 2^(8-E); lo(K) enters the fourth digit at 2^24 times that
        float sc0;
        {
            int E;
            if (NEAR) {
                // the row's largest entry from its nearest source: hi parts of the
                // normalised coordinates differ exactly, and the distance is
                // within sqrt(3) 2^-23 < 2^-22 of theirs; 1/|d| in the exact frame
                // (x 2^-e, 2^e <= s) is at most 1/|d''|.  Rows whose sources span
                // more than 2^12 in distance, or meet a coincident point other
                // than their own, leave the node to the double-float kernel.
                //
                // Every (target, source) pair is visited once: the warps of a
                // target tile and the lanes of a quad split each staged tile.
                // one quad per target row of the pass (warps past the rows sit
                // out); rows past tcount, which the MMA tiles pad with target 0,
                // take row 0's values
                {
                    const int q = tid >> 2;
                    if (warp * 8 < tcount) {
                        const int64_t qpt = toff + tb + (q < tcount ? q : 0);
                        const float4 qx = *reinterpret_cast<const float4 *>(a.xt + qpt * 8);
                        float mn, mx;
                        oz_near_extremes<D>(qx, a, g, e0, e1, t4, a.same ? qpt : -1, mn, mx);
                        if (t4 == 0 && q < tcount) {
                            s_dmin[q] = __float_as_uint(mn);
                            s_dmax[q] = __float_as_uint(mx);
                        }
                    }
                    __syncthreads();
                    if (tid < kOzRows && tid >= tcount) {
                        s_dmin[tid] = s_dmin[0];
                        s_dmax[tid] = s_dmax[0];
                    }
                }
                __syncthreads();
                float dmin2 = __uint_as_float(s_dmin[tr]);
                float dmax2 = __uint_as_float(s_dmax[tr]);
                const float dlo = sqrtf(dmin2) * (1.0f - 0x1p-20f) - 0x1p-22f;
                const bool bad = !(dlo > 0.f) || dmax2 > 0x1p24f * dmin2;
                E = bad ? 0 : ilogbf((1.0f / dlo) * (1.0f + 0x1p-18f)) + 2;
                if (__syncthreads_or(bad)) {
                    if (tid == 0) a.fallback[blockIdx.x] = 1;
                    return;
                }
            } else {
                E = oz_row_exponent(oz_point_gap2<D>(xh, a, e0, e1, t4), kb_node);
            }
            sc0 = ldexpf(1.0f, 8 - E);
            if (active && grp == 0 && t4 == 0) rowE[tr] = E;
        }
        // output o of the lane: right-hand side gq + 8 (o >> 1), target rt * 8 + 2 t4 + (o & 1)
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            acc[(2 * o) * kOzThreads + tid] = 0.f;
            acc[(2 * o + 1) * kOzThreads + tid] = 0.f;
        }
        float C[kOzDigits][4];
#pragma unroll
        for (int L = 0; L < kOzDigits; ++L)
#pragma unroll
            for (int c = 0; c < 4; ++c) C[L][c] = 0.f;

        for (int64_t e = e0; e < e1;) {
            load_partner_chunk<kOzThreads>(pc, e, e1, a.col, a.s_off, a.s_cnt);
            const int nchunk = pc.n, total = pc.pre[pc.n];
            for (int q = tid; q < nchunk; q += kOzThreads) plev[q] = NEAR ? 0 : a.level[a.col[e + q]];
            __syncthreads();
            if (tid == 0) {
                int end = nchunk;
                for (int p = nchunk - 1; p >= 0; --p) {
                    if (p + 1 < nchunk && plev[p + 1] != plev[p]) end = p + 1;
                    runend[p] = end;
                }
            }
            __syncthreads();
            e += nchunk;
            for (int pos = 0; pos < total;) {
                // the partner holding pos; the tile ends with its level run
                int plo = 0, phi = nchunk - 1;
                while (plo < phi) {
                    const int mid = (plo + phi + 1) >> 1;
                    if (pc.pre[mid] <= pos) plo = mid;
                    else phi = mid - 1;
                }
                const int lv = plev[plo];
                const int fill = min(tile, pc.pre[runend[plo]] - pos);
                const int nkb = (fill + 15) >> 4;
                const int fill16 = nkb << 4;
                for (int q = tid; q < fill; q += kOzThreads) sidx[q] = chunk_source(pc, pos + q);
                __syncthreads();
                // coordinates (the pad up to 16 repeats source 0) and digits (zero pad)
                for (int q = tid; q < NF * fill16; q += kOzThreads) {
                    const int b = q / NF, part = q - b * NF;
                    const int64_t src = sidx[b < fill ? b : 0];
                    oz_cp16(sy + part * CAP + b, a.ys + src * 8 + 4 * part);
                }
                constexpr int kPieces = Lay::kDigitBytes / 16;
                for (int q = tid; q < fill * kPieces; q += kOzThreads) {
                    const int b = q / kPieces, p = q - b * kPieces;
                    oz_cp16(sd + (size_t)b * Lay::kStride + 16 * p,
                            reinterpret_cast<const unsigned char *>(a.dig) + sidx[b] * Lay::kDigitBytes + 16 * p);
                }
                for (int q = fill * kPieces + tid; q < fill16 * kPieces; q += kOzThreads) {
                    const int b = q / kPieces, p = q - b * kPieces;
                    *reinterpret_cast<uint4 *>(sd + (size_t)b * Lay::kStride + 16 * p) = make_uint4(0u, 0u, 0u, 0u);
                }
                oz_cp_wait_all();
                __syncthreads();
                if (active) {
                    const uint32_t sd_base = (uint32_t)__cvta_generic_to_shared(sd);
                    for (int kbi = grp; kbi < nkb; kbi += groups) {
                        const int c0 = kbi * 16 + 2 * t4;
                        const int cs[4] = {c0, c0 + 1, c0 + 8, c0 + 9};
                        float kh[4], kl[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if (NEAR)
                                oz_entry_near<KID, D>(xh, xl, x3p, sy[cs[u]], sy[CAP + cs[u]],
                                                      a.ys3 + sidx[cs[u] < fill ? cs[u] : 0] * 12, a.n3h, a.n3l,
                                                      kh[u], kl[u]);
                            else
                                oz_entry<KID, D>(xh, xl, sy[cs[u]], sy[CAP + cs[u]], kh[u], kl[u]);
                        }
                        // q^ digits of the k-block: A fragments of the six planes
                        uint32_t A[kOzDigits][4];
                        const uint32_t rowaddr = sd_base + (uint32_t)((kbi * 16 + lsrc) * Lay::kStride) + 2u * lrhs;
#pragma unroll
                        for (int t = 0; t < kOzDigits; ++t) {
                            const uint32_t ad = rowaddr + (uint32_t)(t * NC * 2);
                            if (NT == 2) {
                                oz_ldsm_x4_trans(ad, A[t][0], A[t][1], A[t][2], A[t][3]);
                            } else {
                                oz_ldsm_x2_trans(ad, A[t][0], A[t][2]);
                                A[t][1] = 0u;
                                A[t][3] = 0u;
                            }
                        }
                        // digits of the 4 entries, most significant first, each
                        // multiplied at once with the vector digits of the levels it reaches
                        float r[4];
#pragma unroll
                        for (int s = 0; s < kOzDigits; ++s) {
                            float dg[4];
#pragma unroll
                            for (int v = 0; v < 4; ++v) dg[v] = oz_digit(s, kh[v], kl[v], sc0, r[v]);
                            const uint32_t b0 = oz_pack(dg[0], dg[1]), b1 = oz_pack(dg[2], dg[3]);
#pragma unroll
                            for (int t = 0; t + s < kOzDigits; ++t)
                                oz_mma(C[s + t], A[t][0], A[t][1], A[t][2], A[t][3], b0, b1);
                        }
                    }
                    // flush: sum_L C_L 2^-8L, scaled to the column's reference
                    // exponent, into the double-float accumulators
#pragma unroll
                    for (int o = 0; o < 4; ++o) {
                        const float fac = ldexpf(1.0f, sfd[lv * 16 + gq + 8 * (o >> 1)]);
                        const float tail = fmaf(C[5][o], 1.0f / 65536.0f, fmaf(C[4][o], 1.0f / 256.0f, C[3][o]));
                        float h, l, e2, e3;
                        two_sum_ordered(C[0][o], C[1][o] * (1.0f / 256.0f), h, l);
                        two_sum_ordered(h, C[2][o] * (1.0f / 65536.0f), h, e2);
                        l = fmaf(tail, 1.0f / 16777216.0f, l + e2);
                        float ah = acc[(2 * o) * kOzThreads + tid], al = acc[(2 * o + 1) * kOzThreads + tid];
                        two_sum_ordered(ah, h * fac, ah, e3);
                        al = al + (e3 + l * fac);
                        fast_two_sum(ah, al, ah, al);
                        acc[(2 * o) * kOzThreads + tid] = ah;
                        acc[(2 * o + 1) * kOzThreads + tid] = al;
#pragma unroll
                        for (int L = 0; L < kOzDigits; ++L) C[L][o] = 0.f;
                    }
                }
                __syncthreads();
                pos += fill;
            }
        }
        // reduce the source groups in a fixed order (red reuses the digit
        // region: every tile of the pass is done), then scale and write
        for (int gg = 0; gg < groups; ++gg) {
            if (active && grp == gg) {
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int c = gq + 8 * (o >> 1);
                    if (c < NC) {
                        const double v =
                            (double)acc[(2 * o) * kOzThreads + tid] + (double)acc[(2 * o + 1) * kOzThreads + tid];
                        double *dst = red + (rt * 8 + 2 * t4 + (o & 1)) * NC + c;
                        *dst = gg == 0 ? v : *dst + v;
                    }
                }
            }
            __syncthreads();
        }
        for (int q = tid; q < tcount * ldq; q += kOzThreads) {
            const int row = q / ldq, c = q - row * ldq;
            a.out[(toff + tb) * ldq + q] = red[row * NC + c] * ldexp(a.scale, rowE[row] - 16) * a.colscale[c];
        }
        __syncthreads();
    }
}

template <int KID, int D, int NT, bool NEAR>
static void launch_oz(const KsumOzArgs &a, int64_t ntn, cudaStream_t s) {
    const size_t smem = OzLayout<8 * NT, NEAR>::kBytes;
    auto kern = ksum_oz_kernel<KID, D, NT, NEAR>;
    allow_max_dynamic_smem((const void *)kern);
    kern<<<(unsigned)ntn, kOzThreads, smem, s>>>(a);
    LAUNCHED();
}

template <int KID, int D, bool NEAR>
static void launch_oz_nt(const KsumOzArgs &a, int64_t ntn, cudaStream_t s) {
    if (a.ldq <= 8)
        launch_oz<KID, D, 1, NEAR>(a, ntn, s);
    else
        launch_oz<KID, D, 2, NEAR>(a, ntn, s);
}

template <bool NEAR>
static void launch_oz_kernel(const smash_h2 *h, int kid, const KsumOzArgs &a, int64_t ntn, cudaStream_t s) {
    if (kid == SMASH_K_CAUCHY1D)
        launch_oz_nt<SMASH_K_CAUCHY1D, 1, NEAR>(a, ntn, s);
    else if (h->dim == 3)
        launch_oz_nt<SMASH_K_INVR, 3, NEAR>(a, ntn, s);
    else if (h->dim == 2)
        launch_oz_nt<SMASH_K_INVR, 2, NEAR>(a, ntn, s);
    else
        launch_oz_nt<SMASH_K_INVR, 1, NEAR>(a, ntn, s);
}

// ------------------------------------------------------------------ tcgen05 variant
// The same digit-split coupling with the digit products issued as tcgen05.mma
// (kind::f16, bf16 digits, FP32 accumulation in tensor memory) by one thread,
// instead of warp MMAs:
//
//  * D_L = sum_{s+t=L} A_s B_t with M = 64 rows, 16 right-hand sides and K =
//    the sources of a stage; the six level sums D_0..D_5 take tensor-memory
//    columns 16 L .. 16 L + 15.  The B planes lie one after another as one
//    K-major tile of 96 rows, so one MMA per entry digit s and K-step,
//    A_s [B_0 .. B_{5-s}] with N = 16 (6 - s) written to columns 16 s .. 95,
//    forms all of A_s's level products (6 MMAs per K-step, not 21).  With
//    M = 64, row i of D sits in lane 32 (i / 16) + i % 16.
//  * A_s (entry digit s) is written to shared memory in the canonical K-major
//    layout without swizzle (8-row x 16-byte core matrices, 128 bytes apart
//    along K).  A plane holds 2048 entries: 64 target rows x 32 sources, or,
//    for a pass of at most 32 targets, 32 rows x 64 sources (the MMA's rows
//    32..63 then read the next plane and are never used), so that the
//    threads stay busy on the small nodes of the lowest level.  One thread
//    evaluates 8 entries of one target row (a source octet) into registers
//    while the previous stage's MMAs run, and stores them, 16 bytes per
//    digit plane, once those have completed (bounded mbarrier wait).
//  * B_t (q^ digit t) comes from the staged q^ digits (per source six planes
//    of 16 bf16, as the warp-MMA kernel reads them) through ldmatrix.trans,
//    which turns source-major 8 x 8 blocks into K-major core matrices.
//  * A window of at most 128 sources of one partner level keeps every level
//    sum below 2^24 (as for the warp-MMA kernel's tiles); at its end the
//    warps holding rows read D_0..D_5 (tcgen05.ld), fold them into
//    double-float running sums kept in tensor-memory columns 96 (hi) and
//    112 (lo), and the next window's first MMA overwrites D.
// Staging of stage i + 1 (cp.async, warp 0, which also publishes the next
// stage's geometry) overlaps stage i, and one CTA barrier per stage hands the
// operands to the issuing thread.  Every wait on the tensor cores is bounded;
// a CTA that gives up counts a timeout, stops (all its threads together),
// frees its tensor memory and returns, and CTAs that start after a timeout
// return at once: the host rejects the result.
constexpr int k5M = 64;            // MMA M: target rows per pass
constexpr int k5N = 16;            // right-hand sides (digits past ldq are zero)
constexpr int k5PlaneEntries = 2048;
constexpr int k5MaxStage = 64;     // sources per stage at most (passes of <= 32 targets)
constexpr int k5Win = 128;         // sources per accumulation window
constexpr int k5RawStride = 192;   // bytes per staged source: 6 planes x 16 bf16 digits
constexpr long k5MaxSpin = 1L << 22;
constexpr uint32_t k5Cols = 128;   // tensor-memory columns: D_L at 16 L, sums at 96 (hi) and 112 (lo)

__device__ int g_oz5_timeouts;

struct Oz5Layout {
    static constexpr int kAPlane = k5PlaneEntries * 2;           // 4 KB per entry-digit plane
    static constexpr int kBPlane = k5N * k5MaxStage * 2;         // 2 KB per q^-digit plane (at most)
    static constexpr int kA = kOzDigits * kAPlane;
    static constexpr int kB = kOzDigits * kBPlane;
    static constexpr int kRaw = k5MaxStage * k5RawStride;
    static constexpr int kY = k5MaxStage * 32;                    // (hi, lo) float4 per source
    static constexpr int kStaging = kRaw + kY;
    static constexpr int kT = k5M * 32;                           // target (hi, lo) float4
    static constexpr int bytes = kA + kB + 2 * kStaging + kT + k5M * 8;
    static_assert(kA % 1024 == 0 && kB % 1024 == 0 && kStaging % 16 == 0, "aligned regions");
};

__device__ __forceinline__ uint32_t oz5_su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, LBO 128 B (next core matrix
// along K), SBO sbo bytes (next 8-row group)
__device__ __forceinline__ uint64_t oz5_desc(uint32_t saddr, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool oz5_wait(uint32_t mbar, uint32_t parity) {
    for (long it = 0; it < k5MaxSpin; ++it) {
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

__device__ __forceinline__ void oz5_ld4(uint32_t taddr, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}

__device__ __forceinline__ void oz5_st4(uint32_t taddr, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(__float_as_uint(v[0])),
                 "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])));
}

// stage geometry at stream position pos of the chunk: its partner level and
// the sources it takes (up to kst, never past the level run)
__device__ __forceinline__ void oz5_stage(const PartnerChunk &pc, const int *plev, const int *runend, int pos,
                                          int kst, int &lv, int &fill) {
    int plo = 0, phi = pc.n - 1;
    while (plo < phi) {
        const int mid = (plo + phi + 1) >> 1;
        if (pc.pre[mid] <= pos) plo = mid;
        else phi = mid - 1;
    }
    lv = plev[plo];
    fill = min(kst, pc.pre[runend[plo]] - pos);
}

// warps 0 and 1 gather a stage: thread k < 64 copies the digits and
// coordinates of source k (when below fill)
__device__ __forceinline__ void oz5_stage_load(const KsumOzArgs &a, const PartnerChunk &pc, int pos, int fill,
                                               unsigned char *buf) {
    const int k = threadIdx.x;
    if (k < fill) {
        const int64_t src = chunk_source(pc, pos + k);
        const unsigned char *dg = reinterpret_cast<const unsigned char *>(a.dig) + src * k5RawStride;
#pragma unroll
        for (int p = 0; p < k5RawStride / 16; ++p) oz_cp16(buf + k * k5RawStride + 16 * p, dg + 16 * p);
        float *y = reinterpret_cast<float *>(buf + Oz5Layout::kRaw) + k * 8;
        oz_cp16(y, a.ys + src * 8);
        oz_cp16(y + 4, a.ys + src * 8 + 4);
    }
}

// fold D_0..D_5 of the lane's row into its double-float sums (lanes 0-15 of
// the warp hold rows; the other lanes fold unused data)
__device__ __forceinline__ void oz5_flush(uint32_t tmem, const int *sfd, int lv) {
    const uint32_t lb = tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < k5N; c0 += 4) {
        uint32_t C[kOzDigits][4], H[4], Lw[4];
#pragma unroll
        for (int L = 0; L < kOzDigits; ++L) oz5_ld4(lb + 16 * L + c0, C[L]);
        oz5_ld4(lb + 96 + c0, H);
        oz5_ld4(lb + 112 + c0, Lw);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float ah[4], al[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float fac = ldexpf(1.0f, sfd[lv * 16 + c0 + j]);
            const float c[kOzDigits] = {__uint_as_float(C[0][j]), __uint_as_float(C[1][j]), __uint_as_float(C[2][j]),
                                        __uint_as_float(C[3][j]), __uint_as_float(C[4][j]), __uint_as_float(C[5][j])};
            const float tail = fmaf(c[5], 1.0f / 65536.0f, fmaf(c[4], 1.0f / 256.0f, c[3]));
            float h, l, e2, e3;
            two_sum_ordered(c[0], c[1] * (1.0f / 256.0f), h, l);
            two_sum_ordered(h, c[2] * (1.0f / 65536.0f), h, e2);
            l = fmaf(tail, 1.0f / 16777216.0f, l + e2);
            float sh = __uint_as_float(H[j]), sl = __uint_as_float(Lw[j]);
            two_sum_ordered(sh, h * fac, sh, e3);
            sl = sl + (e3 + l * fac);
            fast_two_sum(sh, sl, ah[j], al[j]);
        }
        oz5_st4(lb + 96 + c0, ah);
        oz5_st4(lb + 112 + c0, al);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

template <int KID, int D>
__global__ void __launch_bounds__(kOzThreads, 3) ksum_oz5_kernel(KsumOzArgs a) {
    using Lay = Oz5Layout;
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ PartnerChunk pc;
    __shared__ unsigned long long bound_slot;
    __shared__ int runend[kPartnerChunk];
    __shared__ int plev[kPartnerChunk];
    __shared__ int sfd[kOzLevels * 16];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ int s_skip;
    __shared__ int s_geo[2][2];  // (level, fill) of the next stage, by stage parity
    unsigned char *sA = smraw;
    unsigned char *sB = smraw + Lay::kA;
    unsigned char *stg0 = smraw + Lay::kA + Lay::kB;
    float4 *tx = reinterpret_cast<float4 *>(stg0 + 2 * Lay::kStaging);
    float *sc0s = reinterpret_cast<float *>(tx + 2 * k5M);
    int *rowE = reinterpret_cast<int *>(sc0s + k5M);

    const int64_t g = a.tnodes[blockIdx.x];
    const int T = a.t_cnt[g];
    if (threadIdx.x == 0) s_skip = *reinterpret_cast<volatile int *>(&g_oz5_timeouts);
    __syncthreads();
    if (T == 0 || s_skip != 0) return;
    const int64_t toff = a.t_off[g];
    const int64_t e0 = a.ptr[g], e1 = a.ptr[g + 1];
    const int ldq = a.ldq;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kOzLevels * 16; i += kOzThreads) sfd[i] = a.fd[i];
    const double kb_node = oz_node_bound(a, g, e0, e1, &bound_slot);
    if (!(kb_node < INFINITY)) {
        for (int q = tid; q < T * ldq; q += kOzThreads) a.out[toff * ldq + q] = NAN;
        return;
    }
    // operand and staging regions start at 0 (stale contents stay finite)
    for (int i = tid; i < (Lay::kA + Lay::kB + 2 * Lay::kStaging) / 16; i += kOzThreads)
        reinterpret_cast<uint4 *>(smraw)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz5_su32(&mbar)));
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(oz5_su32(&tslot)),
                     "r"(k5Cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tslot;
    const uint32_t mb = oz5_su32(&mbar);
    int nst = 0;             // stages committed by this CTA
    bool pending = false;    // the last committed stage has not been waited for
    bool timed_out = false;  // block-uniform: a wait gave up

    for (int tb = 0; tb < T && !timed_out; tb += k5M) {
        const int tcount = min(k5M, T - tb);
        // plane shape of the pass: rows x kst sources (kst / 16 K-steps)
        const int rows = tcount <= 32 ? 32 : 64;
        const int kst = k5PlaneEntries / rows;
        const uint32_t sbo_a = (uint32_t)(kst / 8) * 128u;  // also B's row-group stride
        const int nitems = tcount * (kst / 8);
        const int row = tid < nitems ? tid % tcount : 0, oct = tid < nitems ? tid / tcount : 0;
        const int fwarps = (tcount + 15) / 16;  // warps whose lanes 0-15 hold rows
        const uint64_t desc_a = oz5_desc(oz5_su32(sA), sbo_a), desc_b = oz5_desc(oz5_su32(sB), sbo_a);
        for (int q = tid; q < 2 * tcount; q += kOzThreads)
            tx[q] = reinterpret_cast<const float4 *>(a.xt + (toff + tb + (q >> 1)) * 8)[q & 1];
        __syncthreads();
        // row exponents: the four lanes of a quad split the row's partners
        for (int r0 = 0; r0 < tcount; r0 += kOzThreads / 4) {
            const int rr = r0 + (tid >> 2);
            const float4 xh = tx[2 * (rr < tcount ? rr : 0)];
            const float gap2 = oz_point_gap2<D>(xh, a, e0, e1, tid & 3);
            if (rr < tcount && (tid & 3) == 0) {
                const int E = oz_row_exponent(gap2, kb_node);
                rowE[rr] = E;
                sc0s[rr] = ldexpf(1.0f, 8 - E);
            }
        }
        // running sums of the pass start at 0
        if (warp < 4) {
            const float z[4] = {0.f, 0.f, 0.f, 0.f};
            const uint32_t lb = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
            for (int c = 96; c < 128; c += 4) oz5_st4(lb + c, z);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        __syncthreads();
        int win = 0, wlv = -1;
        for (int64_t e = e0; e < e1 && !timed_out;) {
            load_partner_chunk<kOzThreads>(pc, e, e1, a.col, a.s_off, a.s_cnt);
            const int nchunk = pc.n, total = pc.pre[pc.n];
            for (int q = tid; q < nchunk; q += kOzThreads) plev[q] = a.level[a.col[e + q]];
            __syncthreads();
            if (tid == 0) {
                int end = nchunk;
                for (int p = nchunk - 1; p >= 0; --p) {
                    if (p + 1 < nchunk && plev[p + 1] != plev[p]) end = p + 1;
                    runend[p] = end;
                }
            }
            __syncthreads();
            e += nchunk;
            int pos = 0, cur = 0, lv, fill;
            oz5_stage(pc, plev, runend, 0, kst, lv, fill);
            oz5_stage_load(a, pc, 0, fill, stg0);
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
            while (pos < total) {
                unsigned char *buf = stg0 + cur * Lay::kStaging;
                const int npos = pos + fill;
                // warp 0: the next stage's geometry (published at this stage's
                // barrier) and its data, into the other buffer (free: its last
                // reads came before the previous stage's barrier)
                if (warp < 2) {
                    int nlv = 0, nfill = 0;
                    if (npos < total) {
                        oz5_stage(pc, plev, runend, npos, kst, nlv, nfill);
                        oz5_stage_load(a, pc, npos, nfill, stg0 + (cur ^ 1) * Lay::kStaging);
                    }
                    if (tid == 0) {
                        s_geo[nst & 1][0] = nlv;
                        s_geo[nst & 1][1] = nfill;
                    }
                }
                const bool fresh = win == 0 || lv != wlv || win + fill > k5Win;
                // the entries of one (row, source octet) per thread, digits packed in registers
                const bool has = tid < nitems;
                uint32_t w[kOzDigits][4];
                if (has) {
                    const float4 xh = tx[2 * row], xl = tx[2 * row + 1];
                    const float sc0 = sc0s[row];
                    const float4 *cy = reinterpret_cast<const float4 *>(buf + Lay::kRaw);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float kh[2], kl[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int k = 8 * oct + 2 * j + u;
                            kh[u] = 0.f;
                            kl[u] = 0.f;
                            if (k < fill) oz_entry<KID, D>(xh, xl, cy[2 * k], cy[2 * k + 1], kh[u], kl[u]);
                        }
                        float r[2];
#pragma unroll
                        for (int s = 0; s < kOzDigits; ++s) {
                            float dg[2];
#pragma unroll
                            for (int u = 0; u < 2; ++u) dg[u] = oz_digit(s, kh[u], kl[u], sc0, r[u]);
                            w[s][j] = oz_pack(dg[0], dg[1]);
                        }
                    }
                }
                // the previous stage's MMAs are done: operands free, D readable
                bool ok = true;
                if (pending) {
                    ok = oz5_wait(mb, (uint32_t)((nst - 1) & 1));
                    pending = false;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (fresh && win > 0 && warp < fwarps) oz5_flush(tmem, sfd, wlv);
                if (fresh) {
                    win = 0;
                    wlv = lv;
                }
                win += fill;
                if (has) {
                    const uint32_t off = (uint32_t)(row >> 3) * sbo_a + (uint32_t)oct * 128u + (uint32_t)(row & 7) * 16u;
#pragma unroll
                    for (int s = 0; s < kOzDigits; ++s)
                        *reinterpret_cast<uint4 *>(sA + s * Lay::kAPlane + off) =
                            make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
                }
                {
                    // B: per (plane t, column octet o, 32-source block) four 8 x 8
                    // source-major matrices, transposed into K-major core matrices;
                    // the 12 (t, o) pairs of a block are spread over the warps
                    const uint32_t src0 = oz5_su32(buf) + (uint32_t)lane * k5RawStride;
                    unsigned char *dst0 = sB + (lane >> 2) * 16 + (lane & 3) * 4;
                    for (int sb = 0; sb < kst / 32; ++sb)
                        for (int to = warp; to < 2 * kOzDigits; to += kOzThreads / 32) {
                            // to = 2 t + o: plane t, column octet o
                            uint32_t R0, R1, R2, R3;
                            oz_ldsm_x4_trans(src0 + (uint32_t)(32 * sb) * k5RawStride + (uint32_t)to * 16, R0, R1,
                                             R2, R3);
                            unsigned char *dst = dst0 + (uint32_t)to * sbo_a + (uint32_t)(4 * sb) * 128u;
                            *reinterpret_cast<uint32_t *>(dst) = R0;
                            *reinterpret_cast<uint32_t *>(dst + 128) = R1;
                            *reinterpret_cast<uint32_t *>(dst + 256) = R2;
                            *reinterpret_cast<uint32_t *>(dst + 384) = R3;
                        }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                asm volatile("cp.async.wait_all;" ::: "memory");  // the next stage's data (warp 0)
                if (__syncthreads_or(!ok)) {
                    timed_out = true;
                    break;
                }
                if (tid == kOzThreads - 1) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    for (int ks = 0; ks < kst / 16; ++ks)
#pragma unroll
                        for (int s = 0; s < kOzDigits; ++s) {
                            // the address field counts 16-byte units (no carry out of it)
                            const uint64_t ad = desc_a + (uint64_t)((s * Lay::kAPlane + ks * 256) >> 4);
                            const uint64_t bd = desc_b + (uint64_t)((ks * 256) >> 4);
                            // BF16 x BF16 -> F32, both K-major, M = 64, N = 16 (6 - s)
                            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                                   ((uint32_t)(k5N * (kOzDigits - s) >> 3) << 17) |
                                                   ((uint32_t)(k5M >> 4) << 24);
                            const uint32_t en = (fresh && ks == 0 && s == 0) ? 0u : 1u;
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                    tmem + (uint32_t)(16 * s)),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(en));
                        }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                        : "memory");
                }
                pending = true;
                pos = npos;
                lv = s_geo[nst & 1][0];
                fill = s_geo[nst & 1][1];
                ++nst;
                cur ^= 1;
            }
        }
        if (timed_out) break;
        // last window of the pass, then the rows' sums scaled out
        bool ok = true;
        if (pending) {
            ok = oz5_wait(mb, (uint32_t)((nst - 1) & 1));
            pending = false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp < fwarps) {
            if (win > 0) oz5_flush(tmem, sfd, wlv);
            const uint32_t lb = tmem + ((uint32_t)(32 * warp) << 16);
            uint32_t H[k5N], Lw[k5N];
#pragma unroll
            for (int c = 0; c < k5N; c += 4) {
                oz5_ld4(lb + 96 + c, H + c);
                oz5_ld4(lb + 112 + c, Lw + c);
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int orow = 16 * warp + lane;
            if (lane < 16 && orow < tcount) {
                const double sc = ldexp(a.scale, rowE[orow] - 16);
#pragma unroll
                for (int c = 0; c < k5N; ++c)
                    if (c < ldq)
                        a.out[(toff + tb + orow) * ldq + c] =
                            ((double)__uint_as_float(H[c]) + (double)__uint_as_float(Lw[c])) * sc * a.colscale[c];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(!ok)) timed_out = true;
    }
    if (timed_out && tid == 0) atomicAdd(&g_oz5_timeouts, 1);
    asm volatile("cp.async.wait_all;" ::: "memory");  // a stopped CTA's prefetch
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(k5Cols));
}

template <int KID, int D>
static void launch_oz5(const KsumOzArgs &a, int64_t ntn, cudaStream_t s) {
    auto kern = ksum_oz5_kernel<KID, D>;
    allow_max_dynamic_smem((const void *)kern);
    kern<<<(unsigned)ntn, kOzThreads, Oz5Layout::bytes, s>>>(a);
    LAUNCHED();
}

int oz5_take_timeouts() {
    int v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_oz5_timeouts, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (v) cudaMemcpyToSymbol(g_oz5_timeouts, &z, sizeof(int));
    return v;
}

bool coupling_oz_supported(const smash_h2 *h, int kid, int ldq) {
    return !dd_exact_coupling(h) && ldq <= 16 && h->tau < 1.0 && h->L < kOzLevels &&
           (kid == SMASH_K_INVR || kid == SMASH_K_CAUCHY1D) && h->nnodes > h->nroots;
}

void coupling_oz(const smash_h2 *h, int kid, const double *qhat, double *zhat, int ldq, cudaStream_t s, bool tc05) {
    const Side &R = h->row;
    const Side &Cs = *h->col;
    const int NC = (ldq <= 8 && !tc05) ? 8 : 16;
    const int64_t nsk = std::max<int64_t>(Cs.total_skel, 1);
    Arena tmp(s);
    unsigned long long *cmax = tmp.alloc<unsigned long long>(kOzLevels * 16);
    int *fd = tmp.alloc<int>(kOzLevels * 16);
    int *fref = tmp.alloc<int>(16);
    double *colscale = tmp.alloc<double>(16);
    __nv_bfloat16 *dig = tmp.alloc<__nv_bfloat16>((size_t)nsk * kOzDigits * NC);
    CK(cudaMemsetAsync(cmax, 0, kOzLevels * 16 * sizeof(unsigned long long), s));
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((h->nnodes + 7) / 8, 8 * (int64_t)h->num_sms));
    oz_colmax_kernel<<<blocks, 256, 0, s>>>(qhat, ldq, h->nnodes, h->level, Cs.k, Cs.sk_off, cmax);
    LAUNCHED();
    oz_scales_kernel<<<1, 32, 0, s>>>(cmax, fd, fref, colscale);
    LAUNCHED();
    oz_digits_kernel<<<blocks, 256, 0, s>>>(qhat, ldq, NC, h->nnodes, h->level, Cs.k, Cs.sk_off, fd, fref, dig);
    LAUNCHED();
    KsumOzArgs a{};
    a.tnodes = h->nonroot_list; a.t_off = R.sk_off; a.t_cnt = R.k;
    a.ptr = h->adm_ptr; a.col = h->adm_col; a.s_off = Cs.sk_off; a.s_cnt = Cs.k;
    a.xt = R.skel_dd; a.ys = Cs.skel_dd; a.dig = dig; a.fd = fd; a.colscale = colscale;
    a.level = h->level; a.cell = h->cell; a.out = zhat; a.scale = 1.0 / h->s; a.ldq = ldq; a.dim = h->dim;
    const int64_t ntn = h->nnodes - h->nroots;
    if (!tc05) launch_oz_kernel<false>(h, kid, a, ntn, s);
    else if (kid == SMASH_K_CAUCHY1D) launch_oz5<SMASH_K_CAUCHY1D, 1>(a, ntn, s);
    else if (h->dim == 3) launch_oz5<SMASH_K_INVR, 3>(a, ntn, s);
    else if (h->dim == 2) launch_oz5<SMASH_K_INVR, 2>(a, ntn, s);
    else launch_oz5<SMASH_K_INVR, 1>(a, ntn, s);
    tmp.release();
}

// ------------------------------------------------------------------ near field
// The near field (3.20) with the same digit-split products: sources are the
// points of the neighbouring leaves, q the sorted input vectors (one exponent
// per column), entries from the normalised two-float coordinates, or from the
// exact three-float ones for the rare pairs closer than 2^-8 of the cube
// (oz_entry_near).  A row's exponent comes from its nearest source; nodes with
// coincident points or a spread of distances above 2^12 are flagged in
// `fallback` and left to the double-float kernel.

// max |q_pc| per column over all points (non-negative doubles order as their bits)
__global__ void oz_colmax_flat_kernel(const double *__restrict__ q, int64_t n, int ldq,
                                      unsigned long long *__restrict__ cmax) {
    __shared__ unsigned long long sm[16];
    if (threadIdx.x < 16) sm[threadIdx.x] = 0ull;
    __syncthreads();
    // the grid stride is a multiple of ldq (a power of two <= 16): one column per thread
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (int)(i % ldq);
    unsigned long long m = 0ull;
    for (; i < n * ldq; i += stride) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(q[i]));
        m = b > m ? b : m;
    }
    if (m) atomicMax(&sm[c], m);
    __syncthreads();
    if (threadIdx.x < ldq && sm[threadIdx.x]) atomicMax(&cmax[threadIdx.x], sm[threadIdx.x]);
}

// dig[(p * 6 + t) * NC + c] = b_t of q_pc 2^-fref_c (zero for c >= ldq)
__global__ void oz_digits_flat_kernel(const double *__restrict__ q, int64_t n, int ldq, int NC,
                                      const int *__restrict__ fref, __nv_bfloat16 *__restrict__ dig) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * NC) return;
    const int64_t p = i / NC;
    const int c = (int)(i % NC);
    double x = c < ldq ? ldexp(q[p * ldq + c], -fref[c]) : 0.0;
#pragma unroll
    for (int u = 0; u < kOzDigits; ++u) {
        x *= 256.0;
        const double d = rint(x);
        x -= d;
        dig[(p * kOzDigits + u) * NC + c] = __float2bfloat16_rn((float)d);
    }
}

bool near_oz_supported(const smash_h2 *h, int kid, int ldq) {
    return ldq <= 16 && (kid == SMASH_K_INVR || kid == SMASH_K_CAUCHY1D) && h->nleaves > 0 && h->xs_dd && h->ys_dd &&
           h->xs_x3 && h->ys_x3;
}

void near_oz(const smash_h2 *h, int kid, const double *qs, double *zs, int ldq, int *fallback, cudaStream_t s) {
    const int NC = ldq <= 8 ? 8 : 16;
    Arena tmp(s);
    unsigned long long *cmax = tmp.alloc<unsigned long long>(kOzLevels * 16);
    int *fd = tmp.alloc<int>(kOzLevels * 16);
    int *fref = tmp.alloc<int>(16);
    double *colscale = tmp.alloc<double>(16);
    __nv_bfloat16 *dig = tmp.alloc<__nv_bfloat16>((size_t)std::max<int64_t>(h->ny, 1) * kOzDigits * NC);
    CK(cudaMemsetAsync(cmax, 0, kOzLevels * 16 * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(fallback, 0, sizeof(int) * (size_t)h->nleaves, s));
    const int64_t work = h->ny * ldq;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 4 * (int64_t)h->num_sms));
    oz_colmax_flat_kernel<<<blocks, 256, 0, s>>>(qs, h->ny, ldq, cmax);
    LAUNCHED();
    oz_scales_kernel<<<1, 32, 0, s>>>(cmax, fd, fref, colscale);
    LAUNCHED();
    const int64_t nd = h->ny * NC;
    oz_digits_flat_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(qs, h->ny, ldq, NC, fref, dig);
    LAUNCHED();
    KsumOzArgs a{};
    a.tnodes = h->leaf_list; a.t_off = h->rs; a.t_cnt = h->rc;
    a.ptr = h->near_ptr; a.col = h->near_col; a.s_off = h->cs; a.s_cnt = h->cc;
    a.xt = h->xs_dd; a.ys = h->ys_dd; a.xt3 = h->xs_x3; a.ys3 = h->ys_x3;
    a.dig = dig; a.fd = fd; a.colscale = colscale; a.level = h->level; a.cell = h->cell;
    a.out = zs; a.scale = 1.0 / h->s; a.ldq = ldq; a.dim = h->dim;
    {
        const double nrm = ldexp(1.0, h->dd_e) / h->s;  // in (1/2, 1]
        a.n3h = (float)nrm;
        a.n3l = (float)(nrm - (double)a.n3h);
    }
    a.fallback = fallback; a.same = h->same; a.boxes = h->nroots == 1;
    launch_oz_kernel<true>(h, kid, a, h->nleaves, s);
    tmp.release();
}

}  // namespace smash

using namespace smash;

// Leaves that the digit-split near field leaves to the double-float kernel:
// the classification of near_oz run on zero right-hand sides (it depends on
// the points only), flags copied back and mapped to global node ids.
extern "C" smash_status smash_near_fallback_leaves(smash_handle h, int32_t *leaves, int64_t cap, int64_t *count) {
    try {
        if (!h || !count) fail(SMASH_EINVAL, "NULL argument");
        if (cap < 0 || (cap > 0 && !leaves)) fail(SMASH_EINVAL, "leaves must hold cap entries");
        *count = 0;
        const int ldq = 8;
        if (!near_oz_supported(h, h->kernel_id, ldq)) return SMASH_OK;
        cudaStream_t s = h->stream;
        Arena tmp(s);
        double *qs = tmp.alloc<double>((size_t)h->ny * ldq);
        double *zs = tmp.alloc<double>((size_t)h->nx * ldq);
        int *fb = tmp.alloc<int>((size_t)std::max<int64_t>(h->nleaves, 1));
        CK(cudaMemsetAsync(qs, 0, sizeof(double) * (size_t)h->ny * ldq, s));
        CK(cudaMemsetAsync(zs, 0, sizeof(double) * (size_t)h->nx * ldq, s));
        near_oz(h, h->kernel_id, qs, zs, ldq, fb, s);
        std::vector<int> flags((size_t)h->nleaves);
        std::vector<int32_t> ids((size_t)h->nleaves);
        CK(cudaMemcpyAsync(flags.data(), fb, sizeof(int) * (size_t)h->nleaves, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(ids.data(), h->leaf_list, sizeof(int32_t) * (size_t)h->nleaves, cudaMemcpyDeviceToHost,
                           s));
        CK(cudaStreamSynchronize(s));
        tmp.release();
        for (int64_t i = 0; i < h->nleaves; ++i) {
            if (!flags[(size_t)i]) continue;
            if (*count < cap) leaves[*count] = ids[(size_t)i];
            ++*count;
        }
        return SMASH_OK;
    } catch (const Error &e) {
        set_last_error(e.msg.c_str());
        return e.status;
    }
}
