// dd_arith.cuh -- double-float (hi + lo float) arithmetic shared by the
// kernel-sum kernels: error-free transformations and the kernel entries
// 1/|d| and 1/d evaluated to ~2^-46 relative precision on the FP32 pipe.
// Every translation unit that includes it is compiled with --fmad=false, so
// each fused operation is an explicit fmaf.
#pragma once

#include <cuda_runtime.h>

#include "../../include/smash.h"

namespace smash {

// ------------------------------------------------------------------ error-free transforms
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    e = b - (s - a);
}

// The same s and e as two_sum: with the operands ordered by magnitude the
// three-operation form above is exact (Dekker), so the error term -- which
// is unique -- comes out bit for bit equal.  The compare and the two selects
// issue on the ALU pipe, leaving three operations on the FP32 pipe instead
// of six.
__device__ __forceinline__ void two_sum_ordered(float a, float b, float &s, float &e) {
    const bool a_big = fabsf(a) >= fabsf(b);
    const float big = a_big ? a : b;
    const float small = a_big ? b : a;
    s = a + b;
    e = small - (s - big);
}

// ------------------------------------------------------------------ differences
// x - y from three-float coordinates, as a normalised double-float
__device__ __forceinline__ void diff3(float xh, float xm, float xl, float yh, float ym, float yl, float &dh,
                                      float &dl) {
    float a, ea, b, eb;
    two_sum_ordered(xh, -yh, a, ea);
    two_sum_ordered(xm, -ym, b, eb);
    float c = xl - yl;
    float s, t;
    two_sum_ordered(a, b, s, t);
    t = t + ((ea + eb) + c);
    fast_two_sum(s, t, dh, dl);
}

// ------------------------------------------------------------------ kernel entries
// kappa'' = 1/|d| (3D/2D/1D) or 1/d (Cauchy, 1D) in double-float; d = (dh + dl) per axis.
template <int KID, int D>
__device__ __forceinline__ void kappa_dd(const float *dh, const float *dl, float &kh, float &kl) {
    if (KID == SMASH_K_CAUCHY1D) {
        float h = dh[0], l = dl[0];
        float dsum, derr;
        fast_two_sum(h, l, dsum, derr);  // |h| >= |l| unless h == 0
        if (dsum == 0.f && derr == 0.f) { kh = 0.f; kl = 0.f; return; }
        float y0 = __frcp_rn(dsum);
        float uh = dsum * y0;
        float ul = fmaf(dsum, y0, -uh);
        ul = fmaf(derr, y0, ul);
        float ee = (1.0f - uh) - ul;
        float c = y0 * ee;
        fast_two_sum(y0, c, kh, kl);
        return;
    }
    // r2 = sum_a (dh + dl)^2 as a double-float
    float p[3], e[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < D) {
            p[a] = dh[a] * dh[a];
            float t = fmaf(dh[a], dh[a], -p[a]);
            t = fmaf(2.0f * dh[a], dl[a], t);
            e[a] = fmaf(dl[a], dl[a], t);
        } else {
            p[a] = 0.f;
            e[a] = 0.f;
        }
    }
    float s1, t1, rh, t2;
    two_sum_ordered(p[0], p[1], s1, t1);
    two_sum_ordered(s1, p[2], rh, t2);
    float rl = ((e[0] + e[1]) + (e[2] + t1)) + t2;
    fast_two_sum(rh, rl, rh, rl);
    if (rh == 0.f) { kh = 0.f; kl = 0.f; return; }
    float y0 = rsqrtf(rh);
    float th = y0 * y0;
    float tl = fmaf(y0, y0, -th);
    float uh = rh * th;
    float ul = fmaf(rh, th, -uh);
    ul = fmaf(rh, tl, ul);
    ul = fmaf(rl, th, ul);
    float ee = (1.0f - uh) - ul;
    float c = y0 * (0.5f * ee);
    fast_two_sum(y0, c, kh, kl);
}

}  // namespace smash
