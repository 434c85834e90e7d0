// kappa_f32.cuh -- kernel entries in FP32 from normalised differences
// d'' = (x - y)/s (the frame of the mixed-precision kernel sums):
// 1/|x-y| = (1/s)/|d''|, 1/(x-y) = (1/s)/d'', log|x-y| = log s + log|d''|,
// exp(-|x-y|)/|x-y| with |x-y| = s|d''|, and the log gradients
// d_a/(2 pi |d|^2) = (1/s) d''_a/(2 pi |d''|^2).  The factor 1/s of 1/r,
// 1/(x-y) and the gradients is applied to the finished sums.  Coincident
// points give 0.
#pragma once

#include "internal.cuh"

namespace smash {

// kernel entry from the FP32 difference d (normalised units); s_f = s,
// inv_s = 1/s (rounded once), log_s = log s
template <int KID, int D>
__device__ __forceinline__ float kappa_f32(const float *d, float s_f, float inv_s, float log_s) {
    if (KID == SMASH_K_CAUCHY1D) return d[0] != 0.f ? __frcp_rn(d[0]) : 0.f;
    float r2 = d[0] * d[0];
    if (D > 1) r2 = fmaf(d[1], d[1], r2);
    if (D > 2) r2 = fmaf(d[2], d[2], r2);
    if (r2 == 0.f) return 0.f;
    // y-gradient of -(1/2pi) log (the factor 1/s is applied to the sums)
    if (KID == SMASH_K_DLP1) return d[0] * (0.15915494309189535f / r2);
    if (KID == SMASH_K_DLP2) return d[1] * (0.15915494309189535f / r2);
    if (KID == SMASH_K_INVR) return rsqrtf(r2);
    if (KID == SMASH_K_LOG) return fmaf(0.5f, __logf(r2), log_s);
    float ri = rsqrtf(r2);
    float r = r2 * ri * s_f;
    return __expf(-r) * (ri * inv_s);  // SMASH_K_YUKAWA
}

}  // namespace smash
