// Generated by fit_normal.py (weighted least-squares fits against SciPy); do not edit.
// Standard normal CDF:  Phi(-a) = exp(-a^2/2) G(u),  u = 2/(1 + 0.3 a) - 1.
// Quantile:  z = sqrt(2) (2p - 1) E,  w = -log(4p(1-p)); E a polynomial in
//   (w - mid)/half for w < 5, else in (sqrt(w) - mid)/half on [sqrt 5, 4] or [4, 9.3].
#pragma once
#define NRM_CDF_C0 0.3f
static __device__ __forceinline__ float nrm_cdf_g(float u) { return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(-2.0718906e-05f, u, 1.8270206e-05f), u, 0.00017996767f), u, -0.00014484004f), u, -0.001497441f), u, -0.0003035786f), u, 0.014788394f), u, 0.057155002f), u, 0.12556458f), u, 0.19327505f), u, 0.11098531f); }
static __device__ __forceinline__ float nrm_ppf_mid(float w) { const float v = (w - 2.5f) * 0.4f; return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(-3.4737714e-05f, v, 3.4992754e-05f), v, 0.00028700175f), v, -0.00084457075f), v, -0.00048637245f), v, 0.008528634f), v, -0.019573683f), v, -0.02610859f), v, 0.6166007f), v, 1.5014094f); }
static __device__ __forceinline__ float nrm_ppf_tail(float s) {
    const bool hi = s >= 4.0f;
    const float v = (s - (hi ? 6.65f : 3.118034f)) * (hi ? 0.3773585f : 1.1338305f);
    return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf((hi ? -2.7808643e-05f : 4.210782e-05f), v, (hi ? 5.1866173e-05f : -6.558183e-05f)), v, (hi ? -6.0726517e-05f : -0.00013075312f)), v, (hi ? 0.00015201076f : 0.00062243326f)), v, (hi ? -0.00032804758f : -0.0013743099f)), v, (hi ? 0.00047616023f : 0.0023428295f)), v, (hi ? -8.1517726e-05f : -0.0037099938f)), v, (hi ? -0.003610334f : 0.0055700787f)), v, (hi ? 2.6737323f : 0.8851585f)), v, (hi ? 6.5159483f : 2.9513285f));
}
