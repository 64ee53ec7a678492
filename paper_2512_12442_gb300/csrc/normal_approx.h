// Generated by fit_normal.py (weighted least-squares fits against SciPy); do not edit.
// Standard normal CDF:  Phi(-a) = exp(-a^2/2) G(u),  u = 2/(1 + 0.3 a) - 1.
// Quantile:  z = (2p - 1) sqrt(2) E,  w = -log(4p(1-p)) = -ln2 lg; sqrt(2) E a polynomial in
//   (w - mid)/half for w < 5, else in (sqrt(w) - mid)/half on [sqrt 5, 4] or [4, 9.3].
#pragma once
#define NRM_CDF_C0 0.3f
#define NRM_PPF_LG_SPLIT -7.213475f
static __device__ __forceinline__ float nrm_cdf_g(float u) { return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(0.00015558592f, u, -0.00012750691f), u, -0.0014855539f), u, -0.00030872854f), u, 0.014785714f), u, 0.05715546f), u, 0.1255648f), u, 0.19327505f), u, 0.1109853f); }
static __device__ __forceinline__ float nrm_ppf_mid_lg(float lg) { const float v = fmaf(lg, -0.27725887f, -1.0f); return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(6.526152e-05f, v, 0.0003015834f), v, -0.0012235859f), v, -0.00061469385f), v, 0.012077982f), v, -0.027700128f), v, -0.036926124f), v, 0.87200636f), v, 2.1233137f); }
static __device__ __forceinline__ float nrm_ppf_tail(float s) {
    const bool hi = s >= 4.0f;
    const float v = fmaf(s, hi ? 0.3773585f : 1.1338305f, hi ? -2.509434f : -3.5353222f);
    return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf((hi ? -3.932736e-05f : 5.9549446e-05f), v, (hi ? 7.3349845e-05f : -9.274671e-05f)), v, (hi ? -8.588027e-05f : -0.00018491283f)), v, (hi ? 0.00021497569f : 0.00088025356f)), v, (hi ? -0.00046392935f : -0.0019435677f)), v, (hi ? 0.00067339226f : 0.0033132613f)), v, (hi ? -0.000115283474f : -0.0052467235f)), v, (hi ? -0.005105783f : 0.007877281f)), v, (hi ? 3.7812285f : 1.2518032f)), v, (hi ? 9.214942f : 4.173809f));
}
