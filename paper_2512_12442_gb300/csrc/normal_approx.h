// Generated by fit_normal.py (minimax-relative-error fits against SciPy); do not edit.
// Standard normal CDF:  Phi(-a) = exp(-a^2/2) G(u),  u = 2/(1 + 0.35 a) - 1.
// Quantile:  z = (2p - 1) sqrt(2) E,  w = -log(4p(1-p)) = -ln2 lg; sqrt(2) E a polynomial in
//   (w - mid)/half for w < 5, else in (sqrt(w) - mid)/half on [sqrt 5, 9.3].
#pragma once
#define NRM_CDF_C0 0.35f
#define NRM_PPF_LG_SPLIT -7.213475f
static __device__ __forceinline__ float nrm_cdf_g(float u) { return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(0.00038237785f, u, -0.0004815742f), u, -0.0033990606f), u, 0.0025471582f), u, 0.040660013f), u, 0.12129871f), u, 0.2123704f), u, 0.12662213f); }
static __device__ __forceinline__ float nrm_ppf_mid_lg(float lg) { const float v = fmaf(lg, -0.27725887f, -1.0f); return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(0.00027242687f, v, -0.0011000016f), v, -0.00056541926f), v, 0.012006258f), v, -0.027723704f), v, -0.03691327f), v, 0.8720091f), v, 2.1233132f); }
static __device__ __forceinline__ float nrm_ppf_tail(float s) {
    const float v = fmaf(s, 0.28312844f, -1.6330944f);
    return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(-0.008913594f, v, -0.02937258f), v, 0.050443884f), v, 0.045742813f), v, -0.057369407f), v, -0.03477084f), v, 0.033149317f), v, 0.0048911464f), v, 0.0002131089f), v, -0.0056126337f), v, -0.0072218487f), v, 5.0440493f), v, 7.955928f);
}
