// Generated by fit_normal.py (minimax-relative-error fits against SciPy); do not edit.
// Standard normal CDF:  Phi(-a) = exp(-a^2/2) G(u),  u = 2/(1 + 0.35 a) - 1.
// Quantile:  z = (2p - 1) sqrt(2) E,  w = -log(4p(1-p)) = -ln2 lg; sqrt(2) E a polynomial in
//   (w - mid)/half for w < 5, else in (sqrt(w) - mid)/half on [sqrt 5, 4] or [4, 9.3].
#pragma once
#define NRM_CDF_C0 0.35f
#define NRM_PPF_LG_SPLIT -7.213475f
static __device__ __forceinline__ float nrm_cdf_g(float u) { return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(0.00038237785f, u, -0.0004815742f), u, -0.0033990606f), u, 0.0025471582f), u, 0.040660013f), u, 0.12129871f), u, 0.2123704f), u, 0.12662213f); }
static __device__ __forceinline__ float nrm_ppf_mid_lg(float lg) { const float v = fmaf(lg, -0.27725887f, -1.0f); return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(6.1595936e-05f, v, 0.00029670962f), v, -0.0012184317f), v, -0.0006072493f), v, 0.012076195f), v, -0.027703274f), v, -0.036926072f), v, 0.87200665f), v, 2.1233137f); }
static __device__ __forceinline__ float nrm_ppf_tail(float s) {
    const bool hi = s >= 4.0f;
    const float v = fmaf(s, hi ? 0.3773585f : 1.1338305f, hi ? -2.509434f : -3.5353222f);
    return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf((hi ? -4.5746387e-05f : 5.8893023e-05f), v, (hi ? 7.33524e-05f : -9.408315e-05f)), v, (hi ? -7.2069895e-05f : -0.00018369175f)), v, (hi ? 0.00021505152f : 0.0008826216f)), v, (hi ? -0.00047378833f : -0.001944278f)), v, (hi ? 0.00067329523f : 0.0033119796f)), v, (hi ? -0.000112690075f : -0.005246588f)), v, (hi ? -0.0051057534f : 0.007877496f)), v, (hi ? 3.7812283f : 1.2518032f)), v, (hi ? 9.214942f : 4.173809f));
}
