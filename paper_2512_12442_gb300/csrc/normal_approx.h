// Generated by fit_normal.py (minimax-relative-error fits against SciPy); do not edit.
// Standard normal CDF:  Phi(-a) = exp(-a^2/2) G(t),  t = 1/(1 + 0.35 a).
// Quantile:  z = (2p - 1) sqrt(2) E,  w = -log(4p(1-p)) = -ln2 lg; sqrt(2) E a polynomial in
//   lg for w < 5, else in (sqrt(w) - mid)/half on [sqrt 5, 9.3].
#pragma once
#define NRM_CDF_C0 0.35f
#define NRM_PPF_LG_SPLIT -7.213475f
static __device__ __forceinline__ float nrm_cdf_g(float t) { return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(0.048944365f, t, -0.20212603f), t, 0.24065024f), t, -0.017030044f), t, 0.15596388f), t, 0.13335471f), t, 0.14027035f), t, -2.7312963e-05f); }
static __device__ __forceinline__ float nrm_ppf_mid_lg(float lg) { return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(-3.4312166e-08f, lg, -1.365981e-06f), lg, -1.9260626e-05f), lg, -6.619455e-05f), lg, 0.0010628646f), lg, 0.007820129f), lg, -0.22744083f), lg, 1.2533138f); }
static __device__ __forceinline__ float nrm_ppf_tail(float s) {
    const float v = fmaf(s, 0.28312844f, -1.6330944f);
    return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(-0.008913594f, v, -0.02937258f), v, 0.050443884f), v, 0.045742813f), v, -0.057369407f), v, -0.03477084f), v, 0.033149317f), v, 0.0048911464f), v, 0.0002131089f), v, -0.0056126337f), v, -0.0072218487f), v, 5.0440493f), v, 7.955928f);
}
