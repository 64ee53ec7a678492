// FP32 standard normal CDF and quantile of the SOV estimator (forward and adjoint sweeps).
#pragma once

#include "normal_approx.h"

// Standard normal CDF in FP32 for the estimator: Phi(-a) = exp(-a^2/2) G(1/(1 + 0.3a)) with G
// a polynomial fitted by fit_normal.py; relative error about 1e-6 where Phi > 1e-7 (below 1e-5
// down to 1e-30: the FP32 rounding of a^2/2 grows with a), one reciprocal and one exponential
// per call, no branch.
static __device__ __forceinline__ float nrm_cdf(float x)
{
    const float a = fabsf(x);
    const float u = fmaf(2.0f, __fdividef(1.0f, fmaf(NRM_CDF_C0, a, 1.0f)), -1.0f);
    const float e = __expf(-0.5f * a * a) * nrm_cdf_g(u);
    return x < 0.0f ? e : 1.0f - e;
}

// Standard normal quantile in FP32 for p in (0, 1): z = sqrt(2) (2p - 1) E(w), w = -log(4p(1-p))
// (the erfinv variable of Giles, taken from p so the tails keep their relative precision); the
// branch at w = 5 splits off p < 0.0017 (and its mirror).
static __device__ __forceinline__ float nrm_ppf(float p)
{
    const float w = -__logf(4.0f * p * (1.0f - p));
    const float E = w < 5.0f ? nrm_ppf_mid(w) : nrm_ppf_tail(w * rsqrtf(w));
    return 1.41421356f * (2.0f * p - 1.0f) * E;
}
