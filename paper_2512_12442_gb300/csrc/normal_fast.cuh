// FP32 standard normal CDF and quantile of the SOV estimator (forward and adjoint sweeps),
// on the hardware's approximate reciprocal, exp2, log2 and rsqrt (PTX *.approx.ftz.f32).
#pragma once

#include "normal_approx.h"

static __device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
static __device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
static __device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
static __device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Phi(x): Phi(-a) = 2^(-a^2 log2(e) / 2) G(1/(1 + 0.35a)), G a polynomial fitted by
// fit_normal.py.  Relative error about 1e-6 where Phi > 1e-7 (below 1e-5 down to 1e-30: the
// FP32 rounding of a^2/2 grows with a).  No branch.
static __device__ __forceinline__ float nrm_cdf(float x)
{
    const float a = fabsf(x);
    const float t = rcp_approx(fmaf(NRM_CDF_C0, a, 1.0f));
    const float e = ex2_approx(a * (a * -0.72134752f)) * nrm_cdf_g(t);
    return x < 0.0f ? e : 1.0f - e;
}

// Phi(x) and, from the same exponential, the density phi(x) = exp(-x^2/2) / sqrt(2 pi).
static __device__ __forceinline__ float nrm_cdf_pdf(float x, float &pdf)
{
    const float a = fabsf(x);
    const float t = rcp_approx(fmaf(NRM_CDF_C0, a, 1.0f));
    const float g = ex2_approx(a * (a * -0.72134752f));
    pdf = 0.3989422804014327f * g;
    const float e = g * nrm_cdf_g(t);
    return x < 0.0f ? e : 1.0f - e;
}

// Tail piece of the quantile (p < 0.0017 or its mirror), out of line: it is rare, and keeping
// one copy keeps the unrolled estimator loop small enough for the instruction cache.
static __device__ __noinline__ float nrm_ppf_tail_lg(float lg)
{
    const float w = lg * -0.69314718f;
    return nrm_ppf_tail(w * rsqrt_approx(w));
}

// Phi^-1(p), p in (0, 1): z = (2p - 1) sqrt(2) E(w), w = -log(4p(1-p)) (the erfinv variable of
// Giles, taken from p so that the tails keep their relative precision; 4p(1-p) is one FMA, so
// it is correctly rounded).  The branch at w = 5 splits off p < 0.0017 and its mirror.
static __device__ __forceinline__ float nrm_ppf(float p)
{
    const float p4 = 4.0f * p;
    const float lg = lg2_approx(fmaf(-p4, p, p4));
    const float E = lg > NRM_PPF_LG_SPLIT ? nrm_ppf_mid_lg(lg) : nrm_ppf_tail_lg(lg);
    const float t = p + p;
    return fmaf(t, E, -E);
}
