#!/usr/bin/env python
"""Writes normal_approx.h: polynomial coefficients of the estimator's single-precision
standard normal CDF and quantile, fitted here to minimise the maximum relative error (Lawson's
iteratively reweighted least squares) against SciPy's double-precision log_ndtr and ndtri.

  CDF, x = -a <= 0:  Phi(-a) = exp(-a^2/2) * G(t),  t = 1 / (1 + 0.35 a),
                     G a degree-7 polynomial in t itself (a in [0, 13.2]; no shift of the
                     variable to save an instruction, at no cost in accuracy).
  Quantile, p in (0, 1):  z = sqrt(2) (2p - 1) E,  w = -log(4 p (1 - p)),
                     E a polynomial on two pieces: degree 7 in lg = log2(4p(1-p)) itself for
                     w in [0, 5], degree 12 in the scaled s = sqrt(w) on [sqrt(5), 9.3].
The variable w is the one of M. Giles, "Approximating the erfinv function" (GPU Computing
Gems, 2011), written in p so that the tails keep full relative precision; the
coefficients are this script's own fit.  Run it to regenerate the header.
"""
import os

import numpy as np
from scipy.special import log_ndtr, ndtri

HERE = os.path.dirname(os.path.abspath(__file__))
CDF_C0 = 0.35
CDF_DEG = 7
PPF_DEG_MID = 7
PPF_DEG_TAIL = 12
PPF_PIECES = (("w", 0.0, 5.0), ("s", float(np.sqrt(5.0)), 9.3))


def fit(u, f, deg, iters=60):
    """Polynomial in u of the given degree with (nearly) the least maximum relative error:
    Lawson's algorithm, least squares with weights multiplied each round by the errors."""
    V = np.vander(u, deg + 1, increasing=True)
    rel = 1.0 / np.abs(f)
    w = np.full(len(u), 1.0 / len(u))
    for _ in range(iters):
        sw = np.sqrt(w) * rel
        c, *_ = np.linalg.lstsq(V * sw[:, None], f * sw, rcond=None)
        err = np.abs(V @ c - f) * rel
        w = w * err
        w /= w.sum()
    return c


def cdf_coeffs():
    a = np.linspace(0.0, 13.2, 200001)
    G = np.exp(log_ndtr(-a) + 0.5 * a * a)
    t = 1.0 / (1.0 + CDF_C0 * a)
    return fit(t, G, CDF_DEG)


def ppf_coeffs():
    p = np.logspace(-37, np.log10(0.5), 400001)
    x = 1.0 - 2.0 * p
    E = np.where(x > 0, -ndtri(p) / (np.sqrt(2.0) * np.maximum(x, 1e-300)), np.sqrt(np.pi) / 2)
    w = -np.log(4.0 * p * (1.0 - p))
    s = np.sqrt(w)
    out = []
    for var, lo, hi in PPF_PIECES:
        v = w if var == "w" else s
        m = (v >= lo) & (v <= hi)
        mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
        if var == "w":  # central piece: directly in lg = -w / ln 2, the value the kernel has
            out.append((0.0, 1.0, fit(-w[m] / np.log(2.0), E[m], PPF_DEG_MID)))
        else:
            out.append((mid, 1.0 / half, fit((v[m] - mid) / half, E[m], PPF_DEG_TAIL)))
    return out


def fmt(v):
    return f"{np.float32(v)!r}f".replace("np.float32(", "").replace(")", "")


def horner(coeffs, var):
    """C expression: Horner chain in `var`."""
    n = len(coeffs)
    expr = fmt(coeffs[n - 1])
    for k in range(n - 2, -1, -1):
        expr = f"fmaf({expr}, {var}, {fmt(coeffs[k])})"
    return expr


def main(path=None):
    """Writes the header (to `path`, default normal_approx.h beside this script)."""
    c = cdf_coeffs()
    (_, _, p0), (m1, h1, p1) = ppf_coeffs()
    r2 = np.sqrt(2.0)
    p0, p1 = p0 * r2, p1 * r2  # sqrt(2) folded into the quantile polynomials
    ln2 = np.log(2.0)
    lines = [
        "// Generated by fit_normal.py (minimax-relative-error fits against SciPy); do not edit.",
        f"// Standard normal CDF:  Phi(-a) = exp(-a^2/2) G(t),  t = 1/(1 + {CDF_C0} a).",
        "// Quantile:  z = (2p - 1) sqrt(2) E,  w = -log(4p(1-p)) = -ln2 lg; sqrt(2) E a polynomial in",
        "//   lg for w < 5, else in (sqrt(w) - mid)/half on [sqrt 5, 9.3].",
        "#pragma once",
        f"#define NRM_CDF_C0 {fmt(CDF_C0)}",
        f"#define NRM_PPF_LG_SPLIT {fmt(-5.0 / ln2)}",
        "static __device__ __forceinline__ float nrm_cdf_g(float t) { return " + horner(c, "t") + "; }",
        "static __device__ __forceinline__ float nrm_ppf_mid_lg(float lg) { return " + horner(p0, "lg") + "; }",
        "static __device__ __forceinline__ float nrm_ppf_tail(float s) {",
        f"    const float v = fmaf(s, {fmt(h1)}, {fmt(-m1 * h1)});",
        "    return " + horner(p1, "v") + ";",
        "}",
    ]
    with open(path or os.path.join(HERE, "normal_approx.h"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
