"""The estimator's FP32 standard normal CDF and quantile (polynomial fits, fit_normal.py)
against the oracle's FP64 Phi and Phi^-1, evaluated at the same binary32 arguments.

Bounds: CDF |error| <= 5e-7 everywhere, relative <= 2e-6 where Phi > 1e-7 and <= 2e-5 where
Phi > 1e-30 (the exponential's argument a^2/2 is rounded in FP32; an orthant factor that small
moves the estimate by far less than its own size); quantile
|error| <= 1e-6 + 2e-6 |z| for p in [1e-37, 1 - 2^-24].
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _eval(x):
    torch = torch_cuda()
    from paper_2512_12442_gb300._lib import load
    t = torch.tensor(x, dtype=torch.float32, device="cuda")
    cdf = torch.zeros_like(t); ppf = torch.zeros_like(t)
    rc = load().gpr_normal_approx_eval(C.c_void_p(t.data_ptr()), t.numel(), C.c_void_p(cdf.data_ptr()),
                                       C.c_void_p(ppf.data_ptr()), None)
    assert rc == 0
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64), cdf.cpu().numpy().astype(np.float64), ppf.cpu().numpy().astype(np.float64)


def test_cdf_against_oracle():
    x, cdf, _ = _eval(np.concatenate([np.linspace(-14, 9, 12001), [0.0, -1e-30, 1e-30]]))
    ref = np.array([oracle.norm_cdf(v) for v in x])
    assert np.abs(cdf - ref).max() <= 5e-7
    for floor, tol in ((1e-7, 2e-6), (1e-30, 2e-5)):
        m = ref > floor
        rel = np.abs(cdf[m] / ref[m] - 1)
        assert rel.max() <= tol, (floor, rel.max(), x[m][np.argmax(rel)])


def test_ppf_against_oracle():
    lo = np.logspace(-37, np.log10(0.5), 6000)
    p = np.concatenate([lo, 1 - np.logspace(np.log10(2.0 ** -24), np.log10(0.5), 3000), [0.5, 0.25, 0.75]])
    x, _, ppf = _eval(p)
    ok = (x > 0) & (x < 1)
    ref = np.array([oracle.norm_ppf(v) for v in x[ok]])
    err = np.abs(ppf[ok] - ref)
    bound = 1e-6 + 2e-6 * np.abs(ref)
    assert np.all(err <= bound), (err / bound).max()
