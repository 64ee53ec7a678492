"""Tensor-core (tcgen05) whitened contraction: TF32, TF32x3, BF16, BF16x3 against the oracle.

Split precisions (TF32x3, BF16x3) are asserted to the FP32-class tolerance (|dvar| <= 1e-4 sf2,
|dmean| <= 1e-4 max|y|; the mean is the compensated k.alpha in every precision).  Single-pass
TF32 and BF16 are reported (their variance error is large on ill-conditioned models) and only
checked for finiteness and the mean.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_util import model_of, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def g():
    import paper_2512_12442_gb300 as g
    return g


def _recon(g, torch, M, n, prec, lo=(0, 0, 0), hi=(1, 1, 1)):
    grid = g.make_grid(n, lo, hi)
    npts = int(np.prod(n)) if not np.isscalar(n) else n ** 3
    mean = torch.zeros(npts, dtype=torch.float32, device="cuda")
    var = torch.zeros_like(mean)
    g.gpr_reconstruct_dense(M, grid, prec, mean, var, None)
    g.gpr_sync()
    return mean.cpu().numpy().astype(np.float64), var.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", ["ragged_m97", "config1"])
def test_tc_split_precisions_small(torch, g, case):
    if case == "config1":
        w = workloads.config1(); n = (32, 32, 32)
    else:
        w = workloads.small(97, 97, 9, ell=(0.15, 0.2, 0.25)); n = (11, 13, 9)  # 1287 points: ragged tiles
    M = model_of(w)
    ref = oracle.Model.from_workload(w).stats15(n)
    ys = np.abs(w.y).max()
    m32, v32 = _recon(g, torch, M, n, g.GPR_P_FP32)
    for prec in (g.GPR_P_TF32X3, g.GPR_P_BF16X3):
        m, v = _recon(g, torch, M, n, prec)
        assert np.abs(m - ref[:, 0]).max() <= 1e-4 * ys
        assert np.abs(v - ref[:, 1]).max() <= 1e-4 * w.sf2, (prec, np.abs(v - ref[:, 1]).max())
        assert np.abs(v - v32).max() <= 1e-4
    for prec in (g.GPR_P_TF32, g.GPR_P_BF16):
        m, v = _recon(g, torch, M, n, prec)
        assert np.all(np.isfinite(v))
        assert np.abs(m - ref[:, 0]).max() <= 1e-4 * ys


def test_tc_config2_full_grid_sampled(torch, g):
    """The m=500 field on the full 128^3 grid in TF32x3 and BF16x3, sampled against the oracle."""
    w = workloads.config2()
    M = model_of(w)
    n = w.n
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.integers(0, n ** 3, 2500), [0, n ** 3 - 1]])
    P = np.stack([idx % n, (idx // n) % n, idx // (n * n)], 1) / (n - 1)
    mu, vr = oracle.Model.from_workload(w).posterior(P)
    ys = np.abs(w.y).max()
    errs = {}
    for prec in (g.GPR_P_TF32X3, g.GPR_P_BF16X3, g.GPR_P_TF32, g.GPR_P_BF16):
        m, v = _recon(g, torch, M, n, prec)
        errs[prec] = (np.abs(m[idx] - mu).max() / ys, np.abs(v[idx] - vr).max())
    for prec in (g.GPR_P_TF32X3, g.GPR_P_BF16X3):
        assert errs[prec][0] <= 1e-4 and errs[prec][1] <= 1e-4, errs
    print("tensor-core errors (max |dmean|/max|y|, max |dvar|):", errs)


def test_tc_prepass_lcp_equals_fp64(torch, g):
    """The LCP cascade with a tensor-core pre-pass gives the all-FP64 field."""
    w = workloads.config1()
    M = model_of(w)
    th = w.isovalues[0]
    out = {}
    for prec in (g.GPR_P_FP64, g.GPR_P_TF32X3, g.GPR_P_BF16X3):
        f = torch.zeros((w.n - 1) ** 3, dtype=torch.float32, device="cuda")
        g.gpr_lcp_dense(M, g.make_grid(w.n), th, g.lcp_options(prec=prec, exact=g.GPR_EXACT_FP64), f)
        g.gpr_sync()
        out[prec] = f.cpu().numpy()
    assert np.array_equal(out[g.GPR_P_FP64], out[g.GPR_P_TF32X3])
    assert np.array_equal(out[g.GPR_P_FP64], out[g.GPR_P_BF16X3])


@pytest.mark.parametrize("prec", ["TF32", "TF32X3", "BF16", "BF16X3"])
def test_tc_cov13_against_oracle(torch, g, prec):
    """The 13 forward covariances in the tensor-core precisions (their whitened rows written out
    and reduced, cov = k(a, b) - w_a . w_b): NaN exactly where the neighbour is off the grid, and
    within the precision's own error of the oracle elsewhere (split forms 1e-4 sf2, single-pass
    forms 5e-2 sf2, the size of their variance errors at this conditioning)."""
    w = workloads.small(3, 20, 5)
    M = model_of(w)
    n = 5
    mean = torch.zeros(n ** 3, dtype=torch.float32, device="cuda")
    var = torch.zeros_like(mean)
    cov = torch.zeros(n ** 3, 13, dtype=torch.float32, device="cuda")
    g.gpr_reconstruct_dense(M, g.make_grid(n), getattr(g, "GPR_P_" + prec), mean, var, cov)
    g.gpr_sync()
    ref = oracle.Model.from_workload(w).stats15(n)
    c = cov.cpu().numpy().astype(np.float64)
    assert np.array_equal(np.isnan(c), np.isnan(ref[:, 2:]))
    ok = ~np.isnan(c)
    tol = (1e-4 if prec.endswith("X3") else 5e-2) * w.sf2
    np.testing.assert_allclose(c[ok], ref[:, 2:][ok], rtol=0, atol=tol)
    np.testing.assert_allclose(var.cpu().numpy().astype(np.float64), ref[:, 1], rtol=0, atol=tol)


@pytest.mark.parametrize("case", ["config2", "small_m97"])
def test_digit_split_stats_vs_fp64_and_oracle(torch, g, case):
    """FP64-class statistics on the BF16 tensor cores (seven 6-bit digit slices, exact FP32
    accumulation, float-float epilogue) against the FP64 CUDA-core path and the oracle."""
    if case == "config2":
        w = workloads.config2(); n = w.n
    else:
        w = workloads.small(97, 97, 9, ell=(0.15, 0.2, 0.25)); n = 11
    M = model_of(w)
    grid = g.make_grid(n)
    rng = np.random.default_rng(4)
    base = np.unique(rng.integers(0, n ** 3, 600))
    # include full cells so neighbour covariances are exercised
    pts = np.unique(np.concatenate([base, base + 1, base + n, base + n * n]))
    pts = pts[pts < n ** 3]
    t = torch.tensor(pts, dtype=torch.int64, device="cuda")
    a = torch.zeros(len(pts), 15, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    g.gpr_stats_points(M, grid, t, a)
    g.gpr_stats_points_split(M, grid, t, b)
    g.gpr_sync()
    a = a.cpu().numpy(); b = b.cpu().numpy()
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(a)
    d = np.abs(a - b)[ok].max()
    assert d <= 1e-8, d
    ref = oracle.Model.from_workload(w).stats15(n)[pts]
    assert np.abs(b[ok] - ref[ok]).max() <= 1e-8


def test_digit_split_lcp_vs_fp64_config2(torch, g):
    """LCP field of the m=500 field at its median isovalue: digit-split corner statistics vs FP64."""
    w = workloads.config2()
    M = model_of(w)
    th = w.isovalues[1]
    out = {}
    for ex in (g.GPR_EXACT_AUTO, g.GPR_EXACT_FP64):
        f = torch.zeros((w.n - 1) ** 3, dtype=torch.float32, device="cuda")
        g.gpr_lcp_dense(M, g.make_grid(w.n), th, g.lcp_options(prec=g.GPR_P_TF32X3, exact=ex), f)
        g.gpr_sync()
        out[ex] = f.cpu().numpy().astype(np.float64)
    d = np.abs(out[g.GPR_EXACT_AUTO] - out[g.GPR_EXACT_FP64])
    # the two corner statistics differ by ~1e-9; the FP32 estimator turns that into ~1e-6 at most
    assert d.max() <= 1e-5, d.max()


def test_digit_split_stats_m_above_1024(torch, g):
    """More observations than one exact FP32 accumulation holds (m=1500: two K chunks, each
    drained to float-float) against the FP64 CUDA-core path and the oracle."""
    w = workloads.small(11, 1500, 13, ell=(0.12, 0.15, 0.18))
    n = w.n
    M = model_of(w)
    grid = g.make_grid(n)
    rng = np.random.default_rng(8)
    base = np.unique(rng.integers(0, n ** 3, 300))
    pts = np.unique(np.concatenate([base, base + 1, base + n, base + n * n]))
    pts = pts[pts < n ** 3]
    t = torch.tensor(pts, dtype=torch.int64, device="cuda")
    a = torch.zeros(len(pts), 15, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    g.gpr_stats_points(M, grid, t, a)
    g.gpr_stats_points_split(M, grid, t, b)
    g.gpr_sync()
    a = a.cpu().numpy(); b = b.cpu().numpy()
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(a)
    assert np.abs(a - b)[ok].max() <= 1e-8
    ref = oracle.Model.from_workload(w).stats15(n)[pts]
    assert np.abs(b[ok] - ref[ok]).max() <= 1e-8


def test_digit_split_lcp_slab_path(torch, g, monkeypatch):
    """Without cached rows and with a row buffer of a few planes, the digit-split leaf path runs
    in z slabs (rows of planes z0-1..z1, statistics of planes z0..z1-1); its field equals the
    single-buffer one and the cached one bit for bit."""
    w = workloads.small(5, 300, 40, ell=(0.15, 0.2, 0.25))
    th = w.isovalues[0]

    def run(env):
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        M = model_of(w)
        f = torch.zeros((w.n - 1) ** 3, dtype=torch.float32, device="cuda")
        l0 = g.gpr_launch_count()
        g.gpr_lcp_dense(M, g.make_grid(w.n), th, g.lcp_options(prec=g.GPR_P_TF32X3), f)
        g.gpr_sync()
        launches = g.gpr_launch_count() - l0
        for k in env:
            monkeypatch.delenv(k)
        return f.cpu().numpy(), launches

    single, l_single = run({"GPR_WCACHE_BUDGET_MB": "0"})
    slabs, l_slabs = run({"GPR_WCACHE_BUDGET_MB": "0", "GPR_ROW_BUDGET_MB": "16"})
    cached, _ = run({})
    assert l_slabs > l_single + 20  # one plane per slab: two compactions and two kernels each
    assert (single > 0).sum() > 100
    assert np.array_equal(single, slabs)
    assert np.array_equal(single, cached)
