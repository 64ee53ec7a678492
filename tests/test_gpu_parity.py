"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Tolerances:
  - FP64 paths: mean/var/cov within 1e-9 of the field scale (rounding order only).
  - FP32-class mean/var: 1e-4 of the field scale (max|y| for the mean, sf2 for var).
  - cell LCP (SOV): |dLCP| <= 1e-4 absolute (LCP in [0,1]).
  - cell LCP (MC): per cell at most 3 samples of 1600 differ (FP32 vs FP64 sampling
    can flip a draw that lands within rounding of theta), mean |dLCP| <= 1e-4.
"""
import math

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


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("m,seed", [(1, 3), (33, 4), (97, 5), (500, 1)])
def test_model_setup_factors(torch, g, m, seed):
    """A0: FP64 blocked Cholesky, L^-1 y, Kt^-1 y and the latent posterior at the observations."""
    w = workloads.config2() if m == 500 else workloads.small(seed, m, 9)
    M = model_of(w)
    dev = g.gpr_model_export(M)
    ref = oracle.Model.from_workload(w).factors()
    np.testing.assert_allclose(dev["L"], ref["L"], rtol=1e-9, atol=1e-12)
    scale = np.abs(ref["alpha"]).max()
    np.testing.assert_allclose(dev["alpha"], ref["alpha"], rtol=1e-6, atol=1e-9 * scale)
    np.testing.assert_allclose(dev["vy"], ref["vy"], rtol=1e-8, atol=1e-10 * np.abs(ref["vy"]).max())
    np.testing.assert_allclose(dev["mu_obs"], ref["mu_obs"], rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(dev["var_obs"], ref["var_obs"], rtol=1e-5, atol=1e-12)


def test_not_positive_definite_reported(torch, g):
    X = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.5], [0.1, 0.2, 0.3]])
    with pytest.raises(g.GPRError) as e:
        g.gpr_model_create(X, np.array([1.0, 2.0, 0.0]), 0, (0.2, 0.2, 0.2), 1.0, 0.0)
    assert e.value.status == g.GPR_ERR_NOT_PD


@pytest.mark.parametrize("case", ["config1", "ragged", "matern", "box"])
def test_reconstruct_fp64_full_grid(torch, g, case):
    """A1-A3 in FP64: mean, variance and the 13 forward covariances at every grid point."""
    if case == "config1":
        w = workloads.config1(); n = (32, 32, 32); lo, hi = (0, 0, 0), (1, 1, 1)
    elif case == "ragged":
        w = workloads.small(12, 70, 9); n = (13, 7, 5); lo, hi = (0, 0, 0), (1, 1, 1)
    elif case == "matern":
        w = workloads.small(13, 65, 9, ell=(0.15, 0.2, 0.3), kernel=workloads.MATERN52, sn2=1e-6); n = (9, 10, 11)
        lo, hi = (0, 0, 0), (1, 1, 1)
    else:
        w = workloads.small(14, 40, 9); n = (6, 9, 8); lo, hi = (0.1, -0.2, 0.3), (0.7, 1.1, 0.9)
    M = model_of(w)
    grid = g.make_grid(n, lo, hi)
    npts = int(np.prod(n))
    mean = torch.zeros(npts, dtype=torch.float64, device="cuda")
    var = torch.zeros_like(mean)
    cov = torch.zeros(npts, 13, dtype=torch.float64, device="cuda")
    g.gpr_reconstruct_dense(M, grid, g.GPR_P_FP64, mean, var, cov)
    g.gpr_sync()
    om = oracle.Model.from_workload(w)
    ref = om.stats15(n, (0, 0, 0), n, lo, hi)
    ys = np.abs(w.y).max()
    np.testing.assert_allclose(_np(mean), ref[:, 0], rtol=0, atol=1e-9 * ys)
    np.testing.assert_allclose(_np(var), ref[:, 1], rtol=0, atol=1e-10 * w.sf2)
    c = _np(cov)
    assert np.array_equal(np.isnan(c), np.isnan(ref[:, 2:]))
    ok = ~np.isnan(c)
    np.testing.assert_allclose(c[ok], ref[:, 2:][ok], rtol=0, atol=1e-10 * w.sf2)


def test_reconstruct_fp32_meanvar_full_size(torch, g):
    """A1-A3 in FP32 on the full 128^3 grid of the paper-scale field (m=500), sampled
    points against the oracle: |dmu| <= 1e-4 max|y|, |dvar| <= 1e-4 sf2."""
    w = workloads.config2()
    M = model_of(w)
    n = w.n
    grid = g.make_grid(n)
    mean = torch.zeros(n ** 3, dtype=torch.float32, device="cuda")
    var = torch.zeros_like(mean)
    g.gpr_reconstruct_dense(M, grid, g.GPR_P_FP32, mean, var, None)
    g.gpr_sync()
    rng = np.random.default_rng(0)
    idx = rng.integers(0, n ** 3, 3000)
    idx = np.concatenate([idx, [0, n ** 3 - 1, n - 1, n * n * (n - 1)]])
    P = np.stack([idx % n, (idx // n) % n, idx // (n * n)], 1) / (n - 1)
    mu, vr = oracle.Model.from_workload(w).posterior(P)
    ys = np.abs(w.y).max()
    dm = np.abs(_np(mean)[idx] - mu).max() / ys
    dv = np.abs(_np(var)[idx] - vr).max() / w.sf2
    assert dm <= 1e-4 and dv <= 1e-4, (dm, dv)
    # with cov13 through the stored-W route: the same mean/var
    mean2 = torch.zeros_like(mean); var2 = torch.zeros_like(mean)
    cov = torch.zeros(n ** 3, 13, dtype=torch.float32, device="cuda")
    g.gpr_reconstruct_dense(M, grid, g.GPR_P_FP32, mean2, var2, cov)
    g.gpr_sync()
    assert np.abs(_np(mean2)[idx] - mu).max() / ys <= 1e-4
    assert np.abs(_np(var2)[idx] - vr).max() <= 1e-4


def test_stats_points_gather(torch, g):
    """Gather mode: stats15 of a listed point set; covariances to unlisted neighbours are NaN."""
    w = workloads.small(21, 80, 11)
    M = model_of(w)
    n = 11
    grid = g.make_grid(n)
    rng = np.random.default_rng(2)
    pts = np.unique(rng.integers(0, n ** 3, 300))
    t_pts = torch.tensor(pts, dtype=torch.int64, device="cuda")
    out = torch.zeros(len(pts), 15, dtype=torch.float64, device="cuda")
    g.gpr_stats_points(M, grid, t_pts, out)
    g.gpr_sync()
    ref = oracle.Model.from_workload(w).stats15(n)[pts]
    o = _np(out)
    np.testing.assert_allclose(o[:, :2], ref[:, :2], atol=1e-9)
    s = set(pts.tolist())
    offs = [(1, -1, -1), (1, -1, 0), (1, -1, 1), (1, 0, -1), (1, 0, 0), (1, 0, 1), (1, 1, -1), (1, 1, 0), (1, 1, 1),
            (0, 1, -1), (0, 1, 0), (0, 1, 1), (0, 0, 1)]
    for r, p in enumerate(pts):
        i, j, k = p % n, (p // n) % n, p // (n * n)
        for e, (a, b, c) in enumerate(offs):
            q = (i + a) + n * ((j + b) + n * (k + c))
            inside = 0 <= i + a < n and 0 <= j + b < n and 0 <= k + c < n
            if inside and q in s:
                assert o[r, 2 + e] == pytest.approx(ref[r, 2 + e], abs=1e-10)
            else:
                assert math.isnan(o[r, 2 + e])


def _lcp_dense_gpu(g, torch, M, n, theta, **kw):
    grid = g.make_grid(n)
    out = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    st = g.gpr_lcp_dense(M, grid, theta, g.lcp_options(**kw), out)
    g.gpr_sync()
    return _np(out).astype(np.float64), st


def test_lcp_dense_config1_sov_full(torch, g):
    """A4 on the config-1 field (m=64, 32^3, SE l=0.2): every cell against the oracle."""
    w = workloads.config1()
    M = model_of(w)
    th = w.isovalues[0]
    gpu, st = _lcp_dense_gpu(g, torch, M, w.n, th, prec=g.GPR_P_FP64)
    ref = oracle.Model.from_workload(w).lcp_dense(w.n, th)
    assert np.abs(gpu - ref).max() <= 1e-4, np.abs(gpu - ref).max()
    assert st["cells_estimated"] > 100


def test_lcp_prepass_equals_all_fp64(torch, g):
    """The FP32 pre-classification changes nothing: with FP64 corner statistics the field equals the
    all-FP64 one bit for bit; with the tensor-core digit split it agrees within 1e-6."""
    w = workloads.config1()
    M = model_of(w)
    th = w.isovalues[0]
    a, sa = _lcp_dense_gpu(g, torch, M, w.n, th, prec=g.GPR_P_FP64)
    b, sb = _lcp_dense_gpu(g, torch, M, w.n, th, prec=g.GPR_P_FP32, exact=g.GPR_EXACT_FP64)
    assert np.array_equal(a, b)
    assert sb["recon_points"] <= w.n ** 3
    c, sc = _lcp_dense_gpu(g, torch, M, w.n, th, prec=g.GPR_P_FP32)
    assert np.abs(a - c).max() <= 1e-5


def test_lcp_dense_config1_mc(torch, g):
    """The paper's MC estimator (1600 samples) with the shared counter-based streams."""
    w = workloads.config1()
    M = model_of(w)
    th = w.isovalues[0]
    gpu, _ = _lcp_dense_gpu(g, torch, M, w.n, th, prec=g.GPR_P_FP64, est=g.GPR_EST_MC)
    ref = oracle.Model.from_workload(w).lcp_dense(w.n, th, est=oracle.EST_MC)
    d = np.abs(gpu - ref)
    assert d.max() <= 3 / 1600 + 1e-7, d.max()
    assert d.mean() <= 1e-4


def test_lcp_dense_config2_full_size_subblock(torch, g):
    """Paper-scale field (m=500, 128^3) at the three isovalues, launched exactly as the bench
    does; a 12^3-cell block straddling the surface and the corners of the domain are
    compared with the oracle cell by cell."""
    w = workloads.config2()
    M = model_of(w)
    om = oracle.Model.from_workload(w)
    n = w.n
    for th in w.isovalues:
        gpu, st = _lcp_dense_gpu(g, torch, M, n, th, prec=g.GPR_P_FP32)
        f = gpu.reshape(n - 1, n - 1, n - 1)  # [k][j][i]
        ref = om.lcp_block(n, th, (50, 60, 40), (62, 72, 52)).reshape(12, 12, 12)
        d = np.abs(f[40:52, 60:72, 50:62] - ref)
        assert d.max() <= 1e-4, (th, d.max())
        for c0 in ((0, 0, 0), (n - 5, n - 5, n - 5)):
            r2 = om.lcp_block(n, th, c0, tuple(v + 4 for v in c0)).reshape(4, 4, 4)
            assert np.abs(f[c0[2]:c0[2] + 4, c0[1]:c0[1] + 4, c0[0]:c0[0] + 4] - r2).max() <= 1e-4
        assert 0.0 <= gpu.min() and gpu.max() <= 1.0


@pytest.mark.parametrize("est", ["indep", "edge"])
def test_lcp_closed_form_estimators_config1(torch, g, est):
    """The closed-form cell estimators (independent corners; Pothkow et al.'s edge maximum) on the
    config-1 field, every cell against the oracle.  Tolerance 2e-5: the GPU evaluates them in FP32
    with this library's Phi (absolute error <= 5e-7 per evaluation, at most 8 factors of a product)
    and Owen's T by a 12-point Gauss-Legendre rule."""
    w = workloads.config1()
    M = model_of(w)
    th = w.isovalues[0]
    e_gpu = g.GPR_EST_INDEP if est == "indep" else g.GPR_EST_EDGE_MAX
    e_or = oracle.EST_INDEP if est == "indep" else oracle.EST_EDGE
    gpu, st = _lcp_dense_gpu(g, torch, M, w.n, th, prec=g.GPR_P_FP64, est=e_gpu)
    ref = oracle.Model.from_workload(w).lcp_dense(w.n, th, est=e_or)
    assert np.abs(gpu - ref).max() <= 2e-5, np.abs(gpu - ref).max()
    assert st["cells_estimated"] > 100 and (ref > 0.01).sum() > 100
    if est == "edge":
        # a crossed edge crosses the cell: against a 16,384-point SOV field (lattice error ~3e-3)
        sov, _ = _lcp_dense_gpu(g, torch, M, w.n, th, prec=g.GPR_P_FP64, n_samples=1 << 14)
        assert np.all(gpu <= sov + 5e-3), float((gpu - sov).max())


def test_lcp_closed_form_estimators_paper_scale_adaptive(torch, g):
    """The edge-maximum estimator on the paper-scale field (m=500, 128^3), adaptive as the bench runs
    fields: equal to the dense field on S, and a 12^3 block against the oracle."""
    w = workloads.config2()
    M = model_of(w)
    n, th = w.n, w.isovalues[1]
    grid = g.make_grid(n)
    opts = g.lcp_options(est=g.GPR_EST_EDGE_MAX)
    ad = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    de = torch.zeros_like(ad)
    sa = g.gpr_lcp_adaptive(M, grid, th, w.max_depth, opts, ad)
    g.gpr_lcp_dense(M, grid, th, opts, de)
    g.gpr_sync()
    a, d = _np(ad), _np(de)
    nz = a != 0
    assert np.array_equal(a[nz], d[nz]) and sa["cells_estimated"] > 1000
    ref = oracle.Model.from_workload(w).lcp_block(n, th, (50, 60, 40), (62, 72, 52), est=oracle.EST_EDGE)
    f = d.reshape(n - 1, n - 1, n - 1)[40:52, 60:72, 50:62].reshape(-1)
    assert np.abs(f - ref).max() <= 2e-5


@pytest.mark.parametrize("n", [2, 3])
def test_lcp_tiny_grids(torch, g, n):
    """Degenerate grids: one cell (n=2) and 8 cells (n=3)."""
    w = workloads.small(31, 10, n, ell=(0.5, 0.5, 0.5))
    M = model_of(w)
    th = float(np.median(w.y))
    gpu, _ = _lcp_dense_gpu(g, torch, M, n, th, prec=g.GPR_P_FP64)
    ref = oracle.Model.from_workload(w).lcp_dense(n, th)
    assert np.abs(gpu - ref).max() <= 1e-4


def test_cell_lcp_from_stats_entry(torch, g):
    """The estimator entry point on oracle-made stats15 (selected cells, output by position)."""
    w = workloads.small(41, 50, 10)
    om = oracle.Model.from_workload(w)
    n = 10
    st = om.stats15(n)
    th = float(np.median(w.y))
    cells = np.array([0, 5, 77, 300, (n - 1) ** 3 - 1], np.int64)
    out = torch.zeros(len(cells), dtype=torch.float32, device="cuda")
    g.gpr_cell_lcp_from_stats(g.make_grid(n), torch.tensor(st, device="cuda"), th, g.lcp_options(),
                              torch.tensor(cells, device="cuda"), out)
    g.gpr_sync()
    ref = om.lcp_dense(n, th)[cells]
    assert np.abs(_np(out) - ref).max() <= 1e-4


def test_invalid_arguments_on_gpu(torch, g):
    w = workloads.small(1, 10, 5)
    M = model_of(w)
    out = torch.zeros(10, dtype=torch.float32, device="cuda")
    with pytest.raises(g.GPRError) as e:
        g.gpr_lcp_dense(M, g.make_grid((1, 4, 4)), 0.0, g.lcp_options(), out)
    assert e.value.status == g.GPR_ERR_ARG
    with pytest.raises(g.GPRError) as e:
        g.gpr_lcp_dense(M, g.make_grid(4), float("nan"), g.lcp_options(), out)
    assert e.value.status == g.GPR_ERR_ARG
    with pytest.raises(g.GPRError) as e:
        g.gpr_lcp_dense(M, g.make_grid(4), 0.0, g.lcp_options(n_samples=0), out)
    assert e.value.status == g.GPR_ERR_ARG
