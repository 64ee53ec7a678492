"""GPU parity for the general stored model of Sec. 3 (sparse GP: inducing sites with a stored
N(mu_M, A_M)), whose posterior is Eq. 1.  The device folds Eq. 1 into a lower-triangular factor of
K_MM^-1 - K_MM^-1 A_M K_MM^-1 and runs the plain-GPR kernels; the oracle evaluates Eq. 1 term by term.

Inputs: workloads.sgpr, the optimal inducing distribution (Titsias 2009) fitted to training samples
of the paper-scale field (GPy stands in for the paper's fitting, which is out of scope).
Tolerances as in test_gpu_parity: FP64 statistics within 1e-9 of the field scale (variances within
1e-10 of the signal variance, 1e-8 for the paper-scale model: its K_MM carries only the fitting jitter
1e-6, so kappa(K_MM) ~ 5e7 against kappa(Kt) ~ 4e5 for the plain models and both sides round ~100x
more); cell LCP within 1e-4 absolute; octree decisions as in test_gpu_adaptive (p-test exact, bound decisions may differ
only where the oracle's bound lies within a factor 3 of alpha).
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


@pytest.fixture(scope="module")
def small():
    return workloads.sgpr(seed=3, m=60, n_train=400, n=17)


@pytest.fixture(scope="module")
def paper_scale():
    return workloads.sgpr()  # m = 500 inducing sites, 4000 training samples, ARD SE, 128^3


def _np(t):
    return t.detach().cpu().numpy()


def test_sgpr_model_factors(torch, g, small):
    """K_MM's Cholesky factor, alpha = K_MM^-1 mu_M and the p-test inputs (mu_M, diag A_M)."""
    M = model_of(small)
    dev = g.gpr_model_export(M)
    ref = oracle.Model.from_workload(small).factors()
    np.testing.assert_allclose(dev["L"], ref["L"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(dev["alpha"], ref["alpha"], rtol=1e-7, atol=1e-9 * np.abs(ref["alpha"]).max())
    np.testing.assert_array_equal(dev["mu_obs"], small.y)
    np.testing.assert_allclose(dev["var_obs"], ref["var_obs"], rtol=1e-15, atol=0)


@pytest.mark.parametrize("n", [(9, 10, 11), (17, 17, 17)])
def test_sgpr_reconstruct_fp64_full_grid(torch, g, small, n):
    """Eq. 1 in FP64 at every grid point: mean, variance and the 13 forward covariances."""
    M = model_of(small)
    grid = g.make_grid(n)
    npts = int(np.prod(n))
    mean = torch.zeros(npts, dtype=torch.float64, device="cuda")
    var = torch.zeros_like(mean)
    cov = torch.zeros(npts, 13, dtype=torch.float64, device="cuda")
    g.gpr_reconstruct_dense(M, grid, g.GPR_P_FP64, mean, var, cov)
    g.gpr_sync()
    ref = oracle.Model.from_workload(small).stats15(n, (0, 0, 0), n)
    ys = np.abs(small.y).max()
    np.testing.assert_allclose(_np(mean), ref[:, 0], rtol=0, atol=1e-9 * ys)
    np.testing.assert_allclose(_np(var), ref[:, 1], rtol=0, atol=1e-10 * small.sf2)
    c = _np(cov)
    assert np.array_equal(np.isnan(c), np.isnan(ref[:, 2:]))
    ok = ~np.isnan(c)
    np.testing.assert_allclose(c[ok], ref[:, 2:][ok], rtol=0, atol=1e-10 * small.sf2)


def test_sgpr_lcp_dense_small(torch, g, small):
    """Cell LCP of an SGPR field: every cell against the oracle, and the FP32 pre-classification
    cascade equals the all-FP64 field bit for bit."""
    M = model_of(small)
    n, th = small.n, small.isovalues[1]
    grid = g.make_grid(n)
    outs = {}
    for key, kw in (("fp64", dict(prec=g.GPR_P_FP64)), ("fp32", dict(prec=g.GPR_P_FP32, exact=g.GPR_EXACT_FP64)),
                    ("default", {})):
        out = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
        g.gpr_lcp_dense(M, grid, th, g.lcp_options(**kw), out)
        g.gpr_sync()
        outs[key] = _np(out).astype(np.float64)
    ref = oracle.Model.from_workload(small).lcp_dense(n, th)
    assert np.abs(outs["fp64"] - ref).max() <= 1e-4
    assert np.array_equal(outs["fp64"], outs["fp32"])
    assert np.abs(outs["default"] - ref).max() <= 1e-4
    assert (ref > 1e-3).sum() > 50


def test_sgpr_octree_levels_and_adaptive_field(torch, g, small):
    """Algorithm 1 on an SGPR model: level decisions against the oracle (whose p-test reads mu_M and
    diag A_M), and the adaptive field equals the dense field on S and is 0 elsewhere."""
    M = model_of(small)
    om = oracle.Model.from_workload(small)
    n, D, th = small.n, small.max_depth, small.isovalues[1]
    grid = g.make_grid(n)
    opts = g.lcp_options()
    mism, seen = 0, 0
    for l in range(D + 1):
        nodes, dec, bnd = g.gpr_octree_trace(M, grid, th, D, opts, l)
        odec, obnd, _ = om.octree_level(n, D, l, th, nodes)
        assert np.array_equal(odec == 1, dec == 1), l
        bad = (odec > 0) != (dec > 0)
        near = (obnd >= 1e-3 / 3) & (obnd <= 3e-3)
        assert np.all(near[bad]), (l, obnd[bad & ~near][:8])
        mism += int(bad.sum()); seen += len(nodes)
    assert seen > 50 and mism <= max(2, seen // 100)
    field = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    st = g.gpr_lcp_adaptive(M, grid, th, D, opts, field)
    dense = torch.zeros_like(field)
    g.gpr_lcp_dense(M, grid, th, opts, dense)
    g.gpr_sync()
    f, d = _np(field), _np(dense)
    nodes, dec, _ = g.gpr_octree_trace(M, grid, th, D, opts, D)
    leaf = nodes[dec > 0]
    lin = (leaf & 0x1FFFFF) + (n - 1) * (((leaf >> 21) & 0x1FFFFF) + (n - 1) * ((leaf >> 42) & 0x1FFFFF))
    inS = np.zeros(f.size, bool); inS[lin] = True
    assert st["leaf_cells"] == inS.sum() > 0
    assert np.array_equal(f[inS], d[inS]) and np.all(f[~inS] == 0.0)


def test_sgpr_paper_scale_full_grid(torch, g, paper_scale):
    """The paper-scale SGPR model (m = 500 inducing sites fitted to 4000 samples, ARD SE, 128^3) run
    as the bench runs fields (default options: TF32x3 pre-pass, FP64-class digit-split corner
    statistics): sampled FP64 statistics, and a 12^3-cell block straddling the surface plus the
    domain corners against the oracle, at the median isovalue."""
    w = paper_scale
    M = model_of(w)
    om = oracle.Model.from_workload(w)
    n, th = w.n, w.isovalues[1]
    grid = g.make_grid(n)
    rng = np.random.default_rng(4)
    pts = np.unique(np.concatenate([rng.integers(0, n ** 3, 400), [0, n ** 3 - 1]]))
    out = torch.zeros(len(pts), 15, dtype=torch.float64, device="cuda")
    g.gpr_stats_points(M, grid, torch.tensor(pts, device="cuda"), out)
    g.gpr_sync()
    P = np.stack([pts % n, (pts // n) % n, pts // (n * n)], 1) / (n - 1)
    mu, var = om.posterior(P)
    o = _np(out)
    assert np.abs(o[:, 0] - mu).max() <= 1e-9 * np.abs(w.y).max()
    assert np.abs(o[:, 1] - var).max() <= 1e-8 * w.sf2
    field = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    st = g.gpr_lcp_dense(M, grid, th, g.lcp_options(), field)
    g.gpr_sync()
    f = _np(field).astype(np.float64).reshape(n - 1, n - 1, n - 1)
    ref = om.lcp_block(n, th, (50, 60, 40), (62, 72, 52)).reshape(12, 12, 12)
    assert np.abs(f[40:52, 60:72, 50:62] - ref).max() <= 1e-4
    assert (ref > 1e-3).sum() > 20
    for c0 in ((0, 0, 0), (n - 5, n - 5, n - 5)):
        r2 = om.lcp_block(n, th, c0, tuple(v + 4 for v in c0)).reshape(4, 4, 4)
        assert np.abs(f[c0[2]:c0[2] + 4, c0[1]:c0[1] + 4, c0[0]:c0[0] + 4] - r2).max() <= 1e-4
    assert st["cells_estimated"] > 10000


def test_sgpr_rejections(torch, g, small):
    """A_M not below K_MM (here A_M = K_MM + I) is not a distribution conditioned on data: the
    reversed-order factorisation fails and the call reports GPR_ERR_NOT_PD; the adjoint is written
    for plain GPR models and reports GPR_ERR_UNSUPPORTED for SGPR ones."""
    X = small.X[:20]
    d = (X[:, None, :] - X[None, :, :]) / np.asarray(small.ell)
    K = np.exp(-0.5 * (d ** 2).sum(-1))
    with pytest.raises(g.GPRError) as e:
        g.gpr_model_create_sgpr(X, np.zeros(20), K + np.eye(20), g.GPR_K_SE, small.ell, 1.0, 1e-6)
    assert e.value.status == g.GPR_ERR_NOT_PD
    M = model_of(small)
    dl = torch.ones((small.n - 1) ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(g.GPRError) as e:
        g.gpr_lcp_backward(M, g.make_grid(small.n), small.isovalues[1], g.lcp_options(), dl)
    assert e.value.status == g.GPR_ERR_UNSUPPORTED
