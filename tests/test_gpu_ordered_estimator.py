"""GPR_EST_SOV_ORDERED on the GPU against the oracle's ordered estimator (Sec. 4's cell LCP with
each orthant's corners in ascending order of their standardised thresholds), through the C ABI.

Tolerance |dLCP| <= 1e-4 as for the index-order estimator (the GPU runs the recursion in FP32 with
its own Phi / Phi^-1; the order is decided in FP64 on both sides).  Also: the adaptive field equals
the dense one on S, the batched call equals the single-field call bit for bit, the perfectly
correlated closed form through the cell entry point, and the calls that do not support the
ordered estimator say so.
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


def _dense(g, torch, M, n, th, **kw):
    out = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    st = g.gpr_lcp_dense(M, g.make_grid(n), th, g.lcp_options(est=g.GPR_EST_SOV_ORDERED, **kw), out)
    g.gpr_sync()
    return out.cpu().numpy().astype(np.float64), st


def test_ordered_dense_config1_every_cell(torch, g):
    """Config-1 field (m=64, 32^3): every cell against the oracle."""
    w = workloads.config1()
    M = model_of(w)
    th = w.isovalues[0]
    gpu, st = _dense(g, torch, M, w.n, th, prec=g.GPR_P_FP64)
    ref = oracle.Model.from_workload(w).lcp_dense(w.n, th, est=oracle.EST_SOV_ORD)
    d = np.abs(gpu - ref)
    assert d.max() <= 1e-4, d.max()
    assert st["cells_estimated"] > 100


@pytest.mark.parametrize("iso,c0", [(0, (50, 60, 40)), (1, (68, 44, 44))])
def test_ordered_paper_scale_block(torch, g, iso, c0):
    """Paper-scale field (m=500, 128^3), launched as the bench launches the dense path: a 12^3-cell
    block across the surface against the oracle cell by cell (185 cells with LCP in (0.01, 0.99)
    at the first isovalue, 1300 at the median one)."""
    w = workloads.config2()
    M = model_of(w)
    n = w.n
    th = w.isovalues[iso]
    gpu, _ = _dense(g, torch, M, n, th, prec=g.GPR_P_FP32)
    f = gpu.reshape(n - 1, n - 1, n - 1)
    ref = oracle.Model.from_workload(w).lcp_block(n, th, c0, tuple(v + 12 for v in c0),
                                                 est=oracle.EST_SOV_ORD).reshape(12, 12, 12)
    assert np.sum((ref > 0.01) & (ref < 0.99)) >= 150
    d = np.abs(f[c0[2]:c0[2] + 12, c0[1]:c0[1] + 12, c0[0]:c0[0] + 12] - ref)
    assert d.max() <= 1e-4, d.max()
    assert 0.0 <= gpu.min() and gpu.max() <= 1.0


def test_ordered_adaptive_equals_dense_and_batched_equals_single(torch, g):
    """Algorithm 1 with the ordered estimator: the adaptive field equals the dense field on the leaf
    cells S; the batched call (two isovalues, shared estimator launch) equals single calls."""
    w = workloads.small(22, 300, 33, ell=(0.15, 0.2, 0.25))
    M = model_of(w)
    opts = g.lcp_options(est=g.GPR_EST_SOV_ORDERED)
    grid = g.make_grid(w.n)
    ths = [w.isovalues[0], float(np.percentile(w.y, 25.0))]
    singles = []
    for th in ths:
        a = torch.zeros((w.n - 1) ** 3, dtype=torch.float32, device="cuda")
        g.gpr_lcp_adaptive(M, grid, th, w.max_depth, opts, a)
        g.gpr_sync()
        singles.append(a.cpu().numpy())
        dense, _ = _dense(g, torch, M, w.n, th)
        on = singles[-1] > 0
        assert np.array_equal(singles[-1][on], dense[on].astype(np.float32))
    outs = [torch.full(((w.n - 1) ** 3,), -1.0, dtype=torch.float32, device="cuda") for _ in ths]
    g.gpr_lcp_adaptive_batched([M, M], [grid, grid], ths, [w.max_depth] * 2, opts, outs)
    g.gpr_sync()
    for a, b in zip(singles, outs):
        assert np.array_equal(a, b.cpu().numpy())


def test_ordered_cell_entry_perfect_correlation(torch, g):
    """Through gpr_cell_lcp_from_stats: corners sharing one normal variable (covariances equal to
    the variance) with distinct means have LCP = Phi(z_max) - Phi(z_min); the ordered estimator
    reaches it in FP32 (5e-6), the index-order one does not need to."""
    from scipy.special import ndtr
    n = 3
    grid = g.make_grid(n)
    rng = np.random.default_rng(4)
    sd = 0.2
    mu = rng.normal(0.0, 0.1, n ** 3)
    st = np.zeros((n ** 3, 15))
    st[:, 0] = mu
    st[:, 1] = sd * sd
    st[:, 2:] = sd * sd
    th = float(np.median(mu))
    s15 = torch.tensor(st, dtype=torch.float64, device="cuda")
    out = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    g.gpr_cell_lcp_from_stats(grid, s15, th, g.lcp_options(est=g.GPR_EST_SOV_ORDERED, skip_eps=0.0), None, out)
    g.gpr_sync()
    got = out.cpu().numpy()
    for c in range((n - 1) ** 3):
        i, j, k = c % (n - 1), (c // (n - 1)) % (n - 1), c // ((n - 1) ** 2)
        corners = [(i + (q & 1)) + n * ((j + ((q >> 1) & 1)) + n * (k + (q >> 2))) for q in range(8)]
        z = (th - mu[corners]) / sd
        assert got[c] == pytest.approx(ndtr(z.max()) - ndtr(z.min()), abs=5e-6), c


def test_ordered_estimator_unsupported_where_documented(torch, g):
    """The backward calls and the allocation-free entry point reject the ordered estimator."""
    w = workloads.small(21, 40, 9)
    M = model_of(w)
    grid = g.make_grid(w.n)
    opts = g.lcp_options(est=g.GPR_EST_SOV_ORDERED)
    dl = torch.ones((w.n - 1) ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(g.GPRError) as e:
        g.gpr_lcp_backward(M, grid, w.isovalues[0], opts, dl)
    assert e.value.status == g.GPR_ERR_UNSUPPORTED
    s15 = torch.zeros((w.n ** 3, 15), dtype=torch.float64, device="cuda")
    s15[:, 1] = 1.0
    out = torch.zeros((w.n - 1) ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(g.GPRError) as e:
        g.gpr_cell_lcp_from_stats_noalloc(grid, s15, 0.0, opts, None, out)
    assert e.value.status == g.GPR_ERR_UNSUPPORTED

