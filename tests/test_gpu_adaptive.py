"""GPU parity of the adaptive path (Algorithm 1 + leaf reconstruction) against the oracle
and against the GPU dense field.

Node decisions: the p-test decisions (FP64 on both sides) must agree exactly; bound decisions
may differ only where the oracle's bound lies within a factor 3 of alpha (the device evaluates
mu, sigma and their gradients in FP32 and its minimiser path can differ near the threshold).
Fields: equal to the dense field on S (same FP64 statistics, bit for bit) and 0 elsewhere.
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


def _compare_level(om, n, D, l, th, nodes, dec, bnd, alpha=1e-3, sample=None, seed=0, bound_tol=None):
    """Decisions of one level against the oracle; with bound_tol = (max, median) also the bounds
    of nodes both sides minimised in full, as |log(bound / oracle bound)| (where the bound can
    decide, >= alpha / 10; None skips that statistic)."""
    idx = np.argsort(nodes, kind="stable")  # the frontier's order is not deterministic: sample by code
    if sample is not None and len(idx) > sample:
        idx = idx[np.sort(np.random.default_rng(seed).choice(len(idx), sample, replace=False))]
    odec, obnd, _ = om.octree_level(n, D, l, th, nodes[idx], alpha=alpha)
    gd = dec[idx]
    # p-test decisions agree exactly
    assert np.array_equal(odec == 1, gd == 1), (l, np.sum((odec == 1) != (gd == 1)))
    keep_o = odec > 0
    keep_g = gd > 0
    mism = keep_o != keep_g
    near = (obnd >= alpha / 3) & (obnd <= 3 * alpha)
    assert np.all(near[mism]), (l, obnd[mism & ~near][:10], bnd[idx][mism & ~near][:10])
    both0 = (odec == 0) & (gd == 0) & (obnd >= alpha / 10)
    if bound_tol is not None and both0.any():
        lr = np.abs(np.log(bnd[idx][both0] / obnd[both0]))
        if bound_tol[0] is not None:
            assert lr.max() <= bound_tol[0], (l, lr.max())
        if bound_tol[1] is not None:
            assert np.median(lr) <= bound_tol[1], (l, np.median(lr))
    return int(mism.sum()), len(idx)


@pytest.mark.parametrize("case,prec", [("small", "fp32"), ("config1", "fp32"), ("small", "tf32x3"),
                                       ("config1", "tf32x3"), ("matern", "tf32x3")])
def test_octree_levels_match_oracle(torch, g, case, prec):
    if case == "small":
        w = workloads.small(5, 60, 17, ell=(0.2, 0.2, 0.2))
    elif case == "matern":
        w = workloads.small(5, 60, 17, ell=(0.2, 0.25, 0.3), kernel=workloads.MATERN52)
    else:
        w = workloads.config1()
    M = model_of(w)
    om = oracle.Model.from_workload(w)
    n, D, th = w.n, w.max_depth, w.isovalues[0]
    grid = g.make_grid(n)
    p = g.GPR_P_FP32 if prec == "fp32" else g.GPR_P_TF32X3
    total_mism = 0
    for l in range(D + 1):
        nodes, dec, bnd = g.gpr_octree_trace(M, grid, th, D, g.lcp_options(prec=p), l)
        if len(nodes) == 0:
            break
        # well-conditioned models: the FP32-class evaluations follow the oracle's minimiser path,
        # so the bounds agree to 1% (measured: < 0.05%)
        mm, cnt = _compare_level(om, n, D, l, th, nodes, dec, bnd, bound_tol=(1e-2, None))
        total_mism += mm
    assert total_mism <= 0.01 * (n - 1) ** 3 + 2


def _fields(g, torch, M, n, D, th, **kw):
    grid = g.make_grid(n)
    a = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    d = torch.zeros_like(a)
    sa = g.gpr_lcp_adaptive(M, grid, th, D, g.lcp_options(**kw), a)
    sd = g.gpr_lcp_dense(M, grid, th, g.lcp_options(**kw), d)
    g.gpr_sync()
    return a.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64), sa, sd


@pytest.mark.parametrize("case", ["small", "config1"])
def test_adaptive_field_vs_dense_and_oracle(torch, g, case):
    """Adaptive = dense on S and 0 elsewhere; against the oracle's adaptive field within 1e-4
    except on cells whose membership of S differs near alpha (their LCP is below ~alpha)."""
    w = workloads.small(5, 60, 17, ell=(0.2, 0.2, 0.2)) if case == "small" else workloads.config1()
    M = model_of(w)
    n, D, th = w.n, w.max_depth, w.isovalues[0]
    a, d, sa, sd = _fields(g, torch, M, n, D, th)
    nz = a != 0
    assert np.array_equal(a[nz], d[nz])
    assert sa["leaf_cells"] <= (n - 1) ** 3 and sa["leaf_cells"] > 0
    om = oracle.Model.from_workload(w)
    fo, leaves, _ = om.lcp_adaptive(n, D, th)
    lin = (leaves & 0x1FFFFF) + (n - 1) * (((leaves >> 21) & 0x1FFFFF) + (n - 1) * ((leaves >> 42) & 0x1FFFFF))
    in_o = np.zeros(a.size, bool); in_o[lin] = True
    diff = np.abs(a - fo)
    # cells the oracle kept and the GPU dropped (or vice versa) carry an LCP below a few alpha
    assert diff.max() <= 5e-3, diff.max()
    assert np.sum(diff > 1e-4) <= 0.01 * a.size + 2
    # RMSE adaptive vs dense (the paper's accuracy metric, Sec. 6.2): small
    assert np.sqrt(np.mean((a - d) ** 2)) < 2e-3


@pytest.mark.parametrize("m,n", [(1, 2), (1, 5), (3, 3), (3, 9)])
def test_adaptive_degenerate_models_and_grids(torch, g, m, n):
    """One or three observations, grids of 1, 8, 64 and 512 cells (max depth 0 .. 3): the adaptive
    field equals the dense field on the GPU's S and 0 elsewhere, and the oracle's adaptive field
    within 1e-4 where both keep the cell (the evaluations and the bound run on padded 64-column
    operands with m = 1)."""
    w = workloads.small(50 + m, m, n, ell=(0.4, 0.5, 0.6))
    M = model_of(w)
    om = oracle.Model.from_workload(w)
    th = float(np.median(w.y)) if m > 1 else float(w.y[0]) + 0.05
    D = w.max_depth
    a, d, sa, _ = _fields(g, torch, M, n, D, th)
    keep = a != 0
    assert np.array_equal(a[keep], d[keep])
    of, _, _ = om.lcp_adaptive(n, D, th)
    both = keep & (of != 0)
    if both.any():
        assert np.abs(a[both] - of[both]).max() <= 1e-4
    assert sa["leaf_cells"] <= (n - 1) ** 3


def test_adaptive_config2_full_size_sampled_nodes(torch, g):
    """Paper-scale field (m=500, 128^3, D=7): sampled nodes of the deepest four levels against the
    oracle's per-node decision (each node's decision depends only on the node)."""
    w = workloads.config2()
    M = model_of(w)
    om = oracle.Model.from_workload(w)
    th = w.isovalues[1]
    grid = g.make_grid(w.n)
    for l in (2, 4, 5, 6, 7):
        nodes, dec, bnd = g.gpr_octree_trace(M, grid, th, w.max_depth, g.lcp_options(prec=g.GPR_P_TF32X3), l)
        assert len(nodes) > 0
        # ill-conditioned model (var down to 4e-5 sf2): the FP32-class variances (|dvar| up to ~4e-5
        # sf2 in the TF32x3 pre-pass and the evaluations) move g by up to a few per cent, a few times
        # that in the Phi tails the bound sits in, and the local minimiser can end at another point:
        # the median bound agrees within 25 % (measured 2-10 %), single nodes by less (one node of 93
        # by a factor 12)
        mm, cnt = _compare_level(om, w.n, w.max_depth, l, th, nodes, dec, bnd, sample=150 if l >= 5 else None,
                                 seed=l, bound_tol=(None, 0.25))
        assert mm <= max(3, 0.03 * cnt)


def test_adaptive_config2_full_field(torch, g):
    """Full adaptive field at the three isovalues, launched as the bench does: equal to the dense
    field on S, zero elsewhere, RMSE vs dense small, and fewer reconstructed points."""
    w = workloads.config2()
    M = model_of(w)
    for th in w.isovalues:
        a, d, sa, sd = _fields(g, torch, M, w.n, w.max_depth, th)
        nz = a != 0
        assert np.array_equal(a[nz], d[nz])
        assert np.sqrt(np.mean((a - d) ** 2)) < 1e-3
        assert sa["leaf_cells"] <= sd["leaf_cells"]  # |S| vs the dense cascade's kept cells
        assert sum(sa["nodes_per_level"]) > 0


def test_adaptive_argument_checks(torch, g):
    w = workloads.small(1, 10, 9)
    M = model_of(w)
    out = torch.zeros(512, dtype=torch.float32, device="cuda")
    with pytest.raises(g.GPRError) as e:
        g.gpr_lcp_adaptive(M, g.make_grid(9), 0.0, 2, g.lcp_options(), out)  # 2^2 < 8 cells
    assert e.value.status == g.GPR_ERR_ARG


@pytest.mark.parametrize("kind", ["gpr", "sgpr"])
def test_local_model_levels_match_oracle(torch, g, kind):
    """Sec. 5.2's local model (beta >= 0): nodes whose enlarged box (beta * l_d per axis) leaves some
    observations out are bounded on the model of the rest.  Plain GPR: nodes with equal local sets
    share one FP64 factorisation and are evaluated in FP32 (as the full model's bound is); SGPR: FP64
    per node.  Level by level against the oracle's FP64 local model: p-test decisions equal, bound
    decisions equal except within a factor 3 of alpha, and the bounds of nodes both sides minimised
    fully agree to 1e-6 relative (SGPR, FP64), or to 5e-2 where they are >= alpha / 10 (plain, FP32
    evaluations: the whitened FP32 variance carries ~6e-6 of sf2 against node variances of ~2e-4
    of sf2, a few per cent in the Phi tails the bound sits in; far smaller bounds differ more in
    relative terms and decide nothing)."""
    w = workloads.config2() if kind == "gpr" else workloads.sgpr(n=33)
    beta = 1.0
    M = model_of(w)
    om = oracle.Model.from_workload(w)
    n, D, th = 33, 5, w.isovalues[1]
    grid = g.make_grid(n)
    opts = g.lcp_options(beta=beta)
    seen = 0
    for l in range(1, D + 1):
        nodes, dec, bnd = g.gpr_octree_trace(M, grid, th, D, opts, l)
        if len(nodes) == 0:
            break
        odec, obnd, _ = om.octree_level(n, D, l, th, nodes, beta=beta)
        assert np.array_equal(odec == 1, dec == 1), l
        bad = (odec > 0) != (dec > 0)
        near = (obnd >= 1e-3 / 3) & (obnd <= 3e-3)
        assert np.all(near[bad]), (l, obnd[bad & ~near][:8], bnd[bad & ~near][:8])
        both0 = (odec == 0) & (dec == 0)
        if kind == "sgpr" and both0.any():
            np.testing.assert_allclose(bnd[both0], obnd[both0], rtol=1e-6, atol=1e-300)
        near_a = both0 & (obnd >= 1e-4)  # FP32 evaluations: compare the bounds that decide
        if kind == "gpr" and near_a.any():
            np.testing.assert_allclose(bnd[near_a], obnd[near_a], rtol=5e-2, atol=1e-300)
        seen += len(nodes)
    assert seen > 100
    # a beta whose boxes cover the domain gives the full model's decisions exactly
    for l in (2, 3):
        a = g.gpr_octree_trace(M, grid, th, D, g.lcp_options(beta=50.0), l)
        b = g.gpr_octree_trace(M, grid, th, D, g.lcp_options(), l)
        ia, ib = np.argsort(a[0]), np.argsort(b[0])  # the frontier order is not deterministic
        np.testing.assert_array_equal(a[0][ia], b[0][ib]); np.testing.assert_array_equal(a[1][ia], b[1][ib])


def test_local_model_adaptive_field(torch, g):
    """With the local model the adaptive field still equals the dense field on its S (the paper-scale
    field on a 33^3 grid, beta = 1: about half of the cells are kept)."""
    w = workloads.config2()
    M = model_of(w)
    n, D, th = 33, 5, w.isovalues[1]
    grid = g.make_grid(n)
    opts = g.lcp_options(beta=1.0)
    a = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    d = torch.zeros_like(a)
    st = g.gpr_lcp_adaptive(M, grid, th, D, opts, a)
    g.gpr_lcp_dense(M, grid, th, opts, d)
    g.gpr_sync()
    nodes, dec, _ = g.gpr_octree_trace(M, grid, th, D, opts, D)
    leaf = nodes[dec > 0]
    lin = (leaf & 0x1FFFFF) + (n - 1) * (((leaf >> 21) & 0x1FFFFF) + (n - 1) * ((leaf >> 42) & 0x1FFFFF))
    inS = np.zeros((n - 1) ** 3, bool); inS[lin] = True
    av, dv = a.cpu().numpy(), d.cpu().numpy()
    assert st["leaf_cells"] == inS.sum() and 0 < inS.sum() < inS.size
    assert np.array_equal(av[inS], dv[inS]) and np.all(av[~inS] == 0)


def test_kd_tree_levels_match_oracle_and_field(torch, g):
    """The K-D tree (Sec. 9) on the device: every level against the oracle's K-D levels (p-test
    exact, bound decisions within a factor 3 of alpha), and the adaptive field equal to the dense
    field on its S (the paper-scale field on a 33^3 grid)."""
    w = workloads.config2()
    M = model_of(w)
    om = oracle.Model.from_workload(w)
    n, D, th = 33, 5, w.isovalues[1]
    grid = g.make_grid(n)
    opts = g.lcp_options(tree=g.GPR_TREE_KD)
    seen = 0
    for l in range(3 * D + 1):
        nodes, dec, bnd = g.gpr_octree_trace(M, grid, th, D, opts, l)
        if len(nodes) == 0:
            break
        odec, obnd, _ = om.octree_level(n, D, l, th, nodes, kd=True)
        assert np.array_equal(odec == 1, dec == 1), l
        bad = (odec > 0) != (dec > 0)
        near = (obnd >= 1e-3 / 3) & (obnd <= 3e-3)
        assert np.all(near[bad]), (l, obnd[bad & ~near][:8], bnd[bad & ~near][:8])
        # bounds both sides computed in full: median within 25% (FP32-class evaluations, as for the octree)
        both0 = (odec == 0) & (dec == 0) & (obnd >= 1e-4)
        if both0.sum() >= 5:
            assert np.median(np.abs(np.log(bnd[both0] / obnd[both0]))) <= 0.25, l
        seen += len(nodes)
    assert seen > 1000
    a = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    d = torch.zeros_like(a)
    st = g.gpr_lcp_adaptive(M, grid, th, D, opts, a)
    g.gpr_lcp_dense(M, grid, th, opts, d)
    g.gpr_sync()
    nodes, dec, _ = g.gpr_octree_trace(M, grid, th, D, opts, 3 * D)
    leaf = nodes[dec > 0]
    lin = (leaf & 0x1FFFFF) + (n - 1) * (((leaf >> 21) & 0x1FFFFF) + (n - 1) * ((leaf >> 42) & 0x1FFFFF))
    inS = np.zeros((n - 1) ** 3, bool); inS[lin] = True
    av, dv = a.cpu().numpy(), d.cpu().numpy()
    assert st["leaf_cells"] == inS.sum() and 0 < inS.sum() < inS.size
    assert np.array_equal(av[inS], dv[inS]) and np.all(av[~inS] == 0)



def _eval_points(g, torch, M, P):
    """mu, var, grad mu, grad var at the points P by the bound minimiser's evaluation path."""
    import ctypes as C
    from paper_2512_12442_gb300._lib import load
    xyz = torch.tensor(np.ascontiguousarray(P), dtype=torch.float64, device="cuda")
    out = torch.zeros(len(P), 8, dtype=torch.float32, device="cuda")
    rc = load().gpr_eval_points(C.c_void_p(M.handle), C.c_void_p(xyz.data_ptr()), len(P), 1,
                                C.c_void_p(out.data_ptr()), None)
    assert rc == 0
    g.gpr_sync()
    o = out.cpu().numpy().astype(np.float64)
    return o[:, 0], o[:, 1], o[:, 2:5], o[:, 5:8]


def _oracle_moments(om, P, t1, t2):
    """The same four from the oracle's FP64 g = (t - mu) / sigma and grad g at two isovalues."""
    g1, gr1 = om.eval_g(P, t1, 1)
    g2, gr2 = om.eval_g(P, t2, 1)
    sd = (t2 - t1) / (g2 - g1)
    mu = t1 - g1 * sd
    gvar = -2.0 * sd[:, None] ** 3 * (gr2 - gr1) / (t2 - t1)
    gmu = -sd[:, None] * (gr1 + g1[:, None] * gvar / (2.0 * sd[:, None] ** 2))
    return mu, sd ** 2, gmu, gvar


@pytest.mark.parametrize("kind", ["gpr", "sgpr", "matern"])
def test_bound_evaluations_vs_oracle(torch, g, kind):
    """The bound minimiser's evaluations (TF32x3 tensor-core rows of k and of d k / d x_d, reduced to
    |w|^2 and w . L^-1 d_k k; mean and its gradient by compensated k . alpha) at 2,000 random points
    and 200 points next to observations, against the oracle's FP64 values (recovered from its g and
    grad g at two isovalues).  Tolerances (FP32-class whitened arithmetic, the tolerance of the FP32
    paths): |dmu| <= 1e-4 max|y|, |dvar| <= 1e-4 sf2, |d grad mu| <= 1e-4 max|y| / l_min,
    |d grad var| <= 1e-4 sf2 / l_min for the plain model; 5e-4 for the sparse one, whose
    K_MM + 1e-6 I (condition ~5e7, against ~4e5) amplifies the FP32 rounding of the kernel entries
    more.  The Matern-5/2 case (m=300, l=(0.12, 0.18, 0.25)) checks that kernel's derivative rows."""
    if kind == "gpr":
        w = workloads.config2()
    elif kind == "sgpr":
        w = workloads.sgpr(n=33)
    else:
        w = workloads.small(9, 300, 33, ell=(0.12, 0.18, 0.25), kernel=workloads.MATERN52)
    M = model_of(w)
    om = oracle.Model.from_workload(w)
    rng = np.random.default_rng(21)
    X = np.asarray(w.X)
    P = np.concatenate([rng.random((2000, 3)),
                        np.clip(X[rng.integers(0, len(X), 200)] + rng.normal(0, 0.01, (200, 3)), 0, 1)])
    mu, var, gmu, gvar = _eval_points(g, torch, M, P)
    omu, ovar, ogmu, ogvar = _oracle_moments(om, P, float(w.isovalues[-1]), float(w.isovalues[-1]) + 1.0)
    ys = np.abs(np.asarray(w.y)).max()  # observations, or the inducing means mu_M of the sparse model
    lmin = float(np.min(w.ell))
    err = (np.abs(mu - omu).max() / ys, np.abs(var - ovar).max() / w.sf2,
           np.abs(gmu - ogmu).max() * lmin / ys, np.abs(gvar - ogvar).max() * lmin / w.sf2)
    print(f"\n{kind}: max |dmu|/max|y| {err[0]:.2e}, |dvar|/sf2 {err[1]:.2e}, "
          f"|d grad mu| l/max|y| {err[2]:.2e}, |d grad var| l/sf2 {err[3]:.2e}; "
          f"var range {ovar.min():.2e}..{ovar.max():.2e}, |grad mu| l/max|y| up to "
          f"{np.abs(ogmu).max() * lmin / ys:.2e}, |grad var| l/sf2 up to {np.abs(ogvar).max() * lmin / w.sf2:.2e}")
    tol = 5e-4 if kind == "sgpr" else 1e-4
    assert max(err) <= tol, err
