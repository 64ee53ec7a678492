"""GPU adjoint (gpr_lcp_backward, gpr_lcp_backward_adaptive, LCPFunction) against the FP64 oracle
gradient and central finite differences (h = 1e-3).

Tolerance against the oracle, entry by entry: every dL/dy_i within 2e-3 |oracle_i| + 2e-4 max_j
|oracle_j|, and every dL/dlog l_d within 2e-3 |oracle_d| + 1e-4 sum_d |oracle_d|.  The reverse sweep
runs on FP32 samples with this library's Phi / Phi^-1 (relative error ~1e-6 each), so a cell's
derivative carries a relative error of ~1e-5; dL/dy_i sums such derivatives of both signs over the
cells near observation i, so its absolute error scales with the largest entries, not with entry i
itself (the second term).  Finite differences of the GPU forward: within 3% (the FP32 estimator adds
~1e-7 per cell of noise to the loss)."""
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


def _gpu_grad(g, torch, w, n, th, wts, **kw):
    M = model_of(w)
    dl = torch.tensor(wts, dtype=torch.float32, device="cuda")
    return g.gpr_lcp_backward(M, g.make_grid(n), th, g.lcp_options(**kw), dl)


def _check_entries(dy, dl, ody, odl):
    """Entry-by-entry comparison with the oracle's FP64 gradient (tolerance in the module doc)."""
    ay = 2e-3 * np.abs(ody) + 2e-4 * np.abs(ody).max()
    bad = np.nonzero(np.abs(dy - ody) > ay)[0]
    assert bad.size == 0, (bad[:8], dy[bad[:8]], ody[bad[:8]], float(np.max(np.abs(dy - ody) / np.abs(ody).max())))
    al = 2e-3 * np.abs(odl) + 1e-4 * np.abs(odl).sum()
    assert np.all(np.abs(dl - odl) <= al), (dl, odl)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_backward_small_vs_oracle(torch, g, prec):
    w = workloads.small(5, 30, 9, ell=(0.2, 0.25, 0.3))
    n, th = 9, w.isovalues[0]
    wts = np.random.default_rng(5).random((n - 1) ** 3)
    p = g.GPR_P_FP64 if prec == "fp64" else g.GPR_P_TF32X3
    dy, dl = _gpu_grad(g, torch, w, n, th, wts, prec=p)
    loss, ody, odl = oracle.Model.from_workload(w).lcp_grad(n, th, wts)
    _check_entries(dy, dl, ody, odl)


def test_backward_matern_vs_oracle(torch, g):
    """Matern-5/2: no digit split for its rows, so the FP64 rows, the FP64 GEMMs, the FP64 Zh and
    the FP64 point terms (kernel derivative through r) carry the backward."""
    w = workloads.small(6, 40, 11, ell=(0.25, 0.3, 0.35), kernel=workloads.MATERN52)
    n, th = 11, w.isovalues[0]
    wts = np.random.default_rng(6).random((n - 1) ** 3)
    dy, dl = _gpu_grad(g, torch, w, n, th, wts)
    loss, ody, odl = oracle.Model.from_workload(w).lcp_grad(n, th, wts)
    _check_entries(dy, dl, ody, odl)


@pytest.mark.parametrize("exact", ["auto", "fp64"])
def test_backward_config5_field_32cubed_vs_oracle(torch, g, exact):
    """The differentiation workload's field (m=500, ARD SE, noise 1e-4) on a 32^3 grid with U(0,1)
    cell weights: GPU gradient vs the oracle's FP64 analytic gradient, with the corner rows from
    the tensor-core digit split (auto) and from the FP64 cores."""
    w = workloads.config5()
    n, th = 32, w.isovalues[0]
    wts = np.random.default_rng(5).random((n - 1) ** 3)
    ex = g.GPR_EXACT_AUTO if exact == "auto" else g.GPR_EXACT_FP64
    dy, dl = _gpu_grad(g, torch, w, n, th, wts, exact=ex)
    loss, ody, odl = oracle.Model.from_workload(w).lcp_grad(n, th, wts)
    _check_entries(dy, dl, ody, odl)


def test_backward_config5_grid128_subgrid_vs_oracle(torch, g):
    """The differentiation workload as named (m=500 ARD SE field on the 128^3 grid): the weights are
    the workload's U(0,1) cell weights on the 31^3 cells of a 32^3-point sub-grid and 0 elsewhere,
    so the GPU call runs on the full grid and the oracle's FP64 gradient covers exactly the weighted
    cells.  Entry by entry."""
    w = workloads.config5()
    n, th = 128, w.isovalues[0]
    c0, c1 = (48, 40, 56), (79, 71, 87)
    wfull = w.extra["cell_weights"].reshape(127, 127, 127)  # [k][j][i]
    mask = np.zeros_like(wfull)
    mask[c0[2]:c1[2], c0[1]:c1[1], c0[0]:c1[0]] = 1.0
    wts = (wfull * mask).reshape(-1)
    dy, dl = _gpu_grad(g, torch, w, n, th, wts)
    loss, ody, odl = oracle.Model.from_workload(w).lcp_grad(n, th, wts, c0=c0, c1=c1)
    assert loss > 0.0
    _check_entries(dy, dl, ody, odl)


def test_backward_finite_differences_gpu(torch, g):
    """Central differences of the GPU forward (dense, all-FP64 statistics) on 4 y_i and 3 log l_d."""
    w = workloads.small(9, 40, 13, ell=(0.2, 0.25, 0.3))
    n, th = 13, w.isovalues[0]
    wts = np.random.default_rng(1).random((n - 1) ** 3)
    dy, dl = _gpu_grad(g, torch, w, n, th, wts, prec=g.GPR_P_FP64)

    def loss(y, ell):
        M = g.gpr_model_create(w.X, y, w.kernel, ell, w.sf2, w.sn2)
        out = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
        g.gpr_lcp_dense(M, g.make_grid(n), th, g.lcp_options(prec=g.GPR_P_FP64), out)
        g.gpr_sync()
        return float(np.dot(out.cpu().numpy().astype(np.float64), wts))

    h = 1e-3
    ell = np.array(w.ell)
    for i in (3, 17, 29, 38):
        yp = w.y.copy(); yp[i] += h
        ym = w.y.copy(); ym[i] -= h
        fd = (loss(yp, ell) - loss(ym, ell)) / (2 * h)
        assert abs(dy[i] - fd) <= 0.03 * abs(fd) + 1e-3 * np.abs(dy).max(), (i, dy[i], fd)
    for d in range(3):
        e = np.zeros(3); e[d] = h
        fd = (loss(w.y, ell * np.exp(e)) - loss(w.y, ell * np.exp(-e))) / (2 * h)
        assert abs(dl[d] - fd) <= 0.03 * abs(fd) + 1e-3 * np.abs(dl).max(), (d, dl[d], fd)


def test_autograd_function(torch, g):
    """LCPFunction: torch autograd through the C ABI gives the same gradient as the direct call."""
    from paper_2512_12442_gb300.autograd import lcp_field
    w = workloads.small(5, 30, 9, ell=(0.2, 0.25, 0.3))
    n, th = 9, w.isovalues[0]
    wts = torch.tensor(np.random.default_rng(5).random((n - 1) ** 3), dtype=torch.float32, device="cuda")
    y = torch.tensor(w.y, dtype=torch.float64, requires_grad=True)
    ll = torch.tensor(np.log(w.ell), dtype=torch.float64, requires_grad=True)
    out = lcp_field(y, ll, w.X, n, th, noise_var=w.sn2)
    (out * wts).sum().backward()
    dy, dl = _gpu_grad(g, torch, w, n, th, wts.cpu().numpy())
    np.testing.assert_allclose(y.grad.numpy(), dy, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(ll.grad.numpy(), dl, rtol=1e-6, atol=1e-9)


def test_backward_adaptive_masks_cells_outside_the_leaf_set(torch, g):
    """gpr_lcp_backward_adaptive equals gpr_lcp_backward with the weights of cells outside Algorithm
    1's leaf set S set to 0; S is read from the device octree's last level (gpr_octree_trace), and
    the adaptive forward field is 0 exactly outside S.  The paper-scale field on a 33^3 grid keeps
    about a third of the cells."""
    w = workloads.config2()
    n, th, D = 33, w.isovalues[1], workloads.depth_for(33)
    wts = np.random.default_rng(3).random((n - 1) ** 3)
    M = model_of(w)
    grid, opts = g.make_grid(n), g.lcp_options()
    nodes, dec, _ = g.gpr_octree_trace(M, grid, th, D, opts, D)
    leaf = nodes[dec > 0]
    lin = (leaf & 0x1FFFFF) + (n - 1) * (((leaf >> 21) & 0x1FFFFF) + (n - 1) * ((leaf >> 42) & 0x1FFFFF))
    inS = np.zeros((n - 1) ** 3, bool); inS[lin] = True
    assert 0 < inS.sum() < inS.size
    field = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    g.gpr_lcp_adaptive(M, grid, th, D, opts, field)
    assert np.all(field.cpu().numpy()[~inS] == 0.0)
    dl_t = torch.tensor(wts, dtype=torch.float32, device="cuda")
    dya, dla = g.gpr_lcp_backward_adaptive(M, grid, th, D, opts, dl_t)
    masked = torch.tensor(np.where(inS, wts, 0.0), dtype=torch.float32, device="cuda")
    dym, dlm = g.gpr_lcp_backward(M, grid, th, opts, masked)
    np.testing.assert_allclose(dya, dym, rtol=1e-10, atol=1e-12 * np.abs(dym).max())
    np.testing.assert_allclose(dla, dlm, rtol=1e-10, atol=1e-12 * np.abs(dlm).max())
    dyf, _ = g.gpr_lcp_backward(M, grid, th, opts, dl_t)
    assert np.abs(dyf - dya).max() > 1e-6 * np.abs(dyf).max()  # S does mask something here


def test_autograd_adaptive_field(torch, g):
    """LCPFunction over the adaptive field calls the library's adaptive backward."""
    from paper_2512_12442_gb300.autograd import lcp_field
    w = workloads.small(7, 60, 17, ell=(0.2, 0.25, 0.3))
    n, th, D = 17, w.isovalues[0], workloads.depth_for(17)
    wts = torch.tensor(np.random.default_rng(3).random((n - 1) ** 3), dtype=torch.float32, device="cuda")
    y = torch.tensor(w.y, dtype=torch.float64, requires_grad=True)
    ll = torch.tensor(np.log(w.ell), dtype=torch.float64, requires_grad=True)
    out = lcp_field(y, ll, w.X, n, th, noise_var=w.sn2, adaptive_depth=D)
    (out * wts).sum().backward()
    M = model_of(w)
    dy, dl = g.gpr_lcp_backward_adaptive(M, g.make_grid(n), th, D, g.lcp_options(), wts)
    np.testing.assert_allclose(y.grad.numpy(), dy, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(ll.grad.numpy(), dl, rtol=1e-6, atol=1e-9)


def test_backward_rejects_mc(torch, g):
    w = workloads.small(5, 30, 9)
    M = model_of(w)
    dl = torch.ones(512, dtype=torch.float32, device="cuda")
    with pytest.raises(g.GPRError) as e:
        g.gpr_lcp_backward(M, g.make_grid(9), 0.0, g.lcp_options(est=g.GPR_EST_MC), dl)
    assert e.value.status == g.GPR_ERR_UNSUPPORTED


def test_backward_after_forward_reuses_cache(torch, g):
    """A backward after a forward call on the same model and grid takes the pre-pass table, rows and
    statistics from the model's grid cache; the gradient equals that of a backward on a fresh model
    (up to the order of the FP64 atomic sums)."""
    w = workloads.small(7, 60, 17, ell=(0.2, 0.25, 0.3))
    n, th = 17, w.isovalues[0]
    wts = np.random.default_rng(3).random((n - 1) ** 3)
    dy0, dl0 = _gpu_grad(g, torch, w, n, th, wts)
    M = model_of(w)
    f = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    g.gpr_lcp_dense(M, g.make_grid(n), th, g.lcp_options(), f)
    dl_t = torch.tensor(wts, dtype=torch.float32, device="cuda")
    dy1, dl1 = g.gpr_lcp_backward(M, g.make_grid(n), th, g.lcp_options(), dl_t)
    np.testing.assert_allclose(dy1, dy0, rtol=1e-10, atol=1e-12 * np.abs(dy0).max())
    np.testing.assert_allclose(dl1, dl0, rtol=1e-10, atol=1e-12 * np.abs(dl0).max())


def test_scratch_release_between_calls(torch, g):
    """gpr_batch_release frees the pooled scratch (batch workspaces, digit buffers of the FP64-class
    products); the next call allocates it again and gives the same gradient."""
    w = workloads.small(5, 30, 9, ell=(0.2, 0.25, 0.3))
    n, th = 9, w.isovalues[0]
    wts = np.random.default_rng(5).random((n - 1) ** 3)
    dy0, dl0 = _gpu_grad(g, torch, w, n, th, wts)
    g.gpr_batch_release()
    dy1, dl1 = _gpu_grad(g, torch, w, n, th, wts)
    np.testing.assert_allclose(dy1, dy0, rtol=1e-10, atol=1e-12 * np.abs(dy0).max())
    np.testing.assert_allclose(dl1, dl0, rtol=1e-10, atol=1e-12 * np.abs(dl0).max())
