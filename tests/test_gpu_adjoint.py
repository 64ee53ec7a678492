"""GPU adjoint (gpr_lcp_backward, LCPFunction) against the FP64 oracle gradient and central
finite differences (h = 1e-3).  Tolerance: relative error of the gradient vector <= 2e-3 vs the
oracle (the estimator's reverse sweep runs in FP32 samples); finite differences of the GPU
forward within 3% (the FP32 estimator adds ~1e-7 per cell of noise to the loss)."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_backward_small_vs_oracle(torch, g, prec):
    w = workloads.small(5, 30, 9, ell=(0.2, 0.25, 0.3))
    n, th = 9, w.isovalues[0]
    wts = np.random.default_rng(5).random((n - 1) ** 3)
    p = g.GPR_P_FP64 if prec == "fp64" else g.GPR_P_TF32X3
    dy, dl = _gpu_grad(g, torch, w, n, th, wts, prec=p)
    loss, ody, odl = oracle.Model.from_workload(w).lcp_grad(n, th, wts)
    assert _rel(dy, ody) <= 2e-3, (_rel(dy, ody), dy[:4], ody[:4])
    assert _rel(dl, odl) <= 2e-3, (dl, odl)


def test_backward_matern_vs_oracle(torch, g):
    """Matern-5/2: no digit split for its rows, so the FP64 rows, the FP64 GEMMs, the FP64 Zh and
    the FP64 point terms (kernel derivative through r) carry the backward."""
    w = workloads.small(6, 40, 11, ell=(0.25, 0.3, 0.35), kernel=workloads.MATERN52)
    n, th = 11, w.isovalues[0]
    wts = np.random.default_rng(6).random((n - 1) ** 3)
    dy, dl = _gpu_grad(g, torch, w, n, th, wts)
    loss, ody, odl = oracle.Model.from_workload(w).lcp_grad(n, th, wts)
    assert _rel(dy, ody) <= 2e-3, (_rel(dy, ody), dy[:4], ody[:4])
    assert _rel(dl, odl) <= 2e-3, (dl, odl)


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
    assert _rel(dy, ody) <= 2e-3 and _rel(dl, odl) <= 2e-3, (_rel(dy, ody), dl, odl)


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
