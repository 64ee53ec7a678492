"""Batched adaptive LCP (many fields, one call): every field equals the single-field call.

The batch groups fields by model, runs them on worker streams and estimates every field's
cells in one launch; none of that changes the arithmetic, so fields must agree bit for bit
with gpr_lcp_adaptive.  Also checked: the per-field fallback when the shared record buffer
is full, a single worker, repeated models, uneven grids and m, and argument errors.
"""
import numpy as np
import pytest

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


def _fields():
    """Uneven fields: m from 40 to 700, grids 17^3 to 65^3 (one anisotropic), a Matern model
    (FP64 leaf path), and one model listed twice with two isovalues."""
    ws = [
        workloads.small(21, 40, 17),
        workloads.small(22, 300, 33, ell=(0.15, 0.2, 0.25)),
        workloads.small(23, 700, 65, ell=(0.12, 0.12, 0.12)),
        workloads.small(24, 120, 40, kernel=workloads.MATERN52, ell=(0.2, 0.2, 0.2)),
        workloads.small(25, 200, 24, ell=(0.3, 0.25, 0.2)),
    ]
    items = [(0, None), (1, None), (2, None), (3, None), (4, None), (1, 25.0)]
    return ws, items


def _run_single(g, torch, w, th, opts):
    M = model_of(w)
    f = torch.zeros((w.n - 1) ** 3, dtype=torch.float32, device="cuda")
    s = g.gpr_lcp_adaptive(M, g.make_grid(w.n), th, w.max_depth, opts, f)
    g.gpr_sync()
    return f.cpu().numpy(), s


def _iso(w, q):
    return w.isovalues[0] if q is None else float(np.percentile(w.y, q))


def _run_batch(g, torch, ws, items, opts):
    models = [model_of(w) for w in ws]
    out = [torch.full(((ws[k].n - 1) ** 3,), -1.0, dtype=torch.float32, device="cuda") for k, _ in items]
    stats = g.gpr_lcp_adaptive_batched([models[k] for k, _ in items], [g.make_grid(ws[k].n) for k, _ in items],
                                       [_iso(ws[k], q) for k, q in items], [ws[k].max_depth for k, _ in items], opts, out)
    g.gpr_sync()
    return [o.cpu().numpy() for o in out], stats


@pytest.fixture(scope="module")
def singles(torch, g):
    ws, items = _fields()
    opts = g.lcp_options(prec=g.GPR_P_TF32X3)
    return ws, items, opts, [_run_single(g, torch, ws[k], _iso(ws[k], q), opts) for k, q in items]


@pytest.mark.parametrize("env", [{}, {"GPR_BATCH_WORKERS": "1"}, {"GPR_BATCH_WORKERS": "3", "GPR_BATCH_RECORD_CAP": "2000"}],
                         ids=["default", "one_worker", "record_overflow"])
def test_batched_equals_single(torch, g, singles, monkeypatch, env):
    ws, items, opts, ref = singles
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    got, stats = _run_batch(g, torch, ws, items, opts)
    assert sum((r[0] > 0).sum() for r in ref) > 500
    for i, ((f_ref, s_ref), f, s) in enumerate(zip(ref, got, stats)):
        assert np.array_equal(f_ref, f), (i, np.abs(f_ref - f).max())
        assert s["leaf_cells"] == s_ref["leaf_cells"], i
        assert s["nodes_per_level"] == s_ref["nodes_per_level"], i
        assert s["cells_estimated"] == s_ref["cells_estimated"], i


def test_batched_empty_and_errors(torch, g):
    opts = g.lcp_options()
    assert g.gpr_lcp_adaptive_batched([], [], [], [], opts, []) == []
    w = workloads.small(26, 30, 17)
    M = model_of(w)
    f = torch.zeros((w.n - 1) ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(g.GPRError) as e:  # 2^3 < 16 cells per axis
        g.gpr_lcp_adaptive_batched([M, M], [g.make_grid(w.n)] * 2, [0.1, 0.2], [w.max_depth, 3], opts, [f, f])
    assert e.value.status == g.GPR_ERR_ARG
    with pytest.raises(g.GPRError) as e:
        g.gpr_lcp_adaptive_batched([M], [g.make_grid(w.n)], [float("nan")], [w.max_depth], opts, [f])
    assert e.value.status == g.GPR_ERR_ARG


def test_batched_same_model_concurrent_fields(torch, g):
    """Four isovalue fields of one model on one grid run concurrently (one job each, shared grid
    cache filled idempotently); each equals its single-field call."""
    w = workloads.small(41, 300, 40, ell=(0.15, 0.2, 0.25))
    opts = g.lcp_options(prec=g.GPR_P_TF32X3)
    ths = [float(np.percentile(w.y, q)) for q in (20, 40, 60, 80)]
    ref = [_run_single(g, torch, w, th, opts) for th in ths]
    M = model_of(w)
    out = [torch.full(((w.n - 1) ** 3,), -1.0, dtype=torch.float32, device="cuda") for _ in ths]
    st = g.gpr_lcp_adaptive_batched([M] * 4, [g.make_grid(w.n)] * 4, ths, [w.max_depth] * 4, opts, out)
    g.gpr_sync()
    for (f_ref, s_ref), f, s in zip(ref, out, st):
        assert np.array_equal(f_ref, f.cpu().numpy())
        assert s["leaf_cells"] == s_ref["leaf_cells"]
