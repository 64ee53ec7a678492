"""The allocation-free cell-LCP entry point, for callers that may not allocate
device memory when they call (a plug-in whose host application owns the device
memory pool; a latency-critical loop where cudaFree would synchronise the device).

It must give the same field as gpr_cell_lcp_from_stats on the same inputs, call
after call (its static scratch keeps the previous call's contents), and reject
requests larger than its fixed scratch.  Collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_two_calls_in_a_row():
    import torch
    import paper_2512_12442_gb300 as g
    assert torch.cuda.is_available()
    w = workloads.small(77, 60, 14)
    om = oracle.Model.from_workload(w)
    n = 14
    st = torch.tensor(om.stats15(n), device="cuda")
    grid = g.make_grid(n)
    th = float(np.median(w.y))
    rng = np.random.default_rng(8)
    for call, (est, k) in enumerate(((g.GPR_EST_SOV_QMC, 900), (g.GPR_EST_MC, 700))):
        cells = torch.tensor(np.sort(rng.choice((n - 1) ** 3, k, replace=False)), dtype=torch.int64, device="cuda")
        opts = g.lcp_options(est=est, seed=call + 3)
        ref = torch.full((k,), -1.0, dtype=torch.float32, device="cuda")
        out = torch.full((k,), -1.0, dtype=torch.float32, device="cuda")
        g.gpr_cell_lcp_from_stats(grid, st, th, opts, cells, ref)
        g.gpr_cell_lcp_from_stats_noalloc(grid, st, th, opts, cells, out)
        g.gpr_sync()
        a, b = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(b >= 0.0) and np.all(b <= 1.0)
        assert np.abs(a - b).max() <= 1e-4, (call, np.abs(a - b).max())


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    import paper_2512_12442_gb300 as g
    n = 32  # 29,791 cells > GPR_NOALLOC_MAX_CELLS
    st = torch.zeros(n ** 3, 15, dtype=torch.float64, device="cuda")
    out = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(g.GPRError) as e:
        g.gpr_cell_lcp_from_stats_noalloc(g.make_grid(n), st, 0.0, g.lcp_options(), None, out)
    assert e.value.status == g.GPR_ERR_ARG
    assert g.GPR_NOALLOC_MAX_CELLS == 16384


def test_noalloc_entry_captures_into_a_cuda_graph():
    """The allocation-free entry point queues work only (no allocation, no synchronisation, no
    timing), so it can be captured into a CUDA graph; replays recompute from the current contents
    of the statistics buffer."""
    import torch
    import paper_2512_12442_gb300 as g
    w = workloads.small(78, 60, 14)
    om = oracle.Model.from_workload(w)
    n = 14
    stats_a = torch.tensor(om.stats15(n), device="cuda")
    w2 = workloads.small(79, 60, 14)
    stats_b = torch.tensor(oracle.Model.from_workload(w2).stats15(n), device="cuda")
    grid = g.make_grid(n)
    th = float(np.median(w.y))
    cells = torch.tensor(np.arange(0, (n - 1) ** 3, 3), dtype=torch.int64, device="cuda")
    opts = g.lcp_options(seed=11)
    buf = stats_a.clone()
    direct_a = torch.zeros(len(cells), dtype=torch.float32, device="cuda")
    direct_b = torch.zeros_like(direct_a)
    g.gpr_cell_lcp_from_stats_noalloc(grid, stats_a, th, opts, cells, direct_a)
    g.gpr_cell_lcp_from_stats_noalloc(grid, stats_b, th, opts, cells, direct_b)
    g.gpr_sync()
    out = torch.full_like(direct_a, -1.0)
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        g.gpr_cell_lcp_from_stats_noalloc(grid, buf, th, opts, cells, out, stream=side)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, direct_a)
    buf.copy_(stats_b)
    out.fill_(-1.0)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, direct_b)
    assert (direct_a > 0).sum() > 20
