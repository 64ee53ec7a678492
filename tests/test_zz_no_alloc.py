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


def test_noalloc_reports_cells_off_the_grid_through_sync():
    """A listed cell index off the grid is skipped (its output is left as it was) and reported as
    GPR_ERR_ARG by the next gpr_sync, as the allocating entry point reports it; the other cells are
    estimated as usual."""
    import torch
    import paper_2512_12442_gb300 as g
    w = workloads.small(77, 60, 14)
    n = 14
    st = torch.tensor(oracle.Model.from_workload(w).stats15(n), device="cuda")
    grid = g.make_grid(n)
    th = float(np.median(w.y))
    idx = np.array([5, 100, (n - 1) ** 3 + 7, 900], np.int64)
    cells = torch.tensor(idx, device="cuda")
    g.gpr_sync()
    out = torch.full((4,), -1.0, dtype=torch.float32, device="cuda")
    g.gpr_cell_lcp_from_stats_noalloc(grid, st, th, g.lcp_options(), cells, out)
    with pytest.raises(g.GPRError) as e:
        g.gpr_sync()
    assert e.value.status == g.GPR_ERR_ARG
    g.gpr_sync()  # the status word was cleared by the read
    ok = torch.tensor(idx[[0, 1, 3]], device="cuda")
    ref = torch.full((3,), -1.0, dtype=torch.float32, device="cuda")
    g.gpr_cell_lcp_from_stats(grid, st, th, g.lcp_options(), ok, ref)
    g.gpr_sync()
    o = out.cpu().numpy()
    assert o[2] == -1.0
    assert np.abs(o[[0, 1, 3]] - ref.cpu().numpy()).max() <= 1e-4
