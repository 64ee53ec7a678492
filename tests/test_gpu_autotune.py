"""Autotuner: every alternative of a tuned launch gives the same bits; a tuned call records its
choice per (kernel, size bucket); GPR_TUNE_FILE persists the table across processes."""
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads
from gpu_util import model_of, torch_cuda

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def g():
    import paper_2512_12442_gb300 as g
    return g


def _force(g, name, choice):
    from paper_2512_12442_gb300._lib import load
    load().gpr_autotune_force(name.encode(), int(choice))


@pytest.mark.parametrize("prec,name", [("TF32", "tc_sumsq_tf32"), ("TF32X3", "tc_sumsq_tf32x3"),
                                       ("BF16", "tc_sumsq_bf16"), ("BF16X3", "tc_sumsq_bf16x3")])
def test_tile_widths_give_same_bits(torch, g, prec, name):
    w = workloads.small(31, 300, 21, ell=(0.15, 0.2, 0.25))  # mp = 320: several tiles of every width
    M = model_of(w)
    grid = g.make_grid(w.n)
    out = []
    # tile widths x (plain, warp-specialised), and for TF32 operands the two-CTAs-per-SM variant
    for c in ((0, 1, 2, 3, 4) if prec.startswith("TF32") else (0, 1, 2, 3)):
        _force(g, name, c)
        mean = torch.zeros(w.n ** 3, dtype=torch.float32, device="cuda")
        var = torch.zeros_like(mean)
        g.gpr_reconstruct_dense(M, grid, getattr(g, "GPR_P_" + prec), mean, var, None)
        g.gpr_sync()
        out.append(var.cpu().numpy())
    _force(g, name, -1)
    assert all(np.array_equal(out[0], o) for o in out[1:])


@pytest.mark.parametrize("case", ["ragged", "paper"])
def test_digit_generation_in_the_gemm_gives_same_bits(torch, g, case):
    """The FP64-class rows with the kernel-row digits generated inside the GEMM (choice 0) and staged in
    HBM first (choice 1) are the same bits (same digits, same MMA order): the statistics of a point list
    with rows beyond a 128-row tile and out-of-list neighbours, and of the paper-scale field's points."""
    if case == "ragged":
        w = workloads.small(33, 300, 19, ell=(0.15, 0.2, 0.25)); n = 19
    else:
        w = workloads.config2(); n = 64
    M = model_of(w)
    grid = g.make_grid(n)
    rng = np.random.default_rng(7)
    pts = np.unique(rng.integers(0, n ** 3, 3000 if case == "paper" else 777))
    t_pts = torch.tensor(pts, dtype=torch.int64, device="cuda")
    out = []
    for c in (0, 1):
        _force(g, "oz_w_kernel", c)
        st = torch.zeros(len(pts), 15, dtype=torch.float64, device="cuda")
        g.gpr_stats_points_split(M, grid, t_pts, st)
        g.gpr_sync()
        out.append(st.cpu().numpy())
    _force(g, "oz_w_kernel", -1)
    assert np.array_equal(out[0], out[1], equal_nan=True)
    assert np.isfinite(out[0][:, :2]).all()


def test_estimator_shapes_give_same_bits_and_table(torch, g):
    w = workloads.small(32, 120, 25)
    M = model_of(w)
    grid = g.make_grid(w.n)
    fields = []
    for c in (0, 1, 2, 3):
        _force(g, "sov_shape", c)
        f = torch.zeros((w.n - 1) ** 3, dtype=torch.float32, device="cuda")
        g.gpr_lcp_dense(M, grid, w.isovalues[0], g.lcp_options(prec=g.GPR_P_TF32X3), f)
        g.gpr_sync()
        fields.append(f.cpu().numpy())
    _force(g, "sov_shape", -1)
    assert (fields[0] > 0).sum() > 100
    assert all(np.array_equal(fields[0], f) for f in fields[1:])
    g.gpr_autotune_clear()
    M = model_of(w)  # a fresh model: no cached pre-pass table, so the tensor-core pass runs
    f = torch.zeros((w.n - 1) ** 3, dtype=torch.float32, device="cuda")
    g.gpr_lcp_dense(M, grid, w.isovalues[0], g.lcp_options(prec=g.GPR_P_TF32X3), f)
    g.gpr_sync()
    assert np.array_equal(f.cpu().numpy(), fields[0])
    tab = g.gpr_autotune_table()
    keys = [k for k in tab if k[0] == "tc_sumsq_tf32x3"]
    # TF32x3 pre-pass: two tile widths x (plain, warp-specialised), and two CTAs per SM
    assert keys and all(tab[k] in (0, 1, 2, 3, 4) and k[1] >> 6 == 128 for k in keys)
    assert any(k[0] == "sov_shape" for k in tab)


def test_tune_file_persists(tmp_path):
    path = tmp_path / "tune.txt"
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
            "import numpy as np, torch, workloads, paper_2512_12442_gb300 as g\n"
            "from gpu_util import model_of\n"
            "w = workloads.small(33, 90, 17); M = model_of(w)\n"
            "mean = torch.zeros(w.n ** 3, device='cuda'); var = torch.zeros_like(mean)\n"
            "g.gpr_reconstruct_dense(M, g.make_grid(w.n), g.GPR_P_BF16X3, mean, var, None); g.gpr_sync()\n"
            "print(sorted(g.gpr_autotune_table().items()))\n") % (ROOT, os.path.join(ROOT, "tests"))
    env = dict(os.environ, GPR_TUNE_FILE=str(path))
    r1 = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r1.returncode == 0, r1.stderr[-2000:]
    lines = path.read_text().split()
    assert lines[0] == "tc_sumsq_bf16x3" and int(lines[1]) >> 6 == 128 and lines[2] in ("0", "1", "2", "3")
    r2 = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r2.returncode == 0, r2.stderr[-2000:]
    assert r1.stdout.strip().splitlines()[-1] == r2.stdout.strip().splitlines()[-1]
