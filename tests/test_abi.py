"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU and
exports every function declared in include/gpr_lcp.h; options defaults; no compute."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "gpr_lcp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(gpr_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_12442_gb300 import build
    build.build()
    from paper_2512_12442_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("gpr_model_create", "gpr_model_destroy", "gpr_reconstruct_dense", "gpr_lcp_dense",
                 "gpr_lcp_adaptive", "gpr_cell_lcp_from_stats", "gpr_stats_points", "gpr_sync"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
    from paper_2512_12442_gb300 import _lib
    assert set(_declared_functions()) <= set(_lib.SIGNATURES)


def test_option_defaults_and_status_strings(lib):
    import paper_2512_12442_gb300 as g
    o = g.lcp_options()
    assert (o.alpha, o.beta, o.n_samples, o.jitter, o.skip_eps, o.max_iters_min) == (1e-3, -1.0, 1600, 1e-10, 1e-9, 4)
    assert lib.gpr_status_string(2) == b"kernel matrix not positive definite"


def test_host_argument_checks_need_no_gpu(lib):
    """Invalid arguments are rejected on the host before any CUDA call."""
    import numpy as np
    import paper_2512_12442_gb300 as g
    h = ctypes.c_void_p()
    X = np.zeros((4, 3)); y = np.zeros(4); ell = np.array([0.1, -1.0, 0.1])
    rc = lib.gpr_model_create(X.ctypes.data, y.ctypes.data, 4, 0, ell.ctypes.data, 1.0, 1e-4, None, ctypes.byref(h))
    assert rc == g.GPR_ERR_ARG
    rc = lib.gpr_model_create(X.ctypes.data, y.ctypes.data, 0, 0, np.ones(3).ctypes.data, 1.0, 1e-4, None,
                              ctypes.byref(h))
    assert rc == g.GPR_ERR_ARG
    y[1] = float("nan")
    rc = lib.gpr_model_create(X.ctypes.data, y.ctypes.data, 4, 0, np.ones(3).ctypes.data, 1.0, 1e-4, None,
                              ctypes.byref(h))
    assert rc == g.GPR_ERR_ARG
    grid = g.make_grid(1)
    assert lib.gpr_cell_lcp_from_stats(ctypes.byref(grid), 1, 0.0, ctypes.byref(g.lcp_options()), None, 0, 1,
                                       None) == g.GPR_ERR_ARG


def test_noalloc_entry_checks_estimator_options_on_the_host(lib):
    """The allocation-free estimator entry rejects the option values the allocating entry rejects
    (non-finite jitter or skip threshold, bad sample counts) before any CUDA call."""
    import paper_2512_12442_gb300 as g
    grid = g.make_grid(9)
    for kw in ({"jitter": float("inf")}, {"skip_eps": float("inf")}, {"jitter": float("nan")},
               {"n_samples": 0}, {"est": 7}):
        o = g.lcp_options(**kw)
        assert lib.gpr_cell_lcp_from_stats_noalloc(ctypes.byref(grid), 1, 0.0, ctypes.byref(o), None, 0, 1,
                                                   None) == g.GPR_ERR_ARG, kw
        assert lib.gpr_cell_lcp_from_stats(ctypes.byref(grid), 1, 0.0, ctypes.byref(o), None, 0, 1,
                                           None) == g.GPR_ERR_ARG, kw


def test_fault_injection_alloc_reports_oom_without_a_gpu(lib, monkeypatch):
    """GPR_FAULT=alloc makes model creation fail as an allocation failure would (GPR_ERR_OOM),
    on the host, before any device work: the caller's error path can be exercised without a GPU."""
    import numpy as np
    import paper_2512_12442_gb300 as g
    X = np.random.default_rng(0).random((8, 3)); y = np.zeros(8)
    h = ctypes.c_void_p()
    monkeypatch.setenv("GPR_FAULT", "alloc")
    rc = lib.gpr_model_create(X.ctypes.data, y.ctypes.data, 8, 0, np.full(3, 0.2).ctypes.data, 1.0, 1e-4, None,
                              ctypes.byref(h))
    assert rc == g.GPR_ERR_OOM and not h.value
    assert lib.gpr_status_string(rc) == b"out of device memory"


def test_sgpr_model_arguments_checked_on_the_host(lib):
    """gpr_model_create_sgpr rejects bad inducing inputs before any CUDA call."""
    import numpy as np
    import paper_2512_12442_gb300 as g
    X = np.random.default_rng(0).random((6, 3)); mu = np.zeros(6); A = np.eye(6) * 1e-3
    ell = np.full(3, 0.2)
    h = ctypes.c_void_p()
    for (Xa, ma, Aa, jit) in ((X, mu, A, -1.0), (X, mu, A, float("nan")), (X, mu, np.full((6, 6), np.inf), 0.0)):
        rc = lib.gpr_model_create_sgpr(Xa.ctypes.data, ma.ctypes.data, Aa.ctypes.data, 6, 0, ell.ctypes.data, 1.0,
                                       jit, None, ctypes.byref(h))
        assert rc == g.GPR_ERR_ARG
    assert lib.gpr_model_create_sgpr(X.ctypes.data, mu.ctypes.data, None, 6, 0, ell.ctypes.data, 1.0, 0.0, None,
                                     ctypes.byref(h)) == g.GPR_ERR_ARG


def test_product_package_does_not_import_the_oracle():
    """The product path never routes through the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2512_12442_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "gpr_oracle" not in txt, f


def test_tune_file_is_read_without_a_gpu(tmp_path):
    """The autotuner's table file (GPR_TUNE_FILE, "kernel bucket choice" lines) is parsed on the
    host: a fresh process sees the entries through gpr_autotune_table, and gpr_autotune_clear
    empties the table (no GPU involved)."""
    import subprocess
    import sys
    path = tmp_path / "tune.txt"
    path.write_text("sov_shape 2097152 3\ntc_sumsq_tf32x3 32772 1\n")
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_2512_12442_gb300 as g\n"
            "t = g.gpr_autotune_table(); print(sorted(t.items()))\n"
            "g.gpr_autotune_clear(); print(len(g.gpr_autotune_table()))\n") % ROOT
    env = dict(os.environ, GPR_TUNE_FILE=str(path))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    out = r.stdout.strip().splitlines()
    assert out[-2] == "[(('sov_shape', 2097152), 3), (('tc_sumsq_tf32x3', 32772), 1)]"
    assert out[-1] == "0"


def test_batched_binding_checks_list_lengths(lib):
    """The batched call's per-field lists must have one entry per field (checked before any call)."""
    import paper_2512_12442_gb300 as g
    with pytest.raises(ValueError):
        g.gpr_lcp_adaptive_batched([], [g.make_grid(9)], [0.0], [3], g.lcp_options(), [])
