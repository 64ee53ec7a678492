"""The estimator's normal CDF / quantile coefficients (normal_approx.h) are exactly what the
committed fitting script produces (CPU; the GPU accuracy of the fits is tests/test_gpu_normal_approx.py)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_12442_gb300", "csrc")


def test_header_matches_fitting_script(tmp_path):
    pytest.importorskip("scipy")
    spec = importlib.util.spec_from_file_location("fit_normal", os.path.join(CSRC, "fit_normal.py"))
    fn = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(fn)
    out = tmp_path / "normal_approx.h"
    fn.main(str(out))
    with open(os.path.join(CSRC, "normal_approx.h")) as f:
        committed = f.read()
    assert out.read_text() == committed
