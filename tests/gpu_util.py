"""Shared helpers of the GPU parity tests."""
import numpy as np


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def model_of(w, stream=None):
    import paper_2512_12442_gb300 as g
    if "A_M" in w.extra:
        return g.gpr_model_create_sgpr(w.X, w.y, w.extra["A_M"], w.kernel, w.ell, w.sf2, w.extra["kmm_jitter"],
                                       stream=stream)
    return g.gpr_model_create(w.X, w.y, w.kernel, w.ell, w.sf2, w.sn2, stream=stream)


def cell_linear(i, j, k, n):
    return i + (n - 1) * (j + (n - 1) * k)
