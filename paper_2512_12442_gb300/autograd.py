"""torch.autograd.Function over the C ABI: the LCP field as a differentiable function of the
observation values y and the log length scales (forward: gpr_model_create + gpr_lcp_dense or
gpr_lcp_adaptive; backward: gpr_lcp_backward or gpr_lcp_backward_adaptive).  Marshalling only: both passes run in
libgprlcp.so."""
from __future__ import annotations

import numpy as np
import torch

from . import api


class LCPFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, log_len, X, n, isovalue, kernel=api.GPR_K_SE, signal_var=1.0, noise_var=1e-4,
                adaptive_depth=None, opts_kw=None):
        opts = api.lcp_options(**(opts_kw or {}))
        ell = np.exp(log_len.detach().cpu().double().numpy())
        model = api.gpr_model_create(np.asarray(X, np.float64), y.detach().cpu().double().numpy(), kernel, ell,
                                     signal_var, noise_var)
        grid = api.make_grid(n)
        nc = (n - 1) ** 3
        out = torch.zeros(nc, dtype=torch.float32, device="cuda")
        if adaptive_depth is None:
            api.gpr_lcp_dense(model, grid, isovalue, opts, out)
        else:
            api.gpr_lcp_adaptive(model, grid, isovalue, adaptive_depth, opts, out)
        ctx.model, ctx.grid, ctx.theta, ctx.opts = model, grid, float(isovalue), opts
        ctx.depth = adaptive_depth
        ctx.y_meta = (y.device, y.dtype)
        ctx.l_meta = (log_len.device, log_len.dtype)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.detach().to(device="cuda", dtype=torch.float32).contiguous()
        if ctx.depth is None:
            dy, dl = api.gpr_lcp_backward(ctx.model, ctx.grid, ctx.theta, ctx.opts, g)
        else:
            dy, dl = api.gpr_lcp_backward_adaptive(ctx.model, ctx.grid, ctx.theta, ctx.depth, ctx.opts, g)
        gy = torch.from_numpy(dy).to(device=ctx.y_meta[0], dtype=ctx.y_meta[1])
        gl = torch.from_numpy(dl).to(device=ctx.l_meta[0], dtype=ctx.l_meta[1])
        return gy, gl, None, None, None, None, None, None, None, None


def lcp_field(y, log_len, X, n, isovalue, **kw):
    """Differentiable LCP field (cells of an n^3 grid on [0,1]^3)."""
    return LCPFunction.apply(y, log_len, X, n, isovalue, kw.get("kernel", api.GPR_K_SE), kw.get("signal_var", 1.0),
                             kw.get("noise_var", 1e-4), kw.get("adaptive_depth"), kw.get("opts_kw"))
