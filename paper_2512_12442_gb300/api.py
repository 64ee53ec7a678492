"""Thin Python binding of the C ABI (include/gpr_lcp.h): same names, argument
marshalling only.  Device buffers are torch CUDA tensors (or raw integer device
pointers); every computation runs in libgprlcp.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._lib import AdaptiveStatsC, GridC, LcpOptionsC, load

GPR_K_SE, GPR_K_MATERN52 = 0, 1
GPR_P_FP64, GPR_P_FP32, GPR_P_TF32, GPR_P_TF32X3, GPR_P_BF16, GPR_P_BF16X3 = range(6)
GPR_EST_SOV_QMC, GPR_EST_MC, GPR_EST_INDEP, GPR_EST_EDGE_MAX, GPR_EST_SOV_ORDERED = 0, 1, 2, 3, 4
GPR_EXACT_AUTO, GPR_EXACT_FP64 = 0, 1
GPR_TREE_OCTREE, GPR_TREE_KD = 0, 1
GPR_OK, GPR_ERR_ARG, GPR_ERR_NOT_PD, GPR_ERR_CUDA, GPR_ERR_OOM, GPR_ERR_TIMEOUT, GPR_ERR_UNSUPPORTED = range(7)


class GPRError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        msg = load().gpr_status_string(int(status)).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def _check(rc: int, where: str):
    if rc != GPR_OK:
        raise GPRError(rc, where)


def _ptr(t, dtype=None, allow_none=False):
    """Device pointer of a torch CUDA tensor (contiguous) or an int pointer."""
    if t is None:
        if allow_none:
            return None
        raise ValueError("buffer required")
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_grid(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> GridC:
    if np.isscalar(n):
        n = (n, n, n)
    g = GridC()
    for d in range(3):
        g.lo[d], g.hi[d], g.n[d] = float(lo[d]), float(hi[d]), int(n[d])
    return g


def lcp_options(**kw) -> LcpOptionsC:
    o = LcpOptionsC()
    load().gpr_lcp_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Model:
    """Owns a gpr_model handle; destroyed with the object."""

    def __init__(self, handle: int):
        self.handle = handle

    @property
    def m(self) -> int:
        return int(load().gpr_model_m(self.handle))

    def close(self):
        if self.handle:
            load().gpr_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gpr_model_create(obs_xyz, y, kernel=GPR_K_SE, length_scales=(0.2, 0.2, 0.2), signal_var=1.0,
                     noise_var=1e-4, stream=None) -> Model:
    X = np.ascontiguousarray(obs_xyz, np.float64).reshape(-1, 3)
    yy = np.ascontiguousarray(y, np.float64).reshape(-1)
    ell = np.ascontiguousarray(length_scales, np.float64).reshape(3)
    h = C.c_void_p()
    rc = load().gpr_model_create(X.ctypes.data, yy.ctypes.data, yy.shape[0], int(kernel), ell.ctypes.data,
                                 float(signal_var), float(noise_var), _stream(stream), C.byref(h))
    _check(rc, "gpr_model_create")
    return Model(h.value)


def gpr_model_create_sgpr(inducing_xyz, mu_M, A_M, kernel=GPR_K_SE, length_scales=(0.2, 0.2, 0.2),
                          signal_var=1.0, kmm_jitter=0.0, stream=None) -> Model:
    """Sparse-GP model from m inducing sites and their stored distribution N(mu_M, A_M) (Eq. 1)."""
    X = np.ascontiguousarray(inducing_xyz, np.float64).reshape(-1, 3)
    mu = np.ascontiguousarray(mu_M, np.float64).reshape(-1)
    m = mu.shape[0]
    A = np.ascontiguousarray(A_M, np.float64).reshape(m, m)
    ell = np.ascontiguousarray(length_scales, np.float64).reshape(3)
    h = C.c_void_p()
    rc = load().gpr_model_create_sgpr(X.ctypes.data, mu.ctypes.data, A.ctypes.data, m, int(kernel), ell.ctypes.data,
                                      float(signal_var), float(kmm_jitter), _stream(stream), C.byref(h))
    _check(rc, "gpr_model_create_sgpr")
    return Model(h.value)


def gpr_reconstruct_dense(model: Model, grid: GridC, prec, mean, var, cov13=None, stream=None):
    rc = load().gpr_reconstruct_dense(model.handle, C.byref(grid), int(prec), _ptr(mean), _ptr(var),
                                      _ptr(cov13, allow_none=True), _stream(stream))
    _check(rc, "gpr_reconstruct_dense")


def gpr_stats_points(model: Model, grid: GridC, point_idx, stats, stream=None):
    n = 0 if point_idx is None else int(point_idx.numel())
    rc = load().gpr_stats_points(model.handle, C.byref(grid), _ptr(point_idx, allow_none=True), n,
                                 _ptr(stats, allow_none=True), _stream(stream))
    _check(rc, "gpr_stats_points")


def gpr_cell_lcp_from_stats(grid: GridC, stats15, isovalue, opts: LcpOptionsC, cell_idx, lcp, stream=None):
    n = 0 if cell_idx is None else int(cell_idx.numel())
    rc = load().gpr_cell_lcp_from_stats(C.byref(grid), _ptr(stats15), float(isovalue), C.byref(opts),
                                        _ptr(cell_idx, allow_none=True), n, _ptr(lcp), _stream(stream))
    _check(rc, "gpr_cell_lcp_from_stats")


GPR_NOALLOC_MAX_CELLS = 16384


def gpr_cell_lcp_from_stats_noalloc(grid: GridC, stats15, isovalue, opts: LcpOptionsC, cell_idx, lcp, stream=None):
    """As gpr_cell_lcp_from_stats, for callers that may not allocate device memory
    (the library's static scratch serves at most GPR_NOALLOC_MAX_CELLS cells per call)."""
    n = 0 if cell_idx is None else int(cell_idx.numel())
    rc = load().gpr_cell_lcp_from_stats_noalloc(C.byref(grid), _ptr(stats15), float(isovalue), C.byref(opts),
                                                _ptr(cell_idx, allow_none=True), n, _ptr(lcp), _stream(stream))
    _check(rc, "gpr_cell_lcp_from_stats_noalloc")


def _stats_dict(s: AdaptiveStatsC) -> dict:
    return {"nodes_per_level": list(s.nodes_per_level), "subdiv_per_level": list(s.subdiv_per_level),
            "leaf_cells": s.leaf_cells, "recon_points": s.recon_points, "cells_estimated": s.cells_estimated}


def gpr_lcp_dense(model: Model, grid: GridC, isovalue, opts: LcpOptionsC, lcp, stream=None) -> dict:
    s = AdaptiveStatsC()
    rc = load().gpr_lcp_dense(model.handle, C.byref(grid), float(isovalue), C.byref(opts), _ptr(lcp), C.byref(s),
                              _stream(stream))
    _check(rc, "gpr_lcp_dense")
    return _stats_dict(s)


def gpr_lcp_adaptive(model: Model, grid: GridC, isovalue, max_depth, opts: LcpOptionsC, lcp, stream=None) -> dict:
    s = AdaptiveStatsC()
    rc = load().gpr_lcp_adaptive(model.handle, C.byref(grid), float(isovalue), int(max_depth), C.byref(opts),
                                 _ptr(lcp), C.byref(s), _stream(stream))
    _check(rc, "gpr_lcp_adaptive")
    return _stats_dict(s)


def gpr_lcp_adaptive_batched(models, grids, isovalues, max_depths, opts: LcpOptionsC, lcps, stream=None) -> list:
    """Many adaptive fields in one call (field i as gpr_lcp_adaptive(models[i], grids[i], ...));
    returns the per-field statistics."""
    n = len(models)
    if not (len(grids) == len(isovalues) == len(max_depths) == len(lcps) == n):
        raise ValueError("gpr_lcp_adaptive_batched: per-field lists differ in length")
    hm = (C.c_void_p * n)(*[m.handle for m in models])
    hg = (GridC * n)(*grids)
    hi = (C.c_double * n)(*[float(v) for v in isovalues])
    hd = (C.c_int32 * n)(*[int(d) for d in max_depths])
    hl = (C.c_void_p * n)(*[_ptr(t) for t in lcps])
    st = (AdaptiveStatsC * n)()
    rc = load().gpr_lcp_adaptive_batched(hm, hg, hi, hd, n, C.byref(opts), hl, st, _stream(stream))
    _check(rc, "gpr_lcp_adaptive_batched")
    return [_stats_dict(st[i]) for i in range(n)]


def gpr_batch_release() -> None:
    _check(load().gpr_batch_release(), "gpr_batch_release")


def gpr_lcp_backward(model: Model, grid: GridC, isovalue, opts: LcpOptionsC, dL_dlcp, stream=None):
    """Adjoint of sum_c dL_dlcp[c] LCP_c: returns (dL/dy (m,), dL/dlog l (3,)) as numpy float64."""
    dy = np.zeros(model.m); dl = np.zeros(3)
    rc = load().gpr_lcp_backward(model.handle, C.byref(grid), float(isovalue), C.byref(opts), _ptr(dL_dlcp),
                                 dy.ctypes.data, dl.ctypes.data, _stream(stream))
    _check(rc, "gpr_lcp_backward")
    return dy, dl


def gpr_lcp_backward_adaptive(model: Model, grid: GridC, isovalue, max_depth, opts: LcpOptionsC, dL_dlcp,
                              stream=None):
    """Adjoint of sum_c dL_dlcp[c] LCP_c for the adaptive field: (dL/dy, dL/dlog l) as numpy float64."""
    dy = np.zeros(model.m); dl = np.zeros(3)
    rc = load().gpr_lcp_backward_adaptive(model.handle, C.byref(grid), float(isovalue), int(max_depth),
                                          C.byref(opts), _ptr(dL_dlcp), dy.ctypes.data, dl.ctypes.data,
                                          _stream(stream))
    _check(rc, "gpr_lcp_backward_adaptive")
    return dy, dl


def gpr_sync(stream=None):
    _check(load().gpr_sync(_stream(stream)), "gpr_sync")


def gpr_octree_trace(model: Model, grid: GridC, isovalue, max_depth, opts: LcpOptionsC, level, capacity=1 << 22,
                     stream=None):
    """Test hook: (node codes, decisions, bounds) of one level of the device octree."""
    nodes = np.zeros(capacity, np.int64); dec = np.zeros(capacity, np.int8); bnd = np.zeros(capacity)
    cnt = C.c_int64()
    _check(load().gpr_octree_trace(model.handle, C.byref(grid), float(isovalue), int(max_depth), C.byref(opts),
                                   int(level), nodes.ctypes.data, dec.ctypes.data, bnd.ctypes.data, capacity,
                                   C.byref(cnt), _stream(stream)), "gpr_octree_trace")
    c = min(cnt.value, capacity)
    return nodes[:c], dec[:c], bnd[:c]


def gpr_stats_points_split(model: Model, grid: GridC, point_idx, stats, stream=None):
    """Test hook: stats15 through the tensor-core digit-split path."""
    rc = load().gpr_stats_points_split(model.handle, C.byref(grid), _ptr(point_idx), int(point_idx.numel()),
                                       _ptr(stats), _stream(stream))
    _check(rc, "gpr_stats_points_split")


def gpr_oz_mul_tn_test(A, B, kchunk=0, nsplit=19, stream=None):
    """Test hook: C = A^T B (device FP64 K x nc tensors) by the tensor-core digit split."""
    K, nc = A.shape
    out = A.new_zeros((nc, nc))
    _check(load().gpr_oz_mul_tn_test(_ptr(A), _ptr(B), K, nc, int(kchunk), int(nsplit), _ptr(out), _stream(stream)),
           "gpr_oz_mul_tn_test")
    return out


def gpr_oz_mul_linv_test(model: Model, X, stream=None):
    """Test hook: X L^-1 (device FP64 rows x m) by the tensor-core digit split."""
    out = X.new_zeros(X.shape)
    _check(load().gpr_oz_mul_linv_test(model.handle, _ptr(X), int(X.shape[0]), _ptr(out), _stream(stream)),
           "gpr_oz_mul_linv_test")
    return out


def gpr_model_export(model: Model):
    """Test hook: FP64 factors of the device model as numpy arrays."""
    m = model.m
    L = np.zeros((m, m)); a = np.zeros(m); vy = np.zeros(m); mo = np.zeros(m); vo = np.zeros(m)
    _check(load().gpr_model_export(model.handle, L.ctypes.data, a.ctypes.data, vy.ctypes.data, mo.ctypes.data,
                                   vo.ctypes.data), "gpr_model_export")
    return {"L": L, "alpha": a, "vy": vy, "mu_obs": mo, "var_obs": vo}


def gpr_profile_enable(on: bool = True):
    load().gpr_profile_enable(1 if on else 0)


def gpr_profile_reset():
    load().gpr_profile_reset()


def gpr_profile_read(name: str):
    """(total milliseconds, launches) recorded for kernel group `name`."""
    t = C.c_double(); n = C.c_int64()
    load().gpr_profile_read(name.encode(), C.byref(t), C.byref(n))
    return t.value, n.value


def gpr_profile_units(name: str) -> float:
    """Work units (rows, points, estimator orthants) behind the recorded time of `name`."""
    u = C.c_double()
    load().gpr_profile_units(name.encode(), C.byref(u))
    return u.value


def gpr_autotune_table() -> dict:
    """The autotuner's choices: {(kernel, bucket): choice}."""
    lib = load()
    n = int(lib.gpr_autotune_table(None, 0))
    buf = C.create_string_buffer(n + 1)
    lib.gpr_autotune_table(buf, n + 1)
    out = {}
    for line in buf.value.decode().splitlines():
        k, b, c = line.split()
        out[(k, int(b))] = int(c)
    return out


def gpr_autotune_clear() -> None:
    load().gpr_autotune_clear()


def gpr_launch_count() -> int:
    return int(load().gpr_launch_count())
