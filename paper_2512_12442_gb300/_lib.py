"""ctypes loader and signatures of libgprlcp.so (the C ABI of include/gpr_lcp.h).

There is no fallback: if the CUDA library is missing, importing raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgprlcp.so")


class GridC(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("n", C.c_int32 * 3)]


class LcpOptionsC(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("est", C.c_int), ("n_samples", C.c_int32),
                ("seed", C.c_uint64), ("jitter", C.c_double), ("skip_eps", C.c_double), ("prec", C.c_int),
                ("max_iters_min", C.c_int32), ("exact", C.c_int), ("tree", C.c_int)]


class AdaptiveStatsC(C.Structure):
    _fields_ = [("nodes_per_level", C.c_int64 * 24), ("subdiv_per_level", C.c_int64 * 24),
                ("leaf_cells", C.c_int64), ("recon_points", C.c_int64), ("cells_estimated", C.c_int64)]


# name -> (restype, argtypes); every symbol declared in include/gpr_lcp.h
SIGNATURES = {
    "gpr_lcp_options_default": (None, [C.POINTER(LcpOptionsC)]),
    "gpr_status_string": (C.c_char_p, [C.c_int]),
    "gpr_model_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_double,
                                   C.c_double, C.c_void_p, C.POINTER(C.c_void_p)]),
    "gpr_model_create_sgpr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p,
                                        C.c_double, C.c_double, C.c_void_p, C.POINTER(C.c_void_p)]),
    "gpr_model_destroy": (C.c_int, [C.c_void_p]),
    "gpr_model_m": (C.c_int64, [C.c_void_p]),
    "gpr_reconstruct_dense": (C.c_int, [C.c_void_p, C.POINTER(GridC), C.c_int, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p]),
    "gpr_stats_points": (C.c_int, [C.c_void_p, C.POINTER(GridC), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "gpr_cell_lcp_from_stats": (C.c_int, [C.POINTER(GridC), C.c_void_p, C.c_double, C.POINTER(LcpOptionsC),
                                          C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "gpr_cell_lcp_from_stats_noalloc": (C.c_int, [C.POINTER(GridC), C.c_void_p, C.c_double,
                                                  C.POINTER(LcpOptionsC), C.c_void_p, C.c_int64, C.c_void_p,
                                                  C.c_void_p]),
    "gpr_lcp_dense": (C.c_int, [C.c_void_p, C.POINTER(GridC), C.c_double, C.POINTER(LcpOptionsC), C.c_void_p,
                                C.POINTER(AdaptiveStatsC), C.c_void_p]),
    "gpr_lcp_adaptive": (C.c_int, [C.c_void_p, C.POINTER(GridC), C.c_double, C.c_int32, C.POINTER(LcpOptionsC),
                                   C.c_void_p, C.POINTER(AdaptiveStatsC), C.c_void_p]),
    "gpr_lcp_adaptive_batched": (C.c_int, [C.c_void_p, C.POINTER(GridC), C.c_void_p, C.c_void_p, C.c_int32,
                                           C.POINTER(LcpOptionsC), C.c_void_p, C.POINTER(AdaptiveStatsC),
                                           C.c_void_p]),
    "gpr_batch_release": (C.c_int, []),
    "gpr_lcp_backward": (C.c_int, [C.c_void_p, C.POINTER(GridC), C.c_double, C.POINTER(LcpOptionsC), C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "gpr_lcp_backward_adaptive": (C.c_int, [C.c_void_p, C.POINTER(GridC), C.c_double, C.c_int32,
                                            C.POINTER(LcpOptionsC), C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p]),
    "gpr_sync": (C.c_int, [C.c_void_p]),
    "gpr_profile_enable": (None, [C.c_int]),
    "gpr_profile_reset": (None, []),
    "gpr_profile_read": (C.c_int, [C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "gpr_profile_units": (C.c_int, [C.c_char_p, C.POINTER(C.c_double)]),
    "gpr_launch_count": (C.c_int64, []),
    "gpr_autotune_table": (C.c_int64, [C.c_char_p, C.c_int64]),
    "gpr_autotune_clear": (None, []),
    # test hooks (not in the public header)
    "gpr_model_export": (C.c_int, [C.c_void_p] + [C.c_void_p] * 5),
    "gpr_stats_points_split": (C.c_int, [C.c_void_p, C.POINTER(GridC), C.c_void_p, C.c_int64, C.c_void_p,
                                         C.c_void_p]),
    "gpr_normal_approx_eval": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gpr_autotune_force": (None, [C.c_char_p, C.c_int]),
    "gpr_oz_mul_tn_test": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_void_p,
                                     C.c_void_p]),
    "gpr_oz_mul_linv_test": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "gpr_eval_points": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]),
    "gpr_octree_trace": (C.c_int, [C.c_void_p, C.POINTER(GridC), C.c_double, C.c_int32, C.POINTER(LcpOptionsC),
                                   C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                   C.POINTER(C.c_int64), C.c_void_p]),
}

_lib = None


def load() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
