"""ctypes declarations of libdg's C ABI (``include/dg.h``).

Argument marshalling only: every step of the solver runs in libdg's CUDA
kernels.  Loading fails loudly when the library has not been built; there is
no fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdg.so")

c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_size_t = ctypes.c_size_t
c_void_p = ctypes.c_void_p
c_float = ctypes.c_float
c_double = ctypes.c_double

DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA, DG_EINFEASIBLE, DG_EFORCED, DG_ETIMEOUT, DG_ESTATE = range(8)
DG_SWEEP_ENERGY, DG_SWEEP_COSTS_OUT, DG_SWEEP_COSTS_IN = 1, 2, 4  # dg_sweep flags
STATUS_NAMES = {0: "DG_OK", 1: "DG_EINVAL", 2: "DG_ENOMEM", 3: "DG_ECUDA", 4: "DG_EINFEASIBLE",
                5: "DG_EFORCED", 6: "DG_ETIMEOUT", 7: "DG_ESTATE"}


class dg_rows(ctypes.Structure):
    _fields_ = [("num_inst", c_int32), ("inst_row_ptr", c_void_p), ("inst_var_ptr", c_void_p),
                ("n", c_int32), ("m", c_int64), ("row_ptr", c_void_p), ("col", c_void_p),
                ("coef", c_void_p), ("sense", c_void_p), ("rhs", c_void_p), ("c", c_void_p)]


class dg_options(ctypes.Structure):
    _fields_ = [("tile_nodes", c_int32), ("tile_slots", c_int32), ("block_threads", c_int32),
                ("renorm_every", c_int32), ("omega", c_float), ("num_threads", c_int32),
                ("host_mb_limit", c_int32), ("chunk_rows", c_int32), ("group_ratio_pct", c_int32),
                ("long_lanes", c_int32), ("reserved", c_int32 * 4)]


class dg_sizes(ctypes.Structure):
    _fields_ = [("arena_bytes", c_size_t), ("num_slots", c_int64), ("num_lambda", c_int64),
                ("num_nodes", c_int64), ("num_nodes_padded", c_int64), ("n", c_int32), ("m", c_int64),
                ("num_inst", c_int32), ("num_tiles", c_int32), ("max_hops", c_int32), ("max_width", c_int32),
                ("smem_bytes", c_size_t), ("num_launch_groups", c_int32), ("num_long_bdds", c_int64),
                ("num_long_nodes", c_int64)]


class dg_stats(ctypes.Structure):
    _fields_ = [("sizes", dg_sizes), ("num_arcs", c_int64), ("bytes_per_iter", c_double),
                ("actual_bytes_per_iter", c_double), ("hop_histogram", c_int64 * 64)]


P = c_void_p
PP = ctypes.POINTER(c_void_p)

# name -> (restype, argtypes); every function declared in include/dg.h
SIGNATURES = {
    "dg_last_error": (ctypes.c_char_p, []),
    "dg_plan": (c_int32, [ctypes.POINTER(dg_rows), ctypes.POINTER(dg_options), PP, ctypes.POINTER(dg_sizes)]),
    "dg_build": (c_int32, [ctypes.POINTER(dg_rows), ctypes.POINTER(dg_options), PP, ctypes.POINTER(dg_sizes)]),
    "dg_bind": (c_int32, [P, P, c_size_t, P, PP]),
    "dg_plan_free": (None, [P]),
    "dg_destroy": (None, [P]),
    "dg_get_sizes": (c_int32, [P, ctypes.POINTER(dg_sizes)]),
    "dg_get_stats": (c_int32, [P, ctypes.POINTER(dg_stats)]),
    "dg_slot_map": (c_int32, [P, P]),
    "dg_launch_group": (c_int32, [P, c_int32, P, P, P, P]),
    "dg_bdd_export": (c_int32, [P, c_int64, P, P, P, ctypes.POINTER(c_int32)]),
    "dg_init_lambda": (c_int32, [P, P, P, P]),
    "dg_iterate": (c_int32, [P, P, P, P, P, P, c_int32, c_int32, P, ctypes.POINTER(dg_options)]),
    "dg_sum_M": (c_int32, [P, P, P, P, P, c_int32, c_int32]),
    "dg_sweep": (c_int32, [P, P, P, P, P, P, c_int32, c_int32, c_int32, ctypes.POINTER(dg_options)]),
    "dg_bound_from_energies": (c_int32, [P, P, P]),
    "dg_min_marginals": (c_int32, [P, P, P, P, P]),
    "dg_lower_bound": (c_int32, [P, P, P, P, P, P]),
    "dg_lb_seed": (c_int32, [P, P, P, P, P, P]),
    "dg_lower_bound_noalloc": (c_int32, [P, P, P, P, P]),
    "dg_backward_workspace_bytes": (c_size_t, [P, c_int32, c_int32]),
    "dg_backward": (c_int32, [P, P, P, P, P, P, c_int32, c_int32, c_int32, P, P, P, P, P, P, P, c_size_t,
                              ctypes.POINTER(dg_options)]),
    "dg_iterate_checkpointed": (c_int32, [P, P, P, P, P, P, c_int32, c_int32, c_int32, P, c_size_t, P,
                                          ctypes.POINTER(dg_options)]),
    "dg_backward_checkpointed": (c_int32, [P, P, P, P, c_int32, c_int32, c_int32, P, P, P, P, P, P, P, c_size_t,
                                           ctypes.POINTER(dg_options)]),
    "dg_plan_validate": (c_int32, [P]),
    "dg_graph_create": (c_int32, [P, P, P, P, P, P, c_int32, c_int32, P, ctypes.POINTER(dg_options), PP]),
    "dg_graph_replay": (c_int32, [P, P]),
    "dg_graph_destroy": (None, [P]),
    "dg_iterate_launches": (c_int32, [P, c_int32, c_int32, ctypes.POINTER(dg_options)]),
    "dg_wait": (c_int32, [P, c_int32]),
    "dg_smoothed_dual": (c_int32, [P, P, P, c_float, P, P]),
    "dg_nonparam_update": (c_int32, [P, P, P, P]),
    "dg_nonparam_backward": (c_int32, [P, P, P, P]),
    "dg_param_transform": (c_int32, [P, P, P, P, P, P, P, P]),
    "dg_param_transform_backward": (c_int32, [P, P, P, P, P, P, P, P, P, P]),
    "dg_autotune": (c_int32, [P, P, P, P, c_int32, P]),
}

_lib = None


def load():
    """Loads libdg.so (built by ``paper_2205_11638_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libdg is not built ({LIB_PATH} missing); run paper_2205_11638_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class DgError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().dg_last_error()
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg.decode() if msg else ''}")
        self.status = status


def check(status: int, where: str):
    if status != DG_OK:
        raise DgError(status, where)
