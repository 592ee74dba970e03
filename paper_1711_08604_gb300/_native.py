"""ctypes view of ``lib/libafd.so`` (the C ABI of ``include/afd.h``).

Only loading and signatures live here.  If the library has not been built
this raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libafd.so")

c_int, c_double, c_void_p, c_char_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_char_p
c_ll, c_size_t, c_u64 = ctypes.c_longlong, ctypes.c_size_t, ctypes.c_uint64
P = ctypes.POINTER


class PlanOpts(ctypes.Structure):
    _fields_ = [("precision", c_int), ("guard_tau", c_double), ("guard_cap", c_int),
                ("force_a1_zero", c_int), ("device", c_int), ("stream", c_void_p),
                ("use_graph", c_int), ("persistent", c_int), ("renormalise", c_int),
                ("autotune", c_int), ("grid_variant", c_int), ("offgrid_iters", c_int)]


class Result(ctypes.Structure):
    _fields_ = [("K_cap", c_int), ("a", c_void_p), ("coeff", c_void_p), ("delta", c_void_p),
                ("idx", c_void_p), ("steps", c_int), ("status", c_int), ("latency_ms", c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_ulonglong), ("completed", ctypes.c_ulonglong),
                ("failed", ctypes.c_ulonglong), ("ticks", ctypes.c_ulonglong),
                ("kernel_launches", c_ll), ("queued", c_int), ("active", c_int),
                ("bytes_reserved", c_size_t), ("bytes_in_use", c_size_t),
                ("suspended", ctypes.c_ulonglong)]


# name -> (restype, argtypes)
SIGNATURES = {
    "afd_plan_opts_default": (None, [P(PlanOpts)]),
    "afd_status_str": (c_char_p, [c_int]),
    "afd_last_error": (c_char_p, []),
    "afd_version": (c_char_p, []),
    "afd_plan_create": (c_int, [P(c_void_p), c_int, c_void_p, c_int, P(PlanOpts)]),
    "afd_plan_create_nonuniform": (c_int, [P(c_void_p), c_int, c_void_p, c_void_p, c_int, c_void_p, c_int,
                                           P(PlanOpts)]),
    "afd_plan_destroy": (c_int, [c_void_p]),
    "afd_decompose": (c_int, [c_void_p, c_void_p, c_int, c_double, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_void_p]),
    "afd_decompose_from": (c_int, [c_void_p, c_void_p, c_double, c_int, c_double, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "afd_plan_last_info": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "afd_plan_set_profiling": (c_int, [c_void_p, c_int]),
    "afd_plan_counters": (c_int, [c_void_p, P(c_ll), P(c_ll), P(c_double)]),
    "afd_plan_reset_counters": (c_int, [c_void_p]),
    "afd_plan_kernel_times": (c_int, [c_void_p, c_void_p, c_void_p]),
    "afd_plan_phase_cycles": (c_int, [c_void_p, c_void_p, P(c_ll)]),
    "afd_plan_get_stream": (c_int, [c_void_p, P(c_void_p)]),
    "afd_batch_create": (c_int, [P(c_void_p), c_int, c_void_p, c_void_p, c_int, c_int, P(PlanOpts)]),
    "afd_batch_run": (c_int, [c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p]),
    "afd_batch_tuning": (c_int, [c_void_p, c_int, P(c_int), c_void_p, c_void_p, c_void_p]),
    "afd_batch_counters": (c_int, [c_void_p, P(c_ll)]),
    "afd_batch_destroy": (c_int, [c_void_p]),
    "afd_decompose_batch": (c_int, [c_int, c_void_p, c_void_p, c_int, c_void_p, c_int, c_double,
                                    P(PlanOpts), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "afd_synthesize": (c_int, [c_int, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "afd_serve_create": (c_int, [P(c_void_p), c_size_t, P(PlanOpts)]),
    "afd_serve_submit": (c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p, c_int, c_double, P(c_u64)]),
    "afd_serve_poll": (c_int, [c_void_p, c_u64, P(Result)]),
    "afd_serve_wait": (c_int, [c_void_p, c_u64, c_double, P(Result)]),
    "afd_serve_suspend": (c_int, [c_void_p, ctypes.c_uint64, c_double]),
    "afd_serve_resume": (c_int, [c_void_p, ctypes.c_uint64]),
    "afd_serve_get_stats": (c_int, [c_void_p, P(ServeStats)]),
    "afd_serve_destroy": (c_int, [c_void_p]),
    "afd_inner_products_noalloc": (c_int, [c_void_p, c_int, c_void_p, c_int, c_void_p, c_void_p]),
    "afd_selftest_wait_timeout": (c_int, [c_int, c_int, P(c_int), P(c_double)]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load the library (once) and attach the signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(paper_1711_08604_gb300.build.build()); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
