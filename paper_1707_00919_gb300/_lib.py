"""ctypes loader of libmuca.so, the C ABI declared in include/muca.h.

There is no fallback: if the CUDA library has not been built, importing the binding
raises ImportError.  Build it with `python -c "import __graft_entry__ as g; g.build()"`
(or `python paper_1707_00919_gb300/build.py`).
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmuca.so")

MUCA_OK = 0
MUCA_EINVAL = -1
MUCA_ENOMEM = -2
MUCA_ECUDA = -3
MUCA_ETIMEOUT = -4
MUCA_ENOTCONVERGED = -5
MUCA_EDEVICE = -6
MUCA_EIO = -7

MUCA_LAYOUT_INT8 = 0
MUCA_LAYOUT_PACKED = 1
MUCA_LAYOUT_AUTO = 2
MUCA_WPB_TUNE = -1
MUCA_WALKERS_OPTIMAL = -1
MUCA_ORDER_TYPEWRITER = 0
MUCA_ORDER_RANDOM = 1
MUCA_PROBE_XOR = 0
MUCA_PROBE_MAD = 1
MUCA_PROBE_MIXED = 2
MUCA_PROBE_PHILOX = 3
MUCA_PROBE_MIXED_ONE_WARP = 4

MUCA_STOP_MIN_MEAN = 0
MUCA_STOP_KL = 1
MUCA_STOP_CHEBYSHEV = 2

MUCA_SCHEDULE_SWEEPS = 0
MUCA_SCHEDULE_PAPER = 1


class muca_options(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("n_walkers", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("layout", ctypes.c_int32), ("walkers_per_block", ctypes.c_int32),
                ("first_walker", ctypes.c_int64)]


class muca_params(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("stop_rule", ctypes.c_int32),
                ("flat_threshold", ctypes.c_double), ("therm_sweeps", ctypes.c_uint64),
                ("sweeps_per_iter", ctypes.c_uint64), ("f_therm", ctypes.c_double),
                ("z", ctypes.c_double), ("factor", ctypes.c_double), ("growth", ctypes.c_double),
                ("max_iterations", ctypes.c_int32), ("deadline_s", ctypes.c_double), ("resume", ctypes.c_int32)]


class muca_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("last_metric", ctypes.c_double), ("attempts_per_walker", ctypes.c_uint64),
                ("seconds", ctypes.c_double)]


class muca_request(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("n_walkers", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("layout", ctypes.c_int32), ("walkers_per_block", ctypes.c_int32), ("params", muca_params)]


class muca_request_status(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("code", ctypes.c_int32), ("stats", muca_stats),
                ("seconds_queued", ctypes.c_double), ("seconds_total", ctypes.c_double)]


MUCA_REQ_QUEUED = 0
MUCA_REQ_ACTIVE = 1
MUCA_REQ_DONE = 2


class muca_raw_instance(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("layout", ctypes.c_int32), ("n_walkers", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("t0", ctypes.c_uint64), ("lattice", ctypes.c_void_p),
                ("energy", ctypes.c_void_p), ("table", ctypes.c_void_p), ("hist", ctypes.c_void_p),
                ("err", ctypes.c_void_p)]


MUCA_NOALLOC_MAX_INSTANCES = 64
MUCA_NOALLOC_SCRATCH_BYTES = 256

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

# name -> (restype, argtypes), the symbols of include/muca.h
_P = ctypes.POINTER
# muca_histogram_reducer: void (*)(uint64_t *H, size_t n_bins, void *ctx)
REDUCER = ctypes.CFUNCTYPE(None, ctypes.POINTER(ctypes.c_uint64), ctypes.c_size_t, ctypes.c_void_p)
# muca_iteration_observer: void (*)(int32_t, const uint64_t *, size_t, double, uint64_t, uint64_t, void *)
OBSERVER = ctypes.CFUNCTYPE(None, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64), ctypes.c_size_t, ctypes.c_double,
                            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p)
_H = ctypes.c_void_p
SIGNATURES = {
    "muca_default_params": (ctypes.c_int, [_P(muca_params)]),
    "muca_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, _P(_H)]),
    "muca_create_ex": (ctypes.c_int, [_P(muca_options), _P(_H)]),
    "muca_optimal_walkers": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_int64), _P(ctypes.c_int32)]),
    "muca_iterate_device": (ctypes.c_int, [_H, _P(muca_params), ctypes.c_int32, _P(muca_stats)]),
    "muca_set_site_order": (ctypes.c_int, [_H, ctypes.c_int32]),
    "muca_synchronize_timeout": (ctypes.c_int, [_H, ctypes.c_double]),
    "muca_set_iteration_observer": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p]),
    "muca_set_histogram_reducer": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "muca_measure_issue_rate": (ctypes.c_int, [ctypes.c_int32, _P(ctypes.c_double)]),
    "muca_set_lattice": (ctypes.c_int, [_H, _P(ctypes.c_int8), ctypes.c_size_t]),
    "muca_set_attempt_counter": (ctypes.c_int, [_H, ctypes.c_uint64]),
    "muca_save": (ctypes.c_int, [_H, ctypes.c_char_p]),
    "muca_load": (ctypes.c_int, [ctypes.c_char_p, _P(_H)]),
    "muca_get_site_order": (ctypes.c_int, [_H, _P(ctypes.c_int32)]),
    "muca_build_table": (ctypes.c_int, [ctypes.c_int32, _P(ctypes.c_double), ctypes.c_size_t, _P(ctypes.c_uint32)]),
    "muca_update_weights": (ctypes.c_int, [ctypes.c_int32, _P(ctypes.c_double), _P(ctypes.c_uint64), ctypes.c_size_t]),
    "muca_flatness": (ctypes.c_int, [ctypes.c_int32, _P(ctypes.c_uint64), ctypes.c_size_t, ctypes.c_int32,
                                     ctypes.c_int32, _P(ctypes.c_double), _P(ctypes.c_double), _P(ctypes.c_double),
                                     _P(ctypes.c_int32), _P(ctypes.c_int32)]),
    "muca_destroy": (ctypes.c_int, [_H]),
    "muca_set_stream": (ctypes.c_int, [_H, ctypes.c_void_p]),
    "muca_set_allocator": (ctypes.c_int, [ALLOC_FN, RELEASE_FN, ctypes.c_void_p]),
    "muca_set_weights": (ctypes.c_int, [_H, _P(ctypes.c_double), ctypes.c_size_t]),
    "muca_get_weights": (ctypes.c_int, [_H, _P(ctypes.c_double), ctypes.c_size_t]),
    "muca_get_table": (ctypes.c_int, [_H, _P(ctypes.c_uint32), ctypes.c_size_t]),
    "muca_sweep": (ctypes.c_int, [_H, ctypes.c_uint64, ctypes.c_int]),
    "muca_attempts": (ctypes.c_int, [_H, ctypes.c_uint64, ctypes.c_int]),
    "muca_thermalize_and_record": (ctypes.c_int, [_H, ctypes.c_uint64, ctypes.c_uint64]),
    "muca_get_histogram": (ctypes.c_int, [_H, _P(ctypes.c_uint64), ctypes.c_size_t]),
    "muca_reset_histogram": (ctypes.c_int, [_H]),
    "muca_iterate_until_flat": (ctypes.c_int, [_H, _P(muca_params), _P(muca_stats)]),
    "muca_production": (ctypes.c_int, [_H, ctypes.c_uint64, ctypes.c_uint64, _P(ctypes.c_uint64),
                                       _P(ctypes.c_double), ctypes.c_size_t]),
    "muca_production_jackknife": (ctypes.c_int, [_H, ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint64,
                                                 _P(ctypes.c_uint64), _P(ctypes.c_double), _P(ctypes.c_double),
                                                 ctypes.c_size_t]),
    "muca_reweight": (ctypes.c_int, [ctypes.c_int32, _P(ctypes.c_double), ctypes.c_size_t, _P(ctypes.c_double),
                                     ctypes.c_size_t, _P(ctypes.c_double), _P(ctypes.c_double)]),
    "muca_get_energies": (ctypes.c_int, [_H, _P(ctypes.c_int32), ctypes.c_size_t]),
    "muca_get_lattice": (ctypes.c_int, [_H, _P(ctypes.c_int8), ctypes.c_size_t]),
    "muca_get_info": (ctypes.c_int, [_H, _P(ctypes.c_int32), _P(ctypes.c_int64), _P(ctypes.c_uint64),
                                     _P(ctypes.c_int32), _P(ctypes.c_int32)]),
    "muca_synchronize": (ctypes.c_int, [_H]),
    "muca_philox": (ctypes.c_int, [_P(ctypes.c_uint32), _P(ctypes.c_uint32), ctypes.c_size_t,
                                   _P(ctypes.c_uint32)]),
    "muca_batch_create": (ctypes.c_int, [_P(_H), ctypes.c_int32, _P(_H)]),
    "muca_batch_destroy": (ctypes.c_int, [_H]),
    "muca_batch_sweep": (ctypes.c_int, [_H, ctypes.c_uint64, ctypes.c_int]),
    "muca_batch_iterate": (ctypes.c_int, [_H, _P(muca_params), _P(muca_stats)]),
    "muca_batch_info": (ctypes.c_int, [_H, _P(ctypes.c_int32), _P(ctypes.c_int32), _P(ctypes.c_size_t)]),
    "muca_server_create": (ctypes.c_int, [ctypes.c_size_t, _P(_H)]),
    "muca_server_destroy": (ctypes.c_int, [_H]),
    "muca_server_submit": (ctypes.c_int, [_H, _P(muca_request), _P(ctypes.c_int64)]),
    "muca_server_step": (ctypes.c_int, [_H, _P(ctypes.c_int32), _P(ctypes.c_int32)]),
    "muca_server_status": (ctypes.c_int, [_H, ctypes.c_int64, _P(muca_request_status)]),
    "muca_server_weights": (ctypes.c_int, [_H, ctypes.c_int64, _P(ctypes.c_double), ctypes.c_size_t]),
    "muca_server_totals": (ctypes.c_int, [_H, _P(ctypes.c_uint64), _P(ctypes.c_double), _P(ctypes.c_int32),
                                          _P(ctypes.c_size_t)]),
    "muca_batch_sweep_noalloc": (ctypes.c_int, [_P(muca_raw_instance), ctypes.c_int32, ctypes.c_uint64, ctypes.c_int,
                                                ctypes.c_void_p]),
    "muca_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load() -> ctypes.CDLL:
    """Loads libmuca.so and declares every exported symbol; raises ImportError if the
    library is missing (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built: run __graft_entry__.build() (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
