"""Python binding of the C ABI in include/muca.h.

Argument marshalling only: every step of the simulation runs in libmuca.so's CUDA
kernels and host library.  The module-level functions carry the C names; `Muca` wraps
one instance.  PyTorch, when importable, supplies device memory (its caching allocator)
and, optionally, the CUDA stream the instance runs on.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _lib as C
from ._lib import (MUCA_LAYOUT_AUTO, MUCA_LAYOUT_INT8, MUCA_LAYOUT_PACKED, MUCA_OK,  # noqa: F401
                   MUCA_ORDER_RANDOM, MUCA_ORDER_TYPEWRITER, MUCA_PROBE_MAD, MUCA_PROBE_MIXED,
                   MUCA_PROBE_MIXED_ONE_WARP, MUCA_PROBE_PHILOX, MUCA_PROBE_XOR, MUCA_SCHEDULE_PAPER,
                   MUCA_WALKERS_OPTIMAL,
                   MUCA_WPB_TUNE,
                   MUCA_SCHEDULE_SWEEPS, MUCA_STOP_CHEBYSHEV, MUCA_STOP_KL, MUCA_STOP_MIN_MEAN,
                   muca_options, muca_params, muca_stats)


class MucaError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"muca error {code}: {message}")
        self.code = code


def _check(rc: int) -> int:
    if rc != MUCA_OK:
        raise MucaError(rc, C.load().muca_last_error().decode(errors="replace"))
    return rc


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


# ---------------------------------------------------------------------------------
# PyTorch as the device allocator
# ---------------------------------------------------------------------------------
_torch_cb = None


def use_torch_allocator() -> bool:
    """Routes libmuca's device allocations through torch's caching allocator."""
    global _torch_cb
    if _torch_cb is not None:
        return True
    try:
        import torch
    except ImportError:
        return False
    if not torch.cuda.is_available():
        return False

    def _alloc(size, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(size))
        except Exception:
            return None

    def _release(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    cb = (C.ALLOC_FN(_alloc), C.RELEASE_FN(_release))
    _check(C.load().muca_set_allocator(cb[0], cb[1], None))
    _torch_cb = cb
    return True


# ---------------------------------------------------------------------------------
# C names
# ---------------------------------------------------------------------------------
def muca_default_params() -> muca_params:
    p = muca_params()
    _check(C.load().muca_default_params(ctypes.byref(p)))
    return p


def muca_create(L: int, n_walkers: int, seed: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(C.load().muca_create(L, n_walkers, seed, ctypes.byref(h)))
    return h


def muca_create_ex(L: int, n_walkers: int, seed: int, layout: int = MUCA_LAYOUT_INT8,
                   walkers_per_block: int = 0, first_walker: int = 0) -> ctypes.c_void_p:
    o = muca_options(L, n_walkers, seed, layout, walkers_per_block, first_walker)
    h = ctypes.c_void_p()
    _check(C.load().muca_create_ex(ctypes.byref(o), ctypes.byref(h)))
    return h


def muca_set_lattice(h, spins) -> None:
    a = np.ascontiguousarray(spins, dtype=np.int8)
    _check(C.load().muca_set_lattice(h, _p(a, ctypes.c_int8), a.size))


def muca_set_attempt_counter(h, t: int) -> None:
    _check(C.load().muca_set_attempt_counter(h, t))


def muca_save(h, path: str) -> None:
    _check(C.load().muca_save(h, os.fsencode(path)))


def muca_load(path: str) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(C.load().muca_load(os.fsencode(path), ctypes.byref(h)))
    return h


def muca_measure_issue_rate(kind: int) -> float:
    v = ctypes.c_double()
    _check(C.load().muca_measure_issue_rate(kind, ctypes.byref(v)))
    return v.value


def muca_set_histogram_reducer(h, fn, total_walkers: int = 0):
    """fn(H) -> None receives the instance's histogram (a uint64 numpy view) and must
    replace it in place by the sum over the simulation's instances; None removes it.
    Returns the C callback object, which must stay alive while it is set."""
    if fn is None:
        _check(C.load().muca_set_histogram_reducer(h, None, None, 0))
        return None

    def tramp(ptr, n, ctx):
        fn(np.ctypeslib.as_array(ptr, shape=(n,)))

    cb = C.REDUCER(tramp)
    _check(C.load().muca_set_histogram_reducer(h, ctypes.cast(cb, ctypes.c_void_p), None, total_walkers))
    return cb


def muca_set_iteration_observer(h, fn):
    """fn(iteration, H, metric, n_therm, n_updates) is called after every iteration of
    muca_iterate_until_flat (H: a uint64 copy); None removes it.  Returns the C callback
    object, which must stay alive while it is set."""
    if fn is None:
        _check(C.load().muca_set_iteration_observer(h, None, None))
        return None

    def tramp(it, ptr, n, metric, n_therm, n_upd, ctx):
        fn(it, np.ctypeslib.as_array(ptr, shape=(n,)).copy(), metric, n_therm, n_upd)

    cb = C.OBSERVER(tramp)
    _check(C.load().muca_set_iteration_observer(h, ctypes.cast(cb, ctypes.c_void_p), None))
    return cb


def muca_synchronize_timeout(h, seconds: float) -> bool:
    """True when the queued work finished within the limit, False on MUCA_ETIMEOUT."""
    rc = C.load().muca_synchronize_timeout(h, seconds)
    if rc == C.MUCA_ETIMEOUT:
        return False
    _check(rc)
    return True


def muca_set_site_order(h, order: int) -> None:
    _check(C.load().muca_set_site_order(h, order))


def muca_get_site_order(h) -> int:
    o = ctypes.c_int32()
    _check(C.load().muca_get_site_order(h, ctypes.byref(o)))
    return o.value


def muca_optimal_walkers(L: int, layout: int = MUCA_LAYOUT_INT8) -> tuple[int, int]:
    """(walker count of full occupancy, its walkers per block) on the current device."""
    n = ctypes.c_int64()
    wpb = ctypes.c_int32()
    _check(C.load().muca_optimal_walkers(L, layout, ctypes.byref(n), ctypes.byref(wpb)))
    return n.value, wpb.value


def muca_destroy(h) -> None:
    _check(C.load().muca_destroy(h))


def muca_set_stream(h, stream_handle: int | None) -> None:
    _check(C.load().muca_set_stream(h, ctypes.c_void_p(stream_handle or 0)))


def muca_set_weights(h, lnW) -> None:
    a = np.ascontiguousarray(lnW, dtype=np.float64)
    _check(C.load().muca_set_weights(h, _p(a, ctypes.c_double), a.size))


def muca_get_weights(h, n_bins: int) -> np.ndarray:
    a = np.zeros(n_bins, dtype=np.float64)
    _check(C.load().muca_get_weights(h, _p(a, ctypes.c_double), n_bins))
    return a


def muca_get_table(h, n_bins: int) -> np.ndarray:
    a = np.zeros(n_bins * 5, dtype=np.uint32)
    _check(C.load().muca_get_table(h, _p(a, ctypes.c_uint32), a.size))
    return a


def muca_sweep(h, n_sweeps: int, record: bool) -> None:
    _check(C.load().muca_sweep(h, n_sweeps, 1 if record else 0))


def muca_attempts(h, n_attempts: int, record: bool) -> None:
    _check(C.load().muca_attempts(h, n_attempts, 1 if record else 0))


def muca_thermalize_and_record(h, n_therm: int, n_record: int) -> None:
    _check(C.load().muca_thermalize_and_record(h, n_therm, n_record))


def muca_get_histogram(h, n_bins: int) -> np.ndarray:
    a = np.zeros(n_bins, dtype=np.uint64)
    _check(C.load().muca_get_histogram(h, _p(a, ctypes.c_uint64), n_bins))
    return a


def muca_reset_histogram(h) -> None:
    _check(C.load().muca_reset_histogram(h))


def muca_iterate_until_flat(h, params: muca_params | None = None, raise_on_fail: bool = True):
    st = muca_stats()
    rc = C.load().muca_iterate_until_flat(h, ctypes.byref(params) if params is not None else None,
                                           ctypes.byref(st))
    if raise_on_fail:
        _check(rc)
    return rc, st


def muca_iterate_device(h, params: muca_params | None = None, iterations_per_sync: int = 8,
                        raise_on_fail: bool = True):
    st = muca_stats()
    rc = C.load().muca_iterate_device(h, ctypes.byref(params) if params is not None else None,
                                       iterations_per_sync, ctypes.byref(st))
    if raise_on_fail:
        _check(rc)
    return rc, st


def muca_build_table(L: int, lnW) -> np.ndarray:
    w = np.ascontiguousarray(lnW, dtype=np.float64)
    T = np.zeros(5 * w.size, dtype=np.uint32)
    _check(C.load().muca_build_table(L, _p(w, ctypes.c_double), w.size, _p(T, ctypes.c_uint32)))
    return T


def muca_update_weights(L: int, lnW: np.ndarray, H) -> None:
    """Eq. (4) in place on a float64 array."""
    assert lnW.dtype == np.float64 and lnW.flags["C_CONTIGUOUS"]
    h = np.ascontiguousarray(H, dtype=np.uint64)
    _check(C.load().muca_update_weights(L, _p(lnW, ctypes.c_double), _p(h, ctypes.c_uint64), lnW.size))


def muca_flatness(L: int, H, prev_range: tuple[int, int] = (-1, -1),
                  measures: tuple[str, ...] = ("min_over_mean", "kl", "chebyshev")) -> dict:
    """min/mean, d_k (Eq. 6, reference width from prev_range and H's range) and d_c
    (Eq. A.1) of a histogram, and its visited range; only the named measures are
    computed (the others are passed as NULL)."""
    h = np.ascontiguousarray(H, dtype=np.uint64)
    out = {name: ctypes.c_double() for name in ("min_over_mean", "kl", "chebyshev") if name in measures}
    ref = {name: ctypes.byref(v) for name, v in out.items()}
    lo, hi = ctypes.c_int32(), ctypes.c_int32()
    _check(C.load().muca_flatness(L, _p(h, ctypes.c_uint64), h.size, prev_range[0], prev_range[1],
                                  ref.get("min_over_mean"), ref.get("kl"), ref.get("chebyshev"), ctypes.byref(lo),
                                  ctypes.byref(hi)))
    res = {name: v.value for name, v in out.items()}
    res["range"] = (lo.value, hi.value)
    return res


class IterationLog:
    """Per-iteration JSON lines for Muca.set_iteration_observer: iteration, visited
    width w, N_therm and N_updates (attempts per walker), the three flatness measures,
    the stop metric, wall time and attempts per second since the previous line."""

    def __init__(self, path: str, L: int, n_walkers: int):
        import time
        self._time = time.perf_counter
        self.L, self.W = L, n_walkers
        self.f = open(path, "w")
        self.prev = (-1, -1)
        self.t0 = self.t_last = self._time()

    def __call__(self, iteration, H, metric, n_therm, n_updates):
        import json
        now = self._time()
        fl = muca_flatness(self.L, H, self.prev)
        lo, hi = fl["range"]
        rec = {"iteration": int(iteration), "w": hi - lo + 1 if lo >= 0 else 0, "n_therm": int(n_therm),
               "n_updates": int(n_updates), "min_over_mean": fl["min_over_mean"], "d_k": fl["kl"],
               "d_c": fl["chebyshev"], "stop_metric": float(metric), "seconds": now - self.t0,
               "attempts_per_s": self.W * (n_therm + n_updates) / max(now - self.t_last, 1e-12)}
        self.f.write(json.dumps(rec) + "\n")
        self.f.flush()
        self.prev = (lo, hi) if lo >= 0 else (-1, -1)
        self.t_last = now

    def close(self) -> None:
        self.f.close()


def muca_production(h, therm_sweeps: int, n_sweeps: int, n_bins: int):
    H = np.zeros(n_bins, dtype=np.uint64)
    g = np.zeros(n_bins, dtype=np.float64)
    _check(C.load().muca_production(h, therm_sweeps, n_sweeps, _p(H, ctypes.c_uint64),
                                    _p(g, ctypes.c_double), n_bins))
    return H, g


def muca_production_jackknife(h, therm_sweeps: int, n_chunks: int, sweeps_per_chunk: int, n_bins: int):
    Hc = np.zeros((n_chunks, n_bins), dtype=np.uint64)
    g = np.zeros(n_bins)
    err = np.zeros(n_bins)
    _check(C.load().muca_production_jackknife(h, therm_sweeps, n_chunks, sweeps_per_chunk, _p(Hc, ctypes.c_uint64),
                                              _p(g, ctypes.c_double), _p(err, ctypes.c_double), n_bins))
    return Hc, g, err


def muca_reweight(L: int, ln_g, betas):
    g = np.ascontiguousarray(ln_g, dtype=np.float64)
    b = np.ascontiguousarray(np.atleast_1d(betas), dtype=np.float64)
    e = np.zeros(b.size)
    c = np.zeros(b.size)
    _check(C.load().muca_reweight(L, _p(g, ctypes.c_double), g.size, _p(b, ctypes.c_double), b.size,
                                  _p(e, ctypes.c_double), _p(c, ctypes.c_double)))
    return e, c


def muca_get_energies(h, n_walkers: int) -> np.ndarray:
    a = np.zeros(n_walkers, dtype=np.int32)
    _check(C.load().muca_get_energies(h, _p(a, ctypes.c_int32), n_walkers))
    return a


def muca_get_lattice(h, n_walkers: int, N: int) -> np.ndarray:
    a = np.zeros((n_walkers, N), dtype=np.int8)
    _check(C.load().muca_get_lattice(h, _p(a, ctypes.c_int8), a.size))
    return a


def muca_get_info(h):
    L, W, t, lay, wpb = (ctypes.c_int32(), ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_int32(),
                         ctypes.c_int32())
    _check(C.load().muca_get_info(h, ctypes.byref(L), ctypes.byref(W), ctypes.byref(t), ctypes.byref(lay),
                                  ctypes.byref(wpb)))
    return L.value, W.value, t.value, lay.value, wpb.value


def muca_synchronize(h) -> None:
    _check(C.load().muca_synchronize(h))


def muca_philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    n = c.size // 4
    out = np.zeros(4 * n, dtype=np.uint32)
    _check(C.load().muca_philox(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), n, _p(out, ctypes.c_uint32)))
    return out.reshape(n, 4)


def muca_last_error() -> str:
    return C.load().muca_last_error().decode(errors="replace")


# ---------------------------------------------------------------------------------
# object wrapper
# ---------------------------------------------------------------------------------
@dataclass
class IterationStats:
    code: int
    iterations: int
    converged: bool
    last_metric: float
    attempts_per_walker: int
    seconds: float


def make_params(schedule: int = MUCA_SCHEDULE_SWEEPS, stop_rule: int = MUCA_STOP_MIN_MEAN,
                flat_threshold: float = 0.8, therm_sweeps: int = 31, sweeps_per_iter: int = 100,
                f_therm: float = 30.0, z: float = 2.25, factor: float = 6.0, growth: float = 1.1,
                max_iterations: int = 1000, deadline_s: float = 0.0, resume: bool = False) -> muca_params:
    return muca_params(schedule, stop_rule, flat_threshold, therm_sweeps, sweeps_per_iter, f_therm, z,
                       factor, growth, max_iterations, deadline_s, 1 if resume else 0)


class Muca:
    """One multicanonical instance: n_walkers periodic L x L Ising lattices on the GPU."""

    def __init__(self, L: int, n_walkers: int, seed: int, layout: int = MUCA_LAYOUT_INT8,
                 walkers_per_block: int = 0, stream=None, torch_allocator: bool = True, first_walker: int = 0):
        if torch_allocator:
            use_torch_allocator()
        self.L, self.N, self.W = L, L * L, n_walkers
        self.n_bins = self.N + 1
        self._reducer = None
        self._h = muca_create_ex(L, n_walkers, seed, layout, walkers_per_block, first_walker)
        if n_walkers == MUCA_WALKERS_OPTIMAL:
            self.W = muca_get_info(self._h)[1]
        if stream is not None:
            handle = getattr(stream, "cuda_stream", stream)
            muca_set_stream(self._h, int(handle))

    @classmethod
    def load(cls, path: str, stream=None, torch_allocator: bool = True) -> "Muca":
        """An instance restored from a checkpoint written by save()."""
        if torch_allocator:
            use_torch_allocator()
        self = cls.__new__(cls)
        self._reducer = None
        self._h = muca_load(path)
        L, W, _, _, _ = muca_get_info(self._h)
        self.L, self.N, self.W = L, L * L, W
        self.n_bins = self.N + 1
        if stream is not None:
            muca_set_stream(self._h, int(getattr(stream, "cuda_stream", stream)))
        return self

    def synchronize(self, timeout: float | None = None) -> bool:
        """Waits for the queued work (at most `timeout` seconds); False if it is still running."""
        if timeout is None:
            muca_synchronize(self._h)
            return True
        return muca_synchronize_timeout(self._h, timeout)

    def set_iteration_observer(self, fn) -> None:
        """fn(iteration, H, metric, n_therm, n_updates) after every iteration."""
        self._observer = muca_set_iteration_observer(self._h, fn)

    def set_histogram_reducer(self, fn, total_walkers: int = 0) -> None:
        """Sum histograms over the instances of one simulation (see muca.h)."""
        self._reducer = muca_set_histogram_reducer(self._h, fn, total_walkers)

    def save(self, path: str) -> None:
        muca_save(self._h, path)

    def set_lattice(self, spins) -> None:
        """spins[walker][site], +1 / -1; energies are recomputed."""
        muca_set_lattice(self._h, spins)

    def set_attempt_counter(self, t: int) -> None:
        muca_set_attempt_counter(self._h, t)

    # lifetime
    def close(self) -> None:
        if self._h:
            muca_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # calls
    def set_weights(self, lnW) -> None:
        muca_set_weights(self._h, lnW)

    def get_weights(self) -> np.ndarray:
        return muca_get_weights(self._h, self.n_bins)

    def get_table(self) -> np.ndarray:
        return muca_get_table(self._h, self.n_bins)

    def sweep(self, n_sweeps: int, record: bool = True) -> None:
        muca_sweep(self._h, n_sweeps, record)

    def attempts(self, n_attempts: int, record: bool = True) -> None:
        muca_attempts(self._h, n_attempts, record)

    def thermalize_and_record(self, n_therm: int, n_record: int) -> None:
        """Zeroed H, n_therm attempts per walker unrecorded, then n_record recorded."""
        muca_thermalize_and_record(self._h, n_therm, n_record)

    def get_histogram(self) -> np.ndarray:
        return muca_get_histogram(self._h, self.n_bins)

    def reset_histogram(self) -> None:
        muca_reset_histogram(self._h)

    def iterate_until_flat(self, params: muca_params | None = None, raise_on_fail: bool = False) -> IterationStats:
        rc, st = muca_iterate_until_flat(self._h, params, raise_on_fail)
        return IterationStats(rc, st.iterations, bool(st.converged), st.last_metric, st.attempts_per_walker,
                              st.seconds)

    @property
    def site_order(self) -> int:
        return muca_get_site_order(self._h)

    @site_order.setter
    def site_order(self, order: int) -> None:
        muca_set_site_order(self._h, order)

    def iterate_device(self, params: muca_params | None = None, iterations_per_sync: int = 8,
                       raise_on_fail: bool = False) -> IterationStats:
        rc, st = muca_iterate_device(self._h, params, iterations_per_sync, raise_on_fail)
        return IterationStats(rc, st.iterations, bool(st.converged), st.last_metric, st.attempts_per_walker,
                              st.seconds)

    def production(self, therm_sweeps: int, n_sweeps: int):
        return muca_production(self._h, therm_sweeps, n_sweeps, self.n_bins)

    def production_jackknife(self, therm_sweeps: int, n_chunks: int, sweeps_per_chunk: int):
        """(chunk histograms, ln g, jackknife error of ln g)."""
        return muca_production_jackknife(self._h, therm_sweeps, n_chunks, sweeps_per_chunk, self.n_bins)

    def get_energies(self) -> np.ndarray:
        return muca_get_energies(self._h, self.W)

    def get_lattice(self) -> np.ndarray:
        return muca_get_lattice(self._h, self.W, self.N)

    def info(self):
        return muca_get_info(self._h)

    @property
    def attempt_counter(self) -> int:
        return muca_get_info(self._h)[2]


# ---------------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------------
def muca_batch_create(handles) -> ctypes.c_void_p:
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    b = ctypes.c_void_p()
    _check(C.load().muca_batch_create(arr, len(handles), ctypes.byref(b)))
    return b


def muca_batch_destroy(b) -> None:
    _check(C.load().muca_batch_destroy(b))


def muca_batch_sweep(b, n_sweeps: int, record: bool) -> None:
    _check(C.load().muca_batch_sweep(b, n_sweeps, 1 if record else 0))


def muca_batch_iterate(b, n: int, params: muca_params | None = None, raise_on_fail: bool = False):
    st = (muca_stats * n)()
    rc = C.load().muca_batch_iterate(b, ctypes.byref(params) if params is not None else None, st)
    if raise_on_fail:
        _check(rc)
    return rc, [IterationStats(rc, s.iterations, bool(s.converged), s.last_metric, s.attempts_per_walker, s.seconds)
                for s in st]


def muca_batch_info(b):
    n, g, sm = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
    _check(C.load().muca_batch_info(b, ctypes.byref(n), ctypes.byref(g), ctypes.byref(sm)))
    return n.value, g.value, sm.value


class Batch:
    """Several Muca instances advanced together by the batched persistent kernel."""

    def __init__(self, instances):
        self.instances = list(instances)
        self._b = muca_batch_create([m._h for m in self.instances])

    def sweep(self, n_sweeps: int, record: bool = True) -> None:
        muca_batch_sweep(self._b, n_sweeps, record)

    def iterate_until_flat(self, params: muca_params | None = None):
        rc, stats = muca_batch_iterate(self._b, len(self.instances), params)
        return rc, stats

    def info(self):
        return muca_batch_info(self._b)

    def close(self) -> None:
        if self._b:
            muca_batch_destroy(self._b)
            self._b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def muca_batch_sweep_noalloc(instances, n_sweeps: int, record: bool, stream_handle: int | None = None) -> None:
    """instances: muca_raw_instance structures (caller-owned device buffers)."""
    arr = (C.muca_raw_instance * len(instances))(*instances)
    _check(C.load().muca_batch_sweep_noalloc(arr, len(instances), n_sweeps, 1 if record else 0,
                                             ctypes.c_void_p(stream_handle or 0)))


# ---------------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------------
class Server:
    """Continuous batching of weight-iteration requests (muca_server_* in muca.h)."""

    def __init__(self, hbm_budget_bytes: int):
        use_torch_allocator()
        self._s = ctypes.c_void_p()
        _check(C.load().muca_server_create(int(hbm_budget_bytes), ctypes.byref(self._s)))

    def submit(self, L: int, n_walkers: int, seed: int, params: muca_params, layout: int = MUCA_LAYOUT_INT8,
               walkers_per_block: int = 0) -> int:
        r = C.muca_request(L, n_walkers, seed, layout, walkers_per_block, params)
        rid = ctypes.c_int64()
        _check(C.load().muca_server_submit(self._s, ctypes.byref(r), ctypes.byref(rid)))
        return rid.value

    def step(self):
        a, q = ctypes.c_int32(), ctypes.c_int32()
        _check(C.load().muca_server_step(self._s, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def status(self, rid: int) -> C.muca_request_status:
        st = C.muca_request_status()
        _check(C.load().muca_server_status(self._s, rid, ctypes.byref(st)))
        return st

    def weights(self, rid: int, n_bins: int) -> np.ndarray:
        a = np.zeros(n_bins, dtype=np.float64)
        _check(C.load().muca_server_weights(self._s, rid, _p(a, ctypes.c_double), n_bins))
        return a

    def totals(self):
        att, sec, steps, used = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_int32(), ctypes.c_size_t()
        _check(C.load().muca_server_totals(self._s, ctypes.byref(att), ctypes.byref(sec), ctypes.byref(steps),
                                           ctypes.byref(used)))
        return att.value, sec.value, steps.value, used.value

    def close(self) -> None:
        if self._s:
            _check(C.load().muca_server_destroy(self._s))
            self._s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
