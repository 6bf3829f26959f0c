"""ctypes binding of the C oracle (muca_oracle.c, exact_dos.c).

TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the CPU-baseline
leg of the benchmark.  The product package never imports this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "muca_oracle.c"), os.path.join(HERE, "exact_dos.c")]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles liboracle.so with gcc (plain C11, no fast-math, no FMA contraction)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in SOURCES)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp] + SOURCES + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("schedule", ctypes.c_int32),
        ("stop_rule", ctypes.c_int32),
        ("flat_threshold", ctypes.c_double),
        ("therm_sweeps", ctypes.c_uint64),
        ("sweeps_per_iter", ctypes.c_uint64),
        ("f_therm", ctypes.c_double),
        ("z", ctypes.c_double),
        ("factor", ctypes.c_double),
        ("growth", ctypes.c_double),
        ("max_iterations", ctypes.c_int32),
        ("site_order", ctypes.c_int32),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("last_metric", ctypes.c_double),
        ("t", ctypes.c_uint64),
        ("attempts", ctypes.c_uint64),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def build_variant(sources: list[str], path: str) -> str:
    """Compiles other oracle sources (e.g. a copy with a planted mistake, for the tests
    that check the pins catch it) into `path` with the same options."""
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-o", path] + \
        list(sources) + ["-lm"]
    subprocess.run(cmd, check=True)
    return path


class using:
    """Context manager: the binding's functions call the library at `path` inside it."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        with _lock:
            self.saved = _lib
            _lib = _bind(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved


def _bind(path: str):
    """Loads a compiled oracle library and declares its C signatures."""
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    u32, u64, i32, i64, dbl, i8 = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32,
                                   ctypes.c_int64, ctypes.c_double, ctypes.c_int8)
    sig = {
        "orc_philox4x32_10": (None, [P(u32), P(u32), P(u32)]),
        "orc_random_word": (u32, [u64, u32, u32, u64]),
        "orc_energy_index": (i32, [i32, P(i8)]),
        "orc_init": (None, [i32, u64, u32, i64, P(i8), P(i32)]),
        "orc_build_table": (None, [i32, P(dbl), P(u32)]),
        "orc_accept": (ctypes.c_int, [u32, u32]),
        "orc_run": (None, [i32, u64, u32, i64, P(i8), P(i32), P(u32), u64, u64, i32, P(u64)]),
        "orc_run_random": (None, [i32, u64, u32, i64, P(i8), P(i32), P(u32), u64, u64, i32, P(u64)]),
        "orc_random_site": (i32, [i32, u64, u64]),
        "orc_update_weights": (None, [i32, P(dbl), P(u64)]),
        "orc_accessible": (ctypes.c_int, [i32, i32]),
        "orc_min_over_mean": (dbl, [i32, P(u64)]),
        "orc_width": (i32, [i32, P(u64)]),
        "orc_accessible_in_range": (i32, [i32, P(u64)]),
        "orc_kl_support": (i32, [i32, i32, i32, P(u64)]),
        "orc_kullback_leibler": (dbl, [i32, P(u64), dbl]),
        "orc_exp": (dbl, [dbl]),
        "orc_log": (dbl, [dbl]),
        "orc_chebyshev": (dbl, [i32, P(u64)]),
        "orc_iterate": (i32, [i32, i64, u64, P(i8), P(i32), P(dbl), P(u64), P(Params),
                              P(dbl), P(dbl), P(Result)]),
        "orc_iterate_traced": (i32, [i32, i64, u64, P(i8), P(i32), P(dbl), P(u64), P(Params),
                                     P(dbl), P(dbl), P(i64), P(Result)]),
        "orc_ln_dos": (None, [i32, P(dbl), P(u64), P(dbl)]),
        "orc_production": (i32, [i32, i64, u64, P(i8), P(i32), P(dbl), P(u64), u64, u64,
                                 P(u64), P(dbl), i32]),
        "orc_dos_bruteforce": (i32, [i32, P(u64)]),
        "orc_jackknife": (i32, [i32, P(dbl), P(u64), i32, P(dbl), P(dbl)]),
        "orc_canonical": (None, [i32, P(dbl), dbl, P(dbl), P(dbl)]),
        "orc_dos_transfer": (i32, [i32, P(u64), P(u64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def _ptr(a: np.ndarray, ctype):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ----------------------------------------------------------------------------------
# thin numpy wrappers
# ----------------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32))
    return out


def random_word(seed: int, walker: int, tag: int, t: int) -> int:
    return int(lib().orc_random_word(seed, walker, tag, t))


def energy_index(L: int, s: np.ndarray) -> int:
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(lib().orc_energy_index(L, _ptr(s, ctypes.c_int8)))


def init(L: int, seed: int, n_walkers: int, walker0: int = 0):
    """Initial lattices spins[w][N] (int8 +/-1) and energy indices e[w]."""
    N = L * L
    spins = np.zeros((n_walkers, N), dtype=np.int8)
    e = np.zeros(n_walkers, dtype=np.int32)
    lib().orc_init(L, seed, walker0, n_walkers, _ptr(spins, ctypes.c_int8), _ptr(e, ctypes.c_int32))
    return spins, e


def exp(x: float) -> float:
    """The oracle's FP64 exp (reading R8)."""
    return lib().orc_exp(float(x))


def log(x: float) -> float:
    """The oracle's FP64 natural logarithm (reading R8)."""
    return lib().orc_log(float(x))


def random_site(L: int, seed: int, t: int) -> int:
    """Site of attempt t in random shared order (reading R9)."""
    return lib().orc_random_site(L, seed, t)


def build_table(L: int, lnW: np.ndarray) -> np.ndarray:
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    assert lnW.shape == (L * L + 1,)
    T = np.zeros((L * L + 1) * 5, dtype=np.uint32)
    lib().orc_build_table(L, _ptr(lnW, ctypes.c_double), _ptr(T, ctypes.c_uint32))
    return T


def run(L: int, seed: int, spins: np.ndarray, e: np.ndarray, T: np.ndarray, t0: int, n: int,
        record: bool, H: np.ndarray | None = None, walker0: int = 0, site_order: int = 0) -> np.ndarray | None:
    """Advances the walkers in place by n attempts from attempt counter t0 (site_order 0:
    typewriter, reading R1; 1: random shared sites, reading R9)."""
    assert spins.dtype == np.int8 and spins.flags["C_CONTIGUOUS"]
    assert e.dtype == np.int32 and e.flags["C_CONTIGUOUS"]
    nw = spins.shape[0]
    if record and H is None:
        H = np.zeros(L * L + 1, dtype=np.uint64)
    Hp = _ptr(H, ctypes.c_uint64) if H is not None else None
    fn = lib().orc_run_random if site_order == 1 else lib().orc_run
    fn(L, seed, walker0, nw, _ptr(spins, ctypes.c_int8), _ptr(e, ctypes.c_int32),
       _ptr(np.ascontiguousarray(T, dtype=np.uint32), ctypes.c_uint32), t0, n, 1 if record else 0, Hp)
    return H


def update_weights(L: int, lnW: np.ndarray, H: np.ndarray) -> None:
    lib().orc_update_weights(L, _ptr(lnW, ctypes.c_double), _ptr(H, ctypes.c_uint64))


def min_over_mean(L: int, H: np.ndarray) -> float:
    return float(lib().orc_min_over_mean(L, _ptr(np.ascontiguousarray(H, dtype=np.uint64), ctypes.c_uint64)))


def kullback_leibler(L: int, H: np.ndarray, q: float) -> float:
    return float(lib().orc_kullback_leibler(L, _ptr(np.ascontiguousarray(H, dtype=np.uint64), ctypes.c_uint64), q))


def chebyshev(L: int, H: np.ndarray) -> float:
    return float(lib().orc_chebyshev(L, _ptr(np.ascontiguousarray(H, dtype=np.uint64), ctypes.c_uint64)))


def width(L: int, H: np.ndarray) -> int:
    return int(lib().orc_width(L, _ptr(np.ascontiguousarray(H, dtype=np.uint64), ctypes.c_uint64)))


def accessible_in_range(L: int, H: np.ndarray) -> int:
    return int(lib().orc_accessible_in_range(L, _ptr(np.ascontiguousarray(H, dtype=np.uint64), ctypes.c_uint64)))


def make_params(schedule=0, stop_rule=0, flat_threshold=0.8, therm_sweeps=31, sweeps_per_iter=100,
                f_therm=30.0, z=2.25, factor=6.0, growth=1.1, max_iterations=200, site_order=0) -> Params:
    return Params(schedule, stop_rule, flat_threshold, therm_sweeps, sweeps_per_iter, f_therm, z,
                  factor, growth, max_iterations, site_order)


def iterate(L: int, seed: int, spins: np.ndarray, e: np.ndarray, lnW: np.ndarray, t: int,
            params: Params, history: bool = False):
    """Weight iteration; spins, e and lnW are advanced in place.  Returns
    (result, t, lnW_history or None, metric_history or None)."""
    N = L * L
    nw = spins.shape[0]
    tt = ctypes.c_uint64(t)
    res = Result()
    hist = mh = None
    hp = mp = None
    if history:
        hist = np.zeros((params.max_iterations, N + 1), dtype=np.float64)
        mh = np.zeros(params.max_iterations, dtype=np.float64)
        hp, mp = _ptr(hist, ctypes.c_double), _ptr(mh, ctypes.c_double)
    rc = lib().orc_iterate(L, nw, seed, _ptr(spins, ctypes.c_int8), _ptr(e, ctypes.c_int32),
                           _ptr(lnW, ctypes.c_double), ctypes.byref(tt), ctypes.byref(params),
                           hp, mp, ctypes.byref(res))
    if rc != 0:
        raise MemoryError("orc_iterate failed")
    if history:
        hist = hist[: res.iterations]
        mh = mh[: res.iterations]
    return res, int(tt.value), hist, mh


def iterate_schedule(L: int, seed: int, spins: np.ndarray, e: np.ndarray, lnW: np.ndarray, t: int,
                     params: Params):
    """Weight iteration as `iterate`, returning (result, t, schedule) with schedule[n] =
    (thermalization attempts, update attempts, lowest and highest visited energy index)
    of iteration n."""
    nw = spins.shape[0]
    tt = ctypes.c_uint64(t)
    res = Result()
    sched = np.zeros((params.max_iterations, 4), dtype=np.int64)
    rc = lib().orc_iterate_traced(L, nw, seed, _ptr(spins, ctypes.c_int8), _ptr(e, ctypes.c_int32),
                                  _ptr(lnW, ctypes.c_double), ctypes.byref(tt), ctypes.byref(params),
                                  None, None, _ptr(sched, ctypes.c_int64), ctypes.byref(res))
    if rc != 0:
        raise MemoryError("orc_iterate_traced failed")
    return res, int(tt.value), sched[: res.iterations]


def ln_dos(L: int, lnW: np.ndarray, H: np.ndarray) -> np.ndarray:
    out = np.zeros(L * L + 1, dtype=np.float64)
    lib().orc_ln_dos(L, _ptr(np.ascontiguousarray(lnW, dtype=np.float64), ctypes.c_double),
                     _ptr(np.ascontiguousarray(H, dtype=np.uint64), ctypes.c_uint64),
                     _ptr(out, ctypes.c_double))
    return out


def production(L: int, seed: int, spins: np.ndarray, e: np.ndarray, lnW: np.ndarray, t: int,
               therm_sweeps: int, sweeps: int, site_order: int = 0):
    """Returns (H, ln_g, t)."""
    N = L * L
    H = np.zeros(N + 1, dtype=np.uint64)
    ln_g = np.zeros(N + 1, dtype=np.float64)
    tt = ctypes.c_uint64(t)
    rc = lib().orc_production(L, spins.shape[0], seed, _ptr(spins, ctypes.c_int8),
                              _ptr(e, ctypes.c_int32),
                              _ptr(np.ascontiguousarray(lnW, dtype=np.float64), ctypes.c_double),
                              ctypes.byref(tt), therm_sweeps, sweeps, _ptr(H, ctypes.c_uint64),
                              _ptr(ln_g, ctypes.c_double), site_order)
    if rc != 0:
        raise MemoryError("orc_production failed")
    return H, ln_g, int(tt.value)


def dos_bruteforce(L: int) -> list[int]:
    g = np.zeros(L * L + 1, dtype=np.uint64)
    if lib().orc_dos_bruteforce(L, _ptr(g, ctypes.c_uint64)) != 0:
        raise ValueError("brute force supports 2 <= L <= 5")
    return [int(x) for x in g]


def dos_transfer(L: int) -> list[int]:
    lo = np.zeros(L * L + 1, dtype=np.uint64)
    hi = np.zeros(L * L + 1, dtype=np.uint64)
    rc = lib().orc_dos_transfer(L, _ptr(lo, ctypes.c_uint64), _ptr(hi, ctypes.c_uint64))
    if rc != 0:
        raise ValueError(f"transfer matrix failed ({rc})")
    return [int(a) | (int(b) << 64) for a, b in zip(lo, hi)]


def jackknife(L: int, lnW: np.ndarray, Hc: np.ndarray):
    """Hc: [n_chunks][N+1] uint64 -> (ln_g, err)."""
    Hc = np.ascontiguousarray(Hc, dtype=np.uint64)
    B = L * L + 1
    ln_g = np.zeros(B)
    err = np.zeros(B)
    rc = lib().orc_jackknife(L, _ptr(np.ascontiguousarray(lnW, dtype=np.float64), ctypes.c_double),
                             _ptr(Hc, ctypes.c_uint64), Hc.shape[0], _ptr(ln_g, ctypes.c_double),
                             _ptr(err, ctypes.c_double))
    if rc != 0:
        raise MemoryError("orc_jackknife failed")
    return ln_g, err


def canonical(L: int, ln_g: np.ndarray, beta: float):
    e, c = ctypes.c_double(), ctypes.c_double()
    lib().orc_canonical(L, _ptr(np.ascontiguousarray(ln_g, dtype=np.float64), ctypes.c_double), beta,
                        ctypes.byref(e), ctypes.byref(c))
    return e.value, c.value
