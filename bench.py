"""Benchmark of the parallel multicanonical 2D Ising hot path on GB300.

Workload (the headline configuration): periodic 32x32 Ising lattices, 16384 walkers,
int8 interleaved lattices, random +/-1 start (seed 1), 10 recorded sweeps per iteration
after 31 thermalization sweeps, uint64 histogram over the 1025 energies, FP64 weight
recursion; iteration budget 2e4 * L^2 recorded walker-sweeps (125 iterations).

Reported:
  value        spin-flip attempts per second over K weight-iteration steps (one step =
               weights upload + table build, thermalization, zeroed histogram, recorded sweeps,
               histogram read, flatness test and Eq. (4) recursion), device-timed with
               CUDA events, L2 flushed in each timed step before its sweep launch (the
               flush's window is not counted);
  time_to_flat wall time of muca_iterate_until_flat from ln W = 0 until min/mean >= 0.8;
  e2e          the same steps through the C ABI with host weights in and the host
               histogram out (copies inside the timed region), host wall clock;
  roofline     the step's sweep kernel (one launch: 31 thermalization sweeps, then 10
               recorded sweeps) against the integer-issue ceiling (and against the
               measured issue rate of a balanced integer mix);
  cpu_baseline the C oracle on the host cores: one step of the same workload on all cores
               and on one thread, and its whole weight iteration to a flat histogram.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_SIDE = 32
WALKERS = 16384
SEED = 1
THERM_SWEEPS = 31
SWEEPS_PER_ITER = 10
MAX_ITERATIONS = 2 * 10**4 * L_SIDE * L_SIDE // (WALKERS * SWEEPS_PER_ITER)   # 125
# Algorithmic integer operations per attempted flip (Philox4x32-10: 10 rounds of 2
# mul-hi, 2 mul-lo and 2 three-input XORs plus 9 key bumps of 2 adds = 78 per 4 words,
# 19.5 per attempt; the flip: own spin, 4 neighbour compares, count, table address and
# load, compare, conditional flip, energy update, run-length histogram record, about
# 15.5).  Fixed by the method, not measured from the code.
OPS_PER_ATTEMPT = 35.0
# Warp instructions the step's whole-sweep launch issues per attempt and warp (ncu
# count, profiles/sweep_full_kernel_L32_W16384_int8.md): converts an instruction issue
# rate into this roofline's algorithmic operations.
INSTR_PER_ATTEMPT = 31.13
WORKLOAD = (f"muca2d_ising_L{L_SIDE}_W{WALKERS}_int8_therm{THERM_SWEEPS}_rec{SWEEPS_PER_ITER}")


def config_dict():
    return {"workload": WORKLOAD, "L": L_SIDE, "walkers": WALKERS, "layout": "int8 [site][walker]",
            "therm_sweeps": THERM_SWEEPS, "sweeps_per_iter": SWEEPS_PER_ITER, "energy_bins": L_SIDE**2 + 1,
            "stop_rule": "min/mean >= 0.8", "max_iterations": MAX_ITERATIONS,
            "l2": "flushed in every timed step before its sweep launch (256 MiB write, its window not counted)", "parallelism": "independent instance per GPU",
            "arithmetic": "u32 thresholds, random words and counts; int8 spins; u64 histogram; f64 weights"}


def exact_ln_dos(L: int):
    """ln g(e) of the periodic L x L lattice from the committed table (exact closed form,
    tests/golden/exact_dos_L{L}.txt); -inf at the two inaccessible energies."""
    import numpy as np
    vals = []
    with open(os.path.join(ROOT, "tests", "golden", f"exact_dos_L{L}.txt")) as f:
        for line in f:
            if not line.startswith("#"):
                vals.append(float(line.split()[1]))
    return np.array(vals, dtype=np.float64)


def perfect_weights(L: int):
    """ln W = -ln g (the perfect multicanonical weights of Sec. 3.1), 0 where g = 0."""
    import numpy as np
    lng = exact_ln_dos(L)
    return np.where(np.isfinite(lng), -lng, 0.0)


def time_recorded_sweeps(m, stream, sweeps: int, reps: int, lead: int = 0) -> float:
    """Median device time (s) of a launch of `sweeps` recorded sweeps on the instance's
    stream; lead > 0 queues that many thermalization sweeps before each timed launch, so
    that the GPU is busy while the host enqueues it (the window then holds no host time)."""
    import torch
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        if lead:
            m.sweep(lead, record=False)
        a.record(stream)
        m.sweep(sweeps, record=True)
        b.record(stream)
        stream.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
    ts.sort()
    return ts[len(ts) // 2]


# ----------------------------------------------------------------------------------
# distributed plumbing
# ----------------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws):
    if ws <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("gloo")
    return dist


def max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ----------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.times = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "10"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.times.append(time.perf_counter())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def count_between(self, t0: float, t1: float) -> int:
        return sum(1 for t in self.times if t0 <= t <= t1)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# Sources that define the timed whole-sweep kernel at L = 32 (body and launcher).
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1707_00919_gb300", "csrc", f)
                  for f in ("muca_device.cuh", "muca_full.cuh", "muca_full_32.cu")]
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "sweep_full_kernel_L32_W16384_int8.md")


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for path in KERNEL_SOURCES:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes (read + write) per launch of the step's sweep kernel (thermalization and
    recorded sweeps) from the committed ncu summary, or None when the kernel source
    changed since that capture."""
    try:
        text = open(TRAFFIC_PROFILE).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_step_launch"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------------------------
# CPU baseline: the oracle on the host cores
# ----------------------------------------------------------------------------------
def _oracle_shard(args):
    L, seed, w0, nw, lnW, t0, n_therm, n_rec = args
    import numpy as np
    from oracle import oracle
    s, e = oracle.init(L, seed, nw, walker0=w0)
    T = oracle.build_table(L, np.asarray(lnW))
    t = time.perf_counter()
    oracle.run(L, seed, s, e, T, t0, n_therm, False, None, walker0=w0)
    H = oracle.run(L, seed, s, e, T, t0 + n_therm, n_rec, True, None, walker0=w0)
    return time.perf_counter() - t, H


def cpu_baseline(lnW, walkers: int, cores: int | None = None):
    """One step (thermalization + recorded sweeps) of `walkers` walkers by the oracle,
    walkers split across a spawn pool of host processes; returns attempts/s."""
    import multiprocessing as mp
    from oracle import oracle
    oracle.build()
    N = L_SIDE * L_SIDE
    cores = cores or os.cpu_count() or 1
    shard = (walkers + cores - 1) // cores
    jobs = []
    for c in range(cores):
        w0 = c * shard
        nw = min(shard, walkers - w0)
        if nw > 0:
            jobs.append((L_SIDE, SEED, w0, nw, list(lnW), 0, THERM_SWEEPS * N, SWEEPS_PER_ITER * N))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(len(jobs)) as pool:
        res = pool.map(_oracle_shard, jobs)
    wall = time.perf_counter() - t0
    busy = max(r[0] for r in res)
    attempts = walkers * (THERM_SWEEPS + SWEEPS_PER_ITER) * N
    return attempts / busy, len(jobs), wall


def _oracle_worker(conn, L, seed, w0, nw):
    """Holds one shard of walkers for the oracle's weight iteration: for each message
    (thresholds, t0, n_therm, n_rec) it runs the shard's thermalization and recorded
    attempts and sends back the shard's histogram."""
    from oracle import oracle
    s, e = oracle.init(L, seed, nw, walker0=w0)
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg is None:
            break
        T, t0, n_therm, n_rec = msg
        oracle.run(L, seed, s, e, T, t0, n_therm, False, None, walker0=w0)
        conn.send(oracle.run(L, seed, s, e, T, t0 + n_therm, n_rec, True, None, walker0=w0))


def cpu_time_to_flat(walkers: int, cores: int | None = None, max_iterations: int = MAX_ITERATIONS):
    """The oracle's weight iteration of the headline workload from ln W = 0 to
    min/mean >= 0.8: walkers split over host processes (one shard each, kept between
    iterations), histograms summed, the oracle's flatness test, Eq. (4) recursion and
    table on the host.  Returns (seconds, iterations, converged, ln W, processes); the
    clock starts once the shards hold their initial lattices."""
    import multiprocessing as mp
    import numpy as np
    from oracle import oracle
    oracle.build()
    N = L_SIDE * L_SIDE
    cores = cores or os.cpu_count() or 1
    shard = (walkers + cores - 1) // cores
    ctx = mp.get_context("spawn")
    procs, conns = [], []
    for c in range(cores):
        w0, nw = c * shard, min(shard, walkers - c * shard)
        if nw <= 0:
            break
        a, b = ctx.Pipe()
        p = ctx.Process(target=_oracle_worker, args=(b, L_SIDE, SEED, w0, nw), daemon=True)
        p.start()
        procs.append(p)
        conns.append(a)
    for c in conns:
        c.recv()
    lnW = np.zeros(N + 1)
    t, it, converged = 0, 0, False
    n_therm, n_rec = THERM_SWEEPS * N, SWEEPS_PER_ITER * N
    t0 = time.perf_counter()
    while it < max_iterations:
        T = oracle.build_table(L_SIDE, lnW)
        for c in conns:
            c.send((T, t, n_therm, n_rec))
        H = np.zeros(N + 1, dtype=np.uint64)
        for c in conns:
            H += c.recv()
        t += n_therm + n_rec
        it += 1
        if oracle.min_over_mean(L_SIDE, H) >= 0.8:
            converged = True
            break
        oracle.update_weights(L_SIDE, lnW, H)
    seconds = time.perf_counter() - t0
    for c in conns:
        c.send(None)
    for p in procs:
        p.join(timeout=10)
    return seconds, it, converged, lnW, len(procs)


def cpu_single_thread(lnW, walkers: int = 512):
    """The oracle on one host thread: one step (thermalization + recorded sweeps) of
    `walkers` walkers; returns attempts/s."""
    N = L_SIDE * L_SIDE
    busy, _ = _oracle_shard((L_SIDE, SEED, 0, walkers, list(lnW), 0, THERM_SWEEPS * N, SWEEPS_PER_ITER * N))
    return walkers * (THERM_SWEEPS + SWEEPS_PER_ITER) * N / busy


# ----------------------------------------------------------------------------------
# native arm
# ----------------------------------------------------------------------------------
def run_native(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    dist = init_dist(ws)
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    barrier(dist)
    __graft_entry__.build()
    from paper_1707_00919_gb300 import muca as M

    N = L_SIDE * L_SIDE
    stream = torch.cuda.Stream()
    seed = SEED + rank                              # independent simulation per GPU
    m = M.Muca(L_SIDE, WALKERS, seed, layout=M.MUCA_LAYOUT_INT8, stream=stream)

    # clocks sampled from here to the end of the end-to-end steps: the whole stretch runs
    # the same kernels (time to flat, warm-up, timed and end-to-end steps)
    clocks = ClockSampler(dev).__enter__()

    # ---- time to flat histogram (from ln W = 0) ----
    params = M.make_params(therm_sweeps=THERM_SWEEPS, sweeps_per_iter=SWEEPS_PER_ITER,
                           max_iterations=MAX_ITERATIONS)
    barrier(dist)
    t0 = time.perf_counter()
    st = m.iterate_until_flat(params)
    torch.cuda.synchronize()
    ttf = time.perf_counter() - t0
    ttf = max_over_ranks(dist, ttf)

    lnW = m.get_weights()
    ln_w_flat = lnW.copy()
    attempts_per_step = WALKERS * (THERM_SWEEPS + SWEEPS_PER_ITER) * N

    # ---- the same, with the recursion, stop test and table build on the device ----
    with M.Muca(L_SIDE, WALKERS, seed, layout=M.MUCA_LAYOUT_INT8, stream=stream) as md:
        barrier(dist)
        t0 = time.perf_counter()
        st_dev = md.iterate_device(params, 8)
        torch.cuda.synchronize()
        ttf_dev = max_over_ranks(dist, time.perf_counter() - t0)
        same_weights = bool(np.array_equal(md.get_weights(), lnW))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    flat = [False]

    def step(ev=None):
        """One weight iteration through the C ABI (weights upload, the table built on the
        device; zeroed histogram, thermalization and recorded sweeps in one
        muca_thermalize_and_record call, one kernel launch; histogram read; the min/mean
        flatness test and the Eq. (4) recursion, muca_flatness and muca_update_weights).
        ev = five CUDA events
        on the instance's stream: step start, the L2 flush's start and end, after the
        sampling call, after the host recursion.  In a timed step the L2 flush (a 256 MiB
        write) runs between the weights upload and the sampling call: the GPU is busy with
        it while the host enqueues the launch, so that the sampling window holds GPU work
        only; the flush's own window is left out of the step's time."""
        if ev:
            ev[0].record(stream)
        m.set_weights(lnW)
        if ev:
            ev[1].record(stream)
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[2].record(stream)
        m.thermalize_and_record(THERM_SWEEPS * N, SWEEPS_PER_ITER * N)
        if ev:
            ev[3].record(stream)
        H = m.get_histogram()
        flat[0] = M.muca_flatness(L_SIDE, H, measures=("min_over_mean",))["min_over_mean"] >= 0.8
        M.muca_update_weights(L_SIDE, lnW, H)
        if ev:
            ev[4].record(stream)
        return H

    # NVTX range around the warm-up and timed steps, so that a profiler can be limited to
    # them (ncu --nvtx --nvtx-include "bench_steps/")
    torch.cuda.nvtx.range_push("bench_steps")
    for _ in range(args.warmup):
        step()
        with torch.cuda.stream(stream):
            flush.zero_()
    stream.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    barrier(dist)
    torch.cuda.synchronize()
    t_timed0 = time.perf_counter()
    for k in range(args.steps):
        step(evs[k])
    stream.synchronize()
    torch.cuda.synchronize()
    t_timed1 = time.perf_counter()
    torch.cuda.nvtx.range_pop()
    step_ms = [evs[k][0].elapsed_time(evs[k][4]) - evs[k][1].elapsed_time(evs[k][2]) for k in range(args.steps)]
    table_ms = [evs[k][0].elapsed_time(evs[k][1]) for k in range(args.steps)]
    sample_ms = [evs[k][2].elapsed_time(evs[k][3]) for k in range(args.steps)]
    total_s = sum(step_ms) / 1e3
    total_s = max_over_ranks(dist, total_s)
    barrier(dist)

    # ---- end to end through the public API, host buffers, host clock ----
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0)
    clocks.__exit__(None, None, None)
    clock_summary = clocks.summary()
    clock_summary["timed_region_samples"] = clocks.count_between(t_timed0, t_timed1)
    clock_summary["window"] = "time to flat, warm-up, timed and end-to-end steps"

    value = ws * attempts_per_step * args.steps / total_s
    e2e_value = ws * attempts_per_step * args.steps / e2e_s
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    # integer-issue ceiling: every SM sub-partition issues one 32-lane instruction per clock
    peak_tops = sm_count * 4 * 32 * sm_max_mhz * 1e6 / 1e12
    # the sampling window holds the launch and the histogram zeroing before it (an 8 KB
    # memset), which is counted against the kernel
    launch_s = (sum(sample_ms) / len(sample_ms)) / 1e3
    launch_attempts = WALKERS * (THERM_SWEEPS + SWEEPS_PER_ITER) * N
    achieved_tops = OPS_PER_ATTEMPT * launch_attempts / launch_s / 1e12
    traffic = profiled_traffic()
    lattice_bytes = 2 * WALKERS * N   # int8 lattices read and written once per launch
    # measured issue rates of the instruction classes the sweep uses (context for the peak)
    probe = {name: M.muca_measure_issue_rate(kind) / 1e12
             for name, kind in (("xor3_alu", M.MUCA_PROBE_XOR), ("imad", M.MUCA_PROBE_MAD),
                                ("xor3_imad_alternating", M.MUCA_PROBE_MIXED),
                                ("xor3_imad_alternating_one_warp_per_smsp", M.MUCA_PROBE_MIXED_ONE_WARP))}
    philox_words = M.muca_measure_issue_rate(M.MUCA_PROBE_PHILOX)
    # what one warp per sub-partition can issue, on the sub-partitions this walker count
    # occupies (one warp per 32 walkers), as a fraction of the peak in this roofline's units
    smsps = sm_count * 4
    busy = min(WALKERS // 32, smsps) / smsps
    one_warp_frac = (probe["xor3_imad_alternating_one_warp_per_smsp"] * busy * OPS_PER_ATTEMPT / INSTR_PER_ATTEMPT
                     / peak_tops)
    result = {
        "metric": "spin-flip attempts/s (and time-to-flat H) at L=32, 16384 walkers; % of integer-issue roofline",
        "value": value,
        "unit": "attempts/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": sum(step_ms) / len(step_ms),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic: random +/-1 Ising lattices from the seed",
        "config": config_dict(),
        "time_to_flat_s": ttf,
        "iterations_to_flat": st.iterations,
        "time_to_flat_device_iteration_s": ttf_dev,
        "device_iteration_identical": bool(same_weights and st_dev.iterations == st.iterations),
        "flat": bool(st.converged),
        "flat_metric": st.last_metric,
        "table_ms_per_step": sum(table_ms) / len(table_ms),
        "sweep_launch_ms_per_step": sum(sample_ms) / len(sample_ms),
        "e2e": {"value": e2e_value, "unit": "attempts/s",
                "h2d_bytes_per_step": (N + 1) * 8, "d2h_bytes_per_step": (N + 1) * 8 + 4},
        "gpu_launches": 2 * args.steps,   # per step: table_kernel, sweep_full_kernel
        "roofline": {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "Tops/s (int32)",
                     "frac": achieved_tops / peak_tops, "traffic": traffic,
                     "kernel": "sweep_full_kernel<32,int8,record> (31 thermalization + 10 recorded "
                               "sweeps in one launch)",
                     "ops_per_attempt": OPS_PER_ATTEMPT,
                     "peak_basis": f"{sm_count} SMs x 4 issue slots x 32 lanes x {sm_max_mhz:.0f} MHz",
                     "measured_issue_tops": {k: round(v, 3) for k, v in probe.items()},
                     # the same achieved rate against the measured issue rate of a balanced
                     # integer mix (three-input XOR and multiply-add alternating, 16 warps per
                     # sub-partition): what the hardware sustains for such a mix
                     "frac_of_measured_mixed_issue": achieved_tops / probe["xor3_imad_alternating"],
                     "single_warp_issue_frac": one_warp_frac,
                     "measured_philox_words_per_s": philox_words,
                     # lattice traffic of the same launch against HBM (not the bound)
                     "hbm": {"algorithmic_bytes": lattice_bytes, "algorithmic_gbs": lattice_bytes / launch_s / 1e9,
                             "dram_gbs": (traffic / launch_s / 1e9) if traffic else None,
                             "peak_gbs": peaks.get("hbm_gbs"),
                             "frac": (lattice_bytes / launch_s / 1e9 / peaks["hbm_gbs"])
                             if peaks.get("hbm_gbs") else None}},
        "clocks": clock_summary,
    }
    m.close()

    # ---- the paper's hardware protocol (Sec. 3.1): perfect weights, equilibrated ----
    mp_ = M.Muca(L_SIDE, WALKERS, seed, layout=M.MUCA_LAYOUT_INT8, stream=stream)
    mp_.set_weights(perfect_weights(L_SIDE))
    mp_.sweep(THERM_SWEEPS, record=False)
    pp_s = time_recorded_sweeps(mp_, stream, SWEEPS_PER_ITER, 7, lead=3)
    mp_.close()
    pp_rate = WALKERS * SWEEPS_PER_ITER * N / pp_s
    # the paper's random shared site order (Sec. 2.3) on the same workload
    mr = M.Muca(L_SIDE, WALKERS, seed, layout=M.MUCA_LAYOUT_INT8, stream=stream)
    mr.site_order = M.MUCA_ORDER_RANDOM
    mr.set_weights(perfect_weights(L_SIDE))
    mr.sweep(3, record=False)
    rnd_s = time_recorded_sweeps(mr, stream, SWEEPS_PER_ITER, 5)
    mr.close()
    rnd_rate = WALKERS * SWEEPS_PER_ITER * N / rnd_s
    result["paper_protocol"] = {"attempts_per_s": pp_rate, "ns_per_flip": 1e9 / pp_rate,
                                "protocol": f"ln W = -ln g exact, {THERM_SWEEPS} sweeps to equilibrate, "
                                            f"median of 7 launches of {SWEEPS_PER_ITER} recorded sweeps, "
                                            f"each queued behind 3 thermalization sweeps"}
    # the recorded launch alone (the form of the kernel before thermalization and recording
    # shared a launch), for comparison with the step's single launch
    result["roofline"]["recorded_launch_alone"] = {
        "sweeps": SWEEPS_PER_ITER, "ms": pp_s * 1e3,
        "achieved": OPS_PER_ATTEMPT * pp_rate / 1e12, "frac": OPS_PER_ATTEMPT * pp_rate / 1e12 / peak_tops}
    result["random_site_order"] = {"attempts_per_s": rnd_rate, "ns_per_flip": 1e9 / rnd_rate,
                                   # the same integer-issue roofline as the typewriter kernel
                                   "roofline_frac": OPS_PER_ATTEMPT * rnd_rate / 1e12 / peak_tops,
                                   "typewriter_roofline_frac": achieved_tops / peak_tops,
                                   "protocol": f"perfect weights, 3 sweeps to equilibrate, median of 5 launches "
                                               f"of {SWEEPS_PER_ITER} recorded sweeps in random shared site order"}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:   # the oracle baseline at N = 1 only
        rate, cores, wall = cpu_baseline(lnW, WALKERS)
        result["cpu_baseline"] = {"value": rate, "unit": "attempts/s", "cores": cores, "kind": "oracle",
                                  "sample": f"one step ({THERM_SWEEPS}+{SWEEPS_PER_ITER} sweeps) of all "
                                            f"{WALKERS} walkers, split over {cores} processes ({wall:.1f} s)"}
        result["cpu_baseline"]["single_thread_attempts_per_s"] = cpu_single_thread(lnW)
        result["cpu_baseline"]["single_thread_sample"] = (f"one step of 512 walkers on one host thread")
        if not args.no_cpu_time_to_flat:
            secs, its, conv, lnW_cpu, procs = cpu_time_to_flat(WALKERS)
            result["cpu_baseline"].update({
                "time_to_flat_s": secs, "time_to_flat_iterations": its, "time_to_flat_flat": conv,
                "time_to_flat_processes": procs,
                "time_to_flat_identical_weights": bool(np.array_equal(lnW_cpu, ln_w_flat)),
                "time_to_flat_sample": f"the whole iteration from ln W = 0 ({WALKERS} walkers, "
                                       f"{THERM_SWEEPS}+{SWEEPS_PER_ITER} sweeps per iteration) on {procs} processes"})
    if rank == 0:
        print(json.dumps(result))
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args):
    """The oracle, timed on the host cores over steps of the same workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    N = L_SIDE * L_SIDE
    # bounded sample per step: 2048 of the 16384 walkers, one full step each
    sample_walkers = 2048
    lnW = np.zeros(N + 1)
    rates = []
    for _ in range(args.warmup):   # untimed: process pool start-up and first-touch costs
        cpu_baseline(lnW, sample_walkers)
    cores_used = 1
    for _ in range(args.steps):
        rate, cores_used, _ = cpu_baseline(lnW, sample_walkers)
        rates.append(rate)
    value = sum(rates) / len(rates)
    out = {
        "impl": "reference",
        "metric": "spin-flip attempts/s (and time-to-flat H) at L=32, 16384 walkers; % of integer-issue roofline",
        "value": value, "unit": "attempts/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": config_dict(),
        "cpu_baseline": {"value": value, "unit": "attempts/s", "cores": cores_used, "kind": "oracle",
                         "sample": f"{sample_walkers} walkers x ({THERM_SWEEPS}+{SWEEPS_PER_ITER}) sweeps per step"},
        "e2e": {"value": value, "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


# ----------------------------------------------------------------------------------
# extra workloads: the 24-instance batched mix and the served request stream
# ----------------------------------------------------------------------------------
def mix_specs():
    """Configuration 4: 24 instances, L from {16, 24, 32, 48, 64}, walkers uniform in
    512..16384 (seed 1234), instance seeds 1234 + index."""
    import numpy as np
    rng = np.random.default_rng(1234)
    Ls = rng.choice([16, 24, 32, 48, 64], size=24)
    Ws = rng.integers(512, 16385, size=24)
    return [(int(L), int(W), 1234 + i) for i, (L, W) in enumerate(zip(Ls, Ws))]


def run_batch_workload(args):
    """Aggregate attempts/s of the 24-instance mix: each instance iterated alone, one
    after the other (one launch per instance and phase), against all instances in the
    batched persistent kernel (one graph replay per iteration).  Both run the same
    number of weight iterations on identical state, so their results are identical."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00919_gb300 import muca as M
    iters = max(1, args.steps)
    specs = mix_specs()
    p = M.make_params(therm_sweeps=THERM_SWEEPS, sweeps_per_iter=SWEEPS_PER_ITER, max_iterations=iters,
                      flat_threshold=2.0)
    attempts = sum(W * L * L * (THERM_SWEEPS + SWEEPS_PER_ITER) * iters for L, W, _ in specs)
    # plain path
    inst = [M.Muca(L, W, seed) for L, W, seed in specs]
    for m in inst:
        m.sweep(1, record=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m in inst:
        m.iterate_until_flat(p)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain_w = [m.get_weights() for m in inst]
    for m in inst:
        m.close()
    # batched path
    inst = [M.Muca(L, W, seed) for L, W, seed in specs]
    for m in inst:
        m.sweep(1, record=False)
    torch.cuda.synchronize()
    with M.Batch(inst) as b:
        t0 = time.perf_counter()
        b.iterate_until_flat(p)
        torch.cuda.synchronize()
        batch_s = time.perf_counter() - t0
        n, grid, smem = b.info()
    same = all(np.array_equal(m.get_weights(), w) for m, w in zip(inst, plain_w))
    for m in inst:
        m.close()
    print(json.dumps({
        "metric": "aggregate spin-flip attempts/s, 24-instance mix (L 16-64, 512-16384 walkers)",
        "value": attempts / batch_s, "unit": "attempts/s", "n_gpus": 1, "higher_is_better": True,
        "workload": "batched persistent kernel, one CUDA graph per weight iteration",
        "iterations": iters, "plain_value": attempts / plain_s, "speedup_vs_plain": plain_s / batch_s,
        "identical_results": same, "batch_grid": grid, "batch_smem_bytes": smem,
        "config": {"instances": [{"L": L, "walkers": W} for L, W, _ in specs],
                   "therm_sweeps": THERM_SWEEPS, "sweeps_per_iter": SWEEPS_PER_ITER},
        "data": "synthetic"}))


def run_serve_workload(args):
    """Configuration 5: Poisson arrivals (mean 20 per second, seed 7) of weight-iteration
    requests, L uniform over {8, 16, 24, 32, 48, 64}, walkers from {256, 1024, 4096,
    16384}, admitted under a 150 GB budget.  Every request runs the paper's Eq. (7)
    schedule (Sec. 3) to min H / mean H >= 0.8, so every request converges at the same
    accuracy whatever its size.  Reports p50 / p99 time from arrival to converged weights
    (converged requests) and aggregate attempts/s, against a first-come-first-served
    queue of the same requests run one at a time (its latencies computed from each
    request's measured time alone and the same arrival times); each served result is
    compared with the same request run alone."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00919_gb300 import muca as M
    rng = np.random.default_rng(7)
    horizon = float(args.serve_seconds)
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / 20.0)
        if t > horizon:
            break
        L = int(rng.choice([8, 16, 24, 32, 48, 64]))
        W = int(rng.choice([256, 1024, 4096, 16384]))
        reqs.append((t, L, W, 7000 + len(reqs)))
    params = M.make_params(schedule=M.MUCA_SCHEDULE_PAPER, stop_rule=M.MUCA_STOP_MIN_MEAN, flat_threshold=0.8,
                           max_iterations=5000)
    # served
    srv = M.Server(150 * 10**9)
    start = time.perf_counter()
    ids = {}
    k = 0
    while True:
        now = time.perf_counter() - start
        while k < len(reqs) and reqs[k][0] <= now:
            _, L, W, seed = reqs[k]
            ids[k] = srv.submit(L, W, seed, params)
            k += 1
        active, queued = srv.step()
        if k == len(reqs) and active == 0 and queued == 0:
            break
        if active == 0 and queued == 0 and k < len(reqs):
            time.sleep(max(0.0, min(0.01, reqs[k][0] - (time.perf_counter() - start))))
    wall = time.perf_counter() - start
    att, _, steps, _ = srv.totals()
    status = [srv.status(ids[i]) for i in range(len(reqs))]
    served_w = [srv.weights(ids[i], L * L + 1) if status[i].stats.converged else None
                for i, (_, L, _, _) in enumerate(reqs)]
    srv.close()
    conv = np.array([bool(st.stats.converged) for st in status])
    lat = np.array([st.seconds_total for st in status])
    # plain: each request alone, first come first served
    service, attempts_plain, same = [], 0, []
    for i, (_, L, W, seed) in enumerate(reqs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with M.Muca(L, W, seed) as m:
            st = m.iterate_until_flat(params)
            lnW = m.get_weights()
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t0)
        attempts_plain += st.attempts_per_walker * W
        same.append(served_w[i] is not None and bool(np.array_equal(served_w[i], lnW))
                    and st.iterations == status[i].stats.iterations)
    free_at, lat_plain = 0.0, []
    for (arr, _, _, _), s_ in zip(reqs, service):
        begin = max(arr, free_at)
        free_at = begin + s_
        lat_plain.append(free_at - arr)
    lat_plain = np.array(lat_plain)
    print(json.dumps({
        "metric": "time from arrival to converged weights (p50/p99) and aggregate attempts/s, served stream",
        "value": float(np.percentile(lat[conv], 50)), "unit": "s", "higher_is_better": False, "n_gpus": 1,
        "p50_s": float(np.percentile(lat[conv], 50)), "p99_s": float(np.percentile(lat[conv], 99)),
        "aggregate_attempts_per_s": att / wall, "requests": len(reqs), "converged_fraction": float(conv.mean()),
        "identical_to_alone_fraction": float(np.mean(same)), "steps": steps, "wall_s": wall,
        "plain": {"p50_s": float(np.percentile(lat_plain, 50)), "p99_s": float(np.percentile(lat_plain, 99)),
                  "aggregate_attempts_per_s": attempts_plain / sum(service), "busy_s": sum(service)},
        "config": {"arrival_rate_per_s": 20, "arrival_seconds": horizon, "L": [8, 16, 24, 32, 48, 64],
                   "walkers": [256, 1024, 4096, 16384], "budget_bytes": 150 * 10**9,
                   "schedule": "Eq. (7): N_therm = 30 w, N_updates = floor(6 w^2.25 / W) + 1, x1.1 after full width",
                   "stop_rule": "min/mean >= 0.8", "max_iterations": 5000},
        "kernel_source_sha256_16": kernel_source_hash(),
        "data": "synthetic"}))


def run_fliptime_workload(args):
    """Time per attempted flip against the walker count (the Fig. 2 protocol of Sec. 3.1:
    perfect weights, timed after equilibration) for L = 16, 32, 64, up to twice the
    full-occupancy count in steps of one block of 128 walkers (a multiple of it where
    that would exceed 400 points), one instance per point."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00919_gb300 import muca as M
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    out = {}
    with ClockSampler(dev) as clocks:
        for L in (16, 32, 64):
            N = L * L
            lnW = perfect_weights(L)
            n_opt, wpb_opt = M.muca_optimal_walkers(L)
            step = 128 * max(1, math.ceil(2 * n_opt / (128 * 400)))
            sweeps = max(1, 10240 // N)
            Ws, ns = [], []
            for W in sorted(set(range(step, 2 * n_opt + 1, step)) | {n_opt}):
                with M.Muca(L, W, SEED, stream=stream) as m:
                    m.set_weights(lnW)
                    m.sweep(3, record=False)
                    t = time_recorded_sweeps(m, stream, sweeps, 3)
                Ws.append(W)
                ns.append(t * 1e9 / (W * sweeps * N))
            best = int(np.argmin(ns))
            out[f"L{L}"] = {"walkers": Ws, "ns_per_flip": [round(v, 6) for v in ns],
                            "full_occupancy_walkers": n_opt, "full_occupancy_walkers_per_block": wpb_opt,
                            "ns_per_flip_at_full_occupancy": ns[Ws.index(n_opt)] if n_opt in Ws else None,
                            "best_walkers": Ws[best], "best_ns_per_flip": ns[best],
                            "recorded_sweeps_per_point": sweeps, "step_walkers": step}
    print(json.dumps({
        "metric": "time per attempted spin flip vs walkers (perfect weights, after equilibration)",
        "value": out["L32"]["best_ns_per_flip"], "unit": "ns/flip", "higher_is_better": False, "n_gpus": 1,
        "scan": out, "clocks": clocks.summary(), "data": "synthetic: random +/-1 start, exact ln g weights",
        "config": {"workload": "fliptime_scan_L16_L32_L64",
                   "layout": "int8 [site][walker]", "walkers_per_block": "occupancy rule"}}))


def _oracle_production_shard(args):
    """One host process of the CPU leg: its walkers thermalized, then n_chunks recorded
    chunks of sweeps_per_chunk sweeps; returns the chunk histograms [n_chunks][N+1]."""
    L, seed, w0, nw, lnW, therm, n_chunks, sweeps_per_chunk = args
    import numpy as np
    from oracle import oracle
    N = L * L
    s, e = oracle.init(L, seed, nw, walker0=w0)
    T = oracle.build_table(L, np.asarray(lnW))
    oracle.run(L, seed, s, e, T, 0, therm * N, False, None, walker0=w0)
    t = therm * N
    Hc = np.zeros((n_chunks, N + 1), dtype=np.uint64)
    for c in range(n_chunks):
        Hc[c] = oracle.run(L, seed, s, e, T, t, sweeps_per_chunk * N, True, None, walker0=w0)
        t += sweeps_per_chunk * N
    return Hc


def run_production_workload(args):
    """Production accuracy (Sec. 3.3, Fig. 7): walkers at full occupancy, weights
    iterated to min/mean >= 0.8, thermalization for a fifth of the production sweeps,
    then a production run of `--prod-seconds` split into 100 chunks; jackknife error
    epsilon(E) and deviation Delta(E) = |ln g - ln g_exact| per energy.  CPU leg: the oracle on the host cores (one walker per process, the same
    weights, the same wall time), and the statistical gain eps_cpu^2 / eps_gpu^2."""
    import multiprocessing as mp
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00919_gb300 import muca as M
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    chunks = 100
    out = {}

    def summary(g, err, exact):
        acc = np.isfinite(exact)
        d = np.abs(g[acc] - exact[acc])
        ep = err[acc]
        ok = np.isfinite(d) & np.isfinite(ep)   # bins seen in every leave-one-out estimate
        mid = len(d) // 2
        return {"max_delta": float(d[ok].max()), "mean_delta": float(d[ok].mean()), "delta_centre": float(d[mid]),
                "median_eps": float(np.median(ep[ok])), "eps_centre": float(ep[mid]),
                "max_eps": float(ep[ok].max()),
                "frac_delta_within_2eps": float(np.mean(d[ok] <= 2 * ep[ok])), "bins_covered": int(ok.sum()),
                "bins": int(acc.sum())}

    with ClockSampler(dev) as clocks:
        for L in (16, 32, 64):
            N = L * L
            exact = exact_ln_dos(L)
            with M.Muca(L, M.MUCA_WALKERS_OPTIMAL, SEED, stream=stream) as m:
                W = m.W
                t0 = time.perf_counter()
                st = m.iterate_until_flat(M.make_params(therm_sweeps=THERM_SWEEPS,
                                                        sweeps_per_iter=10 if L <= 32 else 4, max_iterations=3000))
                torch.cuda.synchronize()
                flat_s = time.perf_counter() - t0
                t_one = time_recorded_sweeps(m, stream, 4, 3) / 4
                spc = max(1, int(args.prod_seconds / (t_one * chunks)))
                therm = max(100, chunks * spc // 5)   # several round trips through the energy range
                t0 = time.perf_counter()
                _, g, err = m.production_jackknife(therm, chunks, spc)
                prod_s = time.perf_counter() - t0
                lnW = m.get_weights()
            res = {"walkers": W, "iterations": st.iterations, "flat": bool(st.converged), "flat_s": flat_s,
                   "production_s": prod_s, "sweeps_per_chunk": spc, "chunks": chunks, "therm_sweeps": therm,
                   "attempts": W * spc * chunks * N, "gpu": summary(g, err, exact)}
            if not args.no_cpu_baseline:
                from oracle import oracle
                oracle.build()
                cores = os.cpu_count() or 1
                rate_core = 4.0e7                    # calibrated below
                s0, e0 = oracle.init(L, SEED, 1)
                Tq = oracle.build_table(L, lnW)
                tc = time.perf_counter()
                oracle.run(L, SEED, s0, e0, Tq, 0, 20 * N, False)
                rate_core = 20 * N / (time.perf_counter() - tc)
                spc_cpu = max(1, int(args.prod_seconds * rate_core / (chunks * N)))
                jobs = [(L, SEED, w, 1, list(lnW), max(100, chunks * spc_cpu // 5), chunks, spc_cpu)
                        for w in range(cores)]
                tc = time.perf_counter()
                with mp.get_context("spawn").Pool(cores) as pool:
                    parts = pool.map(_oracle_production_shard, jobs)
                cpu_s = time.perf_counter() - tc
                Hc = np.sum(np.stack(parts), axis=0).astype(np.uint64)
                g_c, err_c = oracle.jackknife(L, lnW, Hc)
                both = np.isfinite(exact) & (err > 0) & (err_c > 0) & np.isfinite(err) & np.isfinite(err_c)
                res["cpu"] = summary(g_c, err_c, exact)
                res["cpu"].update({"walkers": cores, "cores": cores, "sweeps_per_chunk": spc_cpu, "seconds": cpu_s})
                res["statistical_gain_eps2"] = float(np.mean(err_c[both] ** 2 / err[both] ** 2)) if both.any() else None
            out[f"L{L}"] = res
    print(json.dumps({
        "metric": "ln g accuracy from a fixed-time production run (jackknife eps vs exact Delta)",
        "value": out["L32"]["gpu"]["max_delta"], "unit": "max |Delta ln g|", "higher_is_better": False,
        "n_gpus": 1, "production": out, "clocks": clocks.summary(),
        "data": "synthetic: random +/-1 start, weights iterated from ln W = 0",
        "config": {"workload": "production_L16_L32_L64", "seconds_per_L": args.prod_seconds,
                   "walkers": "full occupancy (Sec. 3.1 rule)", "chunks": chunks,
                   "stop_rule": "min/mean >= 0.8"}}))


def run_traces_workload(args):
    """Convergence traces of the weight iteration against the thermalization factor (the
    protocol of Fig. A.1): L = 32, 26624 walkers, Eq. (7) schedule with f_therm in
    {5, 10, 20, 30, 50}, stop at d_k < 1e-4; per iteration the Kullback-Leibler divergence
    d_k (Eq. (6), the stop metric) and the Chebyshev distance d_c (Eq. (A.1)) of the
    recorded histogram."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00919_gb300 import muca as M
    L, W = 32, 26624
    N = L * L
    acc = np.ones(N + 1, dtype=bool)
    acc[[1, N - 1]] = False
    stream = torch.cuda.Stream()
    out = {}
    for f in (5, 10, 20, 30, 50):
        dk, dc = [], []

        def observe(it, H, metric, n_therm, n_upd):
            dk.append(metric)
            m = H.sum() / (N - 1)
            dc.append(float(np.max(np.abs(H[acc] / m - 1.0))) if m > 0 else float("inf"))
        with M.Muca(L, W, SEED, stream=stream) as m:
            m.set_iteration_observer(observe)
            t0 = time.perf_counter()
            st = m.iterate_until_flat(M.make_params(schedule=M.MUCA_SCHEDULE_PAPER, stop_rule=M.MUCA_STOP_KL,
                                                    flat_threshold=1e-4, f_therm=float(f), max_iterations=3000))
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
        out[f"f_therm_{f}"] = {"iterations": st.iterations, "converged": bool(st.converged), "seconds": secs,
                               "attempts_per_walker": st.attempts_per_walker,
                               "d_k": [float(f"{v:.4g}") for v in dk], "d_c": [float(f"{v:.4g}") for v in dc],
                               "first_iteration_d_c_below_0.05":
                                   next((i + 1 for i, v in enumerate(dc) if v < 0.05), None)}
    print(json.dumps({
        "metric": "convergence traces d_k and d_c per iteration against f_therm",
        "value": out["f_therm_30"]["iterations"], "unit": "iterations", "higher_is_better": False, "n_gpus": 1,
        "traces": out, "data": "synthetic: random +/-1 start, ln W = 0",
        "config": {"workload": "convergence_traces_L32_W26624", "L": L, "walkers": W,
                   "schedule": "Eq. (7)", "stop_rule": "d_k < 1e-4"}}))


def run_convergence_workload(args):
    """Iterations and time until the weights converge against the walker count (the
    protocol of Figs. 3 and 4, Sec. 3.2): Eq. (7) schedule, stop when d_k < 1e-4
    (Eq. (6)), from ln W = 0, `--seeds` independent seeds per point; mean, standard error
    and median of each."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00919_gb300 import muca as M
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    # The first walker count of each size is the reference of the algorithmic speedup of
    # Fig. 6 (the paper's is its 24-thread CPU run; W = 24 is affordable at L = 16 only:
    # its update count starts large and grows by 1.1 per iteration once the range is
    # covered; fewer seeds there, one warp runs the whole simulation)
    cases = {16: [24, 1024, 2048, 4096, 8192, 16384, 32768], 32: [4096, 8192, 16384, 32768, 65536]}
    params = M.make_params(schedule=M.MUCA_SCHEDULE_PAPER, stop_rule=M.MUCA_STOP_KL, flat_threshold=1e-4,
                           max_iterations=3000)
    out = {}
    with ClockSampler(dev) as clocks:
        for L, Ws in cases.items():
            rows = []
            for W in Ws:
                its, secs, atts, conv = [], [], [], 0
                per_walker = []
                n_seeds = args.seeds if W > 24 else min(args.seeds, 8)
                for seed in range(1, n_seeds + 1):
                    with M.Muca(L, W, seed, stream=stream) as m:
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        st = m.iterate_until_flat(params)
                        torch.cuda.synchronize()
                        secs.append(time.perf_counter() - t0)
                    its.append(st.iterations)
                    atts.append(st.attempts_per_walker * W)
                    per_walker.append(st.attempts_per_walker)
                    conv += int(st.converged)

                def stats(v):
                    v = np.asarray(v, dtype=np.float64)
                    return {"mean": float(v.mean()), "err": float(v.std(ddof=1) / math.sqrt(len(v))) if len(v) > 1
                            else 0.0, "median": float(np.median(v))}
                rows.append({"walkers": W, "iterations": stats(its), "seconds": stats(secs),
                             "attempts": stats(atts), "attempts_per_walker": stats(per_walker),
                             "converged": conv, "runs": n_seeds})
            # Fig. 6: algorithmic speedup N_ref / N_W of the attempts per walker (medians)
            ref = rows[0]
            for r in rows:
                r["algorithmic_speedup"] = ref["attempts_per_walker"]["median"] / r["attempts_per_walker"]["median"]
                r["ideal_speedup"] = r["walkers"] / ref["walkers"]
                r["speedup_reference_walkers"] = ref["walkers"]
            out[f"L{L}"] = rows
    l32 = {r["walkers"]: r for r in out["L32"]}
    print(json.dumps({
        "metric": "time until converged weights vs walkers (Eq. (7) schedule, d_k < 1e-4)",
        "value": l32[16384]["seconds"]["mean"], "unit": "s", "higher_is_better": False, "n_gpus": 1,
        "convergence": out, "clocks": clocks.summary(),
        "data": "synthetic: random +/-1 start per seed, ln W = 0",
        "config": {"workload": "convergence_vs_walkers_L16_L32", "seeds": args.seeds,
                   "schedule": "Eq. (7): N_therm = 30 w, N_upd = floor(6 w^2.25 / W) + 1, x1.1 after full range",
                   "stop_rule": "Kullback-Leibler d_k < 1e-4", "max_iterations": 3000}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-time-to-flat", action="store_true",
                    help="skip the oracle's whole weight iteration (about a minute on 16 host cores)")
    ap.add_argument("--workload", choices=["headline", "batch", "serve", "fliptime", "convergence", "production",
                                           "traces"],
                    default="headline")
    ap.add_argument("--seeds", type=int, default=32)
    ap.add_argument("--prod-seconds", type=float, default=10.0)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    args = ap.parse_args()
    if args.workload == "batch":
        run_batch_workload(args)
        return
    if args.workload == "serve":
        run_serve_workload(args)
        return
    if args.workload == "fliptime":
        run_fliptime_workload(args)
        return
    if args.workload == "convergence":
        run_convergence_workload(args)
        return
    if args.workload == "production":
        run_production_workload(args)
        return
    if args.workload == "traces":
        run_traces_workload(args)
        return
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
