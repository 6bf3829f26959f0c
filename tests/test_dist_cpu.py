"""The method's one exchange step (Sec. 2.2: histograms of independent walkers are
summed, the new weights are redistributed) across processes: world size 2 with gloo on
the CPU, each rank advancing its share of the walkers with the oracle.  The all-reduced
histograms and the weights after every iteration must equal the single-process run
(walker-keyed random streams make the split invisible)."""
import os
import socket

import numpy as np
import pytest

L, W, SEED, ITERS = 8, 48, 5, 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from oracle import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N = L * L
    share = W // world
    s, e = oracle.init(L, SEED, share, walker0=rank * share)
    lnW = np.zeros(N + 1)
    t = 0
    hist = []
    for _ in range(ITERS):
        T = oracle.build_table(L, lnW)
        oracle.run(L, SEED, s, e, T, t, 3 * N, False, None, walker0=rank * share)
        t += 3 * N
        H = oracle.run(L, SEED, s, e, T, t, 5 * N, True, None, walker0=rank * share)
        t += 5 * N
        Ht = torch.from_numpy(H.astype(np.int64))
        dist.all_reduce(Ht, op=dist.ReduceOp.SUM)
        H = Ht.numpy().astype(np.uint64)
        hist.append(H)
        oracle.update_weights(L, lnW, H)
    np.save(os.path.join(out_dir, f"lnW_{rank}.npy"), lnW)
    np.save(os.path.join(out_dir, f"H_{rank}.npy"), np.array(hist))
    dist.destroy_process_group()


def test_sharded_walkers_match_single_process(tmp_path, orc):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    port = _free_port()
    tmp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    N = L * L
    s, e = orc.init(L, SEED, W)
    lnW = np.zeros(N + 1)
    t = 0
    ref_hist = []
    for _ in range(ITERS):
        T = orc.build_table(L, lnW)
        orc.run(L, SEED, s, e, T, t, 3 * N, False)
        t += 3 * N
        H = orc.run(L, SEED, s, e, T, t, 5 * N, True)
        t += 5 * N
        ref_hist.append(H)
        orc.update_weights(L, lnW, H)
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / f"H_{r}.npy"), np.array(ref_hist))
        assert np.array_equal(np.load(tmp_path / f"lnW_{r}.npy"), lnW)


def _bench_rank_main(rank, world, port, out_dir):
    """The benchmark's multi-rank plumbing (rank discovery from the environment, gloo
    group, barrier, max over ranks) as torchrun would drive it."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    ws, r, local = bench.dist_env()
    dist = bench.init_dist(ws)
    bench.barrier(dist)
    value = bench.max_over_ranks(dist, 1.5 + r)
    with open(os.path.join(out_dir, f"max_{rank}.txt"), "w") as f:
        f.write(f"{ws} {r} {local} {value}")
    dist.destroy_process_group()


def test_bench_plumbing_two_ranks(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    port = _free_port()
    tmp.spawn(_bench_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        ws, rank, local, value = (tmp_path / f"max_{r}.txt").read_text().split()
        assert (int(ws), int(rank), int(local)) == (2, r, r)
        assert float(value) == 2.5           # every rank sees the slowest rank's time


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the oracle timed on the host cores, no GPU) prints one
    JSON line with the contract's keys: metric, value, unit, steps, warmup, the oracle as
    cpu_baseline (kind, cores, sample) and an e2e object without host-device traffic."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=root, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "attempts/s" and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["L"] == 32 and d["config"]["walkers"] == 16384


def test_cpu_time_to_flat_is_the_oracle_iteration(orc):
    """The benchmark's CPU time-to-flat (walkers sharded over host processes, histograms
    summed, the oracle's flatness test and Eq. (4) recursion on the host) runs exactly
    the oracle's own weight iteration: the same iteration count and the same final
    weights bit for bit (here L = 8, 128 walkers, 31 + 100 sweeps per iteration)."""
    import numpy as np
    import bench
    saved = (bench.L_SIDE, bench.WALKERS, bench.SWEEPS_PER_ITER)
    try:
        bench.L_SIDE, bench.WALKERS, bench.SWEEPS_PER_ITER = 8, 128, 100
        secs, its, conv, lnW, procs = bench.cpu_time_to_flat(128, cores=3, max_iterations=200)
    finally:
        bench.L_SIDE, bench.WALKERS, bench.SWEEPS_PER_ITER = saved
    s, e = orc.init(8, bench.SEED, 128)
    ref = np.zeros(65)
    p = orc.make_params(schedule=0, stop_rule=0, flat_threshold=0.8, therm_sweeps=bench.THERM_SWEEPS,
                        sweeps_per_iter=100, max_iterations=200)
    res, _, _, _ = orc.iterate(8, bench.SEED, s, e, ref, 0, p)
    assert conv and res.converged == 1 and its == res.iterations and procs == 3
    assert np.array_equal(lnW, ref)
