"""One simulation sharded over two processes through the library (Sec. 2.2: walkers are
split, the histograms are summed before every weight update): each process holds a
walker range (first_walker) and sums its histograms with the other through a gloo
all-reduce inside muca_set_histogram_reducer.  Both ranks must reach the weights,
iteration count, stop metric, production histogram and ln g of one instance holding all
walkers, bit for bit, and their lattices must be that instance's walker ranges."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00919_gb300 import muca
    return muca


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return str(s.getsockname()[1])


@pytest.mark.parametrize("schedule", [0, 1])
def test_two_processes_equal_one_instance(M, tmp_path, schedule):
    L, W, seed, world = 8, 128, 4, 2
    if schedule == 0:
        p = M.make_params(therm_sweeps=31, sweeps_per_iter=100, max_iterations=300)
    else:
        p = M.make_params(schedule=M.MUCA_SCHEDULE_PAPER, stop_rule=M.MUCA_STOP_KL, flat_threshold=1e-4,
                          max_iterations=3000)
    with M.Muca(L, W, seed) as whole:
        sw = whole.iterate_until_flat(p)
        Hw, gw = whole.production(31, 500)
        lnWw, latw = whole.get_weights(), whole.get_lattice()
    port = free_port()
    outs = [str(tmp_path / f"rank{r}.npz") for r in range(world)]
    procs = [subprocess.Popen([sys.executable, os.path.join(HERE, "sharded_rank.py"), str(r), str(world), port,
                               outs[r], str(L), str(W), str(seed), str(schedule)],
                              stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
             for r in range(world)]
    logs = []
    try:
        for pr in procs:
            logs.append(pr.communicate(timeout=300)[0])
    finally:
        for pr in procs:
            if pr.poll() is None:
                pr.kill()
    assert all(pr.returncode == 0 for pr in procs), logs
    ranks = [np.load(o) for o in outs]
    assert sw.converged
    for r in ranks:
        assert bool(r["converged"]) and int(r["iterations"]) == sw.iterations
        assert float(r["metric"]) == sw.last_metric
        assert np.array_equal(r["lnW"], lnWw)
        assert np.array_equal(r["H"], Hw) and np.array_equal(r["g"], gw)
    assert np.array_equal(np.concatenate([r["lattice"] for r in ranks]), latw)
