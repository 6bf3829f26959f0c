"""One rank of a simulation sharded over processes (helper of test_gpu_sharded_procs.py):
the rank holds walkers [rank * W / world, ...) of one simulation (first_walker), sums its
histograms with the other ranks through torch.distributed (gloo) inside the library's
histogram reducer (Sec. 2.2), iterates to flat weights, runs a production, and writes
its weights, statistics and ln g to an .npz file.

usage: python sharded_rank.py RANK WORLD PORT OUT L W SEED SCHEDULE"""
import datetime
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    rank, world, port, out, L, W, seed, schedule = (int(sys.argv[1]), int(sys.argv[2]), sys.argv[3], sys.argv[4],
                                                    int(sys.argv[5]), int(sys.argv[6]), int(sys.argv[7]),
                                                    int(sys.argv[8]))
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = port
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    torch.cuda.set_device(0)
    from paper_1707_00919_gb300 import muca as M
    share = W // world
    w0 = rank * share
    nw = share if rank < world - 1 else W - w0
    if schedule == 0:
        p = M.make_params(therm_sweeps=31, sweeps_per_iter=100, max_iterations=300)
    else:
        p = M.make_params(schedule=M.MUCA_SCHEDULE_PAPER, stop_rule=M.MUCA_STOP_KL, flat_threshold=1e-4,
                          max_iterations=3000)

    def reduce(H):
        t = torch.from_numpy(H.astype(np.int64))
        dist.all_reduce(t)
        H[:] = t.numpy().astype(np.uint64)

    with M.Muca(L, nw, seed, first_walker=w0) as m:
        m.set_histogram_reducer(reduce, total_walkers=W)
        st = m.iterate_until_flat(p)
        H, g = m.production(31, 500)
        np.savez(out, lnW=m.get_weights(), iterations=st.iterations, metric=st.last_metric,
                 converged=st.converged, H=H, g=g, lattice=m.get_lattice())
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
