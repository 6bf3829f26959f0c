"""One simulation spread over several instances (Sec. 2.2: the walkers' histograms are
summed before every weight update), as one instance per GPU would run it: instances
holding disjoint walker ranges (first_walker) reproduce the walkers of one instance
holding them all, and two instances iterated in two host threads with a summing
histogram reducer reach the same weights, iteration count and production estimate as
the single instance, bit for bit."""
import threading

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def muca_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00919_gb300 import muca
    return muca


class SumReducer:
    """All-reduce (sum) of the histograms of n instances iterated in n host threads."""

    def __init__(self, n):
        self.bar = threading.Barrier(n, timeout=120)
        self.parts = [None] * n
        self.total = None

    def member(self, i):
        def fn(H):
            self.parts[i] = H.copy()
            if self.bar.wait() == 0:
                self.total = np.sum(self.parts, axis=0, dtype=np.uint64)
            self.bar.wait()
            H[:] = self.total
            self.bar.wait()
        return fn


def run_threads(*jobs):
    out = [None] * len(jobs)
    errors = []

    def wrap(i, job):
        try:
            out[i] = job()
        except Exception as exc:   # surfaced below
            errors.append(exc)
    threads = [threading.Thread(target=wrap, args=(i, j)) for i, j in enumerate(jobs)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    return out


@pytest.mark.parametrize("L,layout,order", [(8, 0, 0), (32, 1, 0), (16, 0, 1)])
def test_walker_ranges_reproduce_one_instance(muca_mod, L, layout, order):
    M = muca_mod
    N = L * L
    lnW = np.cumsum(np.random.default_rng(L).normal(0, 0.3, N + 1))
    with M.Muca(L, 96, 7, layout=layout) as whole, M.Muca(L, 40, 7, layout=layout) as a, \
            M.Muca(L, 56, 7, layout=layout, first_walker=40) as b:
        for m in (whole, a, b):
            m.site_order = order
            m.set_weights(lnW)
            m.sweep(2, False)
            m.reset_histogram()
            m.attempts(N + 5, True)
        assert np.array_equal(whole.get_lattice(), np.concatenate([a.get_lattice(), b.get_lattice()]))
        assert np.array_equal(whole.get_energies(), np.concatenate([a.get_energies(), b.get_energies()]))
        assert np.array_equal(whole.get_histogram(), a.get_histogram() + b.get_histogram())


@pytest.mark.parametrize("schedule", [0, 1])
def test_sharded_iteration_and_production(muca_mod, schedule):
    M = muca_mod
    L, seed = 8, 4
    if schedule == 0:
        p = M.make_params(therm_sweeps=31, sweeps_per_iter=100, max_iterations=300)
    else:
        p = M.make_params(schedule=M.MUCA_SCHEDULE_PAPER, stop_rule=M.MUCA_STOP_KL, flat_threshold=1e-4,
                          max_iterations=3000)
    with M.Muca(L, 128, seed) as whole:
        sw = whole.iterate_until_flat(p)
        Hw, gw = whole.production(31, 500)
        lnWw = whole.get_weights()
    red = SumReducer(2)
    with M.Muca(L, 48, seed) as a, M.Muca(L, 80, seed, first_walker=48) as b:
        a.set_histogram_reducer(red.member(0), total_walkers=128)
        b.set_histogram_reducer(red.member(1), total_walkers=128)
        sa, sb = run_threads(lambda: a.iterate_until_flat(p), lambda: b.iterate_until_flat(p))
        (Ha, ga), (Hb, gb) = run_threads(lambda: a.production(31, 500), lambda: b.production(31, 500))
        wa, wb = a.get_weights(), b.get_weights()
        with pytest.raises(M.MucaError):
            a.iterate_device(p if schedule == 0 else M.make_params(), 4, raise_on_fail=True)
    assert sw.converged and sa.converged and sb.converged
    assert sw.iterations == sa.iterations == sb.iterations
    assert sw.last_metric == sa.last_metric == sb.last_metric
    assert np.array_equal(lnWw, wa) and np.array_equal(lnWw, wb)
    assert np.array_equal(Hw, Ha) and np.array_equal(Hw, Hb)
    assert np.array_equal(gw, ga) and np.array_equal(gw, gb)


def test_first_walker_range_checked(muca_mod):
    M = muca_mod
    with pytest.raises(M.MucaError):
        M.Muca(8, 16, 1, first_walker=2 ** 31 - 10)
    with pytest.raises(M.MucaError):
        M.Muca(8, 16, 1, first_walker=-1)
    with M.Muca(8, 16, 1) as m:
        with pytest.raises(M.MucaError):
            m.set_histogram_reducer(lambda H: None, total_walkers=8)
