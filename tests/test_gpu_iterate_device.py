"""The weight iteration with its recursion, stop test and table build on the device
(muca_iterate_device) against the host-driven iteration and the oracle: iteration
counts, metrics, weights, tables, histograms, lattices, energies and attempt counters
bit for bit, for every stop rule, for runs that stop at the iteration limit, and for
every number of iterations enqueued per synchronisation."""
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


def state(m):
    info = m.info()
    return (m.get_weights(), m.get_histogram(), m.get_table(), m.get_energies(), m.get_lattice(), info[2])


def run_pair(M, L, W, seed, params, per_sync, layout=0):
    with M.Muca(L, W, seed, layout=layout) as a, M.Muca(L, W, seed, layout=layout) as b:
        sa = a.iterate_until_flat(params)
        sb = b.iterate_device(params, per_sync)
        A, B = state(a), state(b)
        # the instances go on identically afterwards
        a.sweep(2, True)
        b.sweep(2, True)
        after = np.array_equal(a.get_histogram(), b.get_histogram())
    return sa, sb, A, B, after


def assert_same(sa, sb, A, B, after):
    assert (sa.code, sa.iterations, sa.converged, sa.attempts_per_walker) == \
           (sb.code, sb.iterations, sb.converged, sb.attempts_per_walker)
    assert sa.last_metric == sb.last_metric or (np.isinf(sa.last_metric) and np.isinf(sb.last_metric))
    for x, y in zip(A, B):
        assert np.array_equal(x, y)
    assert after


@pytest.mark.parametrize("rule,thr", [(0, 0.8), (1, 0.01), (2, 0.3)])
@pytest.mark.parametrize("per_sync", [1, 3, 16])
def test_device_iteration_equals_host_iteration(muca_mod, rule, thr, per_sync):
    M = muca_mod
    p = M.make_params(stop_rule=rule, flat_threshold=thr, therm_sweeps=31, sweeps_per_iter=100, max_iterations=300)
    sa, sb, A, B, after = run_pair(M, 8, 128, 3, p, per_sync)
    assert sa.converged
    assert_same(sa, sb, A, B, after)


@pytest.mark.parametrize("L,W,layout", [(12, 64, 0), (32, 1024, 0), (64, 256, 1)])
def test_device_iteration_stops_at_the_limit(muca_mod, L, W, layout):
    M = muca_mod
    p = M.make_params(stop_rule=1, flat_threshold=1e-4, therm_sweeps=2, sweeps_per_iter=3, max_iterations=7)
    sa, sb, A, B, after = run_pair(M, L, W, 11, p, 4, layout)
    assert not sa.converged and sa.iterations == 7
    assert_same(sa, sb, A, B, after)


def test_device_iteration_matches_oracle(muca_mod, orc):
    """Configuration 1 (L = 8, 128 walkers, 100 sweeps per iteration, min/mean >= 0.8)
    run entirely on the device against the oracle's iteration."""
    M = muca_mod
    L, W, seed = 8, 128, 1
    N = L * L
    with M.Muca(L, W, seed) as m:
        st = m.iterate_device(M.make_params(therm_sweeps=31, sweeps_per_iter=100, max_iterations=200), 8)
        lnW = m.get_weights()
        e = m.get_energies()
        lat = m.get_lattice()
        t_dev = m.info()[2]
    s, eo = orc.init(L, seed, W)
    lnWo = np.zeros(N + 1)
    res, t, _, _ = orc.iterate(L, seed, s, eo, lnWo, 0,
                               orc.make_params(therm_sweeps=31, sweeps_per_iter=100, max_iterations=200))
    assert st.converged and res.converged == 1
    assert st.iterations == res.iterations and st.last_metric == res.last_metric
    assert np.array_equal(lnW, lnWo) and np.array_equal(e, eo) and np.array_equal(lat, s) and t_dev == t


def test_device_iteration_rejects_paper_schedule(muca_mod):
    M = muca_mod
    with M.Muca(8, 32, 1) as m:
        with pytest.raises(M.MucaError):
            m.iterate_device(M.make_params(schedule=M.MUCA_SCHEDULE_PAPER), 4, raise_on_fail=True)
        with pytest.raises(M.MucaError):
            m.iterate_device(M.make_params(), 0, raise_on_fail=True)


def test_iteration_observer(muca_mod, orc):
    """The observer sees every iteration once, in order, with the histogram the stop
    metric came from (its total is walkers x recorded attempts) and that metric; the
    oracle's metric history agrees."""
    M = muca_mod
    L, W, seed = 8, 128, 3
    N = L * L
    seen = []
    p = M.make_params(schedule=M.MUCA_SCHEDULE_PAPER, stop_rule=M.MUCA_STOP_KL, flat_threshold=1e-3,
                      max_iterations=400)
    with M.Muca(L, W, seed) as m:
        m.set_iteration_observer(lambda it, H, metric, nt, nu: seen.append((it, int(H.sum()), metric, nt, nu)))
        st = m.iterate_until_flat(p)
        m.set_iteration_observer(None)
    assert [s[0] for s in seen] == list(range(1, st.iterations + 1))
    assert all(total == W * nu for _, total, _, _, nu in seen)
    assert seen[-1][2] == st.last_metric
    assert sum(nt + nu for _, _, _, nt, nu in seen) == st.attempts_per_walker
    s, e = orc.init(L, seed, W)
    lnW = np.zeros(N + 1)
    res, _, _, mh = orc.iterate(L, seed, s, e, lnW, 0,
                                orc.make_params(schedule=1, stop_rule=1, flat_threshold=1e-3, max_iterations=400),
                                history=True)
    assert np.array_equal(np.array([x[2] for x in seen]), mh)
