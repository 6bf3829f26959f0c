"""The batched persistent kernel (many instances of uneven L and walker count in one
launch, per-instance tables and histograms) against the oracle, and the batched weight
iteration (one CUDA graph per iteration) against the same instances iterated alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00919_gb300 import muca
    return muca


def weights(L, seed, scale=0.4):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.normal(0.0, scale, L * L + 1))


def oracle_advance(orc, L, W, seed, lnW, plan, walkers=None):
    """plan: list of (attempts, record); returns (spins, e, H) for the chosen walkers."""
    N = L * L
    T = orc.build_table(L, lnW)
    H = np.zeros(N + 1, dtype=np.uint64)
    if walkers is None:
        s, e = orc.init(L, seed, W)
        t = 0
        for n, rec in plan:
            orc.run(L, seed, s, e, T, t, n, rec, H if rec else None)
            t += n
        return s, e, H
    out_s, out_e = [], []
    for w in walkers:
        s, e = orc.init(L, seed, 1, walker0=w)
        t = 0
        for n, rec in plan:
            orc.run(L, seed, s, e, T, t, n, False, None, walker0=w)
            t += n
        out_s.append(s[0])
        out_e.append(e[0])
    return np.array(out_s), np.array(out_e), None


def test_batch_sweep_bit_exact_mixed(M, orc):
    specs = [(8, 33, 0), (16, 97, 1), (24, 300, 0), (32, 129, 1), (48, 65, 0), (64, 40, 1)]
    inst = []
    for i, (L, W, lay) in enumerate(specs):
        m = M.Muca(L, W, 100 + i, layout=lay)
        m.set_weights(weights(L, i))
        inst.append(m)
    with M.Batch(inst) as b:
        b.sweep(2, record=False)
        for m in inst:
            m.reset_histogram()
        b.sweep(3, record=True)
        res = [(m.get_lattice(), m.get_energies(), m.get_histogram(), m.attempt_counter) for m in inst]
    for i, (L, W, lay) in enumerate(specs):
        N = L * L
        s, e, H = oracle_advance(orc, L, W, 100 + i, weights(L, i), [(2 * N, False), (3 * N, True)])
        lat, ed, Hd, t = res[i]
        assert t == 5 * N
        assert np.array_equal(lat, s), (L, W)
        assert np.array_equal(ed, e), (L, W)
        assert np.array_equal(Hd, H), (L, W)
    for m in inst:
        m.close()


def test_batch_iterate_equals_single(M):
    specs = [(8, 128, 1), (8, 256, 2), (16, 512, 3), (16, 1024, 4), (24, 1024, 5)]
    p = M.make_params(therm_sweeps=31, sweeps_per_iter=100, max_iterations=300)
    alone = []
    for L, W, seed in specs:
        with M.Muca(L, W, seed) as m:
            st = m.iterate_until_flat(p)
            alone.append((st, m.get_weights(), m.get_energies(), m.attempt_counter))
    inst = [M.Muca(L, W, seed) for L, W, seed in specs]
    with M.Batch(inst) as b:
        rc, stats = b.iterate_until_flat(p)
    assert rc == (0 if all(a[0].converged for a in alone) else M.C.MUCA_ENOTCONVERGED)
    assert sum(a[0].converged for a in alone) >= 3
    for i, m in enumerate(inst):
        st, lnW, e, t = alone[i]
        assert stats[i].iterations == st.iterations and stats[i].converged == st.converged
        assert stats[i].last_metric == st.last_metric
        assert np.array_equal(m.get_weights(), lnW)
        assert np.array_equal(m.get_energies(), e)
        assert m.attempt_counter == t
        m.close()


def test_config4_mix_sampled_walkers(M, orc):
    """24 instances, L drawn from {16, 24, 32, 48, 64} and walker counts uniformly from
    512..16384 (seed 1234), instance seeds 1234 + index: one batched thermalization and
    one recorded sweep; sampled walkers of every instance match the oracle exactly and
    every histogram holds W N counts."""
    rng = np.random.default_rng(1234)
    Ls = rng.choice([16, 24, 32, 48, 64], size=24)
    Ws = rng.integers(512, 16385, size=24)
    inst = []
    for i, (L, W) in enumerate(zip(Ls, Ws)):
        m = M.Muca(int(L), int(W), 1234 + i, layout=i % 2)
        m.set_weights(weights(int(L), 50 + i, 0.05))
        inst.append(m)
    with M.Batch(inst) as b:
        b.sweep(1, record=False)
        b.sweep(1, record=True)
        out = [(m.get_lattice(), m.get_energies(), m.get_histogram()) for m in inst]
    for i, (L, W) in enumerate(zip(Ls, Ws)):
        L, W = int(L), int(W)
        N = L * L
        lat, e, H = out[i]
        assert int(H.sum()) == W * N
        pick = [0, W // 2, W - 1]
        s, eo, _ = oracle_advance(orc, L, W, 1234 + i, weights(L, 50 + i, 0.05), [(N, False), (N, True)], pick)
        assert np.array_equal(lat[pick], s) and np.array_equal(e[pick], eo), (i, L, W)
    for m in inst:
        m.close()


@pytest.mark.parametrize("stop_rule,threshold", [(0, 0.8), (1, 1e-4)])
def test_batch_iterate_paper_schedule_equals_single(M, stop_rule, threshold):
    """Eq. (7) schedule (Sec. 3) in the batched iteration: every member follows its own
    visited ranges, its thermalization and recording launches start and end inside
    sweeps, and each member's iteration count, stop metric, weights, energies and
    attempt counter equal the instance iterated alone."""
    specs = [(8, 128, 11), (16, 256, 12), (8, 64, 13), (24, 512, 14), (16, 1024, 15)]
    if stop_rule == 0:   # the 6-word table rows of L = 64 items and L = 48 as well
        specs += [(64, 1024, 16), (48, 256, 17), (32, 256, 18)]
    p = M.make_params(schedule=M.MUCA_SCHEDULE_PAPER, stop_rule=stop_rule, flat_threshold=threshold,
                      max_iterations=400)
    alone = []
    for L, W, seed in specs:
        with M.Muca(L, W, seed) as m:
            st = m.iterate_until_flat(p)
            alone.append((st, m.get_weights(), m.get_energies(), m.attempt_counter))
    inst = [M.Muca(L, W, seed) for L, W, seed in specs]
    with M.Batch(inst) as b:
        rc, stats = b.iterate_until_flat(p)
    for i, m in enumerate(inst):
        st, lnW, e, t = alone[i]
        assert t % (specs[i][0] ** 2) != 0 or st.iterations > 0
        assert stats[i].iterations == st.iterations and stats[i].converged == st.converged, i
        assert stats[i].last_metric == st.last_metric
        assert stats[i].attempts_per_walker == st.attempts_per_walker
        assert np.array_equal(m.get_weights(), lnW)
        assert np.array_equal(m.get_energies(), e)
        assert m.attempt_counter == t
        m.close()


def test_batch_iteration_longer_than_one_recording_launch(M):
    """Members that record more than 0xFFFFFFFF / 256 attempts per walker in one
    iteration (the 32-bit per-block counts of one launch) run several recording launches
    per iteration, of different lengths for members whose counts end at different
    points; each member equals its instance iterated alone."""
    specs = [(8, 32, 21), (8, 64, 22)]
    p = M.make_params(therm_sweeps=31, sweeps_per_iter=262_200, max_iterations=2)
    alone = []
    for L, W, seed in specs:
        with M.Muca(L, W, seed) as m:
            st = m.iterate_until_flat(p)
            alone.append((st, m.get_weights(), m.get_energies(), m.get_lattice(), m.attempt_counter))
    inst = [M.Muca(L, W, seed) for L, W, seed in specs]
    with M.Batch(inst) as b:
        rc, stats = b.iterate_until_flat(p)
    for i, m in enumerate(inst):
        st, lnW, e, lat, t = alone[i]
        assert stats[i].iterations == st.iterations and stats[i].last_metric == st.last_metric
        assert np.array_equal(m.get_weights(), lnW) and np.array_equal(m.get_lattice(), lat)
        assert np.array_equal(m.get_energies(), e) and m.attempt_counter == t
        m.close()


def test_batch_sweep_from_inside_a_sweep(M, orc):
    """Members whose attempt counters lie inside a sweep (after partial launches of their
    own): a batched launch of whole sweeps then starts and ends inside a row for them, and
    every member equals the oracle."""
    specs = [(8, 40, 0, 5), (32, 70, 1, 1024 + 37), (64, 33, 0, 13), (24, 50, 1, 0)]
    inst = []
    for i, (L, W, lay, head) in enumerate(specs):
        m = M.Muca(L, W, 300 + i, layout=lay)
        m.set_weights(weights(L, 60 + i))
        if head:
            m.attempts(head, False)
        m.reset_histogram()
        inst.append(m)
    with M.Batch(inst) as b:
        b.sweep(2, record=True)
        res = [(m.get_lattice(), m.get_energies(), m.get_histogram(), m.attempt_counter) for m in inst]
    for i, (L, W, lay, head) in enumerate(specs):
        N = L * L
        plan = ([(head, False)] if head else []) + [(2 * N, True)]
        s, e, H = oracle_advance(orc, L, W, 300 + i, weights(L, 60 + i), plan)
        lat, ed, Hd, t = res[i]
        assert t == head + 2 * N
        assert np.array_equal(lat, s) and np.array_equal(ed, e) and np.array_equal(Hd, H), (L, W, lay)
    for m in inst:
        m.close()
