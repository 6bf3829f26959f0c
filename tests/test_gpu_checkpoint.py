"""Checkpoint and resume (the state is lattices, energies, ln W, histogram, attempt
counter and site order; the random numbers are a function of seed, walker and counter,
Sec. 2.3): a restored instance continues bit for bit as the saved one; lattices set from
the host get their energies recomputed; attempt counters beyond 2^32 blocks (the high
counter word of Philox) match the oracle."""
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


def e_index(L, s):
    g = s.reshape(L, L).astype(np.int64)
    E = -(g * np.roll(g, -1, 1)).sum() - (g * np.roll(g, -1, 0)).sum()
    return int((E + 2 * L * L) // 4)


def snapshot(m):
    return (m.get_lattice(), m.get_energies(), m.get_weights(), m.get_histogram(), m.info()[2], m.site_order)


@pytest.mark.parametrize("L,W,layout,order", [(32, 300, 0, 0), (64, 70, 1, 0), (16, 130, 0, 1)])
def test_resume_is_bit_exact(muca_mod, tmp_path, L, W, layout, order):
    M = muca_mod
    rng = np.random.default_rng(L)
    lnW = np.cumsum(rng.normal(0, 0.3, L * L + 1))
    p = M.make_params(therm_sweeps=2, sweeps_per_iter=3, max_iterations=3)
    path = str(tmp_path / "state.muca")
    with M.Muca(L, W, 9, layout=layout) as a:
        a.site_order = order
        a.set_weights(lnW)
        a.sweep(2, False)
        a.reset_histogram()
        a.attempts(L * L + 5, True)            # save in the middle of a sweep
        a.save(path)
        before = snapshot(a)
        with M.Muca.load(path) as b:
            for x, y in zip(before, snapshot(b)):
                assert np.array_equal(x, y)
            for m in (a, b):
                m.attempts(2 * L * L + 7, True)
                m.iterate_until_flat(p)
            for x, y in zip(snapshot(a), snapshot(b)):
                assert np.array_equal(x, y)


@pytest.mark.parametrize("L,order", [(32, 0), (12, 0), (32, 1)])
def test_set_lattice_and_large_counter(muca_mod, orc, L, order):
    M = muca_mod
    N = L * L
    W, seed = 77, 2 ** 63 + 11
    rng = np.random.default_rng(5)
    spins = np.where(rng.random((W, N)) < 0.3, -1, 1).astype(np.int8)
    lnW = np.cumsum(rng.normal(0, 0.3, N + 1))
    t0 = 2 ** 40 + (0 if L == 32 and order == 0 else 12345)   # whole sweeps, or a ragged start
    with M.Muca(L, W, seed) as m:
        m.site_order = order
        m.set_lattice(spins)
        assert np.array_equal(m.get_lattice(), spins)
        assert all(m.get_energies()[w] == e_index(L, spins[w]) for w in range(W))
        m.set_attempt_counter(t0)
        m.set_weights(lnW)
        m.attempts(3 * N, True)
        H, e, lat = m.get_histogram(), m.get_energies(), m.get_lattice()
        assert m.info()[2] == t0 + 3 * N
    s = spins.copy()
    eo = np.array([e_index(L, s[w]) for w in range(W)], dtype=np.int32)
    Ho = orc.run(L, seed, s, eo, orc.build_table(L, lnW), t0, 3 * N, True, site_order=order)
    assert np.array_equal(lat, s) and np.array_equal(e, eo) and np.array_equal(H, Ho)


def test_bad_lattice_rejected(muca_mod):
    M = muca_mod
    with M.Muca(8, 4, 1) as m:
        bad = np.ones((4, 64), dtype=np.int8)
        bad[2, 5] = 0
        with pytest.raises(M.MucaError):
            m.set_lattice(bad)
        with pytest.raises(M.MucaError):
            m.set_lattice(np.ones((4, 63), dtype=np.int8))


@pytest.mark.parametrize("schedule", ["paper", "sweeps"])
def test_iteration_resumes_across_calls_and_checkpoints(muca_mod, tmp_path, schedule):
    """A weight iteration cut by max_iterations continues, with params.resume, as one
    uninterrupted call: the same N_therm / N_updates sequence of Sec. 3, the same
    Kullback-Leibler reference width, the same weights bit for bit, in the same instance
    or in one restored from a checkpoint.  Without resume the schedule starts afresh."""
    M = muca_mod
    L, W, seed = 8, 128, 4
    if schedule == "paper":
        kw = dict(schedule=M.MUCA_SCHEDULE_PAPER, stop_rule=M.MUCA_STOP_KL, flat_threshold=1e-4)
    else:
        kw = dict(stop_rule=M.MUCA_STOP_KL, flat_threshold=0.01, therm_sweeps=31, sweeps_per_iter=100)
    p_all = M.make_params(max_iterations=3000, **kw)

    def run(m, p, log):
        m.set_iteration_observer(lambda it, H, metric, nt, nu: log.append((nt, nu, metric)))
        st = m.iterate_until_flat(p)
        m.set_iteration_observer(None)
        return st

    whole = []
    with M.Muca(L, W, seed) as m:
        st = run(m, p_all, whole)
        ref = (m.get_weights(), m.info()[2])
    assert st.converged and st.iterations >= 4
    k = st.iterations // 2
    p_cut = M.make_params(max_iterations=k, **kw)
    p_resume = M.make_params(max_iterations=3000, resume=True, **kw)
    path = str(tmp_path / "cut.muca")
    for restore in (False, True):
        log = []
        with M.Muca(L, W, seed) as m:
            first = run(m, p_cut, log)
            assert not first.converged and first.iterations == k
            m.save(path)
            if restore:
                with M.Muca.load(path) as r:
                    second = run(r, p_resume, log)
                    got = (r.get_weights(), r.info()[2])
            else:
                second = run(m, p_resume, log)
                got = (m.get_weights(), m.info()[2])
        assert second.converged and k + second.iterations == st.iterations
        assert log == whole
        assert np.array_equal(got[0], ref[0]) and got[1] == ref[1]
    fresh = []
    with M.Muca.load(path) as r:
        run(r, M.make_params(max_iterations=1, **kw), fresh)
    if schedule == "paper":
        assert fresh[0][:2] != whole[k][:2]      # N_therm, N_updates of w = 10 again
    else:
        assert fresh[0][:2] == whole[k][:2]      # fixed sweeps; only the KL reference differs


@pytest.mark.parametrize("mode", ["device", "batch"])
def test_device_and_batched_iterations_resume(muca_mod, tmp_path, mode):
    """The device-side and the batched iteration (fixed sweeps, Kullback-Leibler stop of
    Eq. (6), whose reference width comes from the previous iteration's range) cut by
    max_iterations and continued with params.resume, also after a checkpoint, equal one
    uninterrupted run: iterations, stop metric, weights and attempt counter."""
    M = muca_mod
    L, seeds = 8, (4, 5)
    kw = dict(stop_rule=M.MUCA_STOP_KL, flat_threshold=0.01, therm_sweeps=31, sweeps_per_iter=100)

    def run(ms, p):
        if mode == "device":
            return [m.iterate_device(p, 3) for m in ms]
        with M.Batch(ms) as b:
            return b.iterate_until_flat(p)[1]

    def fresh():
        return [M.Muca(L, 128, s) for s in seeds]

    whole = fresh()
    st = run(whole, M.make_params(max_iterations=3000, **kw))
    ref = [(m.get_weights(), m.info()[2]) for m in whole]
    assert all(s.converged and s.iterations >= 4 for s in st)
    for m in whole:
        m.close()
    k = min(s.iterations for s in st) // 2
    path = [str(tmp_path / f"cut{i}.muca") for i in range(len(seeds))]
    for restore in (False, True):
        ms = fresh()
        first = run(ms, M.make_params(max_iterations=k, **kw))
        assert all(not s.converged and s.iterations == k for s in first)
        if restore:
            for m, pth in zip(ms, path):
                m.save(pth)
                m.close()
            ms = [M.Muca.load(pth) for pth in path]
        second = run(ms, M.make_params(max_iterations=3000, resume=True, **kw))
        for m, s_all, s2, (w, t) in zip(ms, st, second, ref):
            assert s2.converged and k + s2.iterations == s_all.iterations
            assert s2.last_metric == s_all.last_metric
            assert np.array_equal(m.get_weights(), w) and m.info()[2] == t
        for m in ms:
            m.close()


def test_earlier_format_loads_with_a_fresh_schedule(muca_mod, tmp_path):
    """A file of the earlier format (magic MUCACKP1, no iteration state after the header)
    restores the same lattices, energies, weights, histogram and counter, with the
    iteration state of a new instance."""
    M = muca_mod
    L, W = 16, 70
    lnW = np.cumsum(np.random.default_rng(3).normal(0, 0.3, L * L + 1))
    v2, v1 = str(tmp_path / "v2.muca"), str(tmp_path / "v1.muca")
    with M.Muca(L, W, 5) as a:
        a.set_weights(lnW)
        a.iterate_until_flat(M.make_params(therm_sweeps=2, sweeps_per_iter=3, max_iterations=2))
        a.save(v2)
        ref = snapshot(a)
    raw = open(v2, "rb").read()
    head = 8 + 4 + 4 + 8 + 8 + 4 + 4 + 8 + 8          # magic .. first_walker
    assert raw[:8] == b"MUCACKP2"
    open(v1, "wb").write(b"MUCACKP1" + raw[8:head] + raw[head + 4 * 4 + 8:])
    with M.Muca.load(v1) as b:
        for x, y in zip(ref, snapshot(b)):
            assert np.array_equal(x, y)
        log = []
        b.set_iteration_observer(lambda it, H, metric, nt, nu: log.append(nu))
        b.iterate_until_flat(M.make_params(schedule=M.MUCA_SCHEDULE_PAPER, stop_rule=M.MUCA_STOP_KL,
                                           flat_threshold=1e-4, max_iterations=1, resume=True))
        b.set_iteration_observer(None)
    # a fresh state: w' = 0, so the first N_updates is Eq. (7) at w = 10
    assert log == [int(np.floor(6.0 * 10 ** 2.25 / W)) + 1]
