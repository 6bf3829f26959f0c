"""Parity of the CUDA path (through the C ABI) with the oracle, element by element on
the same seeded inputs: Philox words, initial lattices, thresholds, lattices / energies /
histograms after updates (bit-exact, integer work), the weight iteration (ln W bitwise,
FP64 host recursion on identical histograms) and the production estimate."""
import numpy as np
import pytest

from conftest import load_exact_ln_dos

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


def rand_weights(L, seed, scale=0.4):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.normal(0.0, scale, L * L + 1))


def e_index(L, s):
    g = s.reshape(L, L).astype(np.int64)
    E = -(g * np.roll(g, -1, 1)).sum() - (g * np.roll(g, -1, 0)).sum()
    return int((E + 2 * L * L) // 4)


def test_device_philox_matches_oracle(muca_mod, orc):
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**32, size=(512, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    key = np.array([0x12345678, 0x9ABCDEF0], dtype=np.uint32)
    got = muca_mod.muca_philox(ctr, key)
    want = np.array([orc.philox4x32_10(c, key) for c in ctr])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("L,W", [(4, 5), (8, 200), (32, 100), (48, 70), (64, 33)])
def test_init_matches_oracle(muca_mod, orc, layout, L, W):
    with muca_mod.Muca(L, W, 1234, layout=layout) as m:
        lat = m.get_lattice()
        e = m.get_energies()
    s, eo = orc.init(L, 1234, W)
    assert np.array_equal(lat, s)
    assert np.array_equal(e, eo)


def test_table_matches_oracle(muca_mod, orc):
    L = 16
    lnW = rand_weights(L, 5, 3.0)
    lnW[10] = lnW[12] - 1e-18                     # exp rounds to 1.0
    lnW[40] = lnW[42] + 70.0                      # threshold underflows to 0
    with muca_mod.Muca(L, 32, 1) as m:
        m.set_weights(lnW)
        T = m.get_table()
        assert np.array_equal(m.get_weights(), lnW)
    assert np.array_equal(T, orc.build_table(L, lnW))


@pytest.mark.parametrize("L", [4, 8, 24, 64])
def test_device_table_equals_host_and_oracle(muca_mod, orc, L):
    """muca_set_weights builds the thresholds on the device; they equal the host's
    muca_build_table and the oracle's bit for bit, including thresholds that round to
    the accept-all word and ones that underflow to 0."""
    lnW = rand_weights(L, 11 * L, 4.0)
    lnW[3] = lnW[5] - 1e-18
    lnW[L] = lnW[L + 2] + 80.0
    with muca_mod.Muca(L, 40, 2) as m:
        m.set_weights(lnW)
        T = m.get_table()
    assert np.array_equal(T, muca_mod.muca_build_table(L, lnW))
    assert np.array_equal(T, orc.build_table(L, lnW))


def run_both(muca_mod, orc, L, W, seed, layout, wpb, lnW, plan):
    """plan: list of (n_attempts, record, reset_before).  Returns device and oracle
    (lattice, energies, histogram)."""
    N = L * L
    with muca_mod.Muca(L, W, seed, layout=layout, walkers_per_block=wpb) as m:
        m.set_weights(lnW)
        for n, rec, reset in plan:
            if reset:
                m.reset_histogram()
            m.attempts(n, rec)
        dev = (m.get_lattice(), m.get_energies(), m.get_histogram(), m.attempt_counter)
    s, e = orc.init(L, seed, W)
    T = orc.build_table(L, lnW)
    H = np.zeros(N + 1, dtype=np.uint64)
    t = 0
    for n, rec, reset in plan:
        if reset:
            H[:] = 0
        orc.run(L, seed, s, e, T, t, n, rec, H if rec else None)
        t += n
    return dev, (s, e, H, t)


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("L,W,wpb", [(4, 7, 32), (8, 200, 64), (16, 130, 32), (24, 65, 64), (32, 96, 32),
                                     (48, 40, 32), (64, 37, 32)])
def test_sweeps_bit_exact(muca_mod, orc, layout, L, W, wpb):
    N = L * L
    lnW = rand_weights(L, L + W)
    plan = [(3 * N, False, True), (4 * N, True, True)]
    (lat, e, H, t), (s, eo, Ho, to) = run_both(muca_mod, orc, L, W, 99, layout, wpb, lnW, plan)
    assert t == to
    assert np.array_equal(lat, s)
    assert np.array_equal(e, eo)
    assert np.array_equal(H, Ho)
    assert int(H.sum()) == W * 4 * N
    assert all(e[w] == e_index(L, lat[w]) for w in range(W))


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("L", [8, 12, 32, 64])
def test_partial_sweeps_bit_exact(muca_mod, orc, layout, L):
    """Launch boundaries inside rows and inside Philox blocks (Eq. 7 asks for attempt
    counts that are not whole sweeps); L = 12 runs the generic kernel."""
    W = 77
    N = L * L
    lnW = rand_weights(L, 1, 0.4 if L <= 12 else 0.05)
    plan = [(5, False, True), (1, True, True), (70, True, False), (3, True, False), (N * 2 + 9, True, False),
            (13, False, False), (N - 1, True, False), (L + 2, True, False), (3 * L - 1, False, False)]
    (lat, e, H, t), (s, eo, Ho, to) = run_both(muca_mod, orc, L, W, 5, layout, 32, lnW, plan)
    assert t == to
    assert np.array_equal(lat, s) and np.array_equal(e, eo) and np.array_equal(H, Ho)


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("L", [8, 24, 32, 64])
def test_counter_high_word_boundary(muca_mod, orc, layout, L):
    """Attempt counters around t = 2^34, where Philox counter word 1 (the high word of
    t >> 2) steps from 0 to 1: whole sweeps, a row and partial launches across the step
    equal the oracle (the sweep kernels take round 1's product of the constant word from
    the keys only while word 1 stays at the launch's first value)."""
    W = 40
    N = L * L
    lnW = rand_weights(L, 2, 0.3)
    t0 = (2**34 // N - 2) * N                         # two sweeps before the step
    with muca_mod.Muca(L, W, 9, layout=layout, walkers_per_block=32) as m:
        m.set_weights(lnW)
        m.set_attempt_counter(t0)
        m.reset_histogram()
        m.sweep(5, True)                                # crosses 2^34 in one launch
        m.attempts(3 * L + 5, True)                     # partial launches after it
        m.attempts(N - 7, False)
        m.set_attempt_counter(2**34 - L - 3)            # a partial launch across the step
        m.attempts(2 * L + 9, True)
        lat, e, H, t = m.get_lattice(), m.get_energies(), m.get_histogram(), m.attempt_counter
    s, eo = orc.init(L, 9, W)
    T = orc.build_table(L, lnW)
    Ho = np.zeros(N + 1, dtype=np.uint64)
    orc.run(L, 9, s, eo, T, t0, 5 * N, True, Ho)
    orc.run(L, 9, s, eo, T, t0 + 5 * N, 3 * L + 5, True, Ho)
    orc.run(L, 9, s, eo, T, t0 + 5 * N + 3 * L + 5, N - 7, False)
    orc.run(L, 9, s, eo, T, 2**34 - L - 3, 2 * L + 9, True, Ho)
    assert t == 2**34 - L - 3 + 2 * L + 9
    assert np.array_equal(lat, s) and np.array_equal(e, eo) and np.array_equal(H, Ho)


def test_all_accept_and_quench_limits(muca_mod, orc):
    L, W = 8, 64
    N = L * L
    for lnW in (np.zeros(N + 1), -100.0 * np.arange(N + 1)):
        plan = [(2 * N + 3, True, True)]
        (lat, e, H, _), (s, eo, Ho, _) = run_both(muca_mod, orc, L, W, 17, 0, 32, lnW, plan)
        assert np.array_equal(lat, s) and np.array_equal(e, eo) and np.array_equal(H, Ho)


def test_config2_full_size_histogram_and_sampled_walkers(muca_mod, orc):
    """L = 32, 16384 walkers (the headline configuration), int8 layout: the histogram of
    two recorded sweeps equals the oracle's over all walkers; lattices and energies of
    sampled walkers equal the oracle's walker by walker."""
    L, W, seed = 32, 16384, 42
    N = L * L
    lng = load_exact_ln_dos(L)
    lnW = np.where(np.isfinite(lng), -lng, 0.0)
    with muca_mod.Muca(L, W, seed) as m:
        m.set_weights(lnW)
        m.sweep(1, record=False)
        m.reset_histogram()
        m.sweep(2, record=True)
        H = m.get_histogram()
        e = m.get_energies()
        lat = m.get_lattice()
    s, eo = orc.init(L, seed, W)
    T = orc.build_table(L, lnW)
    orc.run(L, seed, s, eo, T, 0, N, False)
    Ho = orc.run(L, seed, s, eo, T, N, 2 * N, True)
    assert np.array_equal(H, Ho)
    assert np.array_equal(e, eo)
    idx = np.random.default_rng(0).choice(W, 64, replace=False)
    assert np.array_equal(lat[idx], s[idx])


def test_max_size_sampled_walkers(muca_mod, orc):
    """L = 64 with 32768 walkers (the largest configuration), packed layout: sampled
    walkers are advanced one by one by the oracle and must match exactly."""
    L, W, seed = 64, 32768, 7
    N = L * L
    lnW = rand_weights(L, 2, 0.05)
    with muca_mod.Muca(L, W, seed, layout=1) as m:
        m.set_weights(lnW)
        m.sweep(1, record=True)
        e = m.get_energies()
        lat = m.get_lattice()
        H = m.get_histogram()
    assert int(H.sum()) == W * N
    T = orc.build_table(L, lnW)
    for w in [0, 1, 31, 32, 12345, W - 1]:
        s, eo = orc.init(L, seed, 1, walker0=w)
        orc.run(L, seed, s, eo, T, 0, N, False, walker0=w)
        assert np.array_equal(lat[w], s[0]) and e[w] == eo[0]


def test_iteration_bit_exact_config1(muca_mod, orc):
    """Configuration 1: L = 8, 128 walkers, seed 1, 100 sweeps per iteration, min/mean >=
    0.8; the iteration count, the final weights (bitwise) and the production histogram
    and ln g match the oracle, and ln g is within 0.05 of the exact result."""
    L, W, seed = 8, 128, 1
    N = L * L
    p_dev = muca_mod.make_params(therm_sweeps=31, sweeps_per_iter=100, max_iterations=200)
    with muca_mod.Muca(L, W, seed) as m:
        st = m.iterate_until_flat(p_dev)
        lnW = m.get_weights()
        H, lng = m.production(31, 4000)
        e = m.get_energies()
    s, eo = orc.init(L, seed, W)
    lnWo = np.zeros(N + 1)
    res, t, _, _ = orc.iterate(L, seed, s, eo, lnWo, 0,
                               orc.make_params(therm_sweeps=31, sweeps_per_iter=100, max_iterations=200))
    assert st.converged and res.converged == 1
    assert st.iterations == res.iterations
    assert st.last_metric == res.last_metric
    assert np.array_equal(lnW, lnWo)
    Ho, lngo, _ = orc.production(L, seed, s, eo, lnWo, t, 31, 4000)
    assert np.array_equal(H, Ho) and np.array_equal(e, eo)
    assert np.array_equal(lng, lngo)
    ex = load_exact_ln_dos(L)
    acc = np.isfinite(ex)
    assert np.max(np.abs(lng[acc] - ex[acc])) < 0.05


def test_iteration_bit_exact_paper_schedule(muca_mod, orc):
    """Eq. (7) schedule with f_therm = 30 and the KL stop (Sec. 3), partial sweeps."""
    L, W, seed = 8, 96, 3
    N = L * L
    with muca_mod.Muca(L, W, seed, walkers_per_block=32) as m:
        st = m.iterate_until_flat(muca_mod.make_params(schedule=1, stop_rule=1, flat_threshold=1e-4,
                                                       max_iterations=400))
        lnW = m.get_weights()
        t_dev = m.attempt_counter
    s, eo = orc.init(L, seed, W)
    lnWo = np.zeros(N + 1)
    res, t, _, _ = orc.iterate(L, seed, s, eo, lnWo, 0,
                               orc.make_params(schedule=1, stop_rule=1, flat_threshold=1e-4, max_iterations=400))
    assert st.iterations == res.iterations and st.converged == bool(res.converged)
    assert st.last_metric == res.last_metric
    assert t_dev == t
    assert np.array_equal(lnW, lnWo)


def test_invalid_arguments(muca_mod):
    with pytest.raises(muca_mod.MucaError):
        muca_mod.Muca(10, 8, 1)
    with pytest.raises(muca_mod.MucaError):
        muca_mod.Muca(8, 8, 1, walkers_per_block=48)
    with muca_mod.Muca(8, 8, 1) as m:
        with pytest.raises(muca_mod.MucaError):
            m.set_weights(np.zeros(10))
        bad = np.zeros(65)
        bad[3] = np.nan
        with pytest.raises(muca_mod.MucaError):
            m.set_weights(bad)


@pytest.mark.parametrize("L", [8, 32, 64])
def test_optimal_walkers(muca_mod, orc, L):
    """Default walker count (Sec. 3.1: full occupancy): a whole number of resident blocks
    on every SM, and an instance created with it runs bit-exact (sampled walkers)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n, wpb = muca_mod.muca_optimal_walkers(L)
    assert wpb % 32 == 0 and 32 <= wpb <= 256
    assert n > 0 and n % (sms * wpb) == 0
    n_packed, _ = muca_mod.muca_optimal_walkers(L, muca_mod.MUCA_LAYOUT_PACKED)
    assert n_packed > 0
    if L != 32:
        return
    N = L * L
    lnW = rand_weights(L, 11, 0.05)
    with muca_mod.Muca(L, muca_mod.MUCA_WALKERS_OPTIMAL, 5) as m:
        assert m.W == n
        info = muca_mod.muca_get_info(m._h)
        assert info[1] == n and info[4] == wpb
        m.set_weights(lnW)
        m.sweep(1, False)
        e = m.get_energies()
        lat = m.get_lattice()
    T = orc.build_table(L, lnW)
    for w in (0, n // 2 + 3, n - 1):
        s, eo = orc.init(L, 5, 1, walker0=w)
        orc.run(L, 5, s, eo, T, 0, N, False, None, walker0=w)
        assert np.array_equal(lat[w], s[0]) and e[w] == eo[0] == e_index(L, lat[w])


def test_issue_rate_probe(muca_mod):
    """The integer issue rates the roofline rests on: every class positive and below the
    issue-slot ceiling (SMs x 4 x 32 lanes x the maximum clock); unknown kinds refused."""
    import torch
    M = muca_mod
    props = torch.cuda.get_device_properties(0)
    ceiling = props.multi_processor_count * 4 * 32 * 2.2e9
    rates = {k: M.muca_measure_issue_rate(k) for k in (M.MUCA_PROBE_XOR, M.MUCA_PROBE_MAD, M.MUCA_PROBE_MIXED)}
    for r in rates.values():
        assert 0.05 * ceiling < r < 1.05 * ceiling
    words = M.muca_measure_issue_rate(M.MUCA_PROBE_PHILOX)
    assert 1e11 < words < ceiling
    one = M.muca_measure_issue_rate(M.MUCA_PROBE_MIXED_ONE_WARP)
    assert 0.02 * ceiling < one < 1.05 * ceiling
    with pytest.raises(M.MucaError):
        M.muca_measure_issue_rate(9)


@pytest.mark.parametrize("L,W,layout", [(8, 1, 0), (32, 1, 1), (64, 1, 0), (16, 16, 0), (16, 32, 0), (16, 33, 0),
                                        (24, 48, 1)])
def test_edge_walker_counts_and_empty_launches(muca_mod, orc, L, W, layout):
    """A single walker, half and whole warps, one walker past a warp; launches of zero
    sweeps or attempts change nothing (the counter included)."""
    M = muca_mod
    N = L * L
    lnW = rand_weights(L, 7, 0.1)
    with M.Muca(L, W, 31, layout=layout) as m:
        m.set_weights(lnW)
        m.sweep(0, True)
        m.attempts(0, True)
        assert m.info()[2] == 0 and int(m.get_histogram().sum()) == 0
        m.sweep(2, False)
        m.reset_histogram()
        m.attempts(N + 7, True)
        m.sweep(0, False)
        lat, e, H, t = m.get_lattice(), m.get_energies(), m.get_histogram(), m.info()[2]
    s, eo = orc.init(L, 31, W)
    T = orc.build_table(L, lnW)
    orc.run(L, 31, s, eo, T, 0, 2 * N, False)
    Ho = orc.run(L, 31, s, eo, T, 2 * N, N + 7, True)
    assert t == 3 * N + 7
    assert np.array_equal(lat, s) and np.array_equal(e, eo) and np.array_equal(H, Ho)


def test_bounded_wait(muca_mod):
    """A wait with a time limit returns at the limit while long work is still running (it
    is not interrupted) and reports completion once it is done."""
    M = muca_mod
    with M.Muca(64, 32768, 3) as m:
        m.sweep(200, False)                     # about a second of work on one GPU
        assert m.synchronize(timeout=0.0) is False
        assert m.synchronize(timeout=60.0) is True
        assert m.info()[2] == 200 * 64 * 64
        with pytest.raises(M.MucaError):
            M.muca_synchronize_timeout(m._h, -1.0)


def test_orders_sample_the_same_distribution(muca_mod):
    """Typewriter and random shared site order are both valid Metropolis chains for the
    multicanonical weights (the shared sequence only correlates walkers, Sec. 2.3): with
    the perfect weights of L = 8 both histograms are flat, and they agree within their
    multinomial noise bin by bin."""
    from conftest import load_exact_ln_dos
    M = muca_mod
    L = 8
    N = L * L
    lng = load_exact_ln_dos(L)
    lnW = np.where(np.isfinite(lng), -lng, 0.0)
    Hs = []
    for order in (M.MUCA_ORDER_TYPEWRITER, M.MUCA_ORDER_RANDOM):
        with M.Muca(L, 4096, 17 + order) as m:
            m.site_order = order
            m.set_weights(lnW)
            m.sweep(200, False)
            m.reset_histogram()
            m.sweep(400, True)
            Hs.append(m.get_histogram().astype(np.float64))
    acc = np.isfinite(lng)
    for H in Hs:
        assert H[acc].min() / H[acc].mean() > 0.9
    a, b = Hs[0][acc], Hs[1][acc]
    # counts are autocorrelated (a walker needs many attempts to cross the range), so
    # the bins differ by a few per cent, not by the multinomial 0.1 % (the oracle, which
    # gives these histograms bit for bit, shows at most 3.5 %)
    assert np.max(np.abs(a - b) / (0.5 * (a + b))) < 0.06
