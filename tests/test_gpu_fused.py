"""muca_thermalize_and_record (one weight iteration's sampling, Sec. 3: N_therm
thermalization attempts, then N_updates recorded ones) against the oracle, bit for bit:
the single launch that runs both phases (typewriter order; whole sweeps from a sweep
boundary or any attempt ranges) and the two launches it falls back to (random site
order, no thermalization, a range across a step of Philox counter word 1)."""
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


def oracle_therm_record(orc, L, W, seed, lnW, t0, n_therm, n_record, s=None, e=None, order=0):
    if s is None:
        s, e = orc.init(L, seed, W)
    T = orc.build_table(L, lnW)
    orc.run(L, seed, s, e, T, t0, n_therm, False, site_order=order)
    H = np.zeros(L * L + 1, dtype=np.uint64)
    orc.run(L, seed, s, e, T, t0 + n_therm, n_record, True, H, site_order=order)
    return s, e, H


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("L,W,wpb", [(8, 200, 64), (16, 130, 32), (24, 65, 64), (32, 96, 32), (32, 300, 128),
                                     (48, 40, 32), (64, 37, 32)])
def test_fused_whole_sweeps_equal_oracle(muca_mod, orc, layout, L, W, wpb):
    """One launch for both phases (ragged last block included); the histogram recorded
    before the call is discarded, as the call zeroes it."""
    N = L * L
    lnW = rand_weights(L, L + W, 0.4 if L <= 16 else 0.05)
    with muca_mod.Muca(L, W, 31, layout=layout, walkers_per_block=wpb) as m:
        m.set_weights(lnW)
        m.sweep(1, record=True)                       # something in H before the call
        m.thermalize_and_record(3 * N, 2 * N)
        lat, e, H, t = m.get_lattice(), m.get_energies(), m.get_histogram(), m.attempt_counter
    s, eo = orc.init(L, 31, W)
    T = orc.build_table(L, lnW)
    orc.run(L, 31, s, eo, T, 0, N, True)
    s, eo, Ho = oracle_therm_record(orc, L, W, 31, lnW, N, 3 * N, 2 * N, s, eo)
    assert t == 6 * N
    assert np.array_equal(lat, s) and np.array_equal(e, eo) and np.array_equal(H, Ho)
    assert int(H.sum()) == W * 2 * N


@pytest.mark.parametrize("L", [8, 12, 32, 64])
def test_fused_any_range_and_fallbacks_equal_oracle(muca_mod, orc, L):
    """Attempt counts that are not whole sweeps (the Eq. (7) schedule's) and a start
    inside a sweep run in one launch of the any-range form; a zero thermalization, random
    site order and L = 12 (no whole-sweep kernel) take two launches.  Every case equals
    the oracle."""
    W, seed = 70, 8
    N = L * L
    lnW = rand_weights(L, 3, 0.4 if L <= 8 else 0.05)
    cases = [(0, 2 * N + 5, 3 * N - 1), (N, N + 3, 2 * N), (N + 7, 2 * N, N), (0, 0, 2 * N), (N, 2 * N, 3 * N)]
    for t0, nt, nr in cases:
        for order in (0, 1):
            with muca_mod.Muca(L, W, seed, walkers_per_block=32) as m:
                m.set_weights(lnW)
                if order:
                    m.site_order = muca_mod.MUCA_ORDER_RANDOM
                m.set_attempt_counter(t0)
                m.thermalize_and_record(nt, nr)
                lat, e, H, t = m.get_lattice(), m.get_energies(), m.get_histogram(), m.attempt_counter
            s, eo, Ho = oracle_therm_record(orc, L, W, seed, lnW, t0, nt, nr, order=order)
            assert t == t0 + nt + nr
            assert np.array_equal(lat, s) and np.array_equal(e, eo) and np.array_equal(H, Ho), (t0, nt, nr, order)


@pytest.mark.parametrize("L", [16, 32])
def test_fused_counter_word_boundary(muca_mod, orc, L):
    """Around t = 2^34, where Philox counter word 1 steps: a range that ends exactly at
    the step runs as one launch, one that crosses it as two (the second split again at
    the step), for whole sweeps and for partial ones; all equal the oracle."""
    W, seed = 40, 4
    N = L * L
    lnW = rand_weights(L, 6, 0.2)
    last = 2**34 // N * N                              # the last sweep boundary <= 2^34
    cases = [(last - 5 * N, 3 * N, 2 * N), (last - 3 * N, 2 * N, 3 * N), (last - N, 2 * N, N),
             (2**34 - 2 * N - 5, N + 2, N + 3), (2**34 - N - 3, N, 7), (2**34 - 9, 4, 2 * N + 1)]
    for t0, nt, nr in cases:
        with muca_mod.Muca(L, W, seed, walkers_per_block=32) as m:
            m.set_weights(lnW)
            m.set_attempt_counter(t0)
            m.thermalize_and_record(nt, nr)
            lat, e, H = m.get_lattice(), m.get_energies(), m.get_histogram()
        s, eo, Ho = oracle_therm_record(orc, L, W, seed, lnW, t0, nt, nr)
        assert np.array_equal(lat, s) and np.array_equal(e, eo) and np.array_equal(H, Ho), (t0, nt, nr)


def test_fused_headline_configuration(muca_mod, orc):
    """L = 32, 16384 walkers, int8, perfect weights: 31 thermalization and 10 recorded
    sweeps in one launch (the step the bench times).  The histogram over all walkers and
    the energies equal the oracle's; lattices of sampled walkers too."""
    L, W, seed = 32, 16384, 42
    N = L * L
    lng = load_exact_ln_dos(L)
    lnW = np.where(np.isfinite(lng), -lng, 0.0)
    with muca_mod.Muca(L, W, seed) as m:
        m.set_weights(lnW)
        m.thermalize_and_record(31 * N, 10 * N)
        H, e, lat = m.get_histogram(), m.get_energies(), m.get_lattice()
    s, eo, Ho = oracle_therm_record(orc, L, W, seed, lnW, 0, 31 * N, 10 * N)
    assert np.array_equal(H, Ho)
    assert np.array_equal(e, eo)
    idx = np.random.default_rng(1).choice(W, 64, replace=False)
    assert np.array_equal(lat[idx], s[idx])


def test_fused_equals_separate_calls_in_iteration(muca_mod):
    """The weight iteration and the production run the fused call; their results equal
    those of the separate calls made by hand (thermalize, zero H, record)."""
    L, W, seed = 16, 256, 12
    N = L * L
    lnW = rand_weights(L, 9, 0.3)
    with muca_mod.Muca(L, W, seed) as a, muca_mod.Muca(L, W, seed) as b:
        a.set_weights(lnW)
        b.set_weights(lnW)
        for _ in range(3):
            a.thermalize_and_record(4 * N, 6 * N)
            b.sweep(4, record=False)
            b.reset_histogram()
            b.sweep(6, record=True)
            assert np.array_equal(a.get_histogram(), b.get_histogram())
        assert np.array_equal(a.get_lattice(), b.get_lattice())
        assert np.array_equal(a.get_energies(), b.get_energies())
        assert a.attempt_counter == b.attempt_counter
