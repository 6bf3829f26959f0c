"""Random shared site order (Sec. 2.3; reading R9) on the GPU against the oracle: lattices,
energies and histograms bit for bit after thermalization and recorded updates (several
L, both layouts, ragged walker counts, attempt ranges that end inside site chunks and
Philox blocks, a switch of order in mid-run), the weight iteration on the host and on
the device, and the batched entry points refusing such instances."""
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


def rand_weights(L, seed, scale=0.4):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.normal(0.0, scale, L * L + 1))


@pytest.mark.parametrize("L,W,layout", [(4, 37, 0), (8, 100, 1), (12, 64, 0), (16, 300, 1), (32, 70, 0),
                                        (48, 33, 1), (64, 40, 0)])
def test_updates_bit_exact(muca_mod, orc, L, W, layout):
    M = muca_mod
    N = L * L
    seed = 100 + L
    lnW = rand_weights(L, L)
    with M.Muca(L, W, seed, layout=layout) as m:
        m.site_order = M.MUCA_ORDER_RANDOM
        assert m.site_order == M.MUCA_ORDER_RANDOM
        m.set_weights(lnW)
        m.attempts(N + 3, False)            # ends inside a sweep and a Philox block
        m.reset_histogram()
        m.attempts(2 * N + 1029, True)      # crosses site chunks of 1024 attempts
        H = m.get_histogram()
        e = m.get_energies()
        lat = m.get_lattice()
    s, eo = orc.init(L, seed, W)
    T = orc.build_table(L, lnW)
    orc.run(L, seed, s, eo, T, 0, N + 3, False, site_order=1)
    Ho = orc.run(L, seed, s, eo, T, N + 3, 2 * N + 1029, True, site_order=1)
    assert np.array_equal(lat, s) and np.array_equal(e, eo) and np.array_equal(H, Ho)
    assert int(H.sum()) == W * (2 * N + 1029)


def test_switching_order_mid_run(muca_mod, orc):
    M = muca_mod
    L, W, seed = 8, 96, 5
    N = L * L
    lnW = rand_weights(L, 3)
    with M.Muca(L, W, seed) as m:
        m.set_weights(lnW)
        m.sweep(3, False)
        m.site_order = M.MUCA_ORDER_RANDOM
        m.sweep(2, True)
        m.site_order = M.MUCA_ORDER_TYPEWRITER
        m.sweep(2, True)
        H = m.get_histogram()
        lat = m.get_lattice()
    s, eo = orc.init(L, seed, W)
    T = orc.build_table(L, lnW)
    orc.run(L, seed, s, eo, T, 0, 3 * N, False)
    Ho = orc.run(L, seed, s, eo, T, 3 * N, 2 * N, True, site_order=1)
    Ho = orc.run(L, seed, s, eo, T, 5 * N, 2 * N, True, Ho)
    assert np.array_equal(lat, s) and np.array_equal(H, Ho)


def test_iteration_in_random_order(muca_mod, orc):
    """The weight iteration (host-driven and on the device) in random order against the
    oracle's iteration with the same order."""
    M = muca_mod
    L, W, seed = 8, 128, 2
    N = L * L
    p = M.make_params(therm_sweeps=31, sweeps_per_iter=100, max_iterations=300)
    with M.Muca(L, W, seed) as a, M.Muca(L, W, seed) as b:
        a.site_order = M.MUCA_ORDER_RANDOM
        b.site_order = M.MUCA_ORDER_RANDOM
        sa = a.iterate_until_flat(p)
        sb = b.iterate_device(p, 4)
        wa, wb = a.get_weights(), b.get_weights()
        ea, eb = a.get_energies(), b.get_energies()
    s, eo = orc.init(L, seed, W)
    lnWo = np.zeros(N + 1)
    res, t, _, _ = orc.iterate(L, seed, s, eo, lnWo, 0,
                               orc.make_params(therm_sweeps=31, sweeps_per_iter=100, max_iterations=300,
                                               site_order=1))
    assert sa.converged and res.converged == 1
    assert sa.iterations == sb.iterations == res.iterations
    assert sa.last_metric == sb.last_metric == res.last_metric
    assert np.array_equal(wa, lnWo) and np.array_equal(wb, lnWo)
    assert np.array_equal(ea, eo) and np.array_equal(eb, eo)


def test_order_arguments_and_batch_refusal(muca_mod):
    M = muca_mod
    with M.Muca(16, 64, 1) as m:
        assert m.site_order == M.MUCA_ORDER_TYPEWRITER
        with pytest.raises(M.MucaError):
            m.site_order = 7
        m.site_order = M.MUCA_ORDER_RANDOM
        with pytest.raises(M.MucaError):
            M.Batch([m])


def test_full_size_sampled_walkers(muca_mod, orc):
    """The random-order measurement of bench.py at full size (L = 32, 16384 walkers,
    perfect weights, 3 thermalization and 2 recorded sweeps): sampled walkers, at warp
    and block edges and inside, equal the oracle walker by walker; the histogram counts
    every recorded attempt."""
    from conftest import load_exact_ln_dos
    M = muca_mod
    L, W, seed = 32, 16384, 1
    N = L * L
    lng = load_exact_ln_dos(L)
    lnW = np.where(np.isfinite(lng), -lng, 0.0)
    with M.Muca(L, W, seed) as m:
        m.site_order = M.MUCA_ORDER_RANDOM
        m.set_weights(lnW)
        m.sweep(3, False)
        m.reset_histogram()
        m.sweep(2, True)
        H, e, lat = m.get_histogram(), m.get_energies(), m.get_lattice()
    assert int(H.sum()) == W * 2 * N
    T = orc.build_table(L, lnW)
    for w in [0, 1, 31, 32, 127, 128, 5000, 9999, W - 1]:
        s, eo = orc.init(L, seed, 1, walker0=w)
        orc.run(L, seed, s, eo, T, 0, 3 * N, False, walker0=w, site_order=1)
        orc.run(L, seed, s, eo, T, 3 * N, 2 * N, True, walker0=w, site_order=1)
        assert np.array_equal(lat[w], s[0]) and e[w] == eo[0], w


@pytest.mark.parametrize("L", [8, 32, 64])
def test_counter_high_word_boundary(muca_mod, orc, L):
    """Attempt counters around t = 2^34, where Philox counter word 1 (t >> 34) steps: a
    launch across the step (run as two launches) and launches after it equal the oracle
    in random order (the kernel takes round 1's product of the acceptance stream from
    its keys, valid while word 1 stays at the launch's first value)."""
    M = muca_mod
    N = L * L
    W = 40
    lnW = rand_weights(L, 3, 0.3)
    t0 = 2**34 - 2 * N - 5
    with M.Muca(L, W, 19) as m:
        m.site_order = M.MUCA_ORDER_RANDOM
        m.set_weights(lnW)
        m.set_attempt_counter(t0)
        m.reset_histogram()
        m.attempts(4 * N + 9, True)
        m.attempts(N, False)
        lat, e, H, t = m.get_lattice(), m.get_energies(), m.get_histogram(), m.attempt_counter
    s, eo = orc.init(L, 19, W)
    T = orc.build_table(L, lnW)
    Ho = orc.run(L, 19, s, eo, T, t0, 4 * N + 9, True, site_order=1)
    orc.run(L, 19, s, eo, T, t0 + 4 * N + 9, N, False, site_order=1)
    assert t == t0 + 5 * N + 9
    assert np.array_equal(lat, s) and np.array_equal(e, eo) and np.array_equal(H, Ho)
