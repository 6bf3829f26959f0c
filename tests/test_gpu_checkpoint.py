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
