"""Configuration 3 (L = 64, packed vs int8 chosen by the autotuner) and the tuner at other
sizes: instances created with MUCA_LAYOUT_AUTO and MUCA_WPB_TUNE time the candidate
layouts and block sizes, record the choice (muca_get_info), and then run exactly the
same chain as the oracle (Sec. 2.3: the layout and block size change only how lattices
are stored and how walkers are grouped, never a decision)."""
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


def rand_weights(L, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.normal(0.0, scale, L * L + 1))


@pytest.mark.parametrize("L,W", [(64, 4096), (8, 2048), (32, 1000)])
def test_tuned_instance_matches_oracle(M, orc, L, W):
    N = L * L
    seed = 70 + L
    lnW = rand_weights(L, seed)
    with M.Muca(L, W, seed, layout=M.MUCA_LAYOUT_AUTO, walkers_per_block=M.MUCA_WPB_TUNE) as m:
        L_, W_, t, layout, wpb = m.info()
        assert (L_, W_, t) == (L, W, 0)
        assert layout in (M.MUCA_LAYOUT_INT8, M.MUCA_LAYOUT_PACKED)
        assert wpb % 32 == 0 and 32 <= wpb <= 256
        m.set_weights(lnW)
        m.sweep(3, record=False)
        m.reset_histogram()
        m.sweep(2, record=True)
        lat, e, H = m.get_lattice(), m.get_energies(), m.get_histogram()
        # the tuned choice, given explicitly, runs the same chain
        with M.Muca(L, W, seed, layout=layout, walkers_per_block=wpb) as m2:
            m2.set_weights(lnW)
            m2.sweep(3, record=False)
            m2.reset_histogram()
            m2.sweep(2, record=True)
            assert np.array_equal(m2.get_lattice(), lat) and np.array_equal(m2.get_histogram(), H)
    s, eo = orc.init(L, seed, W)
    T = orc.build_table(L, lnW)
    orc.run(L, seed, s, eo, T, 0, 3 * N, False)
    Ho = orc.run(L, seed, s, eo, T, 3 * N, 2 * N, True)
    assert np.array_equal(lat, s) and np.array_equal(e, eo) and np.array_equal(H, Ho)


def test_configuration3_tuned_sampled_walkers(M, orc):
    """L = 64, 32768 walkers with layout and block size tuned: histogram total and the
    tracked energies are consistent, and sampled walkers equal the oracle walker by
    walker (each advanced alone with its global index)."""
    L, W, seed = 64, 32768, 3
    N = L * L
    lnW = rand_weights(L, seed, 0.05)
    with M.Muca(L, W, seed, layout=M.MUCA_LAYOUT_AUTO, walkers_per_block=M.MUCA_WPB_TUNE) as m:
        _, _, _, layout, wpb = m.info()
        m.set_weights(lnW)
        m.sweep(2, record=False)
        m.reset_histogram()
        m.sweep(1, record=True)
        lat, e, H = m.get_lattice(), m.get_energies(), m.get_histogram()
    assert int(H.sum()) == W * N
    s0, e0 = orc.init(L, seed, W)
    T = orc.build_table(L, lnW)
    for w in (0, 1, 255, 256, 4097, 20000, 32767):
        sw, ew = np.ascontiguousarray(s0[w:w + 1]), np.ascontiguousarray(e0[w:w + 1])
        orc.run(L, seed, sw, ew, T, 0, 2 * N, False, walker0=w)
        orc.run(L, seed, sw, ew, T, 2 * N, N, True, np.zeros(N + 1, np.uint64), walker0=w)
        assert np.array_equal(lat[w], sw[0]) and e[w] == ew[0], (w, layout, wpb)
