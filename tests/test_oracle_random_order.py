"""Pins of the oracle's random shared site order (Sec. 2.3: one random site sequence for
all walkers, acceptance from each walker's own stream; reading R9): the site
definition against the separately pinned Philox, the uniformity of the sites, the
deterministic all-accept and quench limits against an independent numpy walk over the
same sites, detailed balance against the exact density of states, and the iteration
plus production recovering ln g."""
import numpy as np
import pytest

from conftest import load_exact_ln_dos
from test_oracle_chain import e_index, energy_np


def site_reference(orc, L, seed, t):
    """floor(u N / 2^32), u = word t & 3 of Philox(counter (t >> 2, 0xFFFFFFFF, 2), seed)."""
    blk = t >> 2
    words = orc.philox4x32_10([blk & 0xFFFFFFFF, blk >> 32, 0xFFFFFFFF, 2],
                              [seed & 0xFFFFFFFF, seed >> 32])
    return (int(words[t & 3]) * L * L) >> 32


def test_site_definition(orc):
    for L, seed in [(4, 1), (8, 77), (64, 2 ** 40 + 5)]:
        for t in list(range(40)) + [2 ** 33 + 1, 2 ** 45 + 6]:
            assert orc.random_site(L, seed, t) == site_reference(orc, L, seed, t)


def test_sites_are_uniform(orc):
    L, n = 8, 64 * 2000
    N = L * L
    counts = np.bincount([orc.random_site(L, 5, t) for t in range(n)], minlength=N)
    expect = n / N
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < N - 1 + 6 * np.sqrt(2 * (N - 1))        # about 6 sigma
    assert counts.min() > 0


def _random_reference(orc, L, seed, s0, t0, n_attempts, accept):
    """Independent numpy walk over the oracle's site sequence: attempt t flips the site
    if accept(dE), dE from two full energy evaluations; returns the final lattice and
    the recorded energy indices."""
    s = s0.copy()
    rec = []
    for t in range(t0, t0 + n_attempts):
        i = site_reference(orc, L, seed, t)
        e_old = energy_np(L, s)
        s[i] = -s[i]
        if not accept(energy_np(L, s) - e_old):
            s[i] = -s[i]
        rec.append(e_index(L, s))
    return s, rec


def test_all_accept_limit(orc):
    L, W, seed = 4, 3, 6
    N = L * L
    s, e = orc.init(L, seed, W)
    s0 = s.copy()
    T = orc.build_table(L, np.zeros(N + 1))
    H = orc.run(L, seed, s, e, T, 5, 3 * N, True, site_order=1)
    Href = np.zeros(N + 1, dtype=np.uint64)
    for w in range(W):
        fin, rec = _random_reference(orc, L, seed, s0[w], 5, 3 * N, lambda dE: True)
        assert np.array_equal(fin, s[w]) and e[w] == e_index(L, fin)
        for r in rec:
            Href[r] += 1
    assert np.array_equal(H, Href)
    # every walker flipped the same sites: the walkers' flip patterns are identical
    flips = s * s0
    assert all(np.array_equal(flips[0], flips[w]) for w in range(W))


def test_quench_limit(orc):
    L, W, seed = 6, 4, 9
    N = L * L
    T = orc.build_table(L, -100.0 * np.arange(N + 1))
    s, e = orc.init(L, seed, W)
    s0 = s.copy()
    H = orc.run(L, seed, s, e, T, 0, 3 * N, True, site_order=1)
    Href = np.zeros(N + 1, dtype=np.uint64)
    for w in range(W):
        fin, rec = _random_reference(orc, L, seed, s0[w], 0, 3 * N, lambda dE: dE <= 0)
        assert np.array_equal(fin, s[w])
        for r in rec:
            Href[r] += 1
    assert np.array_equal(H, Href)


def test_splits_compose_and_energy_tracked(orc):
    L, W, seed = 8, 5, 4
    N = L * L
    rng = np.random.default_rng(0)
    T = orc.build_table(L, np.cumsum(rng.normal(0, 0.3, N + 1)))
    s1, e1 = orc.init(L, seed, W)
    s2, e2 = s1.copy(), e1.copy()
    H1 = orc.run(L, seed, s1, e1, T, 10, 333, True, site_order=1)
    H2 = orc.run(L, seed, s2, e2, T, 10, 101, True, site_order=1)
    H2 = orc.run(L, seed, s2, e2, T, 111, 232, True, H2, site_order=1)
    assert np.array_equal(s1, s2) and np.array_equal(e1, e2) and np.array_equal(H1, H2)
    assert all(e1[w] == e_index(L, s1[w]) for w in range(W))


def test_detailed_balance_against_exact_dos(orc):
    """Random site selection is symmetric, so P(e) ~ g(e) W(e) as in typewriter order."""
    L, W, seed = 4, 64, 21
    N = L * L
    lng = load_exact_ln_dos(L)
    lnW = np.where(np.isfinite(lng), -lng, 0.0) + 0.35 * (np.arange(N + 1) - N / 2)
    T = orc.build_table(L, lnW)
    s, e = orc.init(L, seed, W)
    orc.run(L, seed, s, e, T, 0, 200 * N, False, site_order=1)
    H = orc.run(L, seed, s, e, T, 200 * N, 4000 * N, True, site_order=1).astype(np.float64)
    logp = np.where(np.isfinite(lng), lng + lnW, -np.inf)
    p = np.exp(logp - logp[np.isfinite(logp)].max())
    p /= p.sum()
    expect = p * H.sum()
    mask = expect > 200
    assert (np.abs(H[mask] - expect[mask]) / expect[mask]).max() < 0.08
    assert H[mask].max() / H[mask].min() > 50


@pytest.mark.parametrize("L", [4, 8])
def test_iteration_and_production_recover_exact_dos(orc, L):
    W, seed = 128, 1
    N = L * L
    s, e = orc.init(L, seed, W)
    lnW = np.zeros(N + 1)
    res, t, _, _ = orc.iterate(L, seed, s, e, lnW, 0,
                               orc.make_params(therm_sweeps=31, sweeps_per_iter=100, max_iterations=300,
                                               site_order=1))
    assert res.converged == 1
    _, lng, _ = orc.production(L, seed, s, e, lnW, t, 31, 12000, site_order=1)
    ex = load_exact_ln_dos(L)
    acc = np.isfinite(ex)
    assert np.max(np.abs(lng[acc] - ex[acc])) < 0.05
