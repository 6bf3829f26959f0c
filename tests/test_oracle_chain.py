"""Pins the oracle's multicanonical chain (Sec. 2.1-2.3, Sec. 3) to what the physics and
the mathematics fix: deterministic limits of the acceptance rule, detailed balance
against the exact density of states, flat histograms under perfect weights, and the
density of states recovered by iteration plus production."""
import ctypes
import math

import numpy as np
import pytest

from conftest import load_exact_ln_dos


def energy_np(L, s):
    """E of Eq. (5) by the plain definition, numpy version."""
    g = s.reshape(L, L).astype(np.int64)
    return int(-(g * np.roll(g, -1, axis=1)).sum() - (g * np.roll(g, -1, axis=0)).sum())


def e_index(L, s):
    return (energy_np(L, s) + 2 * L * L) // 4


# ---------------------------------------------------------------- lattice / energy
def test_energy_index_special_lattices(orc):
    L = 6
    N = L * L
    up = np.ones(N, dtype=np.int8)
    assert orc.energy_index(L, up) == 0
    assert orc.energy_index(L, -up) == 0
    cb = np.array([1 if (x + y) % 2 == 0 else -1 for y in range(L) for x in range(L)], dtype=np.int8)
    assert orc.energy_index(L, cb) == N                # every bond broken: E = +2N
    one = up.copy()
    one[7] = -1
    assert orc.energy_index(L, one) == 2               # four broken bonds: E = -2N + 8


def test_init_lattices(orc):
    L, W = 8, 64
    s, e = orc.init(L, 11, W)
    assert set(np.unique(s)) <= {-1, 1}
    assert abs((s == 1).mean() - 0.5) < 0.03
    for w in range(W):
        assert e[w] == e_index(L, s[w])
    # walker w of a sub-range equals walker w of the full set (walker-keyed streams)
    s2, e2 = orc.init(L, 11, 8, walker0=20)
    assert np.array_equal(s2, s[20:28]) and np.array_equal(e2, e[20:28])


# ---------------------------------------------------------------- table and accept rule
def test_table_rule(orc):
    L = 4
    N = L * L
    lnW = np.zeros(N + 1)
    T = orc.build_table(L, lnW).reshape(N + 1, 5)
    for e in range(N + 1):
        for k in range(5):
            ep = e + 2 - k
            assert T[e, k] == (0xFFFFFFFF if 0 <= ep <= N else 0)
    lnW = np.zeros(N + 1)
    lnW[6] = -math.log(2.0)      # move 5 -> 6 (k = 1): dw = -ln 2
    lnW[9] = -60.0               # move 8 -> 9: dw = -60: exp underflows the 2^-32 grid
    lnW[12] = -1e-18             # move 11 -> 12: exp(dw) rounds to 1.0 -> always accept
    T = orc.build_table(L, lnW).reshape(N + 1, 5)
    assert abs(int(T[5, 1]) - 2**31) <= 1
    assert T[8, 1] == 0
    assert T[11, 1] == 0xFFFFFFFF
    assert T[6, 3] == 0xFFFFFFFF  # 6 -> 5 goes uphill in lnW
    v = math.exp(-2.5)
    lnW = np.zeros(N + 1)
    lnW[3] = -2.5
    T = orc.build_table(L, lnW).reshape(N + 1, 5)
    assert T[2, 1] == math.floor(v * 2**32)


def test_accept_rule(orc):
    assert orc.lib().orc_accept(5, 6) and not orc.lib().orc_accept(6, 6)
    assert not orc.lib().orc_accept(0, 0)
    assert orc.lib().orc_accept(0xFFFFFFFF, 0xFFFFFFFF)
    assert not orc.lib().orc_accept(0xFFFFFFFF, 0xFFFFFFFE)


# ---------------------------------------------------------------- deterministic limits
def _typewriter_reference(L, s0, n_attempts, accept):
    """Independent numpy walk: attempt t flips site t mod N if accept(dE) holds, where dE
    comes from two full energy evaluations; returns final lattice and the recorded e."""
    s = s0.copy()
    rec = []
    N = L * L
    for t in range(n_attempts):
        i = t % N
        e_old = energy_np(L, s)
        s[i] = -s[i]
        dE = energy_np(L, s) - e_old
        if not accept(dE):
            s[i] = -s[i]
        rec.append(e_index(L, s))
    return s, rec


def test_all_accept_limit(orc):
    """ln W = 0 gives T = 0xFFFFFFFF everywhere: every attempt flips, the lattice is
    negated after one sweep and restored after two, and H is the deterministic path."""
    L, W = 4, 3
    N = L * L
    s, e = orc.init(L, 3, W)
    s_start = s.copy()
    T = orc.build_table(L, np.zeros(N + 1))
    H = orc.run(L, 3, s, e, T, 0, N, True)
    assert np.array_equal(s, -s_start)
    H = orc.run(L, 3, s, e, T, N, N, True, H)
    assert np.array_equal(s, s_start)
    assert int(H.sum()) == W * 2 * N
    Href = np.zeros(N + 1, dtype=np.uint64)
    for w in range(W):
        fin, rec = _typewriter_reference(L, s_start[w], 2 * N, lambda dE: True)
        assert np.array_equal(fin, s_start[w])
        for r in rec:
            Href[r] += 1
    assert np.array_equal(H, Href)
    assert all(e[w] == e_index(L, s[w]) for w in range(W))


def test_quench_limit(orc):
    """Weights rising steeply towards low energy accept exactly the moves with dE <= 0:
    a deterministic zero-temperature typewriter quench."""
    L, W = 6, 4
    N = L * L
    lnW = -100.0 * np.arange(N + 1)
    T = orc.build_table(L, lnW)
    s, e = orc.init(L, 9, W)
    s_start = s.copy()
    H = orc.run(L, 9, s, e, T, 0, 3 * N, True)
    Href = np.zeros(N + 1, dtype=np.uint64)
    for w in range(W):
        fin, rec = _typewriter_reference(L, s_start[w], 3 * N, lambda dE: dE <= 0)
        assert np.array_equal(fin, s[w])
        for r in rec:
            Href[r] += 1
    assert np.array_equal(H, Href)


def test_run_splits_compose(orc):
    """Advancing by n1 then n2 attempts equals one run of n1 + n2 (counter-based stream,
    arbitrary split points inside sweeps and Philox blocks)."""
    L, W = 8, 5
    N = L * L
    rng = np.random.default_rng(0)
    lnW = np.cumsum(rng.normal(0, 0.3, N + 1))
    T = orc.build_table(L, lnW)
    s1, e1 = orc.init(L, 4, W)
    s2, e2 = s1.copy(), e1.copy()
    H1 = orc.run(L, 4, s1, e1, T, 10, 333, True)
    H2 = orc.run(L, 4, s2, e2, T, 10, 101, True)
    H2 = orc.run(L, 4, s2, e2, T, 111, 232, True, H2)
    assert np.array_equal(s1, s2) and np.array_equal(e1, e2) and np.array_equal(H1, H2)
    assert int(H1.sum()) == W * 333


def test_tracked_energy_matches_recomputed(orc):
    L, W = 8, 16
    N = L * L
    rng = np.random.default_rng(1)
    lnW = np.cumsum(rng.normal(0, 0.5, N + 1))
    T = orc.build_table(L, lnW)
    s, e = orc.init(L, 2, W)
    orc.run(L, 2, s, e, T, 0, 37 * N + 5, False)
    assert all(e[w] == e_index(L, s[w]) for w in range(W))


# ---------------------------------------------------------------- statistics
def test_detailed_balance_against_exact_dos(orc):
    """With arbitrary fixed weights the chain samples P(e) ~ g(e) W(e) (Sec. 2.1, Eq. 3).
    A flipped sign or a transposed operand in the acceptance fails this test."""
    L, W = 4, 64
    N = L * L
    lng = load_exact_ln_dos(L)
    lnW = -lng.copy()
    lnW[~np.isfinite(lnW)] = 0.0
    lnW += 0.35 * (np.arange(N + 1) - N / 2)          # tilt: strongly non-flat target
    T = orc.build_table(L, lnW)
    s, e = orc.init(L, 21, W)
    orc.run(L, 21, s, e, T, 0, 200 * N, False)
    H = orc.run(L, 21, s, e, T, 200 * N, 4000 * N, True).astype(np.float64)
    logp = np.where(np.isfinite(lng), lng + lnW, -np.inf)
    p = np.exp(logp - logp[np.isfinite(logp)].max())
    p /= p.sum()
    expect = p * H.sum()
    mask = expect > 200
    # Markov-chain samples: allow the relative deviation of a few autocorrelation times
    rel = np.abs(H[mask] - expect[mask]) / expect[mask]
    assert rel.max() < 0.08, rel.max()
    # and the tilt is visible: the histogram is far from flat
    assert H[mask].max() / H[mask].min() > 50


def test_perfect_weights_give_flat_histogram(orc):
    """W = 1/Omega makes every accessible energy equally likely (Sec. 2.1)."""
    L, W = 8, 64
    N = L * L
    lng = load_exact_ln_dos(L)
    lnW = np.where(np.isfinite(lng), -lng, 0.0)
    T = orc.build_table(L, lnW)
    s, e = orc.init(L, 8, W)
    orc.run(L, 8, s, e, T, 0, 200 * N, False)
    H = orc.run(L, 8, s, e, T, 200 * N, 1000 * N, True)
    assert orc.min_over_mean(L, H) > 0.8
    assert orc.chebyshev(L, H) < 0.2


# ---------------------------------------------------------------- recursion and metrics
def test_weight_update(orc):
    L = 4
    N = L * L
    lnW = np.linspace(-1, 1, N + 1)
    H = np.zeros(N + 1, dtype=np.uint64)
    H[[0, 5, 16]] = [1, 7, 123456789]
    ref = lnW.copy()
    ref[5] -= math.log(7)
    ref[16] -= math.log(123456789)
    before = lnW.copy()
    orc.update_weights(L, lnW, H)
    # only visited energies move, each by ln H to within 3 units in the last place of ln H
    assert np.array_equal(lnW[H == 0], before[H == 0])
    for e in (5, 16):
        assert abs((before[e] - lnW[e]) - (before[e] - ref[e])) <= 3 * math.ulp(before[e] - ref[e]) + math.ulp(lnW[e])


def test_flatness_metrics(orc):
    L = 4
    N = L * L
    acc = np.array([orc.lib().orc_accessible(L, e) for e in range(N + 1)], dtype=bool)
    assert acc.sum() == N - 1 and not acc[1] and not acc[N - 1]
    H = np.where(acc, 1000, 0).astype(np.uint64)
    assert orc.min_over_mean(L, H) == pytest.approx(1.0)
    assert orc.chebyshev(L, H) == pytest.approx(0.0, abs=1e-15)
    assert orc.kullback_leibler(L, H, N - 1) == pytest.approx(0.0, abs=1e-15)
    assert orc.width(L, H) == N + 1 and orc.accessible_in_range(L, H) == N - 1
    H2 = H.copy()
    H2[4] = 500
    tot = float(H2.sum())
    assert orc.min_over_mean(L, H2) == pytest.approx(500 / (tot / (N - 1)))
    assert orc.chebyshev(L, H2) == pytest.approx(abs(500 / (tot / (N - 1)) - 1))
    P = H2[H2 > 0] / tot
    assert orc.kullback_leibler(L, H2, N - 1) == pytest.approx(float((P * np.log(P * (N - 1))).sum()))
    H3 = np.zeros(N + 1, dtype=np.uint64)
    H3[[3, 4, 9]] = 1
    assert orc.width(L, H3) == 7 and orc.accessible_in_range(L, H3) == 7


# ---------------------------------------------------------------- the full method
@pytest.mark.parametrize("L", [4, 8])
def test_iteration_and_production_recover_exact_dos(orc, L):
    """Configuration 1 (L = 8, 128 walkers, 100 sweeps per iteration, min/mean >= 0.8)
    and the same at L = 4: the iteration converges and the production run's ln g is
    within 0.05 of the exact density of states on every accessible energy."""
    W = 128
    N = L * L
    s, e = orc.init(L, 1, W)
    lnW = np.zeros(N + 1)
    p = orc.make_params(schedule=0, stop_rule=0, flat_threshold=0.8, therm_sweeps=31,
                        sweeps_per_iter=100, max_iterations=200)
    res, t, _, _ = orc.iterate(L, 1, s, e, lnW, 0, p)
    assert res.converged == 1 and res.last_metric >= 0.8
    H, lng, t = orc.production(L, 1, s, e, lnW, t, 31, 4000)
    ex = load_exact_ln_dos(L)
    acc = np.isfinite(ex)
    assert np.all(H[acc] > 0) and np.all(H[~acc] == 0)
    assert np.max(np.abs(lng[acc] - ex[acc])) < 0.05


def test_paper_schedule_converges_kl(orc):
    """The schedule of Eq. (7) with f_therm = 30 and the KL stop d_k < 1e-4 (Sec. 3)."""
    L, W = 4, 64
    N = L * L
    s, e = orc.init(L, 3, W)
    lnW = np.zeros(N + 1)
    p = orc.make_params(schedule=1, stop_rule=1, flat_threshold=1e-4, max_iterations=300)
    res, t, hist, mh = orc.iterate(L, 3, s, e, lnW, 0, p, history=True)
    assert res.converged == 1 and res.last_metric < 1e-4
    ex = load_exact_ln_dos(L)
    acc = np.isfinite(ex)
    # converged weights approximate -ln g up to a constant
    d = (-lnW[acc]) - ex[acc]
    assert np.max(np.abs(d - d.mean())) < 0.15


def test_paper_schedule_first_iteration_counts(orc):
    """Eq. (7) by hand for the first iteration (no range covered yet, so w = 10):
    N_therm = 30 * 10 = 300 attempts and N_updates = floor(6 * 10^2.25 / 64) + 1 =
    floor(16.67) + 1 = 17 attempts per walker."""
    L, W = 8, 64
    N = L * L
    s, e = orc.init(L, 2, W)
    lnW = np.zeros(N + 1)
    p = orc.make_params(schedule=1, stop_rule=1, flat_threshold=1e-4, max_iterations=1)
    res, t, _, _ = orc.iterate(L, 2, s, e, lnW, 0, p)
    assert res.iterations == 1 and t == 300 + 17 and res.attempts == 317


def _kl_support(orc, L, prev, visited):
    N = L * L
    H = np.zeros(N + 1, dtype=np.uint64)
    H[list(visited)] = 3
    return int(orc.lib().orc_kl_support(L, prev[0], prev[1], H.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))


def test_kl_support_hand_made(orc):
    """Reference support of the Eq. (6) measure (reading 8): the accessible energies in
    the union of the previous iteration's range and the tested histogram's range, at
    least 10.  Expected counts by hand; at L = 4 the inaccessible indices are 1 and 15,
    at L = 8 they are 1 and 63."""
    cases = [
        # L, previous range, visited energies, expected
        (4, (-1, -1), range(3, 10), 10),        # [3, 9]: 7 accessible, floored at 10
        (4, (-1, -1), [0, 16], 15),             # [0, 16]: 17 points less e = 1 and 15
        (4, (0, 14), [4, 8], 14),               # previous range wider: [0, 14] less e = 1
        (4, (5, 9), [2, 12, 16], 14),           # visits beyond both ends: [2, 16] less e = 15
        (4, (7, 8), [7], 10),                   # [7, 8]: 2 accessible, floored at 10
        (4, (1, 15), [8], 13),                  # [1, 15]: 15 points less e = 1 and 15
        (8, (10, 40), [5, 50], 46),             # [5, 50], all accessible
        (8, (-1, -1), [63], 10),                # e = 63 alone is inaccessible: 0, floored
        (8, (0, 64), [30], 63),                 # whole grid: N - 1 accessible energies
    ]
    for L, prev, vis, want in cases:
        assert _kl_support(orc, L, prev, vis) == want, (L, prev, list(vis))


def test_kl_measure_nonnegative_and_zero_when_flat(orc):
    """With the reference support, d_k >= 0 for any histogram (Gibbs' inequality: Q is
    uniform over a set that contains P's support) and d_k = 0 exactly when H is flat
    over that set."""
    rng = np.random.default_rng(12)
    L = 8
    N = L * L
    acc = np.array([orc.lib().orc_accessible(L, e) for e in range(N + 1)], dtype=bool)
    for _ in range(200):
        lo, hi = sorted(rng.integers(0, N + 1, size=2))
        H = np.zeros(N + 1, dtype=np.uint64)
        H[lo:hi + 1] = rng.integers(0, 50, size=hi - lo + 1)
        H[~acc] = 0
        if H.sum() == 0:
            continue
        prev = (-1, -1) if rng.random() < 0.3 else tuple(sorted(rng.integers(0, N + 1, size=2)))
        q = orc.lib().orc_kl_support(L, int(prev[0]), int(prev[1]),
                                     H.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        assert orc.kullback_leibler(L, H, q) >= -1e-15
    # flat over the accessible energies of the union [3, 40] of [3, 20] and [10, 40]
    H = np.zeros(N + 1, dtype=np.uint64)
    H[10:41] = 7
    q = orc.lib().orc_kl_support(L, 3, 20, H.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    assert q == 38
    Hf = np.zeros(N + 1, dtype=np.uint64)
    Hf[3:41] = 7
    assert orc.kullback_leibler(L, Hf, q) == pytest.approx(0.0, abs=1e-15)
    # H covering only part of it: P = 1/31 on 31 energies, Q = 1/38, d_k = ln(38/31)
    assert orc.kullback_leibler(L, H, q) == pytest.approx(math.log(38 / 31), rel=1e-12)


def test_paper_schedule_trace(orc):
    """Eq. (7) schedule of Sec. 3 (f_therm = 30, z = 2.25, factor 6, growth 1.1) over the
    first seven iterations of L = 4, W = 4, seed 1, derived by hand from the visited
    ranges the run records (w = max(w', 10), w' = e_max - e_min + 1 of the previous
    iteration, N_therm = 30 w, N_updates = floor(6 w^2.25 / W) + 1 while the iteration
    starts below the full width N + 1 = 17, that first full-width iteration included;
    floor(1.1 N_prev) + 1 after it):
      it 0: no range yet, w = 10: 300, floor(6 * 177.828 / 4) + 1 = 267; visits [5, 11]
      it 1: w' = 7, w = 10: 300, 267; visits [2, 14]
      it 2: w = 13: 390, floor(6 * 320.90 / 4) + 1 = 482; visits [0, 16]
      it 3: w = 17 = N + 1: 510, floor(6 * 586.83 / 4) + 1 = 881 (still Eq. 7)
      it 4: 510, floor(1.1 * 881) + 1 = 970
      it 5: 510, floor(1.1 * 970) + 1 = 1068
      it 6: 510, floor(1.1 * 1068) + 1 = 1175"""
    L, W, seed = 4, 4, 1
    N = L * L
    s, e = orc.init(L, seed, W)
    lnW = np.zeros(N + 1)
    p = orc.make_params(schedule=1, stop_rule=1, flat_threshold=1e-4, max_iterations=7)
    res, t, sched = orc.iterate_schedule(L, seed, s, e, lnW, 0, p)
    want = [(300, 267, 5, 11), (300, 267, 2, 14), (390, 482, 0, 16), (510, 881, 0, 16),
            (510, 970, 0, 16), (510, 1068, 0, 16), (510, 1175, 0, 16)]
    assert res.iterations == 7
    assert [tuple(int(v) for v in r) for r in sched] == want
    assert t == sum(a + b for a, b, _, _ in want) and res.attempts == t


def test_paper_schedule_trace_recurrence(orc):
    """The same rules over longer runs of other walker counts: each iteration's counts
    follow from the previous iteration's recorded range and counts."""
    for L, W, seed in [(4, 2, 5), (4, 16, 3), (8, 64, 2)]:
        N = L * L
        s, e = orc.init(L, seed, W)
        lnW = np.zeros(N + 1)
        p = orc.make_params(schedule=1, stop_rule=1, flat_threshold=1e-4, max_iterations=14)
        res, t, sched = orc.iterate_schedule(L, seed, s, e, lnW, 0, p)
        full, prev_w, prev_upd = False, 0, 0
        for therm, upd, lo, hi in sched:
            w = max(prev_w, 10)
            assert therm == 30 * w
            if full:
                assert upd == math.floor(1.1 * prev_upd) + 1
            else:
                assert upd == math.floor(6.0 * w ** 2.25 / W) + 1
                full = prev_w == N + 1
            prev_w, prev_upd = hi - lo + 1, upd
        assert full, (L, W)
