"""Pins of the oracle's production analysis: jackknife errors (Sec. 3.3) and
reweighting of ln g to canonical averages (Sec. 2.1, Eq. 1), against brute-force
enumeration, closed forms and invariances."""
import math

import numpy as np
import pytest

from conftest import load_exact_ln_dos


def brute_canonical_L4(beta):
    """<E>/N and beta^2 var(E)/N by summing over all 2^16 states of the 4x4 torus."""
    L, N = 4, 16
    states = np.arange(1 << N, dtype=np.uint32)
    spins = 1 - 2 * ((states[:, None] >> np.arange(N, dtype=np.uint32)) & 1).astype(np.int64)
    s = spins.reshape(-1, L, L)
    E = -(s * np.roll(s, -1, 2)).sum(axis=(1, 2)) - (s * np.roll(s, -1, 1)).sum(axis=(1, 2))
    w = np.exp(-beta * (E - E.min()))
    m = (w * E).sum() / w.sum()
    v = (w * E * E).sum() / w.sum() - m * m
    return m / N, beta * beta * v / N


@pytest.mark.parametrize("beta", [0.05, 0.3, 0.4406868, 0.7, 1.5])
def test_canonical_equals_enumeration(orc, beta):
    e, c = orc.canonical(4, load_exact_ln_dos(4), beta)
    e_ref, c_ref = brute_canonical_L4(beta)
    assert e == pytest.approx(e_ref, rel=1e-10, abs=1e-12)
    assert c == pytest.approx(c_ref, rel=1e-9, abs=1e-12)


def test_canonical_limits(orc):
    for L in (8, 16, 32):
        lg = load_exact_ln_dos(L)
        e0, c0 = orc.canonical(L, lg, 0.0)
        assert abs(e0) < 1e-12 and c0 == 0.0            # g(E) = g(-E)
        # high-temperature expansion, ln Z / N = ln 2 + 2 ln cosh b + t^4 + O(t^6) with
        # t = tanh b (elementary plaquettes), so <E>/N = -2 t - 4 t^3 (1 - t^2) + O(t^5)
        b = 0.01
        t = math.tanh(b)
        e, _ = orc.canonical(L, lg, b)
        assert e == pytest.approx(-2.0 * t - 4.0 * t**3 * (1.0 - t * t), abs=1e-8)
        # low temperature: ground state
        e, c = orc.canonical(L, lg, 5.0)
        assert e == pytest.approx(-2.0, abs=1e-6) and c < 1e-4


def test_jackknife_scale_invariance_and_identical_chunks(orc):
    L = 4
    N = L * L
    lg = load_exact_ln_dos(L)
    lnW = np.where(np.isfinite(lg), -lg, 0.0)
    base = np.where(np.isfinite(lg), 1000, 0).astype(np.uint64)
    ln_g, err = orc.jackknife(L, lnW, np.stack([base] * 5))
    acc = np.isfinite(lg)
    assert np.all(err[acc] == 0.0) and np.all(np.isnan(err[~acc]))
    assert np.allclose(ln_g[acc], lg[acc], atol=1e-12)         # flat H under perfect weights
    ln_g2, err2 = orc.jackknife(L, lnW, np.stack([base, 2 * base, 3 * base]))
    assert np.allclose(err2[acc], 0.0, atol=1e-12) and np.allclose(ln_g2[acc], lg[acc], atol=1e-12)


def test_jackknife_matches_delta_method(orc):
    """One energy's counts fluctuate between chunks (all others fixed and dominant): the
    jackknife error of ln g there approaches sd(H_c) / (sqrt(n) mean(H_c))."""
    L = 8
    N = L * L
    lg = load_exact_ln_dos(L)
    acc = np.isfinite(lg)
    lnW = np.where(acc, -lg, 0.0)
    rng = np.random.default_rng(4)
    n = 200
    Hc = np.tile(np.where(acc, 10**6, 0).astype(np.uint64), (n, 1))
    e0 = 20
    Hc[:, e0] = rng.integers(900, 1101, size=n).astype(np.uint64)
    ln_g, err = orc.jackknife(L, lnW, Hc)
    x = Hc[:, e0].astype(np.float64)
    expect = x.std(ddof=1) / math.sqrt(n) / x.mean()
    assert err[e0] == pytest.approx(expect, rel=0.02)
    assert err[e0 + 2] < 1e-6


def test_jackknife_marks_incomplete_energies(orc):
    L = 4
    lg = load_exact_ln_dos(L)
    lnW = np.where(np.isfinite(lg), -lg, 0.0)
    Hc = np.tile(np.where(np.isfinite(lg), 50, 0).astype(np.uint64), (4, 1))
    Hc[:, 0] = [7, 0, 0, 0]                 # ground state seen in one chunk only
    ln_g, err = orc.jackknife(L, lnW, Hc)
    assert np.isinf(err[0]) and np.isfinite(ln_g[0])
