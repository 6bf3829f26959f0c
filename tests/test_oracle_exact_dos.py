"""Pins the exact density of states (the reference of Sec. 3.3) by three independent
methods and by closed forms that follow from counting low-energy excitations."""
import math

import numpy as np
import pytest

from conftest import load_exact_dos_integers, load_exact_ln_dos


def test_bruteforce_L2_by_hand(orc):
    # 2x2 torus: each site has its right and down neighbour twice -> 8 bonds.
    # all equal: u = 0 (2 states); one flipped: u = 4 (8 states);
    # two flipped in a row or column: u = 4 (4 states); two flipped on a diagonal: u = 8 (2).
    assert orc.dos_bruteforce(2) == [2, 0, 12, 0, 2]


def test_bruteforce_equals_transfer_matrix(orc):
    assert orc.dos_transfer(4) == orc.dos_bruteforce(4)
    assert orc.dos_transfer(3) == orc.dos_bruteforce(3)


@pytest.mark.parametrize("L", [6, 8])
def test_low_energy_closed_forms(orc, L):
    """Excitations above the two ground states for L >= 5: one flipped spin (4 broken
    bonds), a flipped domino (6), and at 8 broken bonds two separated single flips, a
    straight or bent tromino or a 2x2 block; each doubled by the global flip."""
    g = orc.dos_transfer(L)
    N = L * L
    assert g[0] == 2 and g[1] == 0
    assert g[2] == 2 * N
    assert g[3] == 4 * N
    assert g[4] == 2 * (N * (N - 1) // 2 - 2 * N + 2 * N + 4 * N + N)


@pytest.mark.parametrize("L", [4, 6, 8])
def test_invariants(orc, L):
    g = orc.dos_transfer(L)
    N = L * L
    assert sum(g) == 2**N
    assert g == g[::-1]                               # g(E) = g(-E) for even L
    assert [e for e, x in enumerate(g) if x == 0] == [1, N - 1]


@pytest.mark.parametrize("L", [4, 6, 8])
def test_kaufman_equals_exact_enumeration(orc, L):
    from oracle import kaufman
    ref = orc.dos_bruteforce(L) if L == 4 else orc.dos_transfer(L)
    assert kaufman.exact_dos(L) == ref


@pytest.mark.parametrize("L", [16])
def test_kaufman_fixture_integers(L):
    g = load_exact_dos_integers(L)
    N = L * L
    assert sum(g) == 2**N and g == g[::-1]
    assert g[2] == 2 * N and g[3] == 4 * N and g[4] == N * (N - 1) + 10 * N
    assert [e for e, x in enumerate(g) if x == 0] == [1, N - 1]


def test_fixture_L32_log_values():
    lg = load_exact_ln_dos(32)
    N = 1024
    assert lg.shape == (N + 1,)
    assert np.isneginf(lg[1]) and np.isneginf(lg[N - 1])
    fin = np.isfinite(lg)
    m = lg[fin].max()
    total = m + math.log(np.exp(lg[fin] - m).sum())
    assert abs(total - N * math.log(2.0)) < 1e-9 * N
    assert lg[0] == pytest.approx(math.log(2))
    assert lg[2] == pytest.approx(math.log(2 * N))
    assert np.allclose(lg[fin], lg[::-1][fin], rtol=0, atol=1e-12)


@pytest.mark.parametrize("L", [4, 6, 8, 16])
def test_fixture_matches_generator(orc, L):
    lg = load_exact_ln_dos(L)
    g = orc.dos_bruteforce(L) if L == 4 else (orc.dos_transfer(L) if L <= 8 else load_exact_dos_integers(L))
    ref = np.array([math.log(x) if x else -np.inf for x in g])
    assert np.array_equal(lg, ref)


def test_fixture_L64_log_values():
    lg = load_exact_ln_dos(64)
    N = 4096
    assert lg.shape == (N + 1,)
    fin = np.isfinite(lg)
    assert [e for e in range(N + 1) if not fin[e]] == [1, N - 1]
    m = lg[fin].max()
    total = m + math.log(np.exp(lg[fin] - m).sum())
    assert abs(total - N * math.log(2.0)) < 1e-9 * N
    assert lg[0] == pytest.approx(math.log(2))
    assert lg[2] == pytest.approx(math.log(2 * N))
    assert lg[3] == pytest.approx(math.log(4 * N))
    assert lg[4] == pytest.approx(math.log(N * (N - 1) + 10 * N))
    assert np.allclose(lg[fin], lg[::-1][fin], rtol=0, atol=1e-12)
