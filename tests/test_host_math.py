"""The library's host-side arithmetic against the oracle, without a GPU: threshold tables
(Sec. 2.3 rule, FP64 exp of reading R8) and the Eq. (4) recursion (FP64 ln), bit for
bit, on weights that reach every branch of the rule (always accept, exp underflowing the
2^-32 grid, exp rounding to 1, off-grid targets)."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def mm():
    from paper_1707_00919_gb300 import build
    build.build()
    from paper_1707_00919_gb300 import muca
    return muca


@pytest.mark.parametrize("L", [4, 8, 16, 32, 64])
@pytest.mark.parametrize("scale", [1e-9, 0.3, 3.0, 30.0])
def test_table_matches_oracle(mm, orc, L, scale):
    rng = np.random.default_rng(L * 1000 + int(scale * 10))
    lnW = np.cumsum(rng.normal(0.0, scale, L * L + 1))
    T = mm.muca_build_table(L, lnW)
    To = orc.build_table(L, lnW)
    assert np.array_equal(T, To)


def test_table_branches(mm, orc):
    L = 4
    N = L * L
    lnW = np.zeros(N + 1)
    lnW[6] = -math.log(2.0)
    lnW[9] = -60.0
    lnW[12] = -1e-18
    T = mm.muca_build_table(L, lnW).reshape(N + 1, 5)
    assert np.array_equal(T.ravel(), orc.build_table(L, lnW))
    assert T[5, 1] == 2 ** 31 and T[8, 1] == 0 and T[11, 1] == 0xFFFFFFFF and T[0, 4] == 0


@pytest.mark.parametrize("L", [4, 32, 64])
def test_recursion_matches_oracle(mm, orc, L):
    rng = np.random.default_rng(L)
    N = L * L
    lnW = rng.normal(0.0, 5.0, N + 1)
    H = rng.integers(0, 2 ** 40, N + 1).astype(np.uint64)
    H[rng.random(N + 1) < 0.3] = 0
    H[:3] = [1, 2, 2 ** 53]
    a, b = lnW.copy(), lnW.copy()
    mm.muca_update_weights(L, a, H)
    orc.update_weights(L, b, H)
    assert np.array_equal(a, b)
    assert np.array_equal(a[H == 0], lnW[H == 0])


def test_host_helpers_reject_bad_arguments(mm):
    with pytest.raises(mm.MucaError):
        mm.muca_build_table(6, np.zeros(37))
    with pytest.raises(mm.MucaError):
        mm.muca_build_table(4, np.zeros(16))
    bad = np.zeros(17)
    bad[2] = np.inf
    with pytest.raises(mm.MucaError):
        mm.muca_build_table(4, bad)
    with pytest.raises(mm.MucaError):
        mm.muca_update_weights(4, np.zeros(16), np.zeros(16, dtype=np.uint64))


def _kl_support(orc, L, prev, H):
    import ctypes
    h = np.ascontiguousarray(H, dtype=np.uint64)
    return orc.lib().orc_kl_support(L, prev[0], prev[1], h.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))


@pytest.mark.parametrize("L", [4, 8, 32, 64])
def test_flatness_measures_match_oracle(mm, orc, L):
    """min/mean, d_k of Eq. (6) with the reading-R7 reference width, d_c of Eq. (A.1) and
    the visited range, bit for bit against the oracle, on histograms with gaps, a single
    bin, an empty one and flat ones, with and without a previous range."""
    N = L * L
    rng = np.random.default_rng(L)
    cases = []
    for _ in range(6):
        H = rng.integers(0, 1000, N + 1).astype(np.uint64)
        H[rng.random(N + 1) < 0.3] = 0
        cases.append(H)
    one = np.zeros(N + 1, np.uint64)
    one[N // 2] = 7
    flat = np.full(N + 1, 50, np.uint64)
    flat[[1, N - 1]] = 0
    cases += [one, flat, np.zeros(N + 1, np.uint64)]
    for H in cases:
        for prev in [(-1, -1), (0, N // 3), (N // 4, N)]:
            got = mm.muca_flatness(L, H, prev)
            q = _kl_support(orc, L, prev, H)
            nz = np.nonzero(H)[0]
            assert got["range"] == ((int(nz[0]), int(nz[-1])) if nz.size else (-1, -1))
            assert got["min_over_mean"] == orc.min_over_mean(L, H)
            assert got["chebyshev"] == orc.chebyshev(L, H)
            assert got["kl"] == orc.kullback_leibler(L, H, float(q))


def test_flatness_selected_measures(mm):
    """Only the named measures are computed (the others are passed as NULL); each equals
    the value of the call that computes all three, and the range is always returned."""
    L = 16
    N = L * L
    H = np.random.default_rng(5).integers(1, 500, N + 1).astype(np.uint64)
    full = mm.muca_flatness(L, H, (2, N - 3))
    for measures in [("min_over_mean",), ("kl",), ("chebyshev",), ("min_over_mean", "kl")]:
        got = mm.muca_flatness(L, H, (2, N - 3), measures=measures)
        assert set(got) == set(measures) | {"range"}
        assert got["range"] == full["range"]
        for k in measures:
            assert got[k] == full[k]


def test_flatness_rejects_bad_input(mm):
    N = 64
    with pytest.raises(mm.MucaError):
        mm.muca_flatness(8, np.zeros(N, np.uint64))
    with pytest.raises(mm.MucaError):
        mm.muca_flatness(6, np.zeros(37, np.uint64))
    with pytest.raises(mm.MucaError):
        mm.muca_flatness(8, np.zeros(N + 1, np.uint64), (10, 5))
    with pytest.raises(mm.MucaError):
        mm.muca_flatness(8, np.zeros(N + 1, np.uint64), (10, N + 1))
