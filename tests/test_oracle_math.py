"""Pins of the oracle's FP64 exp and ln (reading R8: a fixed sequence of IEEE double
operations used by the threshold table, the Eq. (4) recursion and the Eq. (6) measure)
against the C library's functions, which are an independent implementation, and against
identities that hold exactly."""
import math

import numpy as np
import pytest


def ulps(a: float, b: float) -> float:
    return 0.0 if a == b else abs(a - b) / math.ulp(b)


def test_exp_against_libm(orc):
    rng = np.random.default_rng(7)
    # the table's range (dw in [-23, 0)), the full double range, and tiny arguments
    xs = np.concatenate([rng.uniform(-23.0, 0.0, 20000), rng.uniform(-740.0, 705.0, 5000),
                         -np.logspace(-20, 0, 2000), np.logspace(-20, 0, 2000)])
    worst = max(ulps(orc.exp(float(x)), math.exp(float(x))) for x in xs)
    assert worst <= 1.0


def test_exp_special_values(orc):
    assert orc.exp(0.0) == 1.0
    assert orc.exp(-0.0) == 1.0
    assert orc.exp(-math.log(2.0)) == 0.5            # exp(-ln 2) rounds to 1/2 exactly
    for k in range(-20, 21):                         # near multiples of ln 2 (k = round(x/ln 2)
        x = k * math.log(2.0)                        # is decided at a tie boundary)
        for y in (x, math.nextafter(x, -math.inf), math.nextafter(x, math.inf)):
            assert ulps(orc.exp(y), math.exp(y)) <= 1.0
            assert orc.exp(y) == pytest.approx(2.0 ** k, rel=(abs(k) + 2) * 2 ** -52)
    assert orc.exp(-746.0) == 0.0
    assert orc.exp(710.0) == math.inf
    assert math.isnan(orc.exp(math.nan))
    assert orc.exp(1.0) == pytest.approx(math.e, rel=2 ** -52)


def test_log_against_libm(orc):
    rng = np.random.default_rng(8)
    ys = np.concatenate([np.arange(1, 20001, dtype=np.float64),               # histogram counts
                         rng.integers(1, 2 ** 53, 5000).astype(np.float64),
                         10.0 ** rng.uniform(-300, 300, 5000),
                         rng.uniform(0.5, 2.0, 10000)])                       # P q near 1 (KL)
    worst = max(ulps(orc.log(float(y)), math.log(float(y))) for y in ys)
    assert worst <= 3.0


def test_log_special_values_and_identities(orc):
    assert orc.log(1.0) == 0.0
    assert orc.log(0.0) == -math.inf
    assert math.isnan(orc.log(-1.0))
    assert orc.log(math.inf) == math.inf
    ln2 = math.log(2.0)
    for k in range(-1074, 1024, 37):                 # ln 2^k = k ln 2, subnormals included
        assert orc.log(math.ldexp(1.0, k)) == pytest.approx(k * ln2, rel=4 * 2 ** -52, abs=1e-300)
    rng = np.random.default_rng(9)
    for x in rng.uniform(-20.0, 20.0, 500):          # ln(exp(x)) = x
        assert orc.log(orc.exp(float(x))) == pytest.approx(float(x), rel=1e-15, abs=4e-16)
    for a, b in rng.integers(1, 2 ** 26, size=(500, 2)):   # ln(ab) = ln a + ln b
        assert orc.log(float(a) * float(b)) == pytest.approx(orc.log(float(a)) + orc.log(float(b)), rel=1e-15)


def test_table_uses_the_pinned_exp(orc):
    """Thresholds are floor(exp(dw) 2^32) with the pinned exp; against libm they may only
    differ where exp(dw) 2^32 lies within one ulp of an integer."""
    L = 8
    N = L * L
    rng = np.random.default_rng(10)
    lnW = np.cumsum(rng.normal(0.0, 2.0, N + 1))
    T = orc.build_table(L, lnW).reshape(N + 1, 5)
    for e in range(N + 1):
        for k in range(5):
            ep = e + 2 - k
            if not 0 <= ep <= N:
                assert T[e, k] == 0
                continue
            dw = lnW[ep] - lnW[e]
            if dw >= 0:
                assert T[e, k] == 0xFFFFFFFF
                continue
            assert T[e, k] == min(math.floor(orc.exp(dw) * 2 ** 32), 0xFFFFFFFF)
            v = math.exp(dw) * 2 ** 32
            assert abs(int(T[e, k]) - math.floor(v)) <= (1 if abs(v - round(v)) < 1e-6 else 0)
