"""Exact density of states of the periodic L x L Ising model from Kaufman's closed form.

TEST INFRASTRUCTURE ONLY (part of the oracle; the product path never imports it).

Gross, Zierenberg, Weigel and Janke (arXiv:1707.00919) check their production-run
estimate of ln Omega(E) against the exact finite-lattice density of states of the
model of Eq. (5) (Sec. 3.3, after Beale).  Beale's tables are not available here, so the
integers g(e), e = (E + 2N)/4, are recomputed from Kaufman's partition function of the
m x n torus (m = n = L even, K = beta J):

    Z = 1/2 (2 sinh 2K)^(N/2) (Z1 + Z2 + Z3 + Z4)
    Z1 = prod_{r<n} 2 cosh(m g_{2r+1}/2)    Z2 = prod_{r<n} 2 sinh(m g_{2r+1}/2)
    Z3 = prod_{r<n} 2 cosh(m g_{2r}/2)      Z4 = prod_{r<n} 2 sinh(m g_{2r}/2)
    cosh g_l = cosh 2K coth 2K - cos(pi l / n),  exp(g_0) = exp(2K) tanh K (signed).

Branch-free evaluation: the angles l and 2n - l share cos(pi l/n), so their factors
pair into squares, (2 cosh(m g/2))^2 = 2 + 2 T_m(cosh g) and
(2 sinh(m g/2))^2 = 2 T_m(cosh g) - 2 with the Chebyshev polynomial T_m; only l = 0
and l = n stay single, and for them exp(g_0) = e^{2K} tanh K, exp(g_n) = e^{2K} coth K
with m even give rational powers.  With v = e^{2K} everything is a rational function
of v, and P(z) = sum_e g(e) z^e = Z v^(-N) with z = e^{-4K} = v^(-2).  P is evaluated
at M >= N+1 equally spaced points on the unit circle (M a power of two, offset by half
a step so that the singular point z = 1 is avoided) in high-precision complex
arithmetic, and the inverse discrete Fourier transform, rounded to integers, gives g(e)
(coefficients above e = N must come out zero, a built-in check).  The working precision
is raised until two precisions give identical integers.
"""
from __future__ import annotations

import math

import mpmath


def _chebyshev_T(m: int, c):
    """T_m(c) by the doubling recurrence on (T_k, T_{k+1})."""
    if m == 0:
        return mpmath.mpc(1)
    t0, t1 = mpmath.mpc(1), c  # T_0, T_1
    # binary expansion of m: maintain (T_k, T_{k+1})
    a, b = t0, t1
    for bit in bin(m)[2:]:
        if bit == "0":
            # (T_2k, T_2k+1)
            a, b = 2 * a * a - 1, 2 * a * b - c
        else:
            # (T_2k+1, T_2k+2)
            a, b = 2 * a * b - c, 2 * b * b - 1
    return a


def _P(L: int, v):
    """P(z) = Z(K) e^{-2NK} at v = e^{2K} (any square root of 1/z)."""
    n = m = L
    N = L * L
    one = mpmath.mpc(1)
    c2 = (v + one / v) / 2            # cosh 2K
    s2 = (v - one / v) / 2            # sinh 2K
    A = c2 * c2 / s2                  # cosh 2K coth 2K
    th = (v - one) / (v + one)        # tanh K
    z1 = z2 = z3 = z4 = one
    for l in range(1, n, 2):          # odd l, paired with 2n - l
        T = _chebyshev_T(m, A - mpmath.cospi(mpmath.mpf(l) / n))
        z1 *= 2 + 2 * T
        z2 *= 2 * T - 2
    for l in range(2, n, 2):          # even l in 2 .. n-2, paired with 2n - l
        T = _chebyshev_T(m, A - mpmath.cospi(mpmath.mpf(l) / n))
        z3 *= 2 + 2 * T
        z4 *= 2 * T - 2
    a0 = (v * th) ** (m // 2)         # e^{m g_0 / 2}
    an = (v / th) ** (m // 2)         # e^{m g_n / 2}
    z3 *= (a0 + one / a0) * (an + one / an)
    z4 *= (a0 - one / a0) * (an - one / an)
    Z = (2 * s2) ** (N // 2) * (z1 + z2 + z3 + z4) / 2
    return Z / v ** N


def _fft_inverse(a: list) -> list:
    """Unnormalised inverse DFT, out[e] = sum_j a[j] exp(+2 pi i j e / M), M a power of 2
    (iterative radix-2)."""
    M = len(a)
    out = list(a)
    # bit-reversal permutation
    j = 0
    for i in range(1, M):
        bit = M >> 1
        while j & bit:
            j ^= bit
            bit >>= 1
        j |= bit
        if i < j:
            out[i], out[j] = out[j], out[i]
    size = 2
    while size <= M:
        half = size // 2
        w_step = [mpmath.expjpi(mpmath.mpf(2 * k) / size) for k in range(half)]
        for start in range(0, M, size):
            for k in range(half):
                u = out[start + k]
                t = out[start + k + half] * w_step[k]
                out[start + k] = u + t
                out[start + k + half] = u - t
        size *= 2
    return out


def _dos_at_precision(L: int, bits: int) -> list[int]:
    N = L * L
    M = 1
    while M < N + 1:
        M *= 2
    with mpmath.workprec(bits):
        vals = [None] * M
        for j in range(M):
            if vals[j] is not None:
                continue
            frac = mpmath.mpf(2 * j + 1) / M               # z_j = exp(i pi frac)
            p = _P(L, mpmath.expjpi(-frac / 2))            # v = z^{-1/2}
            vals[j] = p
            jc = M - 1 - j                                  # z_jc = conj(z_j)
            if jc != j:
                vals[jc] = mpmath.conj(p)
        # g(e) = (1/M) sum_j P(z_j) z_j^{-e} with z_j = zeta w^j, zeta = exp(i pi / M),
        # w = exp(2 pi i / M): the sum is zeta^{-e} times the DFT of P_j at -e.
        rev = [vals[0]] + vals[:0:-1]                      # a[j] -> a[-j]: turns +e into -e
        F = _fft_inverse(rev)
        g = []
        for e in range(M):
            val = F[e] * mpmath.expjpi(-mpmath.mpf(e) / M) / M
            g.append(int(mpmath.nint(val.real)))
        if any(g[N + 1:]):
            raise ArithmeticError("coefficients beyond the top energy did not vanish")
        return g[: N + 1]


def exact_dos(L: int, start_bits: int | None = None) -> list[int]:
    """Exact integers g(e), e = 0 .. L*L, for even L >= 4."""
    if L < 4 or L % 2:
        raise ValueError("Kaufman evaluation implemented for even L >= 4")
    N = L * L
    bits = start_bits if start_bits is not None else N + 64
    prev = _dos_at_precision(L, bits)
    while True:
        bits += 64 + bits // 8
        cur = _dos_at_precision(L, bits)
        if cur == prev:
            return cur
        prev = cur


def ln_dos_from_integers(g: list[int]) -> list[float]:
    """ln g(e) in FP64 (-inf where g = 0), exact up to the final rounding."""
    out = []
    for x in g:
        out.append(math.log(x) if x > 0 else float("-inf"))
    return out
