/*
 * muca_oracle.c - plain CPU oracle for the parallel multicanonical (muca) simulation
 * of the 2D Ising model, after Gross, Zierenberg, Weigel and Janke, "Massively
 * parallel multicanonical simulations" (arXiv:1707.00919).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously correct reference the CUDA
 * path is checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  The product library never links, calls or falls back
 * to it, and the two share no code, header, table or constant generator.
 *
 * Every step follows the paper in its own order:
 *   - Ising energy, Eq. (5), periodic L x L lattice, J = 1 (Sec. 3);
 *   - energy grid E in [-2N, 2N] with spacing 4, N = L*L (Sec. 3), indexed by
 *     e = (E + 2N) / 4 in [0, N];
 *   - Metropolis acceptance min(1, exp[w(E') - w(E)]) with w = ln W (Sec. 2.3);
 *   - one shared site sequence for all walkers, an independent acceptance stream per
 *     walker from the counter-based Philox generator (Sec. 2.3);
 *   - p walkers with identical weights whose histograms are summed (Sec. 2.2);
 *   - weight recursion W <- W / H, Eq. (4), in logarithms (Sec. 2.1);
 *   - Kullback-Leibler flatness, Eq. (6); update schedule, Eq. (7); thermalization
 *     phase N_therm = f_therm * w (Sec. 3); Chebyshev distance, Eq. (A.1);
 *   - production run with fixed weights, ln Omega = ln H - ln W normalised so that
 *     the states sum to 2^N (Sec. 3.3).
 *
 * Where the paper is silent these fixed readings apply (the same readings are listed
 * with the design notes of the project):
 *   R1 site order: typewriter, site i = t mod N (x fastest), where t is the walker's
 *      attempt counter, monotone over the whole run (thermalization included).
 *   R2 random word for attempt t of walker w: Philox4x32-10 with key = (seed low 32,
 *      seed high 32) and counter = (low 32 of t>>2, high 32 of t>>2, w, tag), word
 *      t & 3; tag 0 = Metropolis, tag 1 = initial spins.  Initial spin at site i is +1
 *      iff the tag-1 word for t = i has its top bit clear.
 *   R3 integer acceptance: T = 0xFFFFFFFF if dw >= 0, else min(floor(exp(dw)*2^32),
 *      2^32-1) in FP64 with exp as in R8; T = 0 if the target energy is off the grid.
 *      A draw r is accepted iff r < T or T == 0xFFFFFFFF.
 *   R4 recording: after every recorded attempt the post-decision energy is counted.
 *   R5 recursion: ln W(e) -= ln H(e) with raw counts, only where H(e) > 0.
 *   R6 accessible energies: every grid point except e = 1 and e = N - 1.
 *   R7 the KL reference distribution Q is uniform over the accessible energies inside
 *      the union of the range covered in the previous iteration and the range of the
 *      histogram being tested (at least 10 of them), so that Q covers P's support and
 *      d_k >= 0 as Sec. 3 states; the schedule width w is the previous range's extent
 *      e_max - e_min + 1.
 *   R9 random site order (the paper's scheme of Sec. 2.3, an alternative to R1): the
 *      site of attempt t, the same for every walker, is floor(u N / 2^32) with u the
 *      Philox word t & 3 of counter (t >> 2, walker word 0xFFFFFFFF, tag 2); the
 *      acceptance word of walker w is the one of R2.
 *   R8 the exp of the threshold table (R3), the ln of the recursion (R5) and the ln of
 *      the Kullback-Leibler measure are orc_exp and orc_log below: a fixed sequence of
 *      IEEE double operations (Cody-Waite reduction with a Taylor series; an atanh
 *      series), so that a table built on another processor can be the same bit for bit.
 *      The paper evaluates expf in FP32 (Sec. 2.3); the production estimate and the
 *      reweighting keep the C library's exp and log.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TAG_METROPOLIS 0u
#define ORC_TAG_INIT 1u
#define ORC_TAG_SITE 2u
#define ORC_SHARED_STREAM 0xFFFFFFFFu   /* walker word of the site stream (R9) */

/* ---------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64 bit
 * multiplications whose halves are mixed with the other two counter words and the key;
 * the key is bumped by the Weyl constants between rounds.
 * ------------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Reading R2: the 32-bit word a walker draws for attempt t under a given tag. */
uint32_t orc_random_word(uint64_t seed, uint32_t walker, uint32_t tag, uint64_t t)
{
    uint64_t block = t >> 2;
    uint32_t ctr[4] = {(uint32_t)block, (uint32_t)(block >> 32), walker, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[t & 3u];
}

/* ---------------------------------------------------------------------------------
 * Lattice and energy, Eq. (5).  Spins are int8 +1/-1, one walker's lattice stored as
 * s[y*L + x].
 * ------------------------------------------------------------------------------- */
static int orc_site(int L, int x, int y)
{
    x = ((x % L) + L) % L;
    y = ((y % L) + L) % L;
    return y * L + x;
}

/* E = -sum over the 2N nearest-neighbour bonds of s_i s_j; returns e = (E + 2N)/4. */
int32_t orc_energy_index(int32_t L, const int8_t *s)
{
    const int N = L * L;
    long E = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int i = orc_site(L, x, y);
            E -= (long)s[i] * (long)s[orc_site(L, x + 1, y)];
            E -= (long)s[i] * (long)s[orc_site(L, x, y + 1)];
        }
    return (int32_t)((E + 2L * N) / 4);
}

/* Number of the four nearest neighbours of (x, y) antiparallel to s(x, y). */
static int orc_antiparallel(int L, const int8_t *s, int x, int y)
{
    int si = s[orc_site(L, x, y)];
    int k = 0;
    k += s[orc_site(L, x + 1, y)] != si;
    k += s[orc_site(L, x - 1, y)] != si;
    k += s[orc_site(L, x, y + 1)] != si;
    k += s[orc_site(L, x, y - 1)] != si;
    return k;
}

/* Reading R2: initial lattices of walkers walker0 .. walker0+nw-1 into spins[w][N],
 * and their energy indices. */
void orc_init(int32_t L, uint64_t seed, uint32_t walker0, int64_t nw, int8_t *spins, int32_t *e)
{
    const int N = L * L;
    for (int64_t w = 0; w < nw; ++w) {
        int8_t *s = spins + w * (int64_t)N;
        for (int i = 0; i < N; ++i) {
            uint32_t r = orc_random_word(seed, walker0 + (uint32_t)w, ORC_TAG_INIT, (uint64_t)i);
            s[i] = (r >> 31) ? (int8_t)-1 : (int8_t)1;
        }
        e[w] = orc_energy_index(L, s);
    }
}

/* ---------------------------------------------------------------------------------
 * exp and ln in FP64 (reading R8).  Every step is a single IEEE double operation
 * (round to nearest, no fused multiply-add), so any machine evaluates them to the same
 * bits; both stay within a few units in the last place of the C library's functions
 * (checked by the tests).
 * ------------------------------------------------------------------------------- */
static const double ORC_LN2_HEAD = 0x1.62e42fee00000p-1;   /* ln 2 to 31 bits          */
static const double ORC_LN2_TAIL = 0x1.a39ef35793c76p-33;  /* ln 2 - head, rounded     */
static const double ORC_INV_LN2 = 0x1.71547652b82fep+0;    /* 1 / ln 2, rounded        */
static const double ORC_SQRT2 = 0x1.6a09e667f3bcdp+0;      /* sqrt 2, rounded          */

/* 2^k as a double for -1022 <= k <= 1023 (built from its exponent field). */
static double orc_pow2i(int k)
{
    uint64_t b = (uint64_t)(k + 1023) << 52;
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
}

/* exp(x): Cody and Waite's reduction x = k ln 2 + r, k the integer nearest to x / ln 2
 * and ln 2 split into a head whose multiples by k are exact and a tail; exp(r), |r| <=
 * ln(2)/2, from its Taylor series through r^13 / 13! by Horner's rule (the remainder is
 * below 5e-18); the result scaled by 2^k in two exact steps. */
double orc_exp(double x)
{
    if (x != x)
        return x;
    if (x > 709.0)
        return INFINITY;
    if (x < -745.0)
        return 0.0;
    const double kd = floor(x * ORC_INV_LN2 + 0.5);
    const double r = (x - kd * ORC_LN2_HEAD) - kd * ORC_LN2_TAIL;
    /* 1/n! for n = 13 down to 0 */
    const double inv_fact[14] = {1.0 / 6227020800.0, 1.0 / 479001600.0, 1.0 / 39916800.0, 1.0 / 3628800.0,
                                 1.0 / 362880.0,     1.0 / 40320.0,     1.0 / 5040.0,     1.0 / 720.0,
                                 1.0 / 120.0,        1.0 / 24.0,        1.0 / 6.0,        1.0 / 2.0,
                                 1.0,                1.0};
    double p = inv_fact[0];
    for (int i = 1; i < 14; ++i)
        p = p * r + inv_fact[i];
    const int k = (int)kd;
    const int k1 = k / 2, k2 = k - k1;
    return (p * orc_pow2i(k1)) * orc_pow2i(k2);
}

/* ln(x), x > 0: x = 2^k m with m in [1/sqrt 2, sqrt 2], and
 * ln m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), s = (m - 1)/(m + 1), |s| <= 0.172,
 * summed through s^23 / 23 by Horner's rule in s^2 (the remainder is below 1e-18);
 * ln x = k (ln 2 head) + (k (ln 2 tail) + ln m). */
double orc_log(double x)
{
    if (x != x || x < 0.0)
        return NAN;
    if (x == 0.0)
        return -INFINITY;
    if (x == INFINITY)
        return INFINITY;
    int k = 0;
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    if (((b >> 52) & 0x7FFu) == 0u) {   /* subnormal: scale into the normal range */
        x = x * orc_pow2i(54);
        k = -54;
        memcpy(&b, &x, sizeof b);
    }
    k += (int)((b >> 52) & 0x7FFu) - 1023;
    b = (b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    double m;
    memcpy(&m, &b, sizeof m);
    if (m > ORC_SQRT2) {
        m = m * 0.5;
        k += 1;
    }
    const double s = (m - 1.0) / (m + 1.0);
    const double z = s * s;
    /* 1/(2n+1) for n = 11 down to 0 */
    const double inv_odd[12] = {1.0 / 23.0, 1.0 / 21.0, 1.0 / 19.0, 1.0 / 17.0, 1.0 / 15.0, 1.0 / 13.0,
                                1.0 / 11.0, 1.0 / 9.0,  1.0 / 7.0,  1.0 / 5.0,  1.0 / 3.0,  1.0};
    double q = inv_odd[0];
    for (int i = 1; i < 12; ++i)
        q = q * z + inv_odd[i];
    const double ln_m = (s + s) * q;
    const double kd = (double)k;
    return kd * ORC_LN2_HEAD + (kd * ORC_LN2_TAIL + ln_m);
}

/* ---------------------------------------------------------------------------------
 * Acceptance thresholds (Sec. 2.3, reading R3).  T[e*5 + k] is the threshold for a
 * flip at a site with k antiparallel neighbours from energy index e, which moves the
 * walker to e' = e + 2 - k (Delta E = 8 - 4k).
 * ------------------------------------------------------------------------------- */
void orc_build_table(int32_t L, const double *lnW, uint32_t *T)
{
    const int N = L * L;
    for (int e = 0; e <= N; ++e)
        for (int k = 0; k <= 4; ++k) {
            int ep = e + 2 - k;
            uint32_t thr;
            if (ep < 0 || ep > N) {
                thr = 0u;
            } else {
                double dw = lnW[ep] - lnW[e];
                if (dw >= 0.0) {
                    thr = 0xFFFFFFFFu;
                } else {
                    double v = floor(orc_exp(dw) * 4294967296.0);
                    thr = (v >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)v;
                }
            }
            T[e * 5 + k] = thr;
        }
}

int orc_accept(uint32_t r, uint32_t thr)
{
    return (r < thr) || (thr == 0xFFFFFFFFu);
}

/* ---------------------------------------------------------------------------------
 * Multicanonical Metropolis updates (Sec. 2.3, readings R1-R4).  Each walker performs
 * attempts t0 .. t0+n-1 independently; when record is set every post-decision energy
 * index is added to H (the sum over walkers, Sec. 2.2).
 * ------------------------------------------------------------------------------- */
void orc_run(int32_t L, uint64_t seed, uint32_t walker0, int64_t nw, int8_t *spins, int32_t *e,
             const uint32_t *T, uint64_t t0, uint64_t n, int32_t record, uint64_t *H)
{
    const int N = L * L;
    for (int64_t w = 0; w < nw; ++w) {
        const uint32_t walker = walker0 + (uint32_t)w;
        int8_t *s = spins + w * (int64_t)N;
        int32_t ew = e[w];
        uint64_t cached_block = UINT64_MAX;
        uint32_t words[4] = {0, 0, 0, 0};
        for (uint64_t t = t0; t < t0 + n; ++t) {
            /* the four words of one Philox call serve four consecutive attempts */
            if ((t >> 2) != cached_block) {
                cached_block = t >> 2;
                uint32_t ctr[4] = {(uint32_t)cached_block, (uint32_t)(cached_block >> 32), walker,
                                   ORC_TAG_METROPOLIS};
                uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
                orc_philox4x32_10(ctr, key, words);
            }
            const uint32_t r = words[t & 3u];
            const int i = (int)(t % (uint64_t)N);
            const int x = i % L, y = i / L;
            const int k = orc_antiparallel(L, s, x, y);
            if (orc_accept(r, T[ew * 5 + k])) {
                s[i] = (int8_t)(-s[i]);
                ew += 2 - k;
            }
            if (record)
                H[ew] += 1u;
        }
        e[w] = ew;
    }
}

/* Site of attempt t in random order (R9): one shared stream for all walkers. */
int32_t orc_random_site(int32_t L, uint64_t seed, uint64_t t)
{
    const uint32_t u = orc_random_word(seed, ORC_SHARED_STREAM, ORC_TAG_SITE, t);
    return (int32_t)(((uint64_t)u * (uint64_t)(L * L)) >> 32);
}

/* The same updates with the sites of R9 instead of typewriter order (Sec. 2.3: one
 * random site sequence for all walkers, an independent acceptance stream per walker). */
void orc_run_random(int32_t L, uint64_t seed, uint32_t walker0, int64_t nw, int8_t *spins, int32_t *e,
                    const uint32_t *T, uint64_t t0, uint64_t n, int32_t record, uint64_t *H)
{
    const int N = L * L;
    for (int64_t w = 0; w < nw; ++w) {
        const uint32_t walker = walker0 + (uint32_t)w;
        int8_t *s = spins + w * (int64_t)N;
        int32_t ew = e[w];
        for (uint64_t t = t0; t < t0 + n; ++t) {
            const uint32_t r = orc_random_word(seed, walker, ORC_TAG_METROPOLIS, t);
            const int i = orc_random_site(L, seed, t);
            const int x = i % L, y = i / L;
            const int k = orc_antiparallel(L, s, x, y);
            if (orc_accept(r, T[ew * 5 + k])) {
                s[i] = (int8_t)(-s[i]);
                ew += 2 - k;
            }
            if (record)
                H[ew] += 1u;
        }
        e[w] = ew;
    }
}

/* Updates in the order the parameters ask for. */
static void orc_update(int32_t order, int32_t L, uint64_t seed, int64_t nw, int8_t *spins, int32_t *e,
                       const uint32_t *T, uint64_t t0, uint64_t n, int32_t record, uint64_t *H)
{
    if (order == 1)
        orc_run_random(L, seed, 0u, nw, spins, e, T, t0, n, record, H);
    else
        orc_run(L, seed, 0u, nw, spins, e, T, t0, n, record, H);
}

/* ---------------------------------------------------------------------------------
 * Weight recursion, Eq. (4), in logarithms (reading R5).
 * ------------------------------------------------------------------------------- */
void orc_update_weights(int32_t L, double *lnW, const uint64_t *H)
{
    const int N = L * L;
    for (int e = 0; e <= N; ++e)
        if (H[e] > 0u)
            lnW[e] -= orc_log((double)H[e]);
}

/* ---------------------------------------------------------------------------------
 * Flatness measures.
 * ------------------------------------------------------------------------------- */
int orc_accessible(int32_t L, int32_t e)
{
    const int N = L * L;
    return e >= 0 && e <= N && e != 1 && e != N - 1;
}

/* min H / mean H over the N - 1 accessible energies (0 when H is empty). */
double orc_min_over_mean(int32_t L, const uint64_t *H)
{
    const int N = L * L;
    double total = 0.0;
    uint64_t hmin = UINT64_MAX;
    for (int e = 0; e <= N; ++e) {
        if (!orc_accessible(L, e))
            continue;
        total += (double)H[e];
        if (H[e] < hmin)
            hmin = H[e];
    }
    if (total <= 0.0)
        return 0.0;
    double mean = total / (double)(N - 1);
    return (double)hmin / mean;
}

/* Extent e_max - e_min + 1 of the visited energies (0 if none); the "width in units
 * of Delta E" of Sec. 3. */
int32_t orc_width(int32_t L, const uint64_t *H)
{
    const int N = L * L;
    int lo = -1, hi = -1;
    for (int e = 0; e <= N; ++e)
        if (H[e] > 0u) {
            if (lo < 0)
                lo = e;
            hi = e;
        }
    return lo < 0 ? 0 : hi - lo + 1;
}

/* Accessible energies between the lowest and highest visited energy (reading R7). */
int32_t orc_accessible_in_range(int32_t L, const uint64_t *H)
{
    const int N = L * L;
    int lo = -1, hi = -1;
    for (int e = 0; e <= N; ++e)
        if (H[e] > 0u) {
            if (lo < 0)
                lo = e;
            hi = e;
        }
    if (lo < 0)
        return 0;
    int count = 0;
    for (int e = lo; e <= hi; ++e)
        count += orc_accessible(L, e);
    return count;
}

/* Reading R7: accessible energies in the union of [prev_lo, prev_hi] (none if
 * prev_lo < 0) and the visited range of H, at least 10. */
int32_t orc_kl_support(int32_t L, int32_t prev_lo, int32_t prev_hi, const uint64_t *H)
{
    const int N = L * L;
    int lo = prev_lo, hi = prev_hi;
    for (int e = 0; e <= N; ++e)
        if (H[e] > 0u) {
            if (lo < 0 || e < lo)
                lo = e;
            if (hi < 0 || e > hi)
                hi = e;
        }
    int count = 0;
    if (lo >= 0)
        for (int e = lo; e <= hi; ++e)
            count += orc_accessible(L, e);
    return count > 10 ? count : 10;
}

/* Kullback-Leibler divergence, Eq. (6): d_k = sum P ln(P/Q) with P = H / sum(H) and
 * Q = 1/q, empty bins contributing nothing. */
double orc_kullback_leibler(int32_t L, const uint64_t *H, double q)
{
    const int N = L * L;
    double total = 0.0;
    for (int e = 0; e <= N; ++e)
        total += (double)H[e];
    if (total <= 0.0)
        return INFINITY;
    double dk = 0.0;
    for (int e = 0; e <= N; ++e) {
        if (H[e] == 0u)
            continue;
        double P = (double)H[e] / total;
        dk += P * orc_log(P * q);
    }
    return dk;
}

/* Chebyshev distance, Eq. (A.1): max |H/m - 1| over the accessible energies with
 * m = sum(H) / (N - 1). */
double orc_chebyshev(int32_t L, const uint64_t *H)
{
    const int N = L * L;
    double total = 0.0;
    for (int e = 0; e <= N; ++e)
        total += (double)H[e];
    if (total <= 0.0)
        return INFINITY;
    double m = total / (double)(N - 1);
    double dc = 0.0;
    for (int e = 0; e <= N; ++e) {
        if (!orc_accessible(L, e))
            continue;
        double d = fabs((double)H[e] / m - 1.0);
        if (d > dc)
            dc = d;
    }
    return dc;
}

/* ---------------------------------------------------------------------------------
 * Weight iteration (Sec. 2.2 and Sec. 3): thermalize without recording, record a
 * fresh histogram, test flatness, otherwise W <- W / H, Eq. (4).
 * ------------------------------------------------------------------------------- */
typedef struct {
    int32_t schedule;        /* 0: fixed sweeps per iteration; 1: Eq. (7) schedule   */
    int32_t stop_rule;       /* 0: min/mean >= thr; 1: d_k < thr; 2: d_c < thr       */
    double flat_threshold;
    uint64_t therm_sweeps;   /* schedule 0: sweeps (N attempts) without recording    */
    uint64_t sweeps_per_iter;/* schedule 0: recorded sweeps per iteration            */
    double f_therm;          /* schedule 1: N_therm = f_therm * w attempts           */
    double z;                /* schedule 1: N_updates = floor(factor w^z / W) + 1    */
    double factor;
    double growth;           /* schedule 1: after full coverage, floor(growth N) + 1 */
    int32_t max_iterations;
    int32_t site_order;      /* 0: typewriter (R1); 1: random shared sites (R9)      */
} orc_params;

typedef struct {
    int32_t iterations;      /* iterations run                                        */
    int32_t converged;       /* 1 if the stop rule held after the last iteration      */
    double last_metric;      /* the stop-rule metric of the last iteration            */
    uint64_t t;              /* attempt counter after the run                         */
    uint64_t attempts;       /* attempts per walker spent in the run                  */
} orc_result;

static double orc_stop_metric(int32_t L, const uint64_t *H, int32_t rule, double q)
{
    if (rule == 0)
        return orc_min_over_mean(L, H);
    if (rule == 1)
        return orc_kullback_leibler(L, H, q);
    return orc_chebyshev(L, H);
}

static int orc_is_flat(int32_t rule, double metric, double thr)
{
    return rule == 0 ? (metric >= thr) : (metric < thr);
}

/*
 * Runs the weight iteration for nw walkers (walker ids 0 .. nw-1) from the given
 * lattices, energies, weights and attempt counter.  On return lnW holds the weights
 * of the last iteration run (unchanged by the final histogram when it was flat), and
 * t_inout the advanced attempt counter.  lnW_history[n*(N+1) + e] (optional) receives
 * the weights used in iteration n, metric_history[n] (optional) its stop metric, and
 * sched_history[4n .. 4n+3] (optional) its thermalization and update attempts per
 * walker and the lowest and highest energy index its histogram visited (-1 if none).
 */
int32_t orc_iterate_traced(int32_t L, int64_t nw, uint64_t seed, int8_t *spins, int32_t *e, double *lnW,
                           uint64_t *t_inout, const orc_params *p, double *lnW_history,
                           double *metric_history, int64_t *sched_history, orc_result *res)
{
    const int N = L * L;
    uint64_t *H = (uint64_t *)calloc((size_t)N + 1, sizeof(uint64_t));
    uint32_t *T = (uint32_t *)malloc(((size_t)N + 1) * 5 * sizeof(uint32_t));
    if (!H || !T) {
        free(H);
        free(T);
        return -1;
    }
    uint64_t t = *t_inout;
    uint64_t spent = 0;
    int32_t prev_width = 0;      /* width covered in the previous iteration */
    int32_t prev_lo = -1, prev_hi = -1;   /* that range                       */
    int full = 0;                /* the whole range has been covered        */
    uint64_t n_upd_prev = 0;
    int32_t n = 0;
    int converged = 0;
    double metric = 0.0;
    while (n < p->max_iterations) {
        uint64_t n_therm, n_upd;
        if (p->schedule == 0) {
            n_therm = p->therm_sweeps * (uint64_t)N;
            n_upd = p->sweeps_per_iter * (uint64_t)N;
        } else {
            int32_t w = prev_width > 10 ? prev_width : 10;
            n_therm = (uint64_t)(p->f_therm * (double)w);
            if (full) {
                /* every iteration after the first full-width one grows by `growth` */
                n_upd = (uint64_t)floor(p->growth * (double)n_upd_prev) + 1u;
            } else {
                n_upd = (uint64_t)floor(p->factor * pow((double)w, p->z) / (double)nw) + 1u;
                if (prev_width == N + 1)
                    full = 1;
            }
        }
        if (lnW_history)
            memcpy(lnW_history + (size_t)n * (N + 1), lnW, sizeof(double) * (N + 1));
        orc_build_table(L, lnW, T);
        orc_update(p->site_order, L, seed, nw, spins, e, T, t, n_therm, 0, NULL);
        t += n_therm;
        memset(H, 0, sizeof(uint64_t) * (N + 1));
        orc_update(p->site_order, L, seed, nw, spins, e, T, t, n_upd, 1, H);
        t += n_upd;
        spent += n_therm + n_upd;
        const double q = (double)orc_kl_support(L, prev_lo, prev_hi, H);
        metric = orc_stop_metric(L, H, p->stop_rule, q);
        if (metric_history)
            metric_history[n] = metric;
        if (sched_history) {
            int64_t *rec = sched_history + 4 * (size_t)n;
            rec[0] = (int64_t)n_therm;
            rec[1] = (int64_t)n_upd;
            rec[2] = -1;
            rec[3] = -1;
            for (int ei = 0; ei <= N; ++ei)
                if (H[ei] > 0u) {
                    if (rec[2] < 0)
                        rec[2] = ei;
                    rec[3] = ei;
                }
        }
        ++n;
        if (orc_is_flat(p->stop_rule, metric, p->flat_threshold)) {
            converged = 1;
            break;
        }
        orc_update_weights(L, lnW, H);
        prev_width = orc_width(L, H);
        prev_lo = -1;
        prev_hi = -1;
        for (int e = 0; e <= N; ++e)
            if (H[e] > 0u) {
                if (prev_lo < 0)
                    prev_lo = e;
                prev_hi = e;
            }
        n_upd_prev = n_upd;
    }
    *t_inout = t;
    if (res) {
        res->iterations = n;
        res->converged = converged;
        res->last_metric = metric;
        res->t = t;
        res->attempts = spent;
    }
    free(H);
    free(T);
    return 0;
}

int32_t orc_iterate(int32_t L, int64_t nw, uint64_t seed, int8_t *spins, int32_t *e, double *lnW,
                    uint64_t *t_inout, const orc_params *p, double *lnW_history,
                    double *metric_history, orc_result *res)
{
    return orc_iterate_traced(L, nw, seed, spins, e, lnW, t_inout, p, lnW_history, metric_history, NULL, res);
}

/* ---------------------------------------------------------------------------------
 * Production run (Sec. 3.3): fixed weights, a thermalization phase, then recorded
 * updates; ln Omega(e) = ln H(e) - ln W(e) on visited energies, shifted so that
 * sum_e exp(ln Omega(e)) = 2^N.  Unvisited energies get -inf.
 * ------------------------------------------------------------------------------- */
void orc_ln_dos(int32_t L, const double *lnW, const uint64_t *H, double *ln_g)
{
    const int N = L * L;
    double m = -INFINITY;
    for (int e = 0; e <= N; ++e) {
        ln_g[e] = H[e] > 0u ? log((double)H[e]) - lnW[e] : -INFINITY;
        if (ln_g[e] > m)
            m = ln_g[e];
    }
    if (m == -INFINITY)
        return;
    double s = 0.0;
    for (int e = 0; e <= N; ++e)
        if (H[e] > 0u)
            s += exp(ln_g[e] - m);
    double shift = (double)N * log(2.0) - (m + log(s));
    for (int e = 0; e <= N; ++e)
        if (H[e] > 0u)
            ln_g[e] += shift;
}

int32_t orc_production(int32_t L, int64_t nw, uint64_t seed, int8_t *spins, int32_t *e,
                       const double *lnW, uint64_t *t_inout, uint64_t therm_sweeps,
                       uint64_t sweeps, uint64_t *H, double *ln_g, int32_t site_order)
{
    const int N = L * L;
    uint32_t *T = (uint32_t *)malloc(((size_t)N + 1) * 5 * sizeof(uint32_t));
    if (!T)
        return -1;
    uint64_t t = *t_inout;
    orc_build_table(L, lnW, T);
    orc_update(site_order, L, seed, nw, spins, e, T, t, therm_sweeps * (uint64_t)N, 0, NULL);
    t += therm_sweeps * (uint64_t)N;
    memset(H, 0, sizeof(uint64_t) * (N + 1));
    orc_update(site_order, L, seed, nw, spins, e, T, t, sweeps * (uint64_t)N, 1, H);
    t += sweeps * (uint64_t)N;
    orc_ln_dos(L, lnW, H, ln_g);
    *t_inout = t;
    free(T);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Jackknife errors of the production estimate (Sec. 3.3): the recorded updates are
 * split into n chunks with histograms Hc[c][e]; estimate c leaves chunk c out,
 * ln g_(c) = normalised ln(H - Hc[c]) - ln W, and the error of ln g(e) is
 * sqrt((n - 1)/n sum_c (ln g_(c)(e) - mean_c ln g_(c)(e))^2).  ln_g receives the
 * estimate from all chunks.  Energies missing from some leave-one-out histogram get an
 * infinite error; energies never visited get -inf and an error of NaN.
 * ------------------------------------------------------------------------------- */
int32_t orc_jackknife(int32_t L, const double *lnW, const uint64_t *Hc, int32_t n, double *ln_g, double *err)
{
    const int N = L * L;
    const int B = N + 1;
    uint64_t *tot = (uint64_t *)calloc((size_t)B, sizeof(uint64_t));
    uint64_t *Hm = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)B);
    double *est = (double *)malloc(sizeof(double) * (size_t)B * (size_t)n);
    if (!tot || !Hm || !est) {
        free(tot);
        free(Hm);
        free(est);
        return -1;
    }
    for (int c = 0; c < n; ++c)
        for (int e = 0; e < B; ++e)
            tot[e] += Hc[(size_t)c * B + e];
    orc_ln_dos(L, lnW, tot, ln_g);
    for (int c = 0; c < n; ++c) {
        for (int e = 0; e < B; ++e)
            Hm[e] = tot[e] - Hc[(size_t)c * B + e];
        orc_ln_dos(L, lnW, Hm, est + (size_t)c * B);
    }
    for (int e = 0; e < B; ++e) {
        if (tot[e] == 0u) {
            err[e] = NAN;
            continue;
        }
        double mean = 0.0;
        int missing = 0;
        for (int c = 0; c < n; ++c) {
            double v = est[(size_t)c * B + e];
            if (v == -INFINITY)
                missing = 1;
            mean += v;
        }
        if (missing) {
            err[e] = INFINITY;
            continue;
        }
        mean /= (double)n;
        double s = 0.0;
        for (int c = 0; c < n; ++c) {
            double d = est[(size_t)c * B + e] - mean;
            s += d * d;
        }
        err[e] = sqrt((double)(n - 1) / (double)n * s);
    }
    free(tot);
    free(Hm);
    free(est);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Reweighting to the canonical ensemble (Sec. 2.1, Sec. 3.3): with P(E) ~ g(E) e^{-beta E}
 * (Eq. 1) from ln g on the energy grid E = -2N + 4e, the mean energy per spin <E>/N and
 * the specific heat per spin beta^2 (<E^2> - <E>^2) / N, by log-sum-exp.
 * ------------------------------------------------------------------------------- */
void orc_canonical(int32_t L, const double *ln_g, double beta, double *e_per_spin, double *c_per_spin)
{
    const int N = L * L;
    double m = -INFINITY;
    for (int e = 0; e <= N; ++e) {
        if (ln_g[e] == -INFINITY)
            continue;
        double E = -2.0 * N + 4.0 * e;
        double v = ln_g[e] - beta * E;
        if (v > m)
            m = v;
    }
    double z = 0.0, s1 = 0.0, s2 = 0.0;
    for (int e = 0; e <= N; ++e) {
        if (ln_g[e] == -INFINITY)
            continue;
        double E = -2.0 * N + 4.0 * e;
        double w = exp(ln_g[e] - beta * E - m);
        z += w;
        s1 += w * E;
        s2 += w * E * E;
    }
    double mean = s1 / z;
    double var = s2 / z - mean * mean;
    *e_per_spin = mean / (double)N;
    *c_per_spin = beta * beta * var / (double)N;
}
