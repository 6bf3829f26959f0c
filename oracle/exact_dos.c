/*
 * exact_dos.c - exact density of states g(E) of the periodic L x L Ising model,
 * Eq. (5) of Gross, Zierenberg, Weigel and Janke (arXiv:1707.00919), which compare
 * their estimate with the exact finite-lattice result in Sec. 3.3.
 *
 * TEST INFRASTRUCTURE ONLY (part of the oracle; never used by the product path).
 *
 * Two independent exact-integer methods:
 *   orc_dos_bruteforce  enumerates all 2^N configurations (L <= 5);
 *   orc_dos_transfer    sums over the configurations row by row with a site-by-site
 *                       transfer matrix in unsigned 128-bit integers (L <= 8).
 * Both return g indexed by e = u / 2, where u is the number of unsatisfied bonds, so
 * that E = -2N + 4e as in the energy grid of Sec. 3.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Plain enumeration: bit i of the state is the spin at site i (1 = down). */
int32_t orc_dos_bruteforce(int32_t L, uint64_t *g)
{
    if (L < 2 || L > 5)
        return -1;
    const int N = L * L;
    memset(g, 0, sizeof(uint64_t) * (N + 1));
    const uint64_t states = 1ull << N;
    for (uint64_t c = 0; c < states; ++c) {
        int u = 0;
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int i = y * L + x;
                int right = y * L + (x + 1) % L;
                int down = ((y + 1) % L) * L + x;
                int si = (int)((c >> i) & 1u);
                u += si != (int)((c >> right) & 1u);
                u += si != (int)((c >> down) & 1u);
            }
        g[u / 2] += 1u;
    }
    return 0;
}

/*
 * Transfer matrix over the torus.  For every configuration r0 of row 0 the rows
 * 1 .. L-1 are added one site at a time; the state is the "profile" of the L most
 * recently placed sites (bit x = spin at column x of the newest row that reached x)
 * together with the polynomial (in u) of the summed weights.  Bonds are counted as
 * each site is placed: up (profile bit x, previous row), left (bit x-1, same row) and,
 * for the last column, the wrap-around bond to column 0 of the same row.  At the end
 * the vertical bonds between row L-1 and row 0 close the torus.
 * g_lo/g_hi receive the low and high 64 bits of each g(e).
 */
typedef unsigned __int128 u128;

int32_t orc_dos_transfer(int32_t L, uint64_t *g_lo, uint64_t *g_hi)
{
    if (L < 2 || L > 8)
        return -1;
    const int N = L * L;
    const int U = 2 * N + 1;              /* u = 0 .. 2N */
    const int S = 1 << L;                 /* profiles    */
    u128 *cur = (u128 *)calloc((size_t)S * U, sizeof(u128));
    u128 *nxt = (u128 *)calloc((size_t)S * U, sizeof(u128));
    u128 *tot = (u128 *)calloc((size_t)U, sizeof(u128));
    if (!cur || !nxt || !tot) {
        free(cur);
        free(nxt);
        free(tot);
        return -2;
    }
    for (int r0 = 0; r0 < S; ++r0) {
        memset(cur, 0, sizeof(u128) * (size_t)S * U);
        int u0 = 0;
        for (int x = 0; x < L; ++x)
            u0 += ((r0 >> x) & 1) != ((r0 >> ((x + 1) % L)) & 1);
        cur[(size_t)r0 * U + u0] = 1;
        for (int y = 1; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                memset(nxt, 0, sizeof(u128) * (size_t)S * U);
                for (int p = 0; p < S; ++p) {
                    const u128 *src = cur + (size_t)p * U;
                    for (int s = 0; s <= 1; ++s) {
                        int du = 0;
                        du += ((p >> x) & 1) != s;                    /* up   */
                        if (x > 0)
                            du += ((p >> (x - 1)) & 1) != s;          /* left */
                        if (x == L - 1)
                            du += (p & 1) != s;                        /* wrap: column 0 of this row */
                        int q = (p & ~(1 << x)) | (s << x);
                        u128 *dst = nxt + (size_t)q * U;
                        for (int u = 0; u + du < U; ++u)
                            dst[u + du] += src[u];
                    }
                }
                u128 *tmp = cur;
                cur = nxt;
                nxt = tmp;
            }
        for (int p = 0; p < S; ++p) {
            int du = 0;
            for (int x = 0; x < L; ++x)
                du += ((p >> x) & 1) != ((r0 >> x) & 1);
            const u128 *src = cur + (size_t)p * U;
            for (int u = 0; u + du < U; ++u)
                tot[u + du] += src[u];
        }
    }
    for (int e = 0; e <= N; ++e) {
        u128 v = tot[2 * e];
        g_lo[e] = (uint64_t)v;
        g_hi[e] = (uint64_t)(v >> 64);
    }
    /* odd u never occurs on the torus; report a failure if it did */
    int bad = 0;
    for (int u = 1; u < U; u += 2)
        bad |= tot[u] != 0;
    free(cur);
    free(nxt);
    free(tot);
    return bad ? -3 : 0;
}
