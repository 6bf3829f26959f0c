// muca_kernels.cu - sm_103a kernels of the parallel multicanonical 2D Ising update
// (Gross, Zierenberg, Weigel, Janke, arXiv:1707.00919, Sec. 2.3).
//
// One thread runs one walker (Sec. 2.3: one thread per walker, lattices interleaved so
// that a warp's accesses to one site coalesce).  Inside a launch the walker's lattice
// is bit-packed into shared memory, one word per row ([row][walker-in-block], so a
// warp's row loads hit 32 consecutive words), the acceptance thresholds T[e][k] sit in
// shared memory, random words come from an inline Philox4x32-10, and the visited
// energies go run-length encoded into a per-block shared histogram that is added to the
// global uint64 histogram once at the end of the launch.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <type_traits>

#include <cuda_runtime.h>

#include "../../include/muca.h"
#include "muca_internal.h"

namespace muca {
namespace {

// Philox4x32-10 of Salmon et al. (SC'11), the generator of Sec. 2.3.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

constexpr uint32_t kTagMetropolis = 0u;
bool g_use_full_kernel = true;
constexpr uint32_t kTagInit = 1u;

__host__ __device__ constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

template <typename RowT>
__device__ __forceinline__ uint32_t bit_at(RowT w, int x)
{
    return (uint32_t)(w >> x) & 1u;
}

// ---------------------------------------------------------------------------------
// Sweep kernel.  Template: row word type (uint32 for L <= 32, uint64 for L <= 64),
// global lattice layout, and whether visited energies are recorded.
// ---------------------------------------------------------------------------------
template <typename RowT, int LAYOUT, bool RECORD>
__global__ void __launch_bounds__(1024) sweep_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int L = a.L;
    const int N = L * L;
    const int nb = N + 1;
    const int wpb = blockDim.x;
    uint32_t *sT = reinterpret_cast<uint32_t *>(smem);
    uint32_t *sH = sT + nb * 5;
    RowT *sRows = reinterpret_cast<RowT *>(smem + align_up((size_t)(nb * 5 + (RECORD ? nb : 0)) * 4, 16));

    const int tid = threadIdx.x;
    const int64_t w = (int64_t)blockIdx.x * wpb + tid;
    bool active = w < a.W;

    for (int i = tid; i < nb * 5; i += wpb)
        sT[i] = a.table[i];
    if (RECORD)
        for (int i = tid; i < nb; i += wpb)
            sH[i] = 0u;

    RowT *col = sRows + tid;   // this walker's rows: col[y * wpb]
    int32_t e = 0;
    if (active) {
        if (LAYOUT == MUCA_LAYOUT_PACKED) {
            const RowT *g = reinterpret_cast<const RowT *>(a.lattice);
            for (int y = 0; y < L; ++y)
                col[y * wpb] = g[(size_t)y * a.W + w];
        } else {
            const int8_t *g = reinterpret_cast<const int8_t *>(a.lattice);
            for (int y = 0; y < L; ++y) {
                RowT r = 0;
                for (int x = 0; x < L; ++x)
                    r |= (RowT)(g[(size_t)(y * L + x) * a.W + w] < 0) << x;
                col[y * wpb] = r;
            }
        }
        e = a.energy[w];
        if (e < 0 || e > N) {
            atomicOr(a.err, kErrEnergyRange);
            active = false;
        }
    }
    __syncthreads();

    int32_t run_e = e;
    uint32_t run_n = 0;
    if (active) {
        const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
        const uint32_t wid = (uint32_t)w;
        uint64_t t = a.t0;
        const uint64_t tend = a.t0 + a.n;
        while (t < tend) {
            const int i = (int)(t % (uint64_t)N);
            const int y = i / L;
            const int x0 = i - y * L;
            const uint64_t left = tend - t;
            const int x1 = left < (uint64_t)(L - x0) ? x0 + (int)left : L;
            const int yu = (y == 0) ? L - 1 : y - 1;
            const int yd = (y == L - 1) ? 0 : y + 1;
            const RowT U = col[yu * wpb];
            RowT C = col[y * wpb];
            const RowT D = col[yd * wpb];
            // Vertical disagreements: bit x of VU/VD is fixed until site x itself is
            // visited (a flip at x' != x leaves bit x alone), so one XOR per row serves
            // every site of the row.
            const RowT VU = U ^ C;
            const RowT VD = D ^ C;
            const uint64_t tb = t - (uint64_t)x0;   // attempt number of column 0
            for (int xb = x0 & ~3; xb < x1; xb += 4) {
                const uint64_t blk = (tb + (uint64_t)xb) >> 2;
                const uint4 rw = philox4x32_10(make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), wid, kTagMetropolis), k0, k1);
                const uint32_t words[4] = {rw.x, rw.y, rw.z, rw.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int x = xb + u;
                    if (x < x0 || x >= x1)
                        continue;
                    const int xl = (x == 0) ? L - 1 : x - 1;
                    const int xr = (x == L - 1) ? 0 : x + 1;
                    const uint32_t sx = bit_at(C, x);
                    const uint32_t k = bit_at(VU, x) + bit_at(VD, x) + (sx ^ bit_at(C, xl)) + (sx ^ bit_at(C, xr));
                    const uint32_t thr = sT[e * 5 + (int)k];
                    const bool acc = (words[u] < thr) | (thr == 0xFFFFFFFFu);
                    if (acc) {
                        C ^= (RowT)1 << x;
                        e += 2 - (int)k;
                    }
                    if (RECORD) {
                        if (e != run_e) {
                            if (run_n)
                                atomicAdd(&sH[run_e], run_n);
                            run_e = e;
                            run_n = 0u;
                        }
                        ++run_n;
                    }
                }
            }
            col[y * wpb] = C;
            t += (uint64_t)(x1 - x0);
        }
        if (RECORD && run_n)
            atomicAdd(&sH[run_e], run_n);
    }
    __syncthreads();
    if (RECORD)
        for (int i = tid; i < nb; i += wpb) {
            const uint32_t v = sH[i];
            if (v)
                atomicAdd(&a.hist[i], (unsigned long long)v);
        }
    if (active) {
        if (LAYOUT == MUCA_LAYOUT_PACKED) {
            RowT *g = reinterpret_cast<RowT *>(a.lattice);
            for (int y = 0; y < L; ++y)
                g[(size_t)y * a.W + w] = col[y * wpb];
        } else {
            int8_t *g = reinterpret_cast<int8_t *>(a.lattice);
            for (int y = 0; y < L; ++y) {
                const RowT r = col[y * wpb];
                for (int x = 0; x < L; ++x)
                    g[(size_t)(y * L + x) * a.W + w] = bit_at(r, x) ? (int8_t)-1 : (int8_t)1;
            }
        }
        a.energy[w] = e;
    }
}

// ---------------------------------------------------------------------------------
// Initial spins: +1 iff the top bit of the tag-1 word for attempt number t = site is
// clear; the energy index is the number of unsatisfied bonds over two.
// ---------------------------------------------------------------------------------
template <typename RowT, int LAYOUT>
__global__ void init_kernel(int32_t L, int64_t W, uint64_t seed, void *lattice, int32_t *energy)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W)
        return;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const RowT mask = (L == (int)(8 * sizeof(RowT))) ? ~(RowT)0 : (((RowT)1 << L) - 1);
    RowT first = 0, prev = 0;
    int unsat = 0;
    for (int y = 0; y < L; ++y) {
        RowT r = 0;
        for (int x = 0; x < L; x += 4) {
            const uint32_t site = (uint32_t)(y * L + x);
            const uint4 q = philox4x32_10(make_uint4(site >> 2, 0u, (uint32_t)w, kTagInit), k0, k1);
            const uint32_t words[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
                r |= (RowT)(words[u] >> 31) << (x + u);
        }
        const RowT rot = (r >> 1) | ((r & 1) << (L - 1));   // bit x = spin at x+1 (mod L)
        unsat += __popcll((unsigned long long)((r ^ rot) & mask));
        if (y == 0)
            first = r;
        else
            unsat += __popcll((unsigned long long)((r ^ prev) & mask));
        prev = r;
        if (LAYOUT == MUCA_LAYOUT_PACKED) {
            reinterpret_cast<RowT *>(lattice)[(size_t)y * W + w] = r;
        } else {
            int8_t *g = reinterpret_cast<int8_t *>(lattice);
            for (int x = 0; x < L; ++x)
                g[(size_t)(y * L + x) * W + w] = bit_at(r, x) ? (int8_t)-1 : (int8_t)1;
        }
    }
    unsat += __popcll((unsigned long long)((prev ^ first) & mask));   // row L-1 to row 0
    energy[w] = unsat / 2;
}

template <typename RowT, int LAYOUT>
__global__ void unpack_kernel(int32_t L, int64_t W, const void *lattice, int8_t *out)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W)
        return;
    const int N = L * L;
    for (int i = 0; i < N; ++i) {
        int8_t v;
        if (LAYOUT == MUCA_LAYOUT_PACKED) {
            const RowT r = reinterpret_cast<const RowT *>(lattice)[(size_t)(i / L) * W + w];
            v = bit_at(r, i % L) ? (int8_t)-1 : (int8_t)1;
        } else {
            v = reinterpret_cast<const int8_t *>(lattice)[(size_t)i * W + w];
        }
        out[(size_t)w * N + i] = v;
    }
}

__global__ void philox_kernel(const uint32_t *ctr, uint32_t k0, uint32_t k1, size_t n, uint32_t *out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 r = philox4x32_10(c, k0, k1);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

// ---------------------------------------------------------------------------------
// Whole-sweep kernel, specialised on L.  A launch covers whole sweeps starting at a
// sweep boundary.  Every row is unrolled, so bit positions and neighbour columns are
// compile-time constants; the Philox round keys are computed once per thread.
//
// Row representation: the rows above (U), at (C) and below (D) the current row are held
// as nibble words, eight spins per 32-bit register, one spin in bit 0 of each 4-bit
// field (1 = spin down).  Field-parallel arithmetic gives for all sites of a row at once
//   kb = [s != s_up] + [s != s_down] + [s != s_right]    h0 = [s != s_left]
// with the original spins, so the antiparallel count of site x is k0 = kb + h0 if the
// previous attempt (at x - 1) did not flip, else k1 = kb + 1 - h0.  Site 0's left
// neighbour is site L-1 of the same row, not yet visited, so k1 = k0 there; site L-1's
// right neighbour is site 0, so its counts move by one if site 0 flipped.
//
// Shared-memory table: one 28-byte row per energy index e, words 0..4 the acceptance
// thresholds T[e][k], word 5 the block's histogram count of e, word 6 padding (a stride
// of 7 words spreads the rows over all 32 banks; thermalization counts go there).  The energy is carried as the byte
// address E of its row, so a threshold is at E + 4k, the histogram word at E + 20, and
// an accepted flip moves E by 28 (2 - k).
//
// Latency: the threshold an attempt needs depends on whether the previous attempt
// flipped (through E and through k).  Both candidates are loaded two attempts ahead and
// the right one is picked once the previous decision is known, which takes the shared-
// memory latency off the attempt-to-attempt dependency chain (select, compare).
// ---------------------------------------------------------------------------------
template <int L>
struct RowOf {
    using type = typename std::conditional<(L <= 32), uint32_t, unsigned long long>::type;
};

constexpr int kTableStride = 7;   // words per energy row of the shared table
constexpr int kHistSlot = 5;      // word of the row holding the histogram count

struct PhiloxKeys {
    uint32_t k0[10], k1[10];   // round keys
    uint32_t hi_w, lo_w;       // round-0 product of the walker counter word
};

__device__ __forceinline__ PhiloxKeys make_keys(uint64_t seed, uint32_t walker)
{
    PhiloxKeys p;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        p.k0[r] = (uint32_t)seed + (uint32_t)r * 0x9E3779B9u;
        p.k1[r] = (uint32_t)(seed >> 32) + (uint32_t)r * 0xBB67AE85u;
    }
    const unsigned long long pw = (unsigned long long)0xCD9E8D57u * walker;
    p.hi_w = (uint32_t)(pw >> 32);
    p.lo_w = (uint32_t)pw;
    return p;
}

// Philox4x32-10 on counter (c0, c1, walker, tag 0) with precomputed keys; the products
// are formed as 64-bit results so that one wide multiply gives both halves.
__device__ __forceinline__ uint4 philox_walker(uint32_t c0, uint32_t c1, const PhiloxKeys &p)
{
    const unsigned long long q = (unsigned long long)0xD2511F53u * c0;
    uint32_t x0 = p.hi_w ^ c1 ^ p.k0[0];
    uint32_t x1 = p.lo_w;
    uint32_t x2 = (uint32_t)(q >> 32) ^ p.k1[0];
    uint32_t x3 = (uint32_t)q;
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * x0;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * x2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ x1 ^ p.k0[r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ x3 ^ p.k1[r];
        x0 = n0;
        x1 = (uint32_t)p1;
        x2 = n2;
        x3 = (uint32_t)p0;
    }
    return make_uint4(x0, x1, x2, x3);
}

// 32x32 bit transpose across a warp: lane l holds m with bit j = A[l][j]; returns in
// lane j the word with bit l = A[l][j].  Five butterfly stages of shuffles.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t m, int lane)
{
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int s = 16 >> i;
        const uint32_t part = __shfl_xor_sync(0xFFFFFFFFu, m, s);
        m = (lane & s) ? ((m & ~masks[i]) | ((part >> s) & masks[i])) : ((m & masks[i]) | ((part & masks[i]) << s));
    }
    return m;
}

// Sign bits of four int8 spins (-1 = 0xFF, +1 = 0x01) as a nibble.
__device__ __forceinline__ uint32_t gather_signs(uint32_t v) { return ((v & 0x80808080u) * 0x00204081u) >> 28; }

// Nibble of down-spin bits to four int8 spins.
__device__ __forceinline__ uint32_t spread_signs(uint32_t n)
{
    return 0x01010101u | (((n * 0x00204081u) & 0x01010101u) * 0xFEu);
}

// Bit rows of the warp's 32 walkers from the int8 [site][walker] layout, R rows at a
// time so that their loads are in flight together; lane j receives walker w0 + j.
// All 32 walkers must exist and W % 16 == 0.
template <int L, int R, typename RowT>
__device__ __forceinline__ void warp_load_rows_int8(const int8_t *g, int64_t W, int64_t w0, int y0, int lane,
                                                    RowT (&out)[R])
{
    constexpr int HALVES = (L + 31) / 32;
    uint4 a[R][HALVES], b[R][HALVES];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int half = 0; half < HALVES; ++half) {
            const int x = half * 32 + lane;
            if (x < L) {
                const uint4 *p = reinterpret_cast<const uint4 *>(g + (size_t)((y0 + r) * L + x) * (size_t)W + (size_t)w0);
                a[r][half] = p[0];
                b[r][half] = p[1];
            } else {
                a[r][half] = make_uint4(0, 0, 0, 0);
                b[r][half] = make_uint4(0, 0, 0, 0);
            }
        }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        RowT row = 0;
#pragma unroll
        for (int half = 0; half < HALVES; ++half) {
            const uint4 u = a[r][half], v = b[r][half];
            uint32_t m = gather_signs(u.x) | (gather_signs(u.y) << 4) | (gather_signs(u.z) << 8) |
                         (gather_signs(u.w) << 12) | (gather_signs(v.x) << 16) | (gather_signs(v.y) << 20) |
                         (gather_signs(v.z) << 24) | (gather_signs(v.w) << 28);
            m = warp_transpose32(m, lane);
            row |= (RowT)m << (32 * half);
        }
        out[r] = row;
    }
}

template <int L, typename RowT>
__device__ __forceinline__ void warp_store_row_int8(int8_t *g, int64_t W, int64_t w0, int y, int lane, RowT r)
{
#pragma unroll
    for (int half = 0; half < (L + 31) / 32; ++half) {
        const uint32_t m = warp_transpose32((uint32_t)(r >> (32 * half)), lane);
        const int x = half * 32 + lane;
        if (x < L) {
            uint4 *p = reinterpret_cast<uint4 *>(g + (size_t)(y * L + x) * (size_t)W + (size_t)w0);
            p[0] = make_uint4(spread_signs(m & 15u), spread_signs((m >> 4) & 15u), spread_signs((m >> 8) & 15u),
                              spread_signs((m >> 12) & 15u));
            p[1] = make_uint4(spread_signs((m >> 16) & 15u), spread_signs((m >> 20) & 15u),
                              spread_signs((m >> 24) & 15u), spread_signs(m >> 28));
        }
    }
}

// Eight bits -> eight nibbles (bit i to bit 4i), and back.
__device__ __forceinline__ uint32_t spread8(uint32_t b)
{
    uint32_t x = b & 0xFFu;
    x = (x | (x << 12)) & 0x000F000Fu;
    x = (x | (x << 6)) & 0x03030303u;
    x = (x | (x << 3)) & 0x11111111u;
    return x;
}

__device__ __forceinline__ uint32_t pack8(uint32_t x)
{
    x &= 0x11111111u;
    x = (x | (x >> 3)) & 0x03030303u;
    x = (x | (x >> 6)) & 0x000F000Fu;
    x = (x | (x >> 12)) & 0xFFu;
    return x;
}

template <int L>
__device__ __forceinline__ void to_nibbles(typename RowOf<L>::type r, uint32_t (&n)[L / 8])
{
#pragma unroll
    for (int i = 0; i < L / 8; ++i)
        n[i] = spread8((uint32_t)(r >> (8 * i)));
}

template <int L>
__device__ __forceinline__ typename RowOf<L>::type from_nibbles(const uint32_t (&n)[L / 8])
{
    using RowT = typename RowOf<L>::type;
    RowT r = 0;
#pragma unroll
    for (int i = 0; i < L / 8; ++i)
        r |= (RowT)pack8(n[i]) << (8 * i);
    return r;
}

// Row storage in shared memory during a launch.  L <= 32: nibble words,
// [row][walker][L/8], read and written without conversion.  L > 32: bit words
// [row][walker] (a nibble copy would not fit next to the table), converted per row.
template <int L>
struct SmemRows {
    static constexpr bool kNibbles = (L <= 32);
    static constexpr int NW = L / 8;
    using RowT = typename RowOf<L>::type;
    static constexpr size_t bytes_per_walker() { return kNibbles ? (size_t)L * NW * 4 : (size_t)L * sizeof(RowT); }

    unsigned char *base;
    int wpb, tid;

    __device__ __forceinline__ void load(int y, uint32_t (&n)[NW]) const
    {
        if (kNibbles) {
            const uint32_t *p = reinterpret_cast<const uint32_t *>(base) + ((size_t)y * wpb + tid) * NW;
#pragma unroll
            for (int i = 0; i < NW; ++i)
                n[i] = p[i];
        } else {
            to_nibbles<L>(reinterpret_cast<const RowT *>(base)[(size_t)y * wpb + tid], n);
        }
    }
    __device__ __forceinline__ void store(int y, const uint32_t (&n)[NW]) const
    {
        if (kNibbles) {
            uint32_t *p = reinterpret_cast<uint32_t *>(base) + ((size_t)y * wpb + tid) * NW;
#pragma unroll
            for (int i = 0; i < NW; ++i)
                p[i] = n[i];
        } else {
            reinterpret_cast<RowT *>(base)[(size_t)y * wpb + tid] = from_nibbles<L>(n);
        }
    }
    __device__ __forceinline__ void store_bits(int y, RowT r) const
    {
        if (kNibbles) {
            uint32_t n[NW];
            to_nibbles<L>(r, n);
            store(y, n);
        } else {
            reinterpret_cast<RowT *>(base)[(size_t)y * wpb + tid] = r;
        }
    }
    __device__ __forceinline__ RowT load_bits(int y) const
    {
        if (kNibbles) {
            uint32_t n[NW];
            load(y, n);
            return from_nibbles<L>(n);
        }
        return reinterpret_cast<const RowT *>(base)[(size_t)y * wpb + tid];
    }
};

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// Histogram record of one attempt: one count for the post-decision energy, added to the
// histogram word (offset 20) of its table row.  A shared-memory reduction is issued on
// every attempt anyway (a predicated one, which would allow run-length counting, measured
// about 45 cycles slower per attempt), so a plain +1 needs no further arithmetic.
__device__ __forceinline__ void hist_add_one(uint32_t E)
{
    asm volatile("red.shared.add.u32 [%0+20], 1;" :: "r"(E));
}

// Thermalization launches add the same count to the row's padding word (offset 24),
// which nothing reads.  The reduction orders the shared-memory threshold loads of later
// attempts behind it exactly as in a recording launch; without it the compiler's
// schedule was measured 11% slower (72 vs 64 cycles per attempt and warp at L = 32).
__device__ __forceinline__ void pad_add_one(uint32_t E)
{
    asm volatile("red.shared.add.u32 [%0+24], 1;" :: "r"(E));
}

// Byte offset 4k of the count field x (k in 0..4) of a nibble word.
__device__ __forceinline__ uint32_t field_x4(uint32_t w, int f)
{
    return (f == 0 ? (w << 2) : (w >> (4 * f - 2))) & 0x1Cu;
}

// One row of L attempts (typewriter, x = 0 .. L-1) for one walker.  E is the shared
// byte address of the current energy's table row on entry and on exit.
// Random words of the current row: four attempts at a time, already clamped to
// 0xFFFFFFFE so that "r < T" also accepts every attempt when T = 0xFFFFFFFF.
struct PhiloxSource {
    uint64_t blk;            // Philox block of column 0 of the row
    const PhiloxKeys *pk;
    __device__ __forceinline__ uint4 get(int xb) const
    {
        const uint64_t b = blk + (uint64_t)(xb / 4);
        const uint4 rw = philox_walker((uint32_t)b, (uint32_t)(b >> 32), *pk);
        return make_uint4(min(rw.x, 0xFFFFFFFEu), min(rw.y, 0xFFFFFFFEu), min(rw.z, 0xFFFFFFFEu),
                          min(rw.w, 0xFFFFFFFEu));
    }
};

template <int L, bool RECORD, class Src>
__device__ __forceinline__ void process_row(const uint32_t (&U)[L / 8], uint32_t (&C)[L / 8], const uint32_t (&D)[L / 8],
                                            uint32_t &E, const Src &src)
{
    constexpr int NW = L / 8;
    uint32_t K0[NW], K1[NW];
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        const uint32_t cr = __funnelshift_r(C[i], C[(i + 1) % NW], 4);        // field f <- right neighbour
        const uint32_t cl = __funnelshift_l(C[(i + NW - 1) % NW], C[i], 4);   // field f <- left neighbour
        const uint32_t kb = (U[i] ^ C[i]) + (D[i] ^ C[i]) + (C[i] ^ cr);
        const uint32_t h0 = C[i] ^ cl;
        K0[i] = kb + h0;
        K1[i] = kb + 0x11111111u - h0;
    }
    // site L-1: its right neighbour is site 0, whose flip moves the count by -1 if the
    // two disagreed before, +1 if they agreed (in units of 4 bytes here)
    const uint32_t hr_last = ((C[NW - 1] >> 28) ^ C[0]) & 1u;
    const uint32_t adj_if_flip = hr_last ? (uint32_t)-4 : 4u;
    uint32_t adj_last = 0u;

#define MUCA_SITE_J(x, J0v, J1v)                                                         \
    do {                                                                                 \
        J0v = field_x4(K0[(x) >> 3], (x) & 7);                                           \
        J1v = ((x) == 0) ? J0v : field_x4(K1[(x) >> 3], (x) & 7);                        \
        if ((x) == L - 1) {                                                              \
            J0v += adj_last;                                                             \
            J1v += adj_last;                                                             \
        }                                                                                \
    } while (0)

    // attempt 0 (E resolved) and both outcomes of it for attempt 1
    uint32_t J0a, J1a, J0b, J1b;
    MUCA_SITE_J(0, J0a, J1a);
    MUCA_SITE_J(1, J0b, J1b);
    uint32_t d0_cur = 56u - 7u * J0a, d1_cur = d0_cur;               // attempt x
    uint32_t d0_next = 56u - 7u * J0b, d1_next = 56u - 7u * J1b;     // attempt x + 1
    uint32_t T0n = lds_u32(E + J0a), T1n = T0n;                      // candidates of x
    uint32_t T0nn = lds_u32(E + J0b), T1nn = lds_u32(E + d0_cur + J1b);   // of x + 1
    bool prev_acc = false;
    uint32_t Eres = E;

#pragma unroll
    for (int xb = 0; xb < L; xb += 4) {
        const uint4 rw = src.get(xb);
        const uint32_t words[4] = {rw.x, rw.y, rw.z, rw.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int x = xb + u;
            // decision of attempt x
            const uint32_t T = prev_acc ? T1n : T0n;
            const uint32_t dsel = prev_acc ? d1_cur : d0_cur;
            const bool acc = words[u] < T;
            const uint32_t Epost = acc ? Eres + dsel : Eres;
            C[x >> 3] ^= acc ? (1u << (4 * (x & 7))) : 0u;
            if (x == 0)
                adj_last = acc ? adj_if_flip : 0u;
            if (RECORD)
                hist_add_one(Epost);
            else
                pad_add_one(Epost);
            // candidates of attempt x + 2 for both outcomes of attempt x + 1
            T0n = T0nn;
            T1n = T1nn;
            if (x + 2 < L) {
                uint32_t J0c, J1c;
                MUCA_SITE_J(x + 2, J0c, J1c);
                const uint32_t dnext = acc ? d1_next : d0_next;      // energy step of x + 1 if accepted
                T0nn = lds_u32(Epost + J0c);
                T1nn = lds_u32(Epost + dnext + J1c);
                d0_cur = d0_next;
                d1_cur = d1_next;
                d0_next = 56u - 7u * J0c;
                d1_next = 56u - 7u * J1c;
            } else if (x + 1 < L) {
                d0_cur = d0_next;
                d1_cur = d1_next;
            }
            Eres = Epost;
            prev_acc = acc;
        }
    }
#undef MUCA_SITE_J
    E = Eres;
}

// One block's share of a launch: walkers wbase .. wbase + wpb - 1 of the instance in
// `a` (threads tid >= wpb idle), all of the launch's whole sweeps.  Shared memory:
// the table, then the rows of the wpb walkers.  Every thread of the block calls it.
template <int L, int LAYOUT, bool RECORD>
__device__ __forceinline__ void sweep_block(const SweepArgs &a, int64_t wbase, int wpb, unsigned char *smem)
{
    using RowT = typename RowOf<L>::type;
    constexpr int N = L * L;
    constexpr int NB = N + 1;
    constexpr int NW = L / 8;
    constexpr int RB = 4;   // rows per batch of int8 loads
    const int nthr = blockDim.x;
    uint32_t *sTab = reinterpret_cast<uint32_t *>(smem);
    const int tid = threadIdx.x;
    const SmemRows<L> rows{smem + align_up((size_t)NB * kTableStride * 4, 16), wpb, tid};
    const int lane = tid & 31;
    const bool in_item = tid < wpb;
    const int64_t w = wbase + tid;
    const int64_t w0 = w - lane;
    bool active = in_item && w < a.W;
    const bool warp_full = in_item && (w0 + 32 <= a.W) && (a.W % 16 == 0);

    for (int i = tid; i < NB * kTableStride; i += nthr) {
        const int e = i / kTableStride, k = i - e * kTableStride;
        sTab[i] = k < 5 ? a.table[e * 5 + k] : 0u;
    }

    if (LAYOUT == MUCA_LAYOUT_PACKED) {
        if (active)
            for (int y = 0; y < L; ++y)
                rows.store_bits(y, reinterpret_cast<const RowT *>(a.lattice)[(size_t)y * a.W + w]);
    } else if (warp_full) {
        for (int y = 0; y < L; y += RB) {
            RowT r[RB];
            warp_load_rows_int8<L, RB, RowT>(reinterpret_cast<const int8_t *>(a.lattice), a.W, w0, y, lane, r);
#pragma unroll
            for (int i = 0; i < RB; ++i)
                rows.store_bits(y + i, r[i]);
        }
    } else if (active) {
        const int8_t *g = reinterpret_cast<const int8_t *>(a.lattice);
        for (int y = 0; y < L; ++y) {
            RowT r = 0;
            for (int x = 0; x < L; ++x)
                r |= (RowT)(g[(size_t)(y * L + x) * a.W + w] < 0) << x;
            rows.store_bits(y, r);
        }
    }
    int32_t e = 0;
    if (active) {
        e = a.energy[w];
        if (e < 0 || e > N) {
            atomicOr(a.err, kErrEnergyRange);
            active = false;
        }
    }
    __syncthreads();

    if (active) {
        const PhiloxKeys pk = make_keys(a.seed, (uint32_t)w);
        const uint32_t tbase = (uint32_t)__cvta_generic_to_shared(sTab);
        uint64_t blk = a.t0 >> 2;
        const uint64_t nsweeps = a.n / (uint64_t)N;
        uint32_t U[NW], C[NW], D[NW];
        rows.load(L - 1, U);
        rows.load(0, C);
        rows.load(1, D);
        uint32_t E = tbase + (uint32_t)e * (4u * kTableStride);
        for (uint64_t s = 0; s < nsweeps; ++s) {
#pragma unroll 1
            for (int y = 0; y < L; ++y) {
                const PhiloxSource src{blk, &pk};
                process_row<L, RECORD>(U, C, D, E, src);
                rows.store(y, C);
                const int y2 = (y + 2 < L) ? y + 2 : y + 2 - L;
#pragma unroll
                for (int i = 0; i < NW; ++i) {
                    U[i] = C[i];
                    C[i] = D[i];
                }
                rows.load(y2, D);
                blk += (uint64_t)(L / 4);
            }
        }
        e = (int32_t)((E - tbase) / (4u * kTableStride));
    }
    __syncthreads();
    if (RECORD)
        for (int i = tid; i < NB; i += nthr) {
            const uint32_t v = sTab[i * kTableStride + kHistSlot];
            if (v)
                atomicAdd(&a.hist[i], (unsigned long long)v);
        }
    if (LAYOUT == MUCA_LAYOUT_PACKED) {
        if (active)
            for (int y = 0; y < L; ++y)
                reinterpret_cast<RowT *>(a.lattice)[(size_t)y * a.W + w] = rows.load_bits(y);
    } else if (warp_full) {
        // a walker flagged invalid above kept its lattice in shared memory unchanged
        for (int y = 0; y < L; ++y)
            warp_store_row_int8<L, RowT>(reinterpret_cast<int8_t *>(a.lattice), a.W, w0, y, lane, rows.load_bits(y));
    } else if (active) {
        int8_t *g = reinterpret_cast<int8_t *>(a.lattice);
        for (int y = 0; y < L; ++y) {
            const RowT r = rows.load_bits(y);
            for (int x = 0; x < L; ++x)
                g[(size_t)(y * L + x) * a.W + w] = bit_at(r, x) ? (int8_t)-1 : (int8_t)1;
        }
    }
    if (active)
        a.energy[w] = e;
}

template <int L, int LAYOUT, bool RECORD>
__global__ void __launch_bounds__(256, 1) sweep_full_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    sweep_block<L, LAYOUT, RECORD>(a, (int64_t)blockIdx.x * blockDim.x, blockDim.x, smem);
}

// ---------------------------------------------------------------------------------
// Batched persistent kernel: one launch advances many instances (uneven L, walker
// counts, tables and histograms).  The work list holds (instance, first walker, walker
// count) items; each block takes the next item from a global counter, runs it with the
// body of the whole-sweep kernel for that instance's L and layout, and takes another
// until the list is exhausted.  The counter must be zero at launch.
// ---------------------------------------------------------------------------------
template <int L, bool RECORD>
__device__ __forceinline__ void batch_item(const SweepArgs &a, const BatchItem &it, unsigned char *smem)
{
    if (a.layout == MUCA_LAYOUT_PACKED)
        sweep_block<L, MUCA_LAYOUT_PACKED, RECORD>(a, it.wbase, it.wpb, smem);
    else
        sweep_block<L, MUCA_LAYOUT_INT8, RECORD>(a, it.wbase, it.wpb, smem);
}

template <bool RECORD>
__global__ void __launch_bounds__(256, 1) batch_kernel(const SweepArgs *__restrict__ insts,
                                                        const BatchItem *__restrict__ items, int32_t n_items,
                                                        uint32_t *counter)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int32_t s_item;
    for (;;) {
        if (threadIdx.x == 0)
            s_item = (int32_t)atomicAdd(counter, 1u);
        __syncthreads();
        const int32_t k = s_item;
        __syncthreads();
        if (k >= n_items)
            break;
        const BatchItem it = items[k];
        const SweepArgs a = insts[it.inst];
        switch (a.L) {
        case 8: batch_item<8, RECORD>(a, it, smem); break;
        case 16: batch_item<16, RECORD>(a, it, smem); break;
        case 24: batch_item<24, RECORD>(a, it, smem); break;
        case 32: batch_item<32, RECORD>(a, it, smem); break;
        case 48: batch_item<48, RECORD>(a, it, smem); break;
        case 64: batch_item<64, RECORD>(a, it, smem); break;
        default: break;
        }
    }
}

// ---------------------------------------------------------------------------------
// Allocation-free variant of the batched kernel.  Its scratch (instance descriptors,
// walkers per work item, item prefix sums and the work counter) lives in the file-scope
// array g_noalloc_scratch below instead of memory the library allocates; the work list
// is derived from the prefix sums, so the caller passes only the instances' own buffers.
// ---------------------------------------------------------------------------------
template <bool RECORD>
__global__ void __launch_bounds__(256, 1) batch_noalloc_kernel(const unsigned char *scratch, int32_t n)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int32_t s_inst;
    __shared__ int64_t s_wbase;
    const SweepArgs *descs = reinterpret_cast<const SweepArgs *>(scratch);
    const int32_t *wpbs = reinterpret_cast<const int32_t *>(scratch + kNoAllocWpbOffset);
    const int32_t *prefix = wpbs + kNoAllocMaxInstances;
    uint32_t *counter = reinterpret_cast<uint32_t *>(const_cast<unsigned char *>(scratch) + kNoAllocCounterOffset);
    const int32_t total = prefix[n];
    for (;;) {
        if (threadIdx.x == 0) {
            const int32_t k = (int32_t)atomicAdd(counter, 1u);
            int32_t i = -1;
            if (k < total) {
                i = 0;
                while (prefix[i + 1] <= k)
                    ++i;
                s_wbase = (int64_t)(k - prefix[i]) * wpbs[i];
            }
            s_inst = i;
        }
        __syncthreads();
        const int32_t i = s_inst;
        const int64_t wbase = s_wbase;
        __syncthreads();
        if (i < 0)
            break;
        const SweepArgs a = descs[i];
        BatchItem it;
        it.inst = i;
        it.wpb = wpbs[i];
        it.wbase = wbase;
        switch (a.L) {
        case 8: batch_item<8, RECORD>(a, it, smem); break;
        case 16: batch_item<16, RECORD>(a, it, smem); break;
        case 24: batch_item<24, RECORD>(a, it, smem); break;
        case 32: batch_item<32, RECORD>(a, it, smem); break;
        case 48: batch_item<48, RECORD>(a, it, smem); break;
        case 64: batch_item<64, RECORD>(a, it, smem); break;
        default: break;
        }
    }
}

template <int L, int LAYOUT, bool RECORD>
cudaError_t launch_full_t(const SweepArgs &a, int wpb, cudaStream_t s)
{
    const size_t smem = full_smem_bytes(L, wpb, RECORD);
    auto kern = sweep_full_kernel<L, LAYOUT, RECORD>;
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess)
            return err;
        configured = smem;
    }
    const int64_t blocks = (a.W + wpb - 1) / wpb;
    kern<<<(unsigned)blocks, wpb, smem, s>>>(a);
    return cudaGetLastError();
}

template <int L>
cudaError_t launch_full_l(const SweepArgs &a, int wpb, bool record, cudaStream_t s)
{
    if (a.layout == MUCA_LAYOUT_PACKED)
        return record ? launch_full_t<L, MUCA_LAYOUT_PACKED, true>(a, wpb, s)
                      : launch_full_t<L, MUCA_LAYOUT_PACKED, false>(a, wpb, s);
    return record ? launch_full_t<L, MUCA_LAYOUT_INT8, true>(a, wpb, s)
                  : launch_full_t<L, MUCA_LAYOUT_INT8, false>(a, wpb, s);
}

// Dispatches a whole-sweep range to the kernel specialised for L; returns
// cudaErrorNotSupported when L has no specialisation.
cudaError_t launch_full(const SweepArgs &a, int wpb, bool record, cudaStream_t s)
{
    switch (a.L) {
    case 8: return launch_full_l<8>(a, wpb, record, s);
    case 16: return launch_full_l<16>(a, wpb, record, s);
    case 24: return launch_full_l<24>(a, wpb, record, s);
    case 32: return launch_full_l<32>(a, wpb, record, s);
    case 48: return launch_full_l<48>(a, wpb, record, s);
    case 64: return launch_full_l<64>(a, wpb, record, s);
    default: return cudaErrorNotSupported;
    }
}

template <int L, int LAYOUT>
int occupancy_full_t(int wpb)
{
    const size_t smem = full_smem_bytes(L, wpb, true);
    auto kern = sweep_full_kernel<L, LAYOUT, true>;
    if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, wpb, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <int L>
int occupancy_full_l(int layout, int wpb)
{
    return layout == MUCA_LAYOUT_PACKED ? occupancy_full_t<L, MUCA_LAYOUT_PACKED>(wpb)
                                        : occupancy_full_t<L, MUCA_LAYOUT_INT8>(wpb);
}

bool has_full_kernel(int L) { return L == 8 || L == 16 || L == 24 || L == 32 || L == 48 || L == 64; }

template <typename RowT, int LAYOUT, bool RECORD>
cudaError_t launch_sweep_t(const SweepArgs &a, int wpb, cudaStream_t s)
{
    const size_t smem = sweep_smem_bytes(a.L, wpb, RECORD);
    auto kern = sweep_kernel<RowT, LAYOUT, RECORD>;
    static size_t configured = 0;   // dynamic smem limit already granted to this instantiation
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess)
            return err;
        configured = smem;
    }
    const int64_t blocks = (a.W + wpb - 1) / wpb;
    kern<<<(unsigned)blocks, wpb, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename RowT>
cudaError_t launch_sweep_row(const SweepArgs &a, int wpb, bool record, cudaStream_t s)
{
    if (a.layout == MUCA_LAYOUT_PACKED)
        return record ? launch_sweep_t<RowT, MUCA_LAYOUT_PACKED, true>(a, wpb, s)
                      : launch_sweep_t<RowT, MUCA_LAYOUT_PACKED, false>(a, wpb, s);
    return record ? launch_sweep_t<RowT, MUCA_LAYOUT_INT8, true>(a, wpb, s)
                  : launch_sweep_t<RowT, MUCA_LAYOUT_INT8, false>(a, wpb, s);
}

}  // namespace

size_t full_smem_bytes(int L, int wpb, bool record)
{
    (void)record;
    const size_t nb = (size_t)L * L + 1;
    const size_t per_walker = L <= 32 ? (size_t)L * (L / 8) * 4 : (size_t)L * 8;
    return align_up(nb * kTableStride * 4, 16) + per_walker * (size_t)wpb;
}

size_t sweep_smem_bytes(int L, int wpb, bool record)
{
    const size_t nb = (size_t)L * L + 1;
    const size_t row = L <= 32 ? 4 : 8;
    return align_up((nb * 5 + (record ? nb : 0)) * 4, 16) + (size_t)L * wpb * row;
}

size_t sweep_smem_limit()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)v;
}

static cudaError_t launch_generic(const SweepArgs &a, int wpb, bool record, cudaStream_t s)
{
    if (a.n == 0)
        return cudaSuccess;
    if (a.L <= 32)
        return launch_sweep_row<uint32_t>(a, wpb, record, s);
    return launch_sweep_row<unsigned long long>(a, wpb, record, s);
}

cudaError_t launch_sweep(const SweepArgs &a, int wpb, bool record, cudaStream_t s)
{
    if (a.n == 0 || a.W == 0)
        return cudaSuccess;
    const uint64_t N = (uint64_t)a.L * (uint64_t)a.L;
    if (!has_full_kernel(a.L) || !g_use_full_kernel)
        return launch_generic(a, wpb, record, s);
    // head up to the next sweep boundary, whole sweeps, tail
    const uint64_t head = std::min(a.n, (N - a.t0 % N) % N);
    const uint64_t full = (a.n - head) / N * N;
    SweepArgs p = a;
    p.n = head;
    cudaError_t err = launch_generic(p, wpb, record, s);
    if (err != cudaSuccess)
        return err;
    if (full) {
        p.t0 = a.t0 + head;
        p.n = full;
        err = launch_full(p, wpb, record, s);
        if (err != cudaSuccess)
            return err;
    }
    p.t0 = a.t0 + head + full;
    p.n = a.n - head - full;
    return launch_generic(p, wpb, record, s);
}

void set_full_kernel_enabled(bool on) { g_use_full_kernel = on; }

cudaError_t launch_init(int32_t L, int32_t layout, int64_t W, uint64_t seed, void *lattice, int32_t *energy,
                        cudaStream_t s)
{
    const int threads = 128;
    const unsigned blocks = (unsigned)((W + threads - 1) / threads);
    if (L <= 32) {
        if (layout == MUCA_LAYOUT_PACKED)
            init_kernel<uint32_t, MUCA_LAYOUT_PACKED><<<blocks, threads, 0, s>>>(L, W, seed, lattice, energy);
        else
            init_kernel<uint32_t, MUCA_LAYOUT_INT8><<<blocks, threads, 0, s>>>(L, W, seed, lattice, energy);
    } else {
        if (layout == MUCA_LAYOUT_PACKED)
            init_kernel<unsigned long long, MUCA_LAYOUT_PACKED><<<blocks, threads, 0, s>>>(L, W, seed, lattice, energy);
        else
            init_kernel<unsigned long long, MUCA_LAYOUT_INT8><<<blocks, threads, 0, s>>>(L, W, seed, lattice, energy);
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack(int32_t L, int32_t layout, int64_t W, const void *lattice, int8_t *out, cudaStream_t s)
{
    const int threads = 128;
    const unsigned blocks = (unsigned)((W + threads - 1) / threads);
    if (L <= 32) {
        if (layout == MUCA_LAYOUT_PACKED)
            unpack_kernel<uint32_t, MUCA_LAYOUT_PACKED><<<blocks, threads, 0, s>>>(L, W, lattice, out);
        else
            unpack_kernel<uint32_t, MUCA_LAYOUT_INT8><<<blocks, threads, 0, s>>>(L, W, lattice, out);
    } else {
        if (layout == MUCA_LAYOUT_PACKED)
            unpack_kernel<unsigned long long, MUCA_LAYOUT_PACKED><<<blocks, threads, 0, s>>>(L, W, lattice, out);
        else
            unpack_kernel<unsigned long long, MUCA_LAYOUT_INT8><<<blocks, threads, 0, s>>>(L, W, lattice, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, size_t n, uint32_t *out, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    const int threads = 128;
    philox_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(ctr, k0, k1, n, out);
    return cudaGetLastError();
}

int resident_blocks(int L, int layout, int wpb)
{
    switch (L) {
    case 8: return occupancy_full_l<8>(layout, wpb);
    case 16: return occupancy_full_l<16>(layout, wpb);
    case 24: return occupancy_full_l<24>(layout, wpb);
    case 32: return occupancy_full_l<32>(layout, wpb);
    case 48: return occupancy_full_l<48>(layout, wpb);
    case 64: return occupancy_full_l<64>(layout, wpb);
    default: break;
    }
    // the generic kernel: bounded by shared memory and threads
    int dev = 0, smem_sm = 0, thr_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const size_t need = sweep_smem_bytes(L, wpb, true) + 1024;
    return (int)std::min((size_t)smem_sm / need, (size_t)(thr_sm / wpb));
}

cudaError_t configure_batch(size_t smem)
{
    for (auto kern : {batch_kernel<true>, batch_kernel<false>}) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess)
            return err;
    }
    return cudaSuccess;
}

int batch_resident_blocks(size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<true>, kBatchThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_batch(const SweepArgs *insts, const BatchItem *items, int32_t n_items, uint32_t *counter,
                         int grid, size_t smem, bool record, cudaStream_t s)
{
    if (n_items <= 0)
        return cudaSuccess;
    if (record)
        batch_kernel<true><<<grid, kBatchThreads, smem, s>>>(insts, items, n_items, counter);
    else
        batch_kernel<false><<<grid, kBatchThreads, smem, s>>>(insts, items, n_items, counter);
    return cudaGetLastError();
}

// Scratch of the allocation-free batched sweep: every GPU that loads the library holds
// these kNoAllocScratchBytes until the process exits.  Host code must not use the
// symbol's name as an address (it is a host-side stand-in); the device address is
// looked up once per device below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace

cudaError_t launch_batch_noalloc(const SweepArgs *descs, const int32_t *wpbs, int32_t n, size_t smem, bool record,
                                 cudaStream_t s)
{
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess)
        return err;
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return cudaErrorInvalidDevice;
    void *ptr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            // set-up, once per device, with that device current
            err = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_scratch);
            if (err != cudaSuccess) {
                g_noalloc_ptr[dev] = nullptr;
                return err;
            }
        }
        ptr = g_noalloc_ptr[dev];
    }
    // descriptors, walkers per item, prefix sums and a zero counter, staged on the stack
    unsigned char host[kNoAllocCounterOffset + sizeof(uint32_t)];
    std::memset(host, 0, sizeof host);
    std::memcpy(host, descs, sizeof(SweepArgs) * (size_t)n);
    int32_t *hw = reinterpret_cast<int32_t *>(host + kNoAllocWpbOffset);
    int32_t *hp = hw + kNoAllocMaxInstances;
    hp[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        hw[i] = wpbs[i];
        hp[i + 1] = hp[i] + (int32_t)((descs[i].W + wpbs[i] - 1) / wpbs[i]);
    }
    // pageable source: the copy has left the stack buffer when the call returns
    err = cudaMemcpyAsync(ptr, host, sizeof host, cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess)
        return err;
    auto kern = record ? batch_noalloc_kernel<true> : batch_noalloc_kernel<false>;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess)
        return err;
    int sms = 1, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBatchThreads, smem);
    if (err != cudaSuccess)
        return err;
    if (occ < 1)
        return cudaErrorInvalidConfiguration;
    kern<<<sms * occ, kBatchThreads, smem, s>>>(static_cast<const unsigned char *>(ptr), n);
    return cudaGetLastError();
}

size_t lattice_bytes(int32_t L, int32_t layout, int64_t W)
{
    if (layout == MUCA_LAYOUT_PACKED)
        return (size_t)L * (size_t)W * (L <= 32 ? 4 : 8);
    return (size_t)L * L * (size_t)W;
}

}  // namespace muca
