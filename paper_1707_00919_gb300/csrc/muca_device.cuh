// muca_device.cuh - device code of the whole-sweep kernels, shared by the per-L
// translation units (muca_full_L.cu), the batched kernels (muca_batch.cu) and the
// generic kernels (muca_kernels.cu).  Parallel multicanonical 2D Ising update of Gross,
// Zierenberg, Weigel, Janke (arXiv:1707.00919), Sec. 2.3.
#pragma once

#include <cstddef>
#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#include "../../include/muca.h"
#include "muca_internal.h"

namespace muca {
namespace {

__host__ __device__ constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

template <typename RowT>
__device__ __forceinline__ uint32_t bit_at(RowT w, int x)
{
    return (uint32_t)(w >> x) & 1u;
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
// an accepted flip moves E by 28 (2 - k).  The batched kernel's L = 64 items use 6-word
// rows instead (24 bytes, thermalization counts in the histogram word, which such
// launches never read), which lets 256 walkers share an SM with the 4097-row table.
//
// Latency: the threshold an attempt needs depends on whether the previous attempt
// flipped (through E and through k).  Both candidates are loaded two attempts ahead and
// the right one is picked once the previous decision is known, which takes the shared-
// memory latency off the attempt-to-attempt dependency chain.  Both candidates are
// compared with the random word as soon as they arrive, so the decision itself is one
// select of two booleans, and both load addresses of the next-but-one attempt are
// formed before the decision and selected by it.  So is, in the whole-row stream, the
// row address the next attempt moves to if it flips (E + its step for both outcomes of
// the current attempt): one select after a decision instead of a select and an add.
// ---------------------------------------------------------------------------------
template <int L>
struct RowOf {
    using type = typename std::conditional<(L <= 32), uint32_t, unsigned long long>::type;
};


// Philox4x32-10 of Salmon et al. (SC'11), the generator of Sec. 2.3, on counter c with
// key (k0, k1).
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

// Counter tags of the Philox streams: updates, initial spins, random site order.
constexpr uint32_t kTagMetropolis = 0u;
constexpr uint32_t kTagInit = 1u;
constexpr uint32_t kTagSite = 2u;
constexpr uint32_t kSharedStream = 0xFFFFFFFFu;   // walker word of the site stream

struct PhiloxKeys {
    uint32_t k0[10], k1[10];   // round keys
    uint32_t hi_w, lo_w;       // round-0 product of the walker counter word
    uint32_t c1;               // counter word 1 (high word of t >> 2) the next two are for
    uint32_t r1_hi, r1_lo;     // round-1 product of the first word, (hi_w ^ c1 ^ k0) * M0
};

// Round keys of the seed and the products that depend only on the walker and on counter
// word 1: with the tag word 0, round 0 turns (c0, c1, walker, 0) into
// (hi_w ^ c1 ^ k0, lo_w, hi(M0 c0) ^ k1, lo(M0 c0)), so round 1's first product is
// fixed for as long as c1 is (2^34 attempts).
__device__ __forceinline__ PhiloxKeys make_keys(uint64_t seed, uint32_t walker, uint32_t c1 = 0)
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
    p.c1 = c1;
    const unsigned long long p1 = (unsigned long long)0xD2511F53u * (p.hi_w ^ c1 ^ p.k0[0]);
    p.r1_hi = (uint32_t)(p1 >> 32);
    p.r1_lo = (uint32_t)p1;
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

// The same on counter (c0, p.c1, walker, tag 0), with round 1's product of the
// constant word taken from the keys: one wide multiply fewer per call.
__device__ __forceinline__ uint4 philox_walker_c1(uint32_t c0, const PhiloxKeys &p)
{
    const unsigned long long q = (unsigned long long)0xD2511F53u * c0;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * ((uint32_t)(q >> 32) ^ p.k1[0]);
    uint32_t x0 = (uint32_t)(p1 >> 32) ^ p.lo_w ^ p.k0[1];
    uint32_t x1 = (uint32_t)p1;
    uint32_t x2 = p.r1_hi ^ (uint32_t)q ^ p.k1[1];
    uint32_t x3 = p.r1_lo;
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * x0;
        const unsigned long long pp = (unsigned long long)0xCD9E8D57u * x2;
        const uint32_t n0 = (uint32_t)(pp >> 32) ^ x1 ^ p.k0[r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ x3 ^ p.k1[r];
        x0 = n0;
        x1 = (uint32_t)pp;
        x2 = n2;
        x3 = (uint32_t)p0;
    }
    return make_uint4(x0, x1, x2, x3);
}

// Sign bits of four int8 spins (-1 = 0xFF, +1 = 0x01) as a nibble.
__device__ __forceinline__ uint32_t gather_signs(uint32_t v) { return ((v & 0x80808080u) * 0x00204081u) >> 28; }

// Nibble of down-spin bits to four int8 spins.
__device__ __forceinline__ uint32_t spread_signs(uint32_t n)
{
    return 0x01010101u | (((n * 0x00204081u) & 0x01010101u) * 0xFEu);
}

// Butterfly stages 8, 4, 2, 1 of a 32x32 bit transpose across a warp: swaps bits 0-3 of
// the lane index with bits 0-3 of the bit position (bit 4 of each stays in place).
__device__ __forceinline__ uint32_t warp_swap_low4(uint32_t m, int lane)
{
    const uint32_t masks[4] = {0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int s = 8 >> i;
        const uint32_t part = __shfl_xor_sync(0xFFFFFFFFu, m, s);
        m = (lane & s) ? ((m & ~masks[i]) | ((part >> s) & masks[i])) : ((m & masks[i]) | ((part & masks[i]) << s));
    }
    return m;
}

// Sign bits of 16 int8 spins as a 16-bit mask (bit i = byte i).
__device__ __forceinline__ uint32_t gather16(uint4 u)
{
    return gather_signs(u.x) | (gather_signs(u.y) << 4) | (gather_signs(u.z) << 8) | (gather_signs(u.w) << 12);
}

// Bit rows of the warp's 32 walkers from the int8 [site][walker] layout, R rows at a
// time so that their loads are in flight together; lane j receives walker w0 + j.
// Lanes 2p and 2p + 1 read the two halves of one site's 32 walker bytes (sites 32h + p and
// 32h + 16 + p of row half h), so each load instruction covers 16 whole 32-byte sectors.
// Lane 2p + q then holds bit 16r + s = spin of walker 16q + s at site 32h + 16r + p; a
// lane shuffle to lane 16q + p and four butterfly stages (lane bits 0-3 against bit
// positions 0-3) leave in lane 16q + s the spins of walker 16q + s, bit x at site 32h + x.
// All 32 walkers must exist and W % 16 == 0.
template <int L, int R, typename RowT>
__device__ __forceinline__ void warp_load_rows_int8(const int8_t *g, int64_t W, int64_t w0, int y0, int lane,
                                                    RowT (&out)[R])
{
    constexpr int HALVES = (L + 31) / 32;
    const int p = lane >> 1, q = lane & 1;
    uint4 a[R][HALVES], b[R][HALVES];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int half = 0; half < HALVES; ++half) {
            const int xa = half * 32 + p, xb = xa + 16;
            const int8_t *row = g + (size_t)((y0 + r) * L) * (size_t)W + (size_t)w0 + 16 * q;
            a[r][half] = xa < L ? *reinterpret_cast<const uint4 *>(row + (size_t)xa * (size_t)W) : make_uint4(0, 0, 0, 0);
            b[r][half] = xb < L ? *reinterpret_cast<const uint4 *>(row + (size_t)xb * (size_t)W) : make_uint4(0, 0, 0, 0);
        }
    const int src = 2 * (lane & 15) + (lane >> 4);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        RowT row = 0;
#pragma unroll
        for (int half = 0; half < HALVES; ++half) {
            uint32_t m = gather16(a[r][half]) | (gather16(b[r][half]) << 16);
            m = __shfl_sync(0xFFFFFFFFu, m, src);
            m = warp_swap_low4(m, lane);
            row |= (RowT)m << (32 * half);
        }
        out[r] = row;
    }
}

// 16 spins of a 16-bit mask (bit i = byte i, set = -1) as int8.
__device__ __forceinline__ uint4 scatter16(uint32_t h)
{
    return make_uint4(spread_signs(h & 15u), spread_signs((h >> 4) & 15u), spread_signs((h >> 8) & 15u),
                      spread_signs((h >> 12) & 15u));
}

// The inverse of warp_load_rows_int8 for one row: lane j holds walker w0 + j's bits.
template <int L, typename RowT>
__device__ __forceinline__ void warp_store_row_int8(int8_t *g, int64_t W, int64_t w0, int y, int lane, RowT r)
{
    const int p = lane >> 1, q = lane & 1;
    const int src = 16 * q + p;
#pragma unroll
    for (int half = 0; half < (L + 31) / 32; ++half) {
        uint32_t m = warp_swap_low4((uint32_t)(r >> (32 * half)), lane);
        m = __shfl_sync(0xFFFFFFFFu, m, src);
        const int xa = half * 32 + p, xb = xa + 16;
        int8_t *row = g + (size_t)(y * L) * (size_t)W + (size_t)w0 + 16 * q;
        if (xa < L)
            *reinterpret_cast<uint4 *>(row + (size_t)xa * (size_t)W) = scatter16(m & 0xFFFFu);
        if (xb < L)
            *reinterpret_cast<uint4 *>(row + (size_t)xb * (size_t)W) = scatter16(m >> 16);
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

// Thermalization launches add the same count to the row's padding word (offset 24; with
// 6-word rows the histogram word, which such launches never flush), which nothing reads.
// The reduction orders the shared-memory threshold loads of later attempts behind it
// exactly as in a recording launch; without it the compiler's schedule was measured 11%
// slower (72 vs 64 cycles per attempt and warp at L = 32).
template <int STRIDE>
__device__ __forceinline__ void pad_add_one(uint32_t E)
{
    if (STRIDE == 7)
        asm volatile("red.shared.add.u32 [%0+24], 1;" :: "r"(E));
    else
        asm volatile("red.shared.add.u32 [%0+20], 1;" :: "r"(E));
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
    __device__ __forceinline__ void advance() const {}
};

// The same for a row whose Philox blocks all have counter word 1 equal to pk->c1.  The
// words of the row's first block are computed during the previous row (advance(), called
// by process_row during its last block) and kept in *carry, so that a new row does not
// start by waiting for a whole Philox evaluation.
template <int L>
struct PhiloxSourceC1 {
    uint32_t blk;            // counter word 0 of column 0's block
    const PhiloxKeys *pk;
    uint4 *carry;            // clamped words of block blk, then of the next row's first block
    __device__ __forceinline__ static uint4 words(uint32_t b, const PhiloxKeys &k)
    {
        const uint4 rw = philox_walker_c1(b, k);
        return make_uint4(min(rw.x, 0xFFFFFFFEu), min(rw.y, 0xFFFFFFFEu), min(rw.z, 0xFFFFFFFEu),
                          min(rw.w, 0xFFFFFFFEu));
    }
    __device__ __forceinline__ uint4 get(int xb) const { return xb == 0 ? *carry : words(blk + (uint32_t)(xb / 4), *pk); }
    __device__ __forceinline__ void advance() const { *carry = words(blk + (uint32_t)(L / 4), *pk); }
};

// MASKED: only the attempts x in [x_begin, x_end) happen (a launch that starts or ends
// inside the row); the others neither flip nor count, their random words go unused.
template <int L, bool RECORD, bool MASKED, class Src, int STRIDE = kTableStride>
__device__ __forceinline__ void process_row(const uint32_t (&U)[L / 8], uint32_t (&C)[L / 8], const uint32_t (&D)[L / 8],
                                            uint32_t &E, const Src &src, int x_begin = 0, int x_end = L)
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
    // row step of a flip with count k = J / 4: 4 STRIDE (2 - k) bytes
    constexpr uint32_t kD2 = 8u * STRIDE, kDJ = STRIDE;
    uint32_t d0_cur = kD2 - kDJ * J0a, d1_cur = d0_cur;               // attempt x
    uint32_t d0_next = kD2 - kDJ * J0b, d1_next = kD2 - kDJ * J1b;    // attempt x + 1
    uint32_t T0n = lds_u32(E + J0a), T1n = T0n;                      // candidates of x
    uint32_t T0nn = lds_u32(E + J0b), T1nn = lds_u32(E + d0_cur + J1b);   // of x + 1
    bool prev_acc = false;
    uint32_t Eres = E;

#pragma unroll
    for (int xb = 0; xb < L; xb += 4) {
        const uint4 rw = src.get(xb);
        if (xb == L - 4)
            src.advance();
        const uint32_t words[4] = {rw.x, rw.y, rw.z, rw.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int x = xb + u;
            // decision of attempt x
            const uint32_t dsel = prev_acc ? d1_cur : d0_cur;
            const uint32_t Eacc = Eres + dsel;
            const bool c0 = words[u] < T0n, c1 = words[u] < T1n;
            const bool in_range = !MASKED || (x >= x_begin && x < x_end);
            const bool acc = (prev_acc ? c1 : c0) && in_range;
            const uint32_t Epost = acc ? Eacc : Eres;
            C[x >> 3] ^= acc ? (1u << (4 * (x & 7))) : 0u;
            if (x == 0)
                adj_last = acc ? adj_if_flip : 0u;
            if (RECORD) {
                // masked attempts of a recording launch count nothing (with 6-word rows
                // there is no padding word to send them to)
                if (in_range)
                    hist_add_one(Epost);
            } else {
                pad_add_one<STRIDE>(Epost);
            }
            // candidates of attempt x + 2 for both outcomes of attempt x + 1
            T0n = T0nn;
            T1n = T1nn;
            if (x + 2 < L) {
                uint32_t J0c, J1c;
                MUCA_SITE_J(x + 2, J0c, J1c);
                const uint32_t a0 = acc ? Eacc + J0c : Eres + J0c;
                const uint32_t a1 = acc ? Eacc + d1_next + J1c : Eres + d0_next + J1c;
                T0nn = lds_u32(a0);
                T1nn = lds_u32(a1);
                d0_cur = d0_next;
                d1_cur = d1_next;
                d0_next = kD2 - kDJ * J0c;
                d1_next = kD2 - kDJ * J1c;
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

// ---------------------------------------------------------------------------------
// Continuous attempt stream over whole rows (whole-sweep launches).  The two threshold
// candidates of every attempt are loaded two attempts ahead, across row ends as well:
// the first two sites of the next row have as neighbours the current row's first two
// sites (final after its attempts 0 and 1) and rows that the current row does not
// change, so their counts, and the candidates of the next row's attempts 0 and 1, are
// known during the current row's attempts L - 2 and L - 1.  A new row then starts with
// its first two decisions ready instead of waiting for its counts and loads.
// ---------------------------------------------------------------------------------
template <int L, int STRIDE>
struct AttemptStream {
    static constexpr uint32_t kD2 = 8u * STRIDE, kDJ = STRIDE;   // row step 4 STRIDE (2 - k) = kD2 - kDJ J
    uint32_t E;                      // table row address of the current energy
    bool prev_acc;                   // the previous attempt flipped
    uint32_t T0n, T1n, T0nn, T1nn;   // candidates of the next two attempts
    uint32_t Eacc;                   // row address if the current attempt flips
    uint32_t d0_next, d1_next;

    // Counts of the row (U above, C, D below) in nibble fields: K0 if the left
    // neighbour did not flip, K1 if it did.
    __device__ __forceinline__ static void counts(const uint32_t (&U)[L / 8], const uint32_t (&C)[L / 8],
                                                  const uint32_t (&D)[L / 8], uint32_t (&K0)[L / 8],
                                                  uint32_t (&K1)[L / 8])
    {
        constexpr int NW = L / 8;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            const uint32_t cr = __funnelshift_r(C[i], C[(i + 1) % NW], 4);
            const uint32_t cl = __funnelshift_l(C[(i + NW - 1) % NW], C[i], 4);
            const uint32_t kb = (U[i] ^ C[i]) + (D[i] ^ C[i]) + (C[i] ^ cr);
            const uint32_t h0 = C[i] ^ cl;
            K0[i] = kb + h0;
            K1[i] = kb + 0x11111111u - h0;
        }
    }

    // First row of a launch: the candidates of its attempts 0 and 1.
    __device__ __forceinline__ void start(const uint32_t (&U)[L / 8], const uint32_t (&C)[L / 8],
                                          const uint32_t (&D)[L / 8], uint32_t E0)
    {
        uint32_t K0[L / 8], K1[L / 8];
        counts(U, C, D, K0, K1);
        const uint32_t J0a = field_x4(K0[0], 0), J0b = field_x4(K0[0], 1), J1b = field_x4(K1[0], 1);
        E = E0;
        prev_acc = false;
        const uint32_t d0 = kD2 - kDJ * J0a;
        Eacc = E0 + d0;
        d0_next = kD2 - kDJ * J0b;
        d1_next = kD2 - kDJ * J1b;
        T0n = T1n = lds_u32(E + J0a);
        T0nn = lds_u32(E + J0b);
        T1nn = lds_u32(E + d0 + J1b);
    }

    // One row (U above, C updated in place, D below, D2 the row below D); on return the
    // candidates of the next row's attempts 0 and 1 are loaded.
    template <bool RECORD, class Src>
    __device__ __forceinline__ void row(const uint32_t (&U)[L / 8], uint32_t (&C)[L / 8], const uint32_t (&D)[L / 8],
                                        const uint32_t (&D2)[L / 8], const Src &src)
    {
        constexpr int NW = L / 8;
        uint32_t K0[NW], K1[NW];
        counts(U, C, D, K0, K1);
        uint32_t K0n = 0u, K1n = 0u;   // word 0 of the next row's counts (fields 0 and 1 used)
        const uint32_t hr_last = ((C[NW - 1] >> 28) ^ C[0]) & 1u;
        const uint32_t adj_if_flip = hr_last ? (uint32_t)-4 : 4u;
        uint32_t adj_last = 0u;
        uint32_t Eres = E;
#pragma unroll
        for (int xb = 0; xb < L; xb += 4) {
            const uint4 rw = src.get(xb);
            if (xb == L - 4) {
                src.advance();
                // the current row's sites 0 and 1 are final: the next row's first counts
                const uint32_t crn = __funnelshift_r(D[0], D[1 % NW], 4);
                const uint32_t cln = __funnelshift_l(D[NW - 1], D[0], 4);
                const uint32_t kbn = (C[0] ^ D[0]) + (D2[0] ^ D[0]) + (D[0] ^ crn);
                const uint32_t h0n = D[0] ^ cln;
                K0n = kbn + h0n;
                K1n = kbn + 0x11111111u - h0n;
            }
            const uint32_t words[4] = {rw.x, rw.y, rw.z, rw.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int x = xb + u;
                const bool c0 = words[u] < T0n, c1 = words[u] < T1n;
                const bool acc = prev_acc ? c1 : c0;
                const uint32_t Epost = acc ? Eacc : Eres;
                C[x >> 3] ^= acc ? (1u << (4 * (x & 7))) : 0u;
                if (x == 0)
                    adj_last = acc ? adj_if_flip : 0u;
                if (RECORD)
                    hist_add_one(Epost);
                else
                    pad_add_one<STRIDE>(Epost);
                // candidates of attempt x + 2 (in this row or the next) for both outcomes
                // of attempt x + 1
                uint32_t J0c, J1c;
                if (x + 2 < L) {
                    J0c = field_x4(K0[(x + 2) >> 3], (x + 2) & 7);
                    J1c = field_x4(K1[(x + 2) >> 3], (x + 2) & 7);
                    if (x + 2 == L - 1) {
                        J0c += adj_last;
                        J1c += adj_last;
                    }
                } else if (x + 2 == L) {
                    J0c = J1c = field_x4(K0n, 0);   // site 0: its left neighbour comes later
                } else {
                    J0c = field_x4(K0n, 1);
                    J1c = field_x4(K1n, 1);
                }
                T0n = T0nn;
                T1n = T1nn;
                // the next attempt's flipped row, formed from both outcomes before this
                // decision and selected by it
                const uint32_t t1 = Eacc + d1_next, t0 = Eres + d0_next;
                const uint32_t a0 = acc ? Eacc + J0c : Eres + J0c;
                const uint32_t a1 = acc ? t1 + J1c : t0 + J1c;
                T0nn = lds_u32(a0);
                T1nn = lds_u32(a1);
                Eacc = acc ? t1 : t0;
                d0_next = kD2 - kDJ * J0c;
                d1_next = kD2 - kDJ * J1c;
                Eres = Epost;
                prev_acc = acc;
            }
        }
        E = Eres;
    }
};

// nsweeps whole sweeps of one walker from Philox block blk (column 0 of row 0); U, C, D
// hold rows L - 1, 0 and 1 on entry and are left in the same state on exit.
// nrows whole rows of one walker as one continuous attempt stream, from row y0 (wrapping
// to row 0 after row L - 1) whose column 0 lies in Philox block blk; U, C, D hold rows
// y0 - 1, y0 and y0 + 1 on entry and the rows around the next row on exit.  Counter
// word 1 must stay at pk.c1 for the whole range.
template <int L, bool RECORD, int STRIDE>
__device__ __forceinline__ void stream_rows_c1(const SmemRows<L> &rows, uint32_t (&U)[L / 8], uint32_t (&C)[L / 8],
                                               uint32_t (&D)[L / 8], uint32_t &E, uint64_t blk, int y0,
                                               uint64_t nrows, const PhiloxKeys &pk)
{
    constexpr int NW = L / 8;
    uint32_t b = (uint32_t)blk;
    uint4 carry = PhiloxSourceC1<L>::words(b, pk);
    AttemptStream<L, STRIDE> st;
    st.start(U, C, D, E);
    int y = y0;
#pragma unroll 1
    for (uint64_t r = 0; r < nrows; ++r) {
        const int y2 = (y + 2 < L) ? y + 2 : y + 2 - L;
        uint32_t D2[NW];
        rows.load(y2, D2);
        const PhiloxSourceC1<L> src{b, &pk, &carry};
        st.template row<RECORD>(U, C, D, D2, src);
        rows.store(y, C);
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            U[i] = C[i];
            C[i] = D[i];
            D[i] = D2[i];
        }
        b += (uint32_t)(L / 4);
        y = (y + 1 == L) ? 0 : y + 1;
    }
    E = st.E;
}

// Counter word 1 must stay at pk.c1 for the whole range.  The row below the next one is
// loaded from shared memory when a row starts (the current row does not change it), and
// the next row's first Philox block is computed during the current row.
template <int L, bool RECORD, int STRIDE>
__device__ __forceinline__ void whole_sweeps_c1(const SmemRows<L> &rows, uint32_t (&U)[L / 8], uint32_t (&C)[L / 8],
                                                uint32_t (&D)[L / 8], uint32_t &E, uint64_t blk, uint64_t nsweeps,
                                                const PhiloxKeys &pk)
{
    // the same stream as stream_rows_c1, as a loop over sweeps and rows (the row index a
    // loop variable rather than a wrapped counter: measured about 3 % faster)
    constexpr int NW = L / 8;
    uint32_t b = (uint32_t)blk;
    uint4 carry = PhiloxSourceC1<L>::words(b, pk);
    AttemptStream<L, STRIDE> st;
    st.start(U, C, D, E);
    for (uint64_t s = 0; s < nsweeps; ++s) {
#pragma unroll 1
        for (int y = 0; y < L; ++y) {
            const int y2 = (y + 2 < L) ? y + 2 : y + 2 - L;
            uint32_t D2[NW];
            rows.load(y2, D2);
            const PhiloxSourceC1<L> src{b, &pk, &carry};
            st.template row<RECORD>(U, C, D, D2, src);
            rows.store(y, C);
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                U[i] = C[i];
                C[i] = D[i];
                D[i] = D2[i];
            }
            b += (uint32_t)(L / 4);
        }
    }
    E = st.E;
}

// The same with the general generator (any counter range).
template <int L, bool RECORD, int STRIDE>
__device__ __forceinline__ void whole_sweeps(const SmemRows<L> &rows, uint32_t (&U)[L / 8], uint32_t (&C)[L / 8],
                                             uint32_t (&D)[L / 8], uint32_t &E, uint64_t blk, uint64_t nsweeps,
                                             const PhiloxKeys &pk)
{
    constexpr int NW = L / 8;
    for (uint64_t s = 0; s < nsweeps; ++s) {
#pragma unroll 1
        for (int y = 0; y < L; ++y) {
            const PhiloxSource src{blk, &pk};
            process_row<L, RECORD, false, PhiloxSource, STRIDE>(U, C, D, E, src);
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
}

// One block's share of a launch: walkers wbase .. wbase + wpb - 1 of the instance in
// `a` (threads tid >= wpb idle), all of the launch's whole sweeps.  Shared memory:
// the table, then the rows of the wpb walkers.  Every thread of the block calls it.
// The layout only changes the loads and stores around the sweeps; callers with a
// compile-time layout get it folded, the batched kernels pass it at run time.  GUARD
// adds kTableGuard zero rows on both sides of the table, for energies that come from the
// caller and need not match the lattices (the library's own energies always do).
// C1_ONLY: the caller guarantees that counter word 1 (t >> 34) is the same for every
// attempt of the launch, so only the generator that relies on it is compiled in.
template <int L, bool RECORD, bool PARTIAL = false, bool GUARD = false, int STRIDE = kTableStride,
          bool C1_ONLY = false>
__device__ __forceinline__ void sweep_block(const SweepArgs &a, int64_t wbase, int wpb, unsigned char *smem,
                                            const int LAYOUT)
{
    if (a.skip && *a.skip)   // an iteration run on the device has finished
        return;
    using RowT = typename RowOf<L>::type;
    constexpr int N = L * L;
    constexpr int NB = N + 1;
    constexpr int NW = L / 8;
    constexpr int RB = 4;   // rows per batch of int8 loads
    const int nthr = blockDim.x;
    uint32_t *sTab = reinterpret_cast<uint32_t *>(smem);
    const int tid = threadIdx.x;
    constexpr int G = GUARD ? kTableGuard : 0;
    constexpr int NR = NB + 2 * G;   // table rows: energies -G .. N + G
    const SmemRows<L> rows{smem + align_up((size_t)NR * STRIDE * 4, 16), wpb, tid};
    const int lane = tid & 31;
    const bool in_item = tid < wpb;
    const int64_t w = wbase + tid;
    const int64_t w0 = w - lane;
    bool active = in_item && w < a.W;
    const bool warp_full = in_item && (w0 + 32 <= a.W) && (a.W % 16 == 0);

    // the thresholds as asynchronous 4-byte copies (all in flight together and behind the
    // lattice load; waited for before the barrier), the other words of the table zeroed
    {
        const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sTab);
        for (int i = tid; i < NB * 5; i += nthr) {
            const int e = i / 5, k = i - e * 5;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sbase + 4u * (uint32_t)((e + G) * STRIDE + k)),
                         "l"(a.table + i)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        for (int i = tid; i < NR * STRIDE; i += nthr) {
            const int r = i / STRIDE, k = i - r * STRIDE;
            const int e = r - G;
            if (k >= 5 || e < 0 || e > N)
                sTab[i] = 0u;
        }
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
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();

    const PhiloxKeys pk = make_keys(a.seed, a.walker0 + (uint32_t)w, (uint32_t)(a.t0 >> 34));
    const uint32_t tbase = (uint32_t)__cvta_generic_to_shared(sTab) + G * STRIDE * 4u;
    uint32_t U[NW], C[NW], D[NW];
    uint32_t E = tbase + (uint32_t)e * (4u * STRIDE);
    if (C1_ONLY && !PARTIAL) {
        // whole sweeps from a sweep boundary, counter word 1 (t >> 34) fixed for the launch
        // (launch_sweep splits launches at its steps).  A recording launch may carry a
        // thermalization phase in front (n_therm attempts): the same attempt stream, its
        // counts added to the histogram words and cleared before the recorded phase, so
        // that the launch equals a thermalization launch followed by a recording one.
        // Both phases run the one inlined copy of the sweep loop.
        if (active) {
            rows.load(L - 1, U);
            rows.load(0, C);
            rows.load(1, D);
        }
        const bool fused = RECORD && a.n_therm > 0;   // uniform over the launch
        uint64_t blk = a.t0 >> 2;
        uint64_t ns = (fused ? a.n_therm : a.n) / (uint64_t)N;
#pragma unroll 1
        for (int phase = fused ? 0 : 1; phase < 2; ++phase) {
            if (active)
                whole_sweeps_c1<L, RECORD, STRIDE>(rows, U, C, D, E, blk, ns, pk);
            if (phase == 0) {
                __syncthreads();
                for (int i = tid; i < NB; i += nthr)
                    sTab[(i + G) * STRIDE + kHistSlot] = 0u;
                __syncthreads();
                blk += ns * (uint64_t)(N / 4);
                ns = a.n / (uint64_t)N;
            }
        }
    } else {
        // every other form (the general generator, any attempt range, the batched
        // kernels): a recording launch may carry a thermalization phase in front here too
        // (a.n_therm attempts from a.t0, any range), its counts cleared between the phases
        const bool fused = RECORD && a.n_therm > 0;   // uniform over the launch
#pragma unroll 1
        for (int phase = fused ? 0 : 1; phase < 2; ++phase) {
            const uint64_t t0p = phase == 0 ? a.t0 : a.t0 + (fused ? a.n_therm : 0u);
            const uint64_t np = phase == 0 ? a.n_therm : a.n;
            if (active && np > 0) {
                const PhiloxKeys pkp = make_keys(a.seed, a.walker0 + (uint32_t)w, (uint32_t)(t0p >> 34));
                if (!PARTIAL) {
                    // whole sweeps from a sweep boundary; counter word 1 (t >> 34) is the same
                    // for every attempt of the range except in the rare range that crosses a
                    // step of it, which takes the general generator throughout (kernels whose
                    // launches never cross one compile only the first)
                    rows.load(L - 1, U);
                    rows.load(0, C);
                    rows.load(1, D);
                    if (C1_ONLY || (t0p >> 34) == ((t0p + np - 1) >> 34))
                        whole_sweeps_c1<L, RECORD, STRIDE>(rows, U, C, D, E, t0p >> 2, np / (uint64_t)N, pkp);
                    else
                        whole_sweeps<L, RECORD, STRIDE>(rows, U, C, D, E, t0p >> 2, np / (uint64_t)N, pkp);
                } else {
                    // any attempt range: a first row cut by the launch's start and a last row cut
                    // by its end run masked, the whole rows between them as one attempt stream
                    uint64_t t = t0p;
                    const uint64_t tend = t0p + np;
                    int y = (int)((t % (uint64_t)N) / L);
                    const int x0 = (int)((t % (uint64_t)N) % L);
                    uint64_t blk = (t - (uint64_t)x0) >> 2;   // Philox block of column 0 of row y
                    rows.load((y + L - 1) % L, U);
                    rows.load(y, C);
                    rows.load((y + 1) % L, D);
                    bool ended = false;
                    if (x0 != 0 || tend - t < (uint64_t)L) {
                        const uint64_t left = tend - t;
                        const int xe = left < (uint64_t)(L - x0) ? x0 + (int)left : L;
                        const PhiloxSource src{blk, &pkp};
                        process_row<L, RECORD, true, PhiloxSource, STRIDE>(U, C, D, E, src, x0, xe);
                        rows.store(y, C);
                        t += (uint64_t)(xe - x0);
                        ended = xe < L;   // the launch ends inside this row
                        if (!ended) {
                            const int y2 = (y + 2 < L) ? y + 2 : y + 2 - L;
        #pragma unroll
                            for (int i = 0; i < NW; ++i) {
                                U[i] = C[i];
                                C[i] = D[i];
                            }
                            rows.load(y2, D);
                            y = (y + 1 == L) ? 0 : y + 1;
                            blk += (uint64_t)(L / 4);
                        }
                    }
                    const uint64_t nwhole = ended ? 0u : (tend - t) / (uint64_t)L;
                    if (nwhole > 0) {
                        if (C1_ONLY || (t0p >> 34) == ((t0p + np - 1) >> 34)) {
                            stream_rows_c1<L, RECORD, STRIDE>(rows, U, C, D, E, blk, y, nwhole, pkp);
                        } else {
        #pragma unroll 1
                            for (uint64_t r = 0; r < nwhole; ++r) {
                                const PhiloxSource src{blk + r * (uint64_t)(L / 4), &pkp};
                                const int yr = (int)(((uint64_t)y + r) % (uint64_t)L);
                                process_row<L, RECORD, false, PhiloxSource, STRIDE>(U, C, D, E, src);
                                rows.store(yr, C);
                                const int y2 = (yr + 2 < L) ? yr + 2 : yr + 2 - L;
        #pragma unroll
                                for (int i = 0; i < NW; ++i) {
                                    U[i] = C[i];
                                    C[i] = D[i];
                                }
                                rows.load(y2, D);
                            }
                        }
                        t += nwhole * (uint64_t)L;
                        y = (int)(((uint64_t)y + nwhole) % (uint64_t)L);
                        blk += nwhole * (uint64_t)(L / 4);
                    }
                    if (!ended && t < tend) {   // the launch ends inside the next row
                        const PhiloxSource src{blk, &pkp};
                        process_row<L, RECORD, true, PhiloxSource, STRIDE>(U, C, D, E, src, 0, (int)(tend - t));
                        rows.store(y, C);
                    }
                }
            }
            if (phase == 0) {
                __syncthreads();
                for (int i = tid; i < NB; i += nthr)
                    sTab[(i + G) * STRIDE + kHistSlot] = 0u;
                __syncthreads();
            }
        }
    }
    if (active) {
        e = (int32_t)((E - tbase) / (4u * STRIDE));
        if (E < tbase || e > N || (E - tbase) % (4u * STRIDE) != 0u)   // corrupted energy address
            atomicOr(a.err, kErrEnergyRange);
    }
    __syncthreads();
    if (RECORD)
        for (int i = tid; i < NB; i += nthr) {
            const uint32_t v = sTab[(i + G) * STRIDE + kHistSlot];
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

// A batched work item: the whole-sweep body of the item's instance.  ANY_RANGE: the
// item's launch may start or end inside a sweep (the Eq. (7) schedule's attempt
// counts), which then takes the body with the partial-row path.
template <int L, bool RECORD, bool GUARD = false, int STRIDE = kTableStride, bool ANY_RANGE = false>
__device__ __forceinline__ void batch_item(const SweepArgs &a, const BatchItem &it, unsigned char *smem)
{
    constexpr uint64_t N = (uint64_t)L * (uint64_t)L;
    if (!ANY_RANGE || (a.t0 % N == 0 && a.n % N == 0 && a.n_therm % N == 0))
        sweep_block<L, RECORD, false, GUARD, STRIDE>(a, it.wbase, it.wpb, smem, a.layout);
    else
        sweep_block<L, RECORD, true, GUARD, STRIDE>(a, it.wbase, it.wpb, smem, a.layout);
}

}  // namespace
}  // namespace muca
