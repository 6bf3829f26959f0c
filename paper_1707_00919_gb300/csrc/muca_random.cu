// muca_random.cu - updates in random shared site order, the paper's scheme of Sec. 2.3:
// one random site sequence drives all walkers (so a warp's accesses to a site coincide)
// and each walker draws its acceptance from its own stream.  The site of attempt t is
// floor(u N / 2^32) with u the Philox word t & 3 of counter (t >> 2, 0xFFFFFFFF, tag 2);
// the acceptance word is the one of typewriter order (tag 0, the walker's counter).
//
// One thread runs one walker; its lattice sits in shared memory as one bit row per
// lattice row ([row][walker-in-block]); the block draws the sites of a chunk of
// attempts into shared memory together, then every walker runs the chunk.
#include <cstdint>

#include "muca_device.cuh"

namespace muca {
namespace {

// Attempts whose sites are drawn at once: 32-byte records, half as many for 64-bit rows
// so that the larger lattices keep their block size.
template <typename RowT>
__host__ __device__ constexpr int site_chunk()
{
    return sizeof(RowT) == 4 ? 1024 : 512;
}
constexpr int kSpare = 4;          // records past a chunk's end, read by the look-ahead
constexpr uint32_t kCleanBit = 1u << 31;   // in the first record of a clean group (offset word)
constexpr int kRandStride = 6;     // words per table row: thresholds of k = 0..4, histogram count
constexpr int kRandGuard = 2;      // zero rows below energy 0 and above N (speculative loads)

template <typename RowT>
size_t random_smem_bytes_t(int L, int wpb, bool)
{
    const size_t rows = (size_t)L * L + 1 + 2 * kRandGuard;
    return align_up(rows * kRandStride * 4, 16) + (size_t)(site_chunk<RowT>() + kSpare) * 32 +
           (size_t)L * wpb * sizeof(RowT);
}

template <typename RowT>
__device__ __forceinline__ RowT row_mask(uint32_t lo, uint32_t hi)
{
    return sizeof(RowT) == 4 ? (RowT)lo : (RowT)(((unsigned long long)hi << 32) | lo);
}

__device__ __forceinline__ uint32_t popcount(uint32_t v) { return (uint32_t)__popc(v); }
__device__ __forceinline__ uint32_t popcount(unsigned long long v) { return (uint32_t)__popcll(v); }

// Number k of antiparallel neighbours of a site from the rows above (U), at (C) and
// below (D) it; bx holds the site's bit x, mh bits x and x - 1 (mod L).  Bit i of
// C ^ rot(C) compares columns i and i + 1 (mod L), so its bits x and x - 1 are the
// right and left disagreements.  WIDE: L fills the row word, so rot is a plain rotation.
template <typename RowT, bool WIDE>
__device__ __forceinline__ uint32_t site_count(RowT U, RowT C, RowT D, RowT bx, RowT mh, int L)
{
    constexpr int kBits = 8 * (int)sizeof(RowT);
    const RowT rot = WIDE ? (RowT)((C >> 1) | (C << (kBits - 1))) : (RowT)((C >> 1) | ((C & (RowT)1) << (L - 1)));
    return popcount((C ^ rot) & mh) + popcount((U ^ C) & bx) + popcount((D ^ C) & bx);
}

__device__ __forceinline__ uint32_t lds_word(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void hist_count(uint32_t E)
{
    asm volatile("red.shared.add.u32 [%0+20], 1;" ::"r"(E));
}

// Bit rows of a warp's 32 walkers from the int8 [site][walker] layout, four rows at a
// time (their 16-byte loads in flight together): lane j receives walker w0 + j.  As in
// warp_load_rows_int8, lanes 2p and 2p + 1 read the two halves of one site's 32 walker
// bytes, and a lane shuffle plus four butterfly stages complete the transpose.  All 32
// walkers must exist and W % 16 == 0; L is a multiple of 4 up to 64.
template <typename RowT>
__device__ __forceinline__ void warp_load_rows(const int8_t *g, int64_t W, int64_t w0, int L, int y0, int lane,
                                               RowT (&out)[4])
{
    const int p = lane >> 1, q = lane & 1;
    uint4 va[4][2], vb[4][2];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int xa = half * 32 + p, xb = xa + 16;
            const int8_t *row = g + (size_t)((y0 + r) * L) * (size_t)W + (size_t)w0 + 16 * q;
            va[r][half] = xa < L ? *reinterpret_cast<const uint4 *>(row + (size_t)xa * (size_t)W) : make_uint4(0u, 0u, 0u, 0u);
            vb[r][half] = xb < L ? *reinterpret_cast<const uint4 *>(row + (size_t)xb * (size_t)W) : make_uint4(0u, 0u, 0u, 0u);
        }
    const int src = 2 * (lane & 15) + (lane >> 4);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        RowT row = 0;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            if (half * 32 >= L)   // uniform over the warp
                break;
            uint32_t m = gather16(va[r][half]) | (gather16(vb[r][half]) << 16);
            m = __shfl_sync(0xFFFFFFFFu, m, src);
            m = warp_swap_low4(m, lane);
            row |= (RowT)m << (32 * half);
        }
        out[r] = row;
    }
}

template <typename RowT>
__device__ __forceinline__ void warp_store_row(int8_t *g, int64_t W, int64_t w0, int L, int y, int lane, RowT r)
{
    const int p = lane >> 1, q = lane & 1;
    const int src = 16 * q + p;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        if (half * 32 >= L)   // uniform over the warp
            break;
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

template <typename RowT, int LAYOUT, bool RECORD, bool WIDE>
__global__ void __launch_bounds__(256) random_sweep_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    if (a.skip && *a.skip)   // an iteration run on the device has finished
        return;
    const int L = a.L;
    const int N = L * L;
    const int nrows = N + 1 + 2 * kRandGuard;
    const int wpb = blockDim.x;
    // table row r holds energy r - kRandGuard; the guard rows are zero (never accepted)
    uint32_t *sT = reinterpret_cast<uint32_t *>(smem);
    // per site of the chunk: byte offsets of the rows above (plus kCleanBit, see below),
    // at and below it in a walker's column, and x | y << 24; shared by all walkers of the
    // block
    uint4 *sSite = reinterpret_cast<uint4 *>(smem + align_up((size_t)nrows * kRandStride * 4, 16));
    // per site: its bit and its bit plus the left neighbour's, as row masks (lo, hi words)
    constexpr int kChunk = site_chunk<RowT>();
    uint4 *sMask = sSite + (kChunk + kSpare);
    RowT *sRows = reinterpret_cast<RowT *>(sMask + (kChunk + kSpare));
    const int tid = threadIdx.x;
    const int64_t w = (int64_t)blockIdx.x * wpb + tid;
    bool active = w < a.W;

    for (int i = tid; i < nrows * kRandStride; i += wpb) {
        const int r = i / kRandStride, k = i - r * kRandStride;
        const int e = r - kRandGuard;
        sT[i] = (k < 5 && e >= 0 && e <= N) ? a.table[e * 5 + k] : 0u;
    }
    RowT *col = sRows + tid;   // this walker's rows: col[y * wpb]
    unsigned char *cbytes = reinterpret_cast<unsigned char *>(col);
    const int lane = tid & 31;
    const int64_t w0 = w - lane;
    // the whole warp exists and its 32 bytes per site are 16-byte aligned: uniform
    const bool warp_full = LAYOUT == MUCA_LAYOUT_INT8 && w0 + 32 <= a.W && a.W % 16 == 0;
    if (warp_full)
        for (int y = 0; y < L; y += 4) {
            RowT r4[4];
            warp_load_rows<RowT>(reinterpret_cast<const int8_t *>(a.lattice), a.W, w0, L, y, lane, r4);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                col[(y + i) * wpb] = r4[i];
        }
    int32_t e = 0;
    if (active) {
        if (LAYOUT == MUCA_LAYOUT_PACKED) {
            const RowT *g = reinterpret_cast<const RowT *>(a.lattice);
            for (int y = 0; y < L; ++y)
                col[y * wpb] = g[(size_t)y * a.W + w];
        } else if (!warp_full) {
            const int8_t *g = reinterpret_cast<const int8_t *>(a.lattice);
            for (int y = 0; y < L; ++y) {
                RowT r = 0;
#pragma unroll 16
                for (int x = 0; x < L; ++x)   // unrolled: a row's loads are in flight together
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
    constexpr uint32_t kRowBytes = 4u * kRandStride;
    const uint32_t tbase = (uint32_t)__cvta_generic_to_shared(sT) + kRandGuard * kRowBytes;
    uint32_t E = tbase + (uint32_t)e * kRowBytes;   // byte address of the current energy's row
    auto row = [&](uint32_t off) { return *reinterpret_cast<const RowT *>(cbytes + off); };
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const uint32_t wid = a.walker0 + (uint32_t)w;
    const PhiloxKeys pk = make_keys(a.seed, wid, (uint32_t)(a.t0 >> 34));
    const uint64_t tend = a.t0 + a.n;
    const uint32_t rb = (uint32_t)wpb * (uint32_t)sizeof(RowT);   // bytes between rows of a column
    for (uint64_t tc = a.t0; tc < tend; tc += kChunk) {
        const int m = tend - tc < (uint64_t)kChunk ? (int)(tend - tc) : kChunk;
        __syncthreads();   // the previous chunk's sites are consumed (and the setup done)
        for (int j = tid; j < m; j += wpb) {
            const uint64_t t = tc + (uint64_t)j;
            const uint64_t blk = t >> 2;
            const uint4 q = philox4x32_10(make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), kSharedStream, kTagSite),
                                          k0, k1);
            const uint32_t u = (t & 3) == 0 ? q.x : (t & 3) == 1 ? q.y : (t & 3) == 2 ? q.z : q.w;
            const uint32_t i = __umulhi(u, (uint32_t)N);
            const int y = (int)(i / (uint32_t)L), x = (int)i - y * L;
            const int yu = (y == 0) ? L - 1 : y - 1, yd = (y == L - 1) ? 0 : y + 1;
            const int xl = (x == 0) ? L - 1 : x - 1;
            sSite[j] = make_uint4((uint32_t)yu * rb, (uint32_t)y * rb, (uint32_t)yd * rb,
                                  (uint32_t)(x | (y << 24)));
            const unsigned long long bx = 1ull << x, mh = bx | (1ull << xl);
            sMask[j] = make_uint4((uint32_t)bx, (uint32_t)(bx >> 32), (uint32_t)mh, (uint32_t)(mh >> 32));
        }
        if (tid < kSpare) {   // look-ahead records past the chunk's last site: any valid rows
            sSite[m + tid] = make_uint4(0u, 0u, 0u, 0u);
            sMask[m + tid] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        // Groups of four attempts that share a Philox block start at t = 0 mod 4.  A group
        // is clean when none of its sites coincides with or neighbours an earlier site
        // of the group or of the previous group of the chunk: then the neighbour counts
        // read before the previous group's flips are those at its decisions.
        const int j0 = (int)((4u - (uint32_t)(tc & 3)) & 3u);
        const int ngroups = m > j0 ? (m - j0) / 4 : 0;
        for (int gi = tid; gi < ngroups; gi += wpb) {
            const int jb = j0 + 4 * gi;
            const int first = gi > 0 ? jb - 4 : jb;
            bool clean = true;
            for (int a1 = jb; a1 < jb + 4; ++a1) {
                const uint32_t wa = sSite[a1].w;
                const int xa = (int)(wa & 0xFFu), ya = (int)((wa >> 24) & 0x3Fu);
                for (int b1 = first; b1 < a1; ++b1) {
                    const uint32_t wb = sSite[b1].w;
                    int dx = xa - (int)(wb & 0xFFu), dy = ya - (int)((wb >> 24) & 0x3Fu);
                    dx = dx < 0 ? dx + L : dx;
                    dy = dy < 0 ? dy + L : dy;
                    const bool near = (dx == 0 && (dy == 0 || dy == 1 || dy == L - 1)) ||
                                      (dy == 0 && (dx == 1 || dx == L - 1));
                    clean = clean && !near;
                }
            }
            if (clean)
                sSite[jb].x |= kCleanBit;
        }
        __syncthreads();
        if (!active)
            continue;
        auto flip = [&](uint32_t off, RowT bx, bool acc) {
            atomicXor(reinterpret_cast<RowT *>(cbytes + off), acc ? bx : (RowT)0);
        };
        auto count = [&](const uint4 &mk, RowT U, RowT C, RowT D) {
            return site_count<RowT, WIDE>(U, C, D, row_mask<RowT>(mk.x, mk.y), row_mask<RowT>(mk.z, mk.w), L);
        };
        // one attempt on rows read after every earlier flip
        auto single = [&](int jj, uint32_t r) {
            const uint4 rc = sSite[jj], mk = sMask[jj];
            const uint32_t k = count(mk, row(rc.x & ~kCleanBit), row(rc.y), row(rc.z));
            const bool acc = r < lds_word(E + 4u * k);
            flip(rc.y, row_mask<RowT>(mk.x, mk.y), acc);
            E = acc ? E + (2u - k) * kRowBytes : E;
            if (RECORD)
                hist_count(E);
        };
        auto words = [&](uint64_t tt) {
            // the walker's stream of typewriter order (tag 0) with the keys and the products
            // that depend only on the walker and counter word 1 computed once (the launch
            // keeps t >> 34 fixed)
            const uint4 q = philox_walker_c1((uint32_t)(tt >> 2), pk);
            // clamped so that "r < T" also accepts every attempt when T = 0xFFFFFFFF
            return make_uint4(min(q.x, 0xFFFFFFFEu), min(q.y, 0xFFFFFFFEu), min(q.z, 0xFFFFFFFEu),
                              min(q.w, 0xFFFFFFFEu));
        };
        auto word_at = [](const uint4 &q, uint32_t u) { return u == 0 ? q.x : u == 1 ? q.y : u == 2 ? q.z : q.w; };
        int j = 0;
        uint64_t t = tc;
        for (; j < m && (t & 3) != 0; ++j, ++t)   // the head of a launch that starts inside a Philox block
            single(j, word_at(words(t), (uint32_t)(t & 3)));
        if (m - j >= 4) {
            uint4 c0 = sSite[j], c1 = sSite[j + 1], c2 = sSite[j + 2], c3 = sSite[j + 3];
            uint4 b0 = sMask[j], b1 = sMask[j + 1], b2 = sMask[j + 2], b3 = sMask[j + 3];
            uint32_t kc0 = count(b0, row(c0.x & ~kCleanBit), row(c0.y), row(c0.z));
            uint32_t kc1 = count(b1, row(c1.x & ~kCleanBit), row(c1.y), row(c1.z));
            uint32_t kc2 = count(b2, row(c2.x & ~kCleanBit), row(c2.y), row(c2.z));
            uint32_t kc3 = count(b3, row(c3.x & ~kCleanBit), row(c3.y), row(c3.z));
            uint4 qn = words(t);
            for (; m - j >= 4; j += 4, t += 4) {
                const uint4 qg = qn;
                qn = words(t + 4);   // the next group's words, ahead of its decisions
                // the next group's sites and rows, read before this group's flips
                const uint4 n0 = sSite[j + 4], n1 = sSite[j + 5], n2 = sSite[j + 6], n3 = sSite[j + 7];
                const uint4 p0 = sMask[j + 4], p1 = sMask[j + 5], p2 = sMask[j + 6], p3 = sMask[j + 7];
                const RowT u0 = row(n0.x & ~kCleanBit), m0 = row(n0.y), d0r = row(n0.z);
                const RowT u1 = row(n1.x & ~kCleanBit), m1 = row(n1.y), d1r = row(n1.z);
                const RowT u2 = row(n2.x & ~kCleanBit), m2 = row(n2.y), d2r = row(n2.z);
                const RowT u3 = row(n3.x & ~kCleanBit), m3 = row(n3.y), d3r = row(n3.z);
                // the next group's counts; computed inside each branch below, so that the
                // scheduler can place them (and the next group's Philox rounds, started
                // above) between the decisions
                auto next_counts = [&]() {
                    kc0 = count(p0, u0, m0, d0r);
                    kc1 = count(p1, u1, m1, d1r);
                    kc2 = count(p2, u2, m2, d2r);
                    kc3 = count(p3, u3, m3, d3r);
                };
                if (c0.x & kCleanBit) {
                    const uint4 q = qg;
                    // Each decision takes one of two thresholds loaded one attempt
                    // ahead (the previous attempt rejected / flipped); the counts are
                    // known for the whole group.
                    const uint32_t s0 = (2u - kc0) * kRowBytes, s1 = (2u - kc1) * kRowBytes,
                                   s2 = (2u - kc2) * kRowBytes, s3 = (2u - kc3) * kRowBytes;
                    const uint32_t T00 = lds_word(E + 4u * kc0);
                    const uint32_t T10 = lds_word(E + 4u * kc1), T11 = lds_word(E + s0 + 4u * kc1);
                    const bool a0 = q.x < T00;
                    flip(c0.y, row_mask<RowT>(b0.x, b0.y), a0);
                    const uint32_t E1 = a0 ? E + s0 : E;
                    if (RECORD)
                        hist_count(E1);
                    const uint32_t T20 = lds_word(E1 + 4u * kc2), T21 = lds_word(E1 + s1 + 4u * kc2);
                    const bool a1 = q.y < (a0 ? T11 : T10);
                    flip(c1.y, row_mask<RowT>(b1.x, b1.y), a1);
                    const uint32_t E2 = a1 ? E1 + s1 : E1;
                    if (RECORD)
                        hist_count(E2);
                    const uint32_t T30 = lds_word(E2 + 4u * kc3), T31 = lds_word(E2 + s2 + 4u * kc3);
                    const bool a2 = q.z < (a1 ? T21 : T20);
                    flip(c2.y, row_mask<RowT>(b2.x, b2.y), a2);
                    const uint32_t E3 = a2 ? E2 + s2 : E2;
                    if (RECORD)
                        hist_count(E3);
                    const bool a3 = q.w < (a2 ? T31 : T30);
                    flip(c3.y, row_mask<RowT>(b3.x, b3.y), a3);
                    E = a3 ? E3 + s3 : E3;
                    if (RECORD)
                        hist_count(E);
                    next_counts();
                } else {
                    const uint4 q = qg;
                    single(j, q.x);
                    single(j + 1, q.y);
                    single(j + 2, q.z);
                    single(j + 3, q.w);
                    next_counts();
                }
                c0 = n0;
                c1 = n1;
                c2 = n2;
                c3 = n3;
                b0 = p0;
                b1 = p1;
                b2 = p2;
                b3 = p3;
            }
        }
        for (; j < m; ++j, ++t)   // the tail of a launch that ends inside a Philox block
            single(j, word_at(words(t), (uint32_t)(t & 3)));
    }
    if (active) {
        e = (int32_t)((E - tbase) / kRowBytes);
        if (E < tbase || e > N || (E - tbase) % kRowBytes != 0u)   // corrupted energy address
            atomicOr(a.err, kErrEnergyRange);
    }
    __syncthreads();
    if (RECORD)
        for (int i = tid; i <= N; i += wpb) {
            const uint32_t v = sT[(i + kRandGuard) * kRandStride + 5];
            if (v)
                atomicAdd(&a.hist[i], (unsigned long long)v);
        }
    if (warp_full)   // a walker flagged invalid above kept its rows unchanged
        for (int y = 0; y < L; ++y)
            warp_store_row<RowT>(reinterpret_cast<int8_t *>(a.lattice), a.W, w0, L, y, lane, col[y * wpb]);
    if (active) {
        if (LAYOUT == MUCA_LAYOUT_PACKED) {
            RowT *g = reinterpret_cast<RowT *>(a.lattice);
            for (int y = 0; y < L; ++y)
                g[(size_t)y * a.W + w] = col[y * wpb];
        } else if (!warp_full) {
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

template <typename RowT, int LAYOUT, bool RECORD>
cudaError_t launch_random_t(const SweepArgs &a, int wpb, cudaStream_t s)
{
    const size_t smem = random_smem_bytes_t<RowT>(a.L, wpb, RECORD);
    auto kern = a.L == 8 * (int)sizeof(RowT) ? random_sweep_kernel<RowT, LAYOUT, RECORD, true>
                                              : random_sweep_kernel<RowT, LAYOUT, RECORD, false>;
    if (smem > 48 * 1024) {
        const cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess)
            return err;
    }
    const int64_t blocks = (a.W + wpb - 1) / wpb;
    kern<<<(unsigned)blocks, wpb, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename RowT>
cudaError_t launch_random_row(const SweepArgs &a, int wpb, bool record, cudaStream_t s)
{
    if (a.layout == MUCA_LAYOUT_PACKED)
        return record ? launch_random_t<RowT, MUCA_LAYOUT_PACKED, true>(a, wpb, s)
                      : launch_random_t<RowT, MUCA_LAYOUT_PACKED, false>(a, wpb, s);
    return record ? launch_random_t<RowT, MUCA_LAYOUT_INT8, true>(a, wpb, s)
                  : launch_random_t<RowT, MUCA_LAYOUT_INT8, false>(a, wpb, s);
}

}  // namespace

size_t random_smem_bytes(int L, int wpb, bool record)
{
    return L <= 32 ? random_smem_bytes_t<uint32_t>(L, wpb, record)
                   : random_smem_bytes_t<unsigned long long>(L, wpb, record);
}

cudaError_t launch_random_sweep(const SweepArgs &a, int walkers_per_block, bool record, cudaStream_t s)
{
    if (a.n == 0 || a.W == 0)
        return cudaSuccess;
    // the instance's block size (one warp per SM sub-partition where the walker count
    // allows), else the largest block of whole warps whose rows fit next to the table,
    // histogram and site buffer (the walker-to-thread mapping does not affect the result)
    const size_t limit = sweep_smem_limit();
    int wpb = walkers_per_block >= 32 && walkers_per_block <= 256 ? walkers_per_block : 256;
    while (wpb > 32 && random_smem_bytes(a.L, wpb, record) > limit)
        wpb -= 32;
    if (random_smem_bytes(a.L, wpb, record) > limit)
        return cudaErrorInvalidConfiguration;
    // the kernel keeps Philox counter word 1 (t >> 34) fixed within a launch: a range that
    // crosses a multiple of 2^34 runs as two launches
    const uint64_t step = a.t0 >> 34;
    if (((a.t0 + a.n - 1) >> 34) != step) {
        SweepArgs first = a, second = a;
        first.n = ((step + 1) << 34) - a.t0;
        second.t0 = a.t0 + first.n;
        second.n = a.n - first.n;
        cudaError_t err = launch_random_sweep(first, walkers_per_block, record, s);
        return err != cudaSuccess ? err : launch_random_sweep(second, walkers_per_block, record, s);
    }
    if (a.L <= 32)
        return launch_random_row<uint32_t>(a, wpb, record, s);
    return launch_random_row<unsigned long long>(a, wpb, record, s);
}

}  // namespace muca
