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

constexpr int kSiteChunk = 1024;   // attempts whose sites are drawn at once

template <typename RowT>
size_t random_smem_bytes_t(int L, int wpb, bool record)
{
    const size_t nb = (size_t)L * L + 1;
    return align_up((nb * 5 + (record ? nb : 0)) * 4, 16) + (size_t)(kSiteChunk + 1) * 16 + (size_t)L * wpb * sizeof(RowT);
}

template <typename RowT, int LAYOUT, bool RECORD>
__global__ void __launch_bounds__(256) random_sweep_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    if (a.skip && *a.skip)   // an iteration run on the device has finished
        return;
    const int L = a.L;
    const int N = L * L;
    const int nb = N + 1;
    const int wpb = blockDim.x;
    uint32_t *sT = reinterpret_cast<uint32_t *>(smem);
    uint32_t *sH = sT + nb * 5;
    // per site of the chunk: row offsets (row * wpb) of the rows above, at and below,
    // and x | x_left << 8 | x_right << 16; shared by all walkers of the block
    uint4 *sSite = reinterpret_cast<uint4 *>(smem + align_up((size_t)(nb * 5 + (RECORD ? nb : 0)) * 4, 16));
    RowT *sRows = reinterpret_cast<RowT *>(reinterpret_cast<unsigned char *>(sSite) + (size_t)(kSiteChunk + 1) * 16);
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
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const uint32_t wid = a.walker0 + (uint32_t)w;
    const uint64_t tend = a.t0 + a.n;
    for (uint64_t tc = a.t0; tc < tend; tc += kSiteChunk) {
        const int m = tend - tc < (uint64_t)kSiteChunk ? (int)(tend - tc) : kSiteChunk;
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
            const int xl = (x == 0) ? L - 1 : x - 1, xr = (x == L - 1) ? 0 : x + 1;
            sSite[j] = make_uint4((uint32_t)(yu * wpb), (uint32_t)(y * wpb), (uint32_t)(yd * wpb),
                                  (uint32_t)(x | (xl << 8) | (xr << 16)));
        }
        if (tid == 0)   // look-ahead record past the chunk's last site: any valid rows
            sSite[m] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        if (!active)
            continue;
        // The rows of the next attempt's site are loaded before the current attempt
        // decides (its flip is then applied to them where the rows coincide), which
        // takes the row loads off the attempt-to-attempt chain (energy, threshold
        // load, compare).
        uint4 site = sSite[0];
        RowT U = col[site.x], C = col[site.y], D = col[site.z];
        bool pacc = false;
        uint32_t prow = 0xFFFFFFFFu;   // row offset of the previous attempt's site
        RowT pbit = 0;
        int j = 0;
        uint64_t t = tc;
        auto attempt = [&](uint32_t r) {
            if (pacc) {   // the previous attempt flipped a site after these rows were read
                U ^= (site.x == prow) ? pbit : (RowT)0;
                C ^= (site.y == prow) ? pbit : (RowT)0;
                D ^= (site.z == prow) ? pbit : (RowT)0;
            }
            const uint4 nsite = sSite[j + 1];   // j + 1 <= m: the spare record at the end
            const RowT nU = col[nsite.x], nC = col[nsite.y], nD = col[nsite.z];
            const int x = (int)(site.w & 0xFFu), xl = (int)((site.w >> 8) & 0xFFu), xr = (int)(site.w >> 16);
            const uint32_t sx = bit_at(C, x);
            const uint32_t k = (sx ^ bit_at(U, x)) + (sx ^ bit_at(D, x)) + (sx ^ bit_at(C, xl)) + (sx ^ bit_at(C, xr));
            const uint32_t thr = sT[e * 5 + (int)k];
            const bool acc = r < thr || thr == 0xFFFFFFFFu;
            const RowT bx = (RowT)1 << x;
            col[site.y] = C ^ (acc ? bx : (RowT)0);   // unconditional: the row is unchanged on a rejection
            e += acc ? 2 - (int)k : 0;
            if (RECORD)
                asm volatile("red.shared.add.u32 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(sH + e)));
            pacc = acc;
            prow = site.y;
            pbit = bx;
            site = nsite;
            U = nU;
            C = nC;
            D = nD;
            ++j;
            ++t;
        };
        while (j < m) {
            // one Philox call serves the attempts of its block (t & 3 = 0 .. 3)
            const uint64_t blk = t >> 2;
            const uint4 rw = philox4x32_10(make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), wid, kTagMetropolis),
                                           k0, k1);
            const int u0 = (int)(t & 3);
            if (u0 <= 0 && j < m)
                attempt(rw.x);
            if (u0 <= 1 && j < m)
                attempt(rw.y);
            if (u0 <= 2 && j < m)
                attempt(rw.z);
            if (j < m)
                attempt(rw.w);
        }
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

template <typename RowT, int LAYOUT, bool RECORD>
cudaError_t launch_random_t(const SweepArgs &a, int wpb, cudaStream_t s)
{
    const size_t smem = random_smem_bytes_t<RowT>(a.L, wpb, RECORD);
    auto kern = random_sweep_kernel<RowT, LAYOUT, RECORD>;
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
    if (a.L <= 32)
        return launch_random_row<uint32_t>(a, wpb, record, s);
    return launch_random_row<unsigned long long>(a, wpb, record, s);
}

}  // namespace muca
