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

#include "muca_device.cuh"

namespace muca {
namespace {

bool g_use_full_kernel = true;


// ---------------------------------------------------------------------------------
// Sweep kernel.  Template: row word type (uint32 for L <= 32, uint64 for L <= 64),
// global lattice layout, and whether visited energies are recorded.
// ---------------------------------------------------------------------------------
template <typename RowT, int LAYOUT, bool RECORD>
__global__ void __launch_bounds__(1024) sweep_kernel(const SweepArgs a)
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
    __syncthreads();

    int32_t run_e = e;
    uint32_t run_n = 0;
    if (active) {
        const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
        const uint32_t wid = a.walker0 + (uint32_t)w;
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
// Writes a walker's lattice, given row by row (bit x = spin at x is down), in the
// instance's layout, and its energy index: the number of unsatisfied bonds over two.
template <typename RowT, int LAYOUT, class RowSource>
__device__ __forceinline__ void write_lattice(int32_t L, int64_t W, int64_t w, const RowSource &rows, void *lattice,
                                              int32_t *energy)
{
    const RowT mask = (L == (int)(8 * sizeof(RowT))) ? ~(RowT)0 : (((RowT)1 << L) - 1);
    RowT first = 0, prev = 0;
    int unsat = 0;
    for (int y = 0; y < L; ++y) {
        const RowT r = rows(y);
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

template <typename RowT>
struct InitRows {
    int32_t L;
    uint32_t k0, k1, w;
    __device__ RowT operator()(int y) const
    {
        RowT r = 0;
        for (int x = 0; x < L; x += 4) {
            const uint32_t site = (uint32_t)(y * L + x);
            const uint4 q = philox4x32_10(make_uint4(site >> 2, 0u, w, kTagInit), k0, k1);
            const uint32_t words[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
                r |= (RowT)(words[u] >> 31) << (x + u);
        }
        return r;
    }
};

template <typename RowT>
struct GivenRows {
    int32_t L;
    const int8_t *spins;   // this walker's N spins, +1 / -1
    __device__ RowT operator()(int y) const
    {
        RowT r = 0;
        for (int x = 0; x < L; ++x)
            r |= (RowT)(spins[y * L + x] < 0) << x;
        return r;
    }
};

template <typename RowT, int LAYOUT>
__global__ void init_kernel(int32_t L, int64_t W, uint64_t seed, uint32_t walker0, void *lattice, int32_t *energy)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W)
        return;
    const InitRows<RowT> rows{L, (uint32_t)seed, (uint32_t)(seed >> 32), walker0 + (uint32_t)w};
    write_lattice<RowT, LAYOUT>(L, W, w, rows, lattice, energy);
}

// Lattices given as int8 in[walker][site] (+1 / -1) into the layout, energies recomputed.
template <typename RowT, int LAYOUT>
__global__ void pack_kernel(int32_t L, int64_t W, const int8_t *in, void *lattice, int32_t *energy)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W)
        return;
    const GivenRows<RowT> rows{L, in + (size_t)w * (size_t)(L * L)};
    write_lattice<RowT, LAYOUT>(L, W, w, rows, lattice, energy);
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

// Dispatches a whole-sweep range to the kernel specialised for L; returns
// cudaErrorNotSupported when L has no specialisation.
cudaError_t launch_full(const SweepArgs &a, int wpb, bool record, cudaStream_t s)
{
    switch (a.L) {
    case 8: return launch_full_L8(a, wpb, record, s);
    case 16: return launch_full_L16(a, wpb, record, s);
    case 24: return launch_full_L24(a, wpb, record, s);
    case 32: return launch_full_L32(a, wpb, record, s);
    case 48: return launch_full_L48(a, wpb, record, s);
    case 64: return launch_full_L64(a, wpb, record, s);
    default: return cudaErrorNotSupported;
    }
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

size_t full_smem_bytes(int L, int wpb, bool record, bool guard, int stride)
{
    (void)record;
    const size_t rows = (size_t)L * L + 1 + (guard ? 2 * kTableGuard : 0);
    const size_t per_walker = L <= 32 ? (size_t)L * (L / 8) * 4 : (size_t)L * 8;
    return align_up(rows * (size_t)stride * 4, 16) + per_walker * (size_t)wpb;
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
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;   // nothing fits: callers report it
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
    if (!has_full_kernel(a.L) || !g_use_full_kernel)
        return launch_generic(a, wpb, record, s);
    // the whole-sweep kernels keep Philox counter word 1 (t >> 34) fixed within a launch:
    // a range that crosses a multiple of 2^34 runs as two launches
    const uint64_t step = a.t0 >> 34;
    if (((a.t0 + a.n - 1) >> 34) != step) {
        SweepArgs first = a, second = a;
        first.n = ((step + 1) << 34) - a.t0;
        second.t0 = a.t0 + first.n;
        second.n = a.n - first.n;
        cudaError_t err = launch_full(first, wpb, record, s);
        return err != cudaSuccess ? err : launch_sweep(second, wpb, record, s);
    }
    return launch_full(a, wpb, record, s);
}

cudaError_t launch_sweep_fused(const SweepArgs &a, int wpb, cudaStream_t s)
{
    const uint64_t total = a.n_therm + a.n;
    // one launch of the whole-sweep kernel (its whole-sweep form when both phases are
    // whole sweeps from a sweep boundary, else its any-range form), counter word 1
    // (t >> 34) the same for both phases
    if (a.W > 0 && a.n_therm > 0 && a.n > 0 && has_full_kernel(a.L) && g_use_full_kernel && total > a.n &&
        (a.t0 >> 34) == ((a.t0 + total - 1) >> 34))
        return launch_full(a, wpb, true, s);
    SweepArgs therm = a, rec = a;
    therm.n = a.n_therm;
    therm.n_therm = 0;
    rec.t0 = a.t0 + a.n_therm;
    rec.n_therm = 0;
    const cudaError_t err = launch_sweep(therm, wpb, false, s);
    return err != cudaSuccess ? err : launch_sweep(rec, wpb, true, s);
}

void set_full_kernel_enabled(bool on) { g_use_full_kernel = on; }

cudaError_t launch_init(int32_t L, int32_t layout, int64_t W, uint64_t seed, uint32_t walker0, void *lattice,
                        int32_t *energy,
                        cudaStream_t s)
{
    const int threads = 128;
    const unsigned blocks = (unsigned)((W + threads - 1) / threads);
    if (L <= 32) {
        if (layout == MUCA_LAYOUT_PACKED)
            init_kernel<uint32_t, MUCA_LAYOUT_PACKED><<<blocks, threads, 0, s>>>(L, W, seed, walker0, lattice, energy);
        else
            init_kernel<uint32_t, MUCA_LAYOUT_INT8><<<blocks, threads, 0, s>>>(L, W, seed, walker0, lattice, energy);
    } else {
        if (layout == MUCA_LAYOUT_PACKED)
            init_kernel<unsigned long long, MUCA_LAYOUT_PACKED><<<blocks, threads, 0, s>>>(L, W, seed, walker0, lattice, energy);
        else
            init_kernel<unsigned long long, MUCA_LAYOUT_INT8><<<blocks, threads, 0, s>>>(L, W, seed, walker0, lattice, energy);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack(int32_t L, int32_t layout, int64_t W, const int8_t *in, void *lattice, int32_t *energy,
                        cudaStream_t s)
{
    const int threads = 128;
    const unsigned blocks = (unsigned)((W + threads - 1) / threads);
    if (L <= 32) {
        if (layout == MUCA_LAYOUT_PACKED)
            pack_kernel<uint32_t, MUCA_LAYOUT_PACKED><<<blocks, threads, 0, s>>>(L, W, in, lattice, energy);
        else
            pack_kernel<uint32_t, MUCA_LAYOUT_INT8><<<blocks, threads, 0, s>>>(L, W, in, lattice, energy);
    } else {
        if (layout == MUCA_LAYOUT_PACKED)
            pack_kernel<unsigned long long, MUCA_LAYOUT_PACKED><<<blocks, threads, 0, s>>>(L, W, in, lattice, energy);
        else
            pack_kernel<unsigned long long, MUCA_LAYOUT_INT8><<<blocks, threads, 0, s>>>(L, W, in, lattice, energy);
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
    case 8: return occupancy_full_L8(layout, wpb);
    case 16: return occupancy_full_L16(layout, wpb);
    case 24: return occupancy_full_L24(layout, wpb);
    case 32: return occupancy_full_L32(layout, wpb);
    case 48: return occupancy_full_L48(layout, wpb);
    case 64: return occupancy_full_L64(layout, wpb);
    default: break;
    }
    // the generic kernel: bounded by shared memory and threads
    int dev = 0, smem_sm = 0, thr_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return 0;   // no resident block: callers skip this block size
    const size_t need = sweep_smem_bytes(L, wpb, true) + 1024;
    return (int)std::min((size_t)smem_sm / need, (size_t)(thr_sm / wpb));
}

size_t lattice_bytes(int32_t L, int32_t layout, int64_t W)
{
    if (layout == MUCA_LAYOUT_PACKED)
        return (size_t)L * (size_t)W * (L <= 32 ? 4 : 8);
    return (size_t)L * L * (size_t)W;
}

}  // namespace muca
