// muca_full.cuh - the whole-sweep kernel for one lattice size; included by
// muca_full_L.cu with MUCA_L defined, so that the six sizes compile in parallel.
#pragma once

#include "muca_device.cuh"

#ifndef MUCA_L
#error "define MUCA_L before including muca_full.cuh"
#endif

namespace muca {
namespace {

template <int L, int LAYOUT, bool RECORD, bool PARTIAL>
__global__ void __launch_bounds__(256, 1) sweep_full_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // launch_sweep splits launches at the steps of counter word 1
    sweep_block<L, RECORD, PARTIAL, false, kTableStride, true>(a, (int64_t)blockIdx.x * blockDim.x, blockDim.x, smem,
                                                               LAYOUT);
}

template <int L, int LAYOUT, bool RECORD, bool PARTIAL>
cudaError_t launch_full_t(const SweepArgs &a, int wpb, cudaStream_t s)
{
    const size_t smem = full_smem_bytes(L, wpb, RECORD);
    auto kern = sweep_full_kernel<L, LAYOUT, RECORD, PARTIAL>;
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

template <int L, bool PARTIAL>
cudaError_t launch_full_p(const SweepArgs &a, int wpb, bool record, cudaStream_t s)
{
    if (a.layout == MUCA_LAYOUT_PACKED)
        return record ? launch_full_t<L, MUCA_LAYOUT_PACKED, true, PARTIAL>(a, wpb, s)
                      : launch_full_t<L, MUCA_LAYOUT_PACKED, false, PARTIAL>(a, wpb, s);
    return record ? launch_full_t<L, MUCA_LAYOUT_INT8, true, PARTIAL>(a, wpb, s)
                  : launch_full_t<L, MUCA_LAYOUT_INT8, false, PARTIAL>(a, wpb, s);
}

// Any attempt range: whole sweeps from a sweep boundary take the kernel without the
// partial-row path, everything else the one with it.
template <int L>
cudaError_t launch_full_l(const SweepArgs &a, int wpb, bool record, cudaStream_t s)
{
    const uint64_t N = (uint64_t)L * (uint64_t)L;
    if (a.t0 % N == 0 && a.n % N == 0 && a.n_therm % N == 0)
        return launch_full_p<L, false>(a, wpb, record, s);
    return launch_full_p<L, true>(a, wpb, record, s);
}

template <int L, int LAYOUT>
int occupancy_full_t(int wpb)
{
    const size_t smem = full_smem_bytes(L, wpb, true);
    auto kern = sweep_full_kernel<L, LAYOUT, true, false>;
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

}  // namespace

#define MUCA_CAT2(a, b) a##b
#define MUCA_CAT(a, b) MUCA_CAT2(a, b)

cudaError_t MUCA_CAT(launch_full_L, MUCA_L)(const SweepArgs &a, int wpb, bool record, cudaStream_t s)
{
    return launch_full_l<MUCA_L>(a, wpb, record, s);
}

int MUCA_CAT(occupancy_full_L, MUCA_L)(int layout, int wpb)
{
    return occupancy_full_l<MUCA_L>(layout, wpb);
}

}  // namespace muca
