// muca_batch.cuh - the batched persistent kernel: one launch advances many instances of
// uneven L and walker count (work list and counter in library memory).  Included by
// muca_batch.cu (thermalization launches) and muca_batch_rec.cu (recording launches), so
// that the two instantiations, each holding the unrolled row bodies of every L, compile
// in parallel.
#pragma once

#include "muca_device.cuh"

namespace muca {
namespace {

// ---------------------------------------------------------------------------------
// Batched persistent kernel: one launch advances many instances (uneven L, walker
// counts, tables and histograms).  The work list holds (instance, first walker, walker
// count) items; each block takes the next item from a global counter, runs it with the
// body of the whole-sweep kernel for that instance's L and layout (with its partial-row
// path where the instance's launch starts or ends inside a sweep), and takes another
// until the list is exhausted.  The counter must be zero at launch.
// ---------------------------------------------------------------------------------
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
        case 8: batch_item<8, RECORD, false, kTableStride, true>(a, it, smem); break;
        case 16: batch_item<16, RECORD, false, kTableStride, true>(a, it, smem); break;
        case 24: batch_item<24, RECORD, false, kTableStride, true>(a, it, smem); break;
        case 32: batch_item<32, RECORD, false, kTableStride, true>(a, it, smem); break;
        case 48: batch_item<48, RECORD, false, kTableStride, true>(a, it, smem); break;
        case 64: batch_item<64, RECORD, false, batch_table_stride(64), true>(a, it, smem); break;
        default: break;
        }
    }
}

template <bool RECORD>
cudaError_t configure_batch_t(size_t smem)
{
    return cudaFuncSetAttribute(batch_kernel<RECORD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <bool RECORD>
int batch_resident_blocks_t(size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<RECORD>, kBatchThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <bool RECORD>
cudaError_t launch_batch_t(const SweepArgs *insts, const BatchItem *items, int32_t n_items, uint32_t *counter,
                           int grid, size_t smem, cudaStream_t s)
{
    batch_kernel<RECORD><<<grid, kBatchThreads, smem, s>>>(insts, items, n_items, counter);
    return cudaGetLastError();
}

}  // namespace
}  // namespace muca
