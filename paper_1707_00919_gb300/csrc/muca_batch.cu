// muca_batch.cu - the batched persistent kernel's thermalization instantiation and the
// launch interface (the recording instantiation is in muca_batch_rec.cu).
#include <algorithm>

#include "muca_batch.cuh"

namespace muca {

cudaError_t configure_batch(size_t smem)
{
    cudaError_t err = configure_batch_t<false>(smem);
    return err != cudaSuccess ? err : configure_batch_record(smem);
}

int batch_resident_blocks(size_t smem)
{
    return std::min(batch_resident_blocks_t<false>(smem), batch_resident_blocks_record(smem));
}

cudaError_t launch_batch(const SweepArgs *insts, const BatchItem *items, int32_t n_items, uint32_t *counter,
                         int grid, size_t smem, bool record, cudaStream_t s)
{
    if (n_items <= 0)
        return cudaSuccess;
    if (record)
        return launch_batch_record(insts, items, n_items, counter, grid, smem, s);
    return launch_batch_t<false>(insts, items, n_items, counter, grid, smem, s);
}

}  // namespace muca
