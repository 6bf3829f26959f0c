// muca_batch_rec.cu - the batched persistent kernel's recording instantiation.
#include "muca_batch.cuh"

namespace muca {

cudaError_t configure_batch_record(size_t smem) { return configure_batch_t<true>(smem); }

int batch_resident_blocks_record(size_t smem) { return batch_resident_blocks_t<true>(smem); }

cudaError_t launch_batch_record(const SweepArgs *insts, const BatchItem *items, int32_t n_items, uint32_t *counter,
                                int grid, size_t smem, cudaStream_t s)
{
    return launch_batch_t<true>(insts, items, n_items, counter, grid, smem, s);
}

}  // namespace muca
