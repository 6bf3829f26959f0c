// muca_noalloc.cu - allocation-free variant of the batched kernel: its scratch is the
// file-scope device array below, whose device address the host looks up once per
// device; nothing is allocated per call.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "muca_device.cuh"

namespace muca {
namespace {

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
        case 8: batch_item<8, RECORD, true>(a, it, smem); break;
        case 16: batch_item<16, RECORD, true>(a, it, smem); break;
        case 24: batch_item<24, RECORD, true>(a, it, smem); break;
        case 32: batch_item<32, RECORD, true>(a, it, smem); break;
        case 48: batch_item<48, RECORD, true>(a, it, smem); break;
        case 64: batch_item<64, RECORD, true>(a, it, smem); break;
        default: break;
        }
    }
}

}  // namespace

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

}  // namespace muca
