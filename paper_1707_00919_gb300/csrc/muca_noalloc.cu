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
// Allocation-free variant of the batched kernel.  The instance descriptors, walkers per
// work item and the work list's prefix sums travel by value in the launch parameters
// (NoAllocLaunch, a few KiB); its one piece of scratch, the work counter, lives in the
// file-scope array g_noalloc_scratch below instead of memory the library allocates.
// The work list is derived from the prefix sums, so the caller passes only the
// instances' own buffers.
// ---------------------------------------------------------------------------------
struct NoAllocLaunch {
    SweepArgs descs[kNoAllocMaxInstances];
    int32_t wpbs[kNoAllocMaxInstances];
    int32_t prefix[kNoAllocMaxInstances + 1];   // work items before instance i
    int32_t n;
};
// kernel parameters may take 32 764 bytes (CUDA 12.1 and later)
static_assert(sizeof(NoAllocLaunch) + sizeof(uint32_t *) <= 32764, "launch parameters too large");

template <bool RECORD>
__global__ void __launch_bounds__(256, 1) batch_noalloc_kernel(const __grid_constant__ NoAllocLaunch p,
                                                               uint32_t *counter)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int32_t s_inst;
    __shared__ int64_t s_wbase;
    const int32_t total = p.prefix[p.n];
    for (;;) {
        if (threadIdx.x == 0) {
            const int32_t k = (int32_t)atomicAdd(counter, 1u);
            int32_t i = -1;
            if (k >= 0 && k < total) {
                i = 0;
                while (p.prefix[i + 1] <= k)
                    ++i;
                s_wbase = (int64_t)(k - p.prefix[i]) * p.wpbs[i];
            }
            s_inst = i;
        }
        __syncthreads();
        const int32_t i = s_inst;
        const int64_t wbase = s_wbase;
        __syncthreads();
        if (i < 0)
            break;
        const SweepArgs a = p.descs[i];
        BatchItem it;
        it.inst = i;
        it.wpb = p.wpbs[i];
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

cudaError_t launch_batch_noalloc(const SweepArgs *descs, const int32_t *wpbs, const int32_t *prefix, int32_t n,
                                 size_t smem, bool record, cudaStream_t s)
{
    if (n < 1 || n > kNoAllocMaxInstances)
        return cudaErrorInvalidValue;
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
    NoAllocLaunch p;
    std::memset(&p, 0, sizeof p);
    std::memcpy(p.descs, descs, sizeof(SweepArgs) * (size_t)n);
    std::memcpy(p.wpbs, wpbs, sizeof(int32_t) * (size_t)n);
    std::memcpy(p.prefix, prefix, sizeof(int32_t) * (size_t)(n + 1));
    p.n = n;
    auto kern = record ? batch_noalloc_kernel<true> : batch_noalloc_kernel<false>;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess)
        return err;
    int sms = 0, occ = 0;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess)
        return err;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBatchThreads, smem);
    if (err != cudaSuccess)
        return err;
    if (occ < 1 || sms < 1)
        return cudaErrorInvalidConfiguration;
    // the work counter starts at zero in every call
    uint32_t *counter = static_cast<uint32_t *>(ptr);
    err = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    if (err != cudaSuccess)
        return err;
    kern<<<sms * occ, kBatchThreads, smem, s>>>(p, counter);
    return cudaGetLastError();
}

}  // namespace muca
