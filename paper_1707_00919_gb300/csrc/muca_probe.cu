// muca_probe.cu - integer issue-rate measurement for the roofline of the sweep kernels:
// independent streams of one instruction class on every SM sub-partition (16 warps
// each), timed with CUDA events.  Kinds: three-input XOR (the integer ALU pipe),
// 32-bit multiply-add (the multiply pipe), the two alternating, Philox4x32-10 words
// (the generator of the sweep kernels), and the alternating mix with a single warp per
// sub-partition.
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/muca.h"
#include "muca_device.cuh"

namespace muca {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 16;   // independent chains per thread: enough to fill one warp's issue slots

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) probe_kernel(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (KIND == MUCA_PROBE_PHILOX) {
        uint32_t acc = 0;
        for (uint32_t i = 0; i < iters; ++i) {
            const uint4 q = philox4x32_10(make_uint4(i, 0u, tid, 3u), seed, ~seed);
            acc ^= q.x ^ q.y ^ q.z ^ q.w;
        }
        if (acc == 0x12345678u)   // practically never: keeps the work observable
            sink[tid & 1023u] = acc;
        return;
    }
    uint32_t x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = tid * (2 * c + 1) + seed;
#pragma unroll 4
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            const uint32_t o = x[(c + 1) % kChains];
            if (KIND == MUCA_PROBE_XOR || (KIND == MUCA_PROBE_MIXED && (c & 1) == 0)) {
                uint32_t r;
                asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(x[c]), "r"(o), "r"(i));
                x[c] = r;
            } else {
                uint32_t r;
                asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x[c]), "r"(0x9E3779B9u), "r"(o));
                x[c] = r;
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc ^= x[c];
    if (acc == 0x12345678u)
        sink[tid & 1023u] = acc;
}

template <int KIND>
cudaError_t run_probe(int blocks, int threads, uint32_t iters, uint32_t *sink, cudaStream_t s)
{
    probe_kernel<KIND><<<blocks, threads, 0, s>>>(iters, 0x2545F491u, sink);
    return cudaGetLastError();
}

cudaError_t launch_probe(int kind, int blocks, int threads, uint32_t iters, uint32_t *sink, cudaStream_t s)
{
    switch (kind) {
    case MUCA_PROBE_XOR: return run_probe<MUCA_PROBE_XOR>(blocks, threads, iters, sink, s);
    case MUCA_PROBE_MAD: return run_probe<MUCA_PROBE_MAD>(blocks, threads, iters, sink, s);
    case MUCA_PROBE_MIXED:
    case MUCA_PROBE_MIXED_ONE_WARP: return run_probe<MUCA_PROBE_MIXED>(blocks, threads, iters, sink, s);
    default: return run_probe<MUCA_PROBE_PHILOX>(blocks, threads, iters, sink, s);
    }
}

}  // namespace

cudaError_t measure_issue_rate(int kind, double *per_second)
{
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess)
        err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess)
        return err;
    // 2048 threads per SM (16 warps per sub-partition), or 128 (one warp per sub-partition)
    const bool one_warp = kind == MUCA_PROBE_MIXED_ONE_WARP;
    const int threads = one_warp ? 128 : kProbeThreads;
    const int blocks = one_warp ? sms : sms * 8;
    uint32_t *sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    err = cudaMalloc(&sink, 1024 * sizeof(uint32_t));
    if (err == cudaSuccess)
        err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (err == cudaSuccess)
        err = cudaEventCreate(&a);
    if (err == cudaSuccess)
        err = cudaEventCreate(&b);
    // Each pass grows the loop count until a launch takes at least 50 ms.
    uint32_t iters = 1024;
    float ms = 0.0f;
    for (int pass = 0; err == cudaSuccess && pass < 12; ++pass) {
        err = launch_probe(kind, blocks, threads, iters / 4, sink, s);   // warm-up
        if (err == cudaSuccess)
            err = cudaEventRecord(a, s);
        if (err == cudaSuccess)
            err = launch_probe(kind, blocks, threads, iters, sink, s);
        if (err == cudaSuccess)
            err = cudaEventRecord(b, s);
        if (err == cudaSuccess)
            err = cudaEventSynchronize(b);
        if (err == cudaSuccess)
            err = cudaEventElapsedTime(&ms, a, b);
        if (err != cudaSuccess || ms >= 50.0f || iters >= (1u << 30))
            break;
        iters *= 4;
    }
    if (err == cudaSuccess) {
        const double all_threads = (double)blocks * threads;
        // per thread and iteration: kChains instructions, or one Philox call (4 words)
        const double units = kind == MUCA_PROBE_PHILOX ? 4.0 : (double)kChains;
        *per_second = all_threads * (double)iters * units / ((double)ms * 1e-3);
    }
    if (a)
        cudaEventDestroy(a);
    if (b)
        cudaEventDestroy(b);
    if (s)
        cudaStreamDestroy(s);
    if (sink)
        cudaFree(sink);
    return err;
}

}  // namespace muca
