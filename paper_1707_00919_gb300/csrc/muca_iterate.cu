// muca_iterate.cu - the weight iteration's host-side steps run as kernels: stop metric
// (min/mean, Eq. (6) Kullback-Leibler, Eq. (A.1) Chebyshev), the recursion of Eq. (4)
// and the threshold table of the next iteration.  Every floating-point step is the one
// the host library takes, in the same order (muca_math.cuh for exp and ln), so the
// weights, tables and metrics are the host's bit for bit.
#include <climits>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/muca.h"
#include "muca_internal.h"
#include "muca_math.cuh"

namespace muca {
namespace {

constexpr int kMetricThreads = 1024;

__device__ __forceinline__ bool accessible_e(int32_t N, int32_t e) { return e != 1 && e != N - 1; }

__global__ void iter_reset_hist_kernel(unsigned long long *hist, int32_t nb, const IterState *st)
{
    if (st->done)
        return;
    for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < nb; e += gridDim.x * blockDim.x)
        hist[e] = 0ull;
}

// Reduction over the block (every thread calls it; identity fills unused lanes).
template <typename T, typename Op>
__device__ T block_reduce(T v, Op op, T *scratch, T identity)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1)
        v = op(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    __syncthreads();
    if (lane == 0)
        scratch[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nwarps ? scratch[lane] : identity;
        for (int o = 16; o > 0; o >>= 1)
            v = op(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
        if (lane == 0)
            scratch[0] = v;
    }
    __syncthreads();
    const T r = scratch[0];
    __syncthreads();
    return r;
}

struct AddU64 {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a + b; }
};
struct MinU64 {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a < b ? a : b; }
};
struct MinI32 {
    __device__ int operator()(int a, int b) const { return a < b ? a : b; }
};
struct MaxI32 {
    __device__ int operator()(int a, int b) const { return a > b ? a : b; }
};
struct MaxF64 {
    __device__ double operator()(double a, double b) const { return a > b ? a : b; }
};

// One block.  Decides whether the histogram just recorded is flat, and whether the
// recursion and table kernels that follow run (see IterState).
__global__ void __launch_bounds__(kMetricThreads) iter_metric_kernel(IterState *st, int32_t N,
                                                                     const unsigned long long *H, int32_t rule,
                                                                     double flat_threshold, int32_t max_iterations)
{
    extern __shared__ double terms[];   // [N+1] Kullback-Leibler terms
    __shared__ unsigned long long s_u64[32];
    __shared__ int s_i32[32];
    __shared__ double s_f64[32];
    if (st->done) {
        if (threadIdx.x == 0)
            st->update = 0u;
        return;
    }
    unsigned long long sum_all = 0ull, sum_acc = 0ull, mn = ULLONG_MAX;
    int lo = INT_MAX, hi = -1;
    for (int32_t e = threadIdx.x; e <= N; e += blockDim.x) {
        const unsigned long long h = H[e];
        sum_all += h;
        if (accessible_e(N, e)) {
            sum_acc += h;
            mn = h < mn ? h : mn;
        }
        if (h) {
            lo = e < lo ? e : lo;
            hi = e > hi ? e : hi;
        }
    }
    sum_all = block_reduce(sum_all, AddU64(), s_u64, 0ull);
    sum_acc = block_reduce(sum_acc, AddU64(), s_u64, 0ull);
    mn = block_reduce(mn, MinU64(), s_u64, ULLONG_MAX);
    lo = block_reduce(lo, MinI32(), s_i32, INT_MAX);
    hi = block_reduce(hi, MaxI32(), s_i32, -1);
    const double total = (double)sum_all;   // the host's running sum of exact counts

    double metric = 0.0;
    if (rule == MUCA_STOP_MIN_MEAN) {
        const double sacc = (double)sum_acc;
        metric = sacc <= 0.0 ? 0.0 : __ddiv_rn((double)mn, __ddiv_rn(sacc, (double)(N - 1)));
    } else if (rule == MUCA_STOP_CHEBYSHEV) {
        if (total <= 0.0) {
            metric = __longlong_as_double(0x7FF0000000000000ll);
        } else {
            const double m = __ddiv_rn(total, (double)(N - 1));
            double d = 0.0;
            for (int32_t e = threadIdx.x; e <= N; e += blockDim.x)
                if (accessible_e(N, e))
                    d = fmax(d, fabs(__dsub_rn(__ddiv_rn((double)H[e], m), 1.0)));
            metric = block_reduce(d, MaxF64(), s_f64, 0.0);
        }
    } else {
        // reference size: accessible energies in the union of the previous range and
        // the range of this histogram, at least 10
        int ulo = st->prev_lo, uhi = st->prev_hi;
        if (hi >= 0) {
            ulo = ulo < 0 ? lo : (lo < ulo ? lo : ulo);
            uhi = uhi < 0 ? hi : (hi > uhi ? hi : uhi);
        }
        int count = 0;
        if (ulo >= 0)
            count = (uhi - ulo + 1) - ((ulo <= 1 && 1 <= uhi) ? 1 : 0) - ((ulo <= N - 1 && N - 1 <= uhi) ? 1 : 0);
        const double q = (double)(count > 10 ? count : 10);
        if (total <= 0.0) {
            metric = __longlong_as_double(0x7FF0000000000000ll);
        } else {
            for (int32_t e = threadIdx.x; e <= N; e += blockDim.x) {
                const unsigned long long h = H[e];
                double t = 0.0;
                if (h) {
                    const double p = __ddiv_rn((double)h, total);
                    t = __dmul_rn(p, fp64::log(__dmul_rn(p, q)));
                }
                terms[e] = t;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double d = 0.0;   // in energy order, as on the host
                for (int32_t e = 0; e <= N; ++e)
                    if (H[e])
                        d = __dadd_rn(d, terms[e]);
                terms[0] = d;
            }
            __syncthreads();
            metric = terms[0];
        }
    }
    if (threadIdx.x == 0) {
        const bool flat = rule == MUCA_STOP_MIN_MEAN ? metric >= flat_threshold : metric < flat_threshold;
        const int32_t n = st->iterations + 1;
        st->iterations = n;
        st->metric = metric;
        if (flat) {
            st->done = 1u;
            st->update = 0u;
        } else {
            st->update = 1u;
            st->prev_lo = hi >= 0 ? lo : -1;
            st->prev_hi = hi >= 0 ? hi : -1;
            st->done = n >= max_iterations ? 2u : 0u;
        }
    }
}

// Eq. (4) in logarithms on visited energies.
__global__ void iter_recursion_kernel(const IterState *st, int32_t N, double *lnW, const unsigned long long *H)
{
    if (!st->update)
        return;
    const int32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e <= N && H[e])
        lnW[e] = __dsub_rn(lnW[e], fp64::log((double)H[e]));
}

// Threshold T[e][k], i = 5 e + k (the rule of muca.h, the arithmetic of the host's
// build_table).
__device__ __forceinline__ uint32_t table_entry(int32_t N, const double *lnW, int32_t i)
{
    const int32_t e = i / 5, k = i - 5 * e, to = e + 2 - k;
    return (to >= 0 && to <= N) ? fp64::threshold(__dsub_rn(lnW[to], lnW[e])) : 0u;
}

// Thresholds of the next iteration, when the metric kernel asked for them.
__global__ void iter_table_kernel(const IterState *st, int32_t N, const double *lnW, uint32_t *T)
{
    if (!st->update)
        return;
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (N + 1) * 5)
        T[i] = table_entry(N, lnW, i);
}

// Thresholds of the given weights (every weight upload of an instance).
__global__ void table_kernel(int32_t N, const double *lnW, uint32_t *T)
{
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (N + 1) * 5)
        T[i] = table_entry(N, lnW, i);
}

}  // namespace

cudaError_t launch_iter_reset_hist(unsigned long long *hist, int32_t nb, const IterState *st, cudaStream_t s)
{
    iter_reset_hist_kernel<<<(nb + 255) / 256, 256, 0, s>>>(hist, nb, st);
    return cudaGetLastError();
}

cudaError_t configure_iter_metric(int32_t N)
{
    const size_t smem = (size_t)(N + 1) * sizeof(double);
    if (smem <= 48 * 1024)
        return cudaSuccess;
    return cudaFuncSetAttribute(iter_metric_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_iter_metric(IterState *st, int32_t N, const unsigned long long *hist, int32_t stop_rule,
                               double flat_threshold, int32_t max_iterations, cudaStream_t s)
{
    const size_t smem = (size_t)(N + 1) * sizeof(double);
    iter_metric_kernel<<<1, kMetricThreads, smem, s>>>(st, N, hist, stop_rule, flat_threshold, max_iterations);
    return cudaGetLastError();
}

cudaError_t launch_iter_recursion(const IterState *st, int32_t N, double *lnW, const unsigned long long *hist,
                                  cudaStream_t s)
{
    iter_recursion_kernel<<<(N + 1 + 127) / 128, 128, 0, s>>>(st, N, lnW, hist);
    return cudaGetLastError();
}

cudaError_t launch_table(int32_t N, const double *lnW, uint32_t *table, cudaStream_t s)
{
    const int32_t n = (N + 1) * 5;
    table_kernel<<<(n + 127) / 128, 128, 0, s>>>(N, lnW, table);
    return cudaGetLastError();
}

cudaError_t launch_iter_table(const IterState *st, int32_t N, const double *lnW, uint32_t *table, cudaStream_t s)
{
    const int32_t n = (N + 1) * 5;
    iter_table_kernel<<<(n + 127) / 128, 128, 0, s>>>(st, N, lnW, table);
    return cudaGetLastError();
}

}  // namespace muca
