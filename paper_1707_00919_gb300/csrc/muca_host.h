// muca_host.h - shared state and helpers of the host side of the C ABI (muca_api.cu:
// instances, sweeps, state and checkpoints; muca_api_iterate.cu: the weight iteration,
// production and reweighting; muca_api_batch.cu: batches, the allocation-free sweep and
// the request server).  Internal; not installed.
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/muca.h"
#include "muca_internal.h"
#include "muca_math.cuh"

namespace muca_host {

// Error reporting: the message of the last failed call of this host thread.
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t err, const char *what);

// Device allocations go through the caller-set allocator hook when there is one.
struct Allocator {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *ctx = nullptr;
};
extern std::mutex g_alloc_mutex;
extern Allocator g_alloc;
void *device_alloc(const Allocator &a, size_t bytes);
void device_free(const Allocator &a, void *p);

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Largest attempts per walker one recorded launch may take so that a block's 32-bit
// shared histogram bins cannot overflow (each walker adds one count per attempt).
inline uint64_t max_recorded_attempts(int wpb) { return 0xFFFFFFFFull / (uint64_t)std::max(wpb, 256); }

// State of the weight iteration carried from one iteration to the next (Sec. 3):
// extent and range of the energies visited in the previous iteration, whether the whole
// range had been covered, and the previous N_updates.
struct IterSchedule {
    int32_t prev_width = 0, prev_lo = -1, prev_hi = -1, full = 0;
    uint64_t upd_prev = 0;
};

}  // namespace muca_host

struct muca_s {
    int32_t L = 0, N = 0;
    int64_t W = 0;
    uint64_t seed = 0;
    int32_t layout = MUCA_LAYOUT_INT8;
    int32_t wpb = 64;
    muca_host::Allocator alloc;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    void *block = nullptr;           // single device allocation holding all buffers
    void *d_lattice = nullptr;
    int32_t *d_energy = nullptr;
    uint32_t *d_table = nullptr;
    unsigned long long *d_hist = nullptr;
    uint32_t *d_err = nullptr;
    uint32_t *h_table = nullptr;     // pinned staging of the table upload
    unsigned long long *h_hist = nullptr;  // pinned staging of histogram reads
    uint32_t *h_err = nullptr;
    cudaEvent_t table_copied = nullptr;    // last table upload has left h_table
    std::vector<double> lnW;
    void *iter_block = nullptr;      // device iteration state (muca_iterate_device)
    double *d_lnW = nullptr;         // device ln W (in block): the table is built from it
    muca::IterState *d_iter = nullptr;
    muca::IterState *h_iter = nullptr;   // pinned staging of the state
    uint64_t t = 0;                  // attempt counter (tag 0 stream)
    int32_t order = MUCA_ORDER_TYPEWRITER;   // site order of the updates
    uint32_t walker0 = 0;            // global index of walker 0
    muca_histogram_reducer reducer = nullptr;   // sum over the instances of one simulation
    void *reducer_ctx = nullptr;
    int64_t total_walkers = 0;       // walkers of the whole simulation (Eq. (7)), 0 = W
    muca_iteration_observer observer = nullptr;
    void *observer_ctx = nullptr;
    int32_t kl_lo = -1, kl_hi = -1;  // range visited in the previous batched iteration
    muca_host::IterSchedule sched;              // iteration state kept between calls (params.resume)
};

namespace muca_host {

// Instance helpers (muca_api.cu).
// Acceptance thresholds from ln W (Sec. 2.3, integer form): see muca.h.
void build_table(int32_t L, const std::vector<double> &lnW, uint32_t *T);
int upload_table(muca_t h);
int check_device_error(muca_t h);
int sync_and_check(muca_t h);
int run_attempts(muca_t h, uint64_t n, bool record, const uint32_t *skip = nullptr);
// n_therm attempts without recording, then n_record recorded ones (the histogram is not
// zeroed here); one kernel launch where the whole-sweep kernel allows it.
int run_therm_record(muca_t h, uint64_t n_therm, uint64_t n_record, const uint32_t *skip = nullptr);
int read_histogram(muca_t h, std::vector<uint64_t> &H);
// The instance's histogram, or its sum over the instances of the simulation when a reducer is set.
int read_reduced_histogram(muca_t h, std::vector<uint64_t> &H);
int validate(muca_t h);

// Flatness measures and the production estimate (muca_api_iterate.cu, FP64).
inline bool accessible(int32_t N, int32_t e) { return e != 1 && e != N - 1; }
double min_over_mean(int32_t N, const std::vector<uint64_t> &H);
double kullback_leibler(int32_t N, const std::vector<uint64_t> &H, double q);
double chebyshev(int32_t N, const std::vector<uint64_t> &H);
bool visited_range(int32_t N, const std::vector<uint64_t> &H, int32_t &lo, int32_t &hi);
int32_t kl_support(int32_t N, int32_t prev_lo, int32_t prev_hi, const std::vector<uint64_t> &H);
void ln_dos_from_histogram(int32_t N, const std::vector<double> &lnW, const uint64_t *H, double *ln_g);

}  // namespace muca_host

#define MUCA_CUDA(call, what)                              \
    do {                                                   \
        cudaError_t err_ = (call);                         \
        if (err_ != cudaSuccess)                           \
            return muca_host::cuda_fail(err_, (what));     \
    } while (0)
