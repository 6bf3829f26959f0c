// muca_api.cu - host side of the C ABI declared in include/muca.h.
//
// The host owns what the paper does on the host (Sec. 2.2, Sec. 3): the FP64 weight
// recursion of Eq. (4), the flatness tests (min/mean, Eq. 6, Eq. A.1), the update
// schedule of Eq. (7) and the threshold table built from ln W (Sec. 2.3, integer form).
// Everything per attempt runs in the kernels of muca_kernels.cu.
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

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t err, const char *what)
{
    return fail(err == cudaErrorMemoryAllocation ? MUCA_ENOMEM : MUCA_ECUDA, "%s: %s", what,
                cudaGetErrorString(err));
}

#define MUCA_CUDA(call, what)                   \
    do {                                        \
        cudaError_t err_ = (call);              \
        if (err_ != cudaSuccess)                \
            return cuda_fail(err_, (what));     \
    } while (0)

// ---------------------------------------------------------------------------------
// device allocator hook
// ---------------------------------------------------------------------------------
struct Allocator {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *ctx = nullptr;
};
std::mutex g_alloc_mutex;
Allocator g_alloc;

void *device_alloc(const Allocator &a, size_t bytes)
{
    if (a.alloc)
        return a.alloc(bytes, a.ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void device_free(const Allocator &a, void *p)
{
    if (!p)
        return;
    if (a.release)
        a.release(p, a.ctx);
    else
        cudaFree(p);
}

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Largest attempts per walker one recorded launch may take so that a block's 32-bit
// shared histogram bins cannot overflow (each walker adds one count per attempt).
uint64_t max_recorded_attempts(int wpb) { return 0xFFFFFFFFull / (uint64_t)std::max(wpb, 256); }

}  // namespace

// State of the weight iteration carried from one iteration to the next (Sec. 3):
// extent and range of the energies visited in the previous iteration, whether the whole
// range had been covered, and the previous N_updates.
struct IterSchedule {
    int32_t prev_width = 0, prev_lo = -1, prev_hi = -1, full = 0;
    uint64_t upd_prev = 0;
};

struct muca_s {
    int32_t L = 0, N = 0;
    int64_t W = 0;
    uint64_t seed = 0;
    int32_t layout = MUCA_LAYOUT_INT8;
    int32_t wpb = 64;
    Allocator alloc;
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
    void *iter_block = nullptr;      // device ln W and iteration state (muca_iterate_device)
    double *d_lnW = nullptr;
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
    IterSchedule sched;              // iteration state kept between calls (params.resume)
};

namespace {

// Checkpoint files (muca_save / muca_load).
const char kCheckpointMagic[8] = {'M', 'U', 'C', 'A', 'C', 'K', 'P', '2'};
const char kCheckpointMagicV1[8] = {'M', 'U', 'C', 'A', 'C', 'K', 'P', '1'};   // no iteration state

struct FileCloser {
    FILE *f;
    ~FileCloser()
    {
        if (f)
            std::fclose(f);
    }
};

template <typename T>
bool put(FILE *f, const T *v, size_t n)
{
    return std::fwrite(v, sizeof(T), n, f) == n;
}

template <typename T>
bool get(FILE *f, T *v, size_t n)
{
    return std::fread(v, sizeof(T), n, f) == n;
}


// Acceptance thresholds from ln W (Sec. 2.3, integer form): see muca.h.
void build_table(int32_t L, const std::vector<double> &lnW, uint32_t *T)
{
    const int32_t N = L * L;
    for (int32_t e = 0; e <= N; ++e)
        for (int32_t k = 0; k <= 4; ++k) {
            const int32_t to = e + 2 - k;
            uint32_t v = 0u;
            if (to >= 0 && to <= N) {
                v = muca::fp64::threshold(lnW[(size_t)to] - lnW[(size_t)e]);
            }
            T[(size_t)e * 5 + (size_t)k] = v;
        }
}

int upload_table(muca_t h)
{
    MUCA_CUDA(cudaEventSynchronize(h->table_copied), "waiting for the previous table upload");
    build_table(h->L, h->lnW, h->h_table);
    const size_t bytes = (size_t)(h->N + 1) * 5 * sizeof(uint32_t);
    MUCA_CUDA(cudaMemcpyAsync(h->d_table, h->h_table, bytes, cudaMemcpyHostToDevice, h->stream), "table upload");
    MUCA_CUDA(cudaEventRecord(h->table_copied, h->stream), "table upload event");
    return MUCA_OK;
}

int check_device_error(muca_t h)
{
    if (*h->h_err & muca::kErrEnergyRange)
        return fail(MUCA_EDEVICE, "a walker's energy index left the grid [0, N]");
    if (*h->h_err & muca::kErrSyncTimeout)
        return fail(MUCA_EDEVICE, "a bounded wait between warps of a sweep kernel timed out");
    if (*h->h_err)
        return fail(MUCA_EDEVICE, "device error word 0x%x", *h->h_err);
    return MUCA_OK;
}

int sync_and_check(muca_t h)
{
    MUCA_CUDA(cudaMemcpyAsync(h->h_err, h->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream),
              "error word read");
    MUCA_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    return check_device_error(h);
}

int run_attempts(muca_t h, uint64_t n, bool record, const uint32_t *skip = nullptr)
{
    const uint64_t cap = record ? max_recorded_attempts(h->wpb) : UINT64_MAX;
    while (n > 0) {
        const uint64_t chunk = std::min(n, cap);
        muca::SweepArgs a;
        a.L = h->L;
        a.layout = h->layout;
        a.W = h->W;
        a.seed = h->seed;
        a.t0 = h->t;
        a.n = chunk;
        a.lattice = h->d_lattice;
        a.energy = h->d_energy;
        a.table = h->d_table;
        a.hist = h->d_hist;
        a.err = h->d_err;
        a.skip = skip;
        a.walker0 = h->walker0;
        if (h->order == MUCA_ORDER_RANDOM)
            MUCA_CUDA(muca::launch_random_sweep(a, h->wpb, record, h->stream), "random-order sweep launch");
        else
            MUCA_CUDA(muca::launch_sweep(a, h->wpb, record, h->stream), "sweep launch");
        h->t += chunk;
        n -= chunk;
    }
    return MUCA_OK;
}

int read_histogram(muca_t h, std::vector<uint64_t> &H)
{
    const size_t nb = (size_t)h->N + 1;
    MUCA_CUDA(cudaMemcpyAsync(h->h_hist, h->d_hist, nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                              h->stream),
              "histogram read");
    int rc = sync_and_check(h);
    if (rc != MUCA_OK)
        return rc;
    H.assign(h->h_hist, h->h_hist + nb);
    return MUCA_OK;
}

// The histogram as the iteration and the production use it: the instance's own, or its
// sum over all instances of the simulation when a reducer is set.
int read_reduced_histogram(muca_t h, std::vector<uint64_t> &H)
{
    const int rc = read_histogram(h, H);
    if (rc == MUCA_OK && h->reducer)
        h->reducer(H.data(), H.size(), h->reducer_ctx);
    return rc;
}

// ---------------------------------------------------------------------------------
// flatness measures and the update schedule (host, FP64)
// ---------------------------------------------------------------------------------
bool accessible(int32_t N, int32_t e) { return e != 1 && e != N - 1; }

double min_over_mean(int32_t N, const std::vector<uint64_t> &H)
{
    double sum = 0.0;
    uint64_t lo = UINT64_MAX;
    for (int32_t e = 0; e <= N; ++e)
        if (accessible(N, e)) {
            sum += (double)H[(size_t)e];
            lo = std::min(lo, H[(size_t)e]);
        }
    if (sum <= 0.0)
        return 0.0;
    return (double)lo / (sum / (double)(N - 1));
}

double kullback_leibler(int32_t N, const std::vector<uint64_t> &H, double q)
{
    double sum = 0.0;
    for (int32_t e = 0; e <= N; ++e)
        sum += (double)H[(size_t)e];
    if (sum <= 0.0)
        return INFINITY;
    double d = 0.0;
    for (int32_t e = 0; e <= N; ++e)
        if (H[(size_t)e]) {
            const double p = (double)H[(size_t)e] / sum;
            d += p * muca::fp64::log(p * q);
        }
    return d;
}

double chebyshev(int32_t N, const std::vector<uint64_t> &H)
{
    double sum = 0.0;
    for (int32_t e = 0; e <= N; ++e)
        sum += (double)H[(size_t)e];
    if (sum <= 0.0)
        return INFINITY;
    const double m = sum / (double)(N - 1);
    double d = 0.0;
    for (int32_t e = 0; e <= N; ++e)
        if (accessible(N, e))
            d = std::max(d, std::fabs((double)H[(size_t)e] / m - 1.0));
    return d;
}

// Visited range [lo, hi] of a histogram; returns false if H is empty.
bool visited_range(int32_t N, const std::vector<uint64_t> &H, int32_t &lo, int32_t &hi)
{
    lo = -1;
    hi = -1;
    for (int32_t e = 0; e <= N; ++e)
        if (H[(size_t)e]) {
            if (lo < 0)
                lo = e;
            hi = e;
        }
    return lo >= 0;
}

// KL reference size (the Eq. (6) reading): accessible energies in the union of the
// previous iteration's range and the tested histogram's range, at least 10.
int32_t kl_support(int32_t N, int32_t prev_lo, int32_t prev_hi, const std::vector<uint64_t> &H)
{
    int32_t lo = prev_lo, hi = prev_hi, clo, chi;
    if (visited_range(N, H, clo, chi)) {
        lo = lo < 0 ? clo : std::min(lo, clo);
        hi = hi < 0 ? chi : std::max(hi, chi);
    }
    int32_t count = 0;
    if (lo >= 0)
        for (int32_t e = lo; e <= hi; ++e)
            count += accessible(N, e) ? 1 : 0;
    return std::max(count, 10);
}

int validate(muca_t h)
{
    if (!h)
        return fail(MUCA_EINVAL, "NULL instance");
    return MUCA_OK;
}

// Block size for L, layout and W by occupancy: the makespan of a launch is set by the
// most loaded SM sub-partition (one walker per thread, one warp per 32 walkers), so the
// cost of a block size is waves x warps per sub-partition in a full wave; ties go to
// the larger block.
int default_walkers_per_block(int32_t L, int32_t layout, int64_t W)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t limit = muca::sweep_smem_limit();
    int best = 64;
    int64_t best_cost = INT64_MAX;
    for (int wpb = 32; wpb <= 256; wpb += 32) {
        if (std::max(muca::sweep_smem_bytes(L, wpb, true), muca::full_smem_bytes(L, wpb, true)) > limit)
            continue;
        const int occ = muca::resident_blocks(L, layout, wpb);
        if (occ < 1)
            continue;
        const int64_t blocks = (W + wpb - 1) / wpb;
        const int64_t per_wave = (int64_t)sms * occ;
        const int64_t waves = (blocks + per_wave - 1) / per_wave;
        const int64_t first = std::min(blocks, per_wave);
        const int64_t blocks_per_sm = (first + sms - 1) / sms;
        const int64_t warps_per_smsp = (blocks_per_sm * (wpb / 32) + 3) / 4;
        const int64_t cost = waves * warps_per_smsp;
        if (cost < best_cost || (cost == best_cost && wpb > best)) {
            best_cost = cost;
            best = wpb;
        }
    }
    return best;
}

// Measured choice of layout and/or block size: each candidate runs two recorded sweeps
// on a temporary instance of the same size; the fastest is kept.
int tune_options(const muca_options &in, muca_options *out)
{
    *out = in;
    std::vector<int32_t> layouts;
    if (in.layout == MUCA_LAYOUT_AUTO)
        layouts = {MUCA_LAYOUT_INT8, MUCA_LAYOUT_PACKED};
    else
        layouts = {in.layout};
    float best_ms = 1e30f;
    bool found = false;
    for (int32_t lay : layouts) {
        std::vector<int32_t> wpbs;
        if (in.walkers_per_block == MUCA_WPB_TUNE) {
            for (int wpb = 32; wpb <= 256; wpb += 32)
                wpbs.push_back(wpb);
        } else {
            wpbs.push_back(in.walkers_per_block);
        }
        for (int32_t wpb : wpbs) {
            muca_options o = in;
            o.layout = lay;
            o.walkers_per_block = wpb != 0 ? wpb : default_walkers_per_block(in.L, lay, in.n_walkers);
            if (std::max(muca::sweep_smem_bytes(o.L, o.walkers_per_block, true),
                         muca::full_smem_bytes(o.L, o.walkers_per_block, true)) > muca::sweep_smem_limit())
                continue;
            muca_t t = nullptr;
            if (muca_create_ex(&o, &t) != MUCA_OK)
                continue;
            cudaEvent_t a = nullptr, b = nullptr;
            float ms = 1e30f;
            if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess &&
                muca_sweep(t, 1, 1) == MUCA_OK && cudaEventRecord(a, t->stream) == cudaSuccess &&
                muca_sweep(t, 2, 1) == MUCA_OK && cudaEventRecord(b, t->stream) == cudaSuccess &&
                cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) {
                if (ms < best_ms) {
                    best_ms = ms;
                    *out = o;
                    found = true;
                }
            }
            if (a)
                cudaEventDestroy(a);
            if (b)
                cudaEventDestroy(b);
            muca_destroy(t);
        }
    }
    if (!found)
        return fail(MUCA_EINVAL, "no layout / block size fits L = %d", in.L);
    return MUCA_OK;
}

}  // namespace


// ---------------------------------------------------------------------------------
// Batches: many instances advanced by one launch of the batched persistent kernel.
// ---------------------------------------------------------------------------------
struct muca_batch_s {
    std::vector<muca_t> inst;
    std::vector<cudaStream_t> saved_streams;
    std::vector<int32_t> item_wpb;        // walkers per work item, per instance
    Allocator alloc;
    cudaStream_t stream = nullptr;
    void *block = nullptr;
    muca::SweepArgs *d_args = nullptr;    // [2 n]: thermalization launch, recording launch
    muca::BatchItem *d_items = nullptr;   // capacity: all items of all instances
    uint32_t *d_counter = nullptr;        // two work counters
    muca::SweepArgs *h_args = nullptr;    // pinned staging of d_args
    muca::BatchItem *h_items = nullptr;   // pinned staging of d_items
    cudaEvent_t staged = nullptr;         // the last upload of h_args / h_items has completed
    size_t items_capacity = 0;
    int32_t n_items = 0;                  // items of the current member set
    std::vector<int32_t> members;         // instances in the current work list
    size_t smem = 0;
    int grid = 0;
    cudaGraphExec_t exec = nullptr;       // one weight iteration of the current members
    uint64_t g_therm = 0, g_rec = 0;
};

namespace {

bool batchable_L(int32_t L) { return L == 8 || L == 16 || L == 24 || L == 32 || L == 48 || L == 64; }

// Work items of the given member instances (member index j refers to args[j]),
// largest first so that the dynamic schedule ends evenly.
void build_items(muca_batch_t b, const std::vector<int32_t> &members)
{
    std::vector<std::pair<int64_t, muca::BatchItem>> v;
    for (size_t j = 0; j < members.size(); ++j) {
        const muca_t h = b->inst[(size_t)members[j]];
        const int32_t wpb = b->item_wpb[(size_t)members[j]];
        for (int64_t wb = 0; wb < h->W; wb += wpb) {
            muca::BatchItem it;
            it.inst = (int32_t)j;
            it.wpb = wpb;
            it.wbase = wb;
            const int64_t cost = (int64_t)h->N * std::min<int64_t>(wpb, h->W - wb);
            v.emplace_back(cost, it);
        }
    }
    std::stable_sort(v.begin(), v.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
    b->n_items = (int32_t)v.size();
    for (size_t i = 0; i < v.size(); ++i)
        b->h_items[i] = v[i].second;
    b->members = members;
}

muca::SweepArgs make_args(muca_t h, uint64_t t0, uint64_t n)
{
    muca::SweepArgs a;
    a.L = h->L;
    a.layout = h->layout;
    a.W = h->W;
    a.seed = h->seed;
    a.walker0 = h->walker0;
    a.t0 = t0;
    a.n = n;
    a.lattice = h->d_lattice;
    a.energy = h->d_energy;
    a.table = h->d_table;
    a.hist = h->d_hist;
    a.err = h->d_err;
    return a;
}

int stage_wait(muca_batch_t b)
{
    MUCA_CUDA(cudaEventSynchronize(b->staged), "waiting for the previous batch upload");
    return MUCA_OK;
}

int upload_items(muca_batch_t b)
{
    MUCA_CUDA(cudaMemcpyAsync(b->d_items, b->h_items, sizeof(muca::BatchItem) * (size_t)b->n_items,
                              cudaMemcpyHostToDevice, b->stream),
              "batch work list upload");
    MUCA_CUDA(cudaEventRecord(b->staged, b->stream), "batch upload event");
    return MUCA_OK;
}

int check_members(muca_batch_t b)
{
    for (int32_t j : b->members) {
        int rc = check_device_error(b->inst[(size_t)j]);
        if (rc)
            return rc;
    }
    return MUCA_OK;
}

// Captures one weight iteration of the current members: table uploads, the launch
// descriptors, thermalization launch, zeroed histograms, recording launch, histogram
// and error-word reads.  The host refills the pinned buffers before every replay.
int build_graph(muca_batch_t b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    const size_t nm = b->members.size();
    cudaGraph_t g = nullptr;
    MUCA_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
    cudaError_t err = cudaSuccess;
    for (int32_t j : b->members) {
        const muca_t h = b->inst[(size_t)j];
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(h->d_table, h->h_table, sizeof(uint32_t) * 5 * ((size_t)h->N + 1),
                                  cudaMemcpyHostToDevice, b->stream);
    }
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(b->d_args, b->h_args, sizeof(muca::SweepArgs) * 2 * nm, cudaMemcpyHostToDevice,
                              b->stream);
    if (err == cudaSuccess)
        err = cudaMemsetAsync(b->d_counter, 0, 2 * sizeof(uint32_t), b->stream);
    if (err == cudaSuccess)
        err = muca::launch_batch(b->d_args, b->d_items, b->n_items, b->d_counter, b->grid, b->smem, false, b->stream);
    for (int32_t j : b->members) {
        const muca_t h = b->inst[(size_t)j];
        if (err == cudaSuccess)
            err = cudaMemsetAsync(h->d_hist, 0, sizeof(unsigned long long) * ((size_t)h->N + 1), b->stream);
    }
    if (err == cudaSuccess)
        err = muca::launch_batch(b->d_args + nm, b->d_items, b->n_items, b->d_counter + 1, b->grid, b->smem, true,
                                 b->stream);
    for (int32_t j : b->members) {
        const muca_t h = b->inst[(size_t)j];
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(h->h_hist, h->d_hist, sizeof(unsigned long long) * ((size_t)h->N + 1),
                                  cudaMemcpyDeviceToHost, b->stream);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(h->h_err, h->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream);
    }
    cudaError_t end = cudaStreamEndCapture(b->stream, &g);
    if (err == cudaSuccess)
        err = end;
    if (err == cudaSuccess)
        err = cudaGraphInstantiate(&b->exec, g, 0);
    if (g)
        cudaGraphDestroy(g);
    if (err != cudaSuccess) {
        b->exec = nullptr;
        return cuda_fail(err, "batch iteration graph");
    }
    return MUCA_OK;
}


int check_iteration_params(const muca_params &p, muca_t h)
{
    if (p.schedule != MUCA_SCHEDULE_SWEEPS)
        return fail(MUCA_EINVAL, "batched iteration supports the fixed-sweep schedule");
    if (p.stop_rule < MUCA_STOP_MIN_MEAN || p.stop_rule > MUCA_STOP_CHEBYSHEV || p.max_iterations < 1)
        return fail(MUCA_EINVAL, "bad stop rule or max_iterations");
    if (p.resume != 0 && p.resume != 1)
        return fail(MUCA_EINVAL, "resume must be 0 or 1");
    if (p.sweeps_per_iter * (uint64_t)h->N > 0xFFFFFFFFull / 256ull)
        return fail(MUCA_EINVAL, "sweeps_per_iter too large for one recording launch");
    if (h->t % (uint64_t)h->N != 0)
        return fail(MUCA_EINVAL, "batched launches need every member at a sweep boundary");
    return MUCA_OK;
}

// One weight iteration of the members `active` (indices into b->inst): member j
// thermalizes therm[j] sweeps and records rec[j] sweeps, all members in one replay of
// the iteration graph.  Afterwards each member's histogram is in its pinned buffer and
// its attempt counter is advanced.
int batch_run_iteration(muca_batch_t b, const std::vector<int32_t> &active, const std::vector<uint64_t> &therm,
                        const std::vector<uint64_t> &rec)
{
    int rc = stage_wait(b);
    if (rc)
        return rc;
    if (active != b->members || !b->exec) {
        MUCA_CUDA(cudaStreamSynchronize(b->stream), "batch synchronize");
        build_items(b, active);
        rc = upload_items(b);
        if (rc)
            return rc;
        MUCA_CUDA(cudaStreamSynchronize(b->stream), "batch synchronize");
        rc = build_graph(b);
        if (rc)
            return rc;
    }
    const size_t nm = active.size();
    for (size_t j = 0; j < nm; ++j) {
        muca_t h = b->inst[(size_t)active[j]];
        build_table(h->L, h->lnW, h->h_table);
        const uint64_t nt = therm[j] * (uint64_t)h->N, nr = rec[j] * (uint64_t)h->N;
        b->h_args[j] = make_args(h, h->t, nt);
        b->h_args[nm + j] = make_args(h, h->t + nt, nr);
        h->t += nt + nr;
    }
    MUCA_CUDA(cudaGraphLaunch(b->exec, b->stream), "batch iteration launch");
    MUCA_CUDA(cudaStreamSynchronize(b->stream), "batch synchronize");
    return check_members(b);
}

// Host half of one iteration for a member whose histogram is in its pinned buffer:
// stop metric, flatness, Eq. (4) recursion.  Returns true when the member is finished
// (flat, or max_iterations reached).
bool member_update(muca_t h, const muca_params &p, muca_stats &s)
{
    const int32_t N = h->N;
    std::vector<uint64_t> H(h->h_hist, h->h_hist + N + 1);
    s.iterations += 1;
    s.attempts_per_walker += (p.therm_sweeps + p.sweeps_per_iter) * (uint64_t)N;
    double metric;
    if (p.stop_rule == MUCA_STOP_MIN_MEAN)
        metric = min_over_mean(N, H);
    else if (p.stop_rule == MUCA_STOP_KL)
        metric = kullback_leibler(N, H, (double)kl_support(N, h->kl_lo, h->kl_hi, H));
    else
        metric = chebyshev(N, H);
    s.last_metric = metric;
    const bool flat = p.stop_rule == MUCA_STOP_MIN_MEAN ? metric >= p.flat_threshold : metric < p.flat_threshold;
    if (flat) {
        s.converged = 1;
        return true;
    }
    for (int32_t e = 0; e <= N; ++e)
        if (H[(size_t)e])
            h->lnW[(size_t)e] -= muca::fp64::log((double)H[(size_t)e]);
    if (!visited_range(N, H, h->kl_lo, h->kl_hi))
        h->kl_lo = h->kl_hi = -1;
    h->sched.prev_lo = h->kl_lo;
    h->sched.prev_hi = h->kl_hi;
    h->sched.prev_width = h->kl_lo >= 0 ? h->kl_hi - h->kl_lo + 1 : 0;
    h->sched.upd_prev = p.sweeps_per_iter * (uint64_t)N;
    return s.iterations >= p.max_iterations;
}

size_t instance_device_bytes(int32_t L, int32_t layout, int64_t W)
{
    const size_t nb = (size_t)L * L + 1;
    return align256(muca::lattice_bytes(L, layout == MUCA_LAYOUT_PACKED ? MUCA_LAYOUT_PACKED : MUCA_LAYOUT_INT8, W)) +
           align256((size_t)W * sizeof(int32_t)) + align256(nb * 5 * sizeof(uint32_t)) +
           align256(nb * sizeof(unsigned long long)) + 256;
}

// ln g(e) = ln H(e) - ln W(e) on visited energies, shifted so that sum_e exp(ln g) = 2^N
// (Sec. 3.3); -inf elsewhere.
void ln_dos_from_histogram(int32_t N, const std::vector<double> &lnW, const uint64_t *H, double *ln_g)
{
    double top = -INFINITY;
    for (int32_t e = 0; e <= N; ++e) {
        ln_g[e] = H[e] ? std::log((double)H[e]) - lnW[(size_t)e] : -INFINITY;
        top = std::max(top, ln_g[e]);
    }
    if (top == -INFINITY)
        return;
    double s = 0.0;
    for (int32_t e = 0; e <= N; ++e)
        if (H[e])
            s += std::exp(ln_g[e] - top);
    const double shift = (double)N * std::log(2.0) - (top + std::log(s));
    for (int32_t e = 0; e <= N; ++e)
        if (H[e])
            ln_g[e] += shift;
}
}  // namespace

extern "C" {

int muca_default_params(muca_params *p)
{
    if (!p)
        return fail(MUCA_EINVAL, "NULL params");
    std::memset(p, 0, sizeof *p);
    p->schedule = MUCA_SCHEDULE_SWEEPS;
    p->stop_rule = MUCA_STOP_MIN_MEAN;
    p->flat_threshold = 0.8;
    p->therm_sweeps = 31;
    p->sweeps_per_iter = 100;
    p->f_therm = 30.0;
    p->z = 2.25;
    p->factor = 6.0;
    p->growth = 1.1;
    p->max_iterations = 1000;
    p->deadline_s = 0.0;
    return MUCA_OK;
}

int muca_set_allocator(void *(*alloc)(size_t, void *), void (*release)(void *, void *), void *ctx)
{
    if ((alloc == nullptr) != (release == nullptr))
        return fail(MUCA_EINVAL, "allocator and release must be given together");
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.ctx = ctx;
    return MUCA_OK;
}

int muca_create(int32_t L, int64_t n_walkers, uint64_t seed, muca_t *out)
{
    muca_options o;
    std::memset(&o, 0, sizeof o);
    o.L = L;
    o.n_walkers = n_walkers;
    o.seed = seed;
    o.layout = MUCA_LAYOUT_INT8;
    return muca_create_ex(&o, out);
}

int muca_optimal_walkers(int32_t L, int32_t layout, int64_t *n_walkers, int32_t *walkers_per_block)
{
    if (!n_walkers)
        return fail(MUCA_EINVAL, "NULL argument");
    if (L < 4 || L > 64 || L % 4 != 0)
        return fail(MUCA_EINVAL, "L = %d: must be a multiple of 4 in [4, 64]", L);
    if (layout != MUCA_LAYOUT_INT8 && layout != MUCA_LAYOUT_PACKED)
        return fail(MUCA_EINVAL, "layout %d: must be MUCA_LAYOUT_INT8 or MUCA_LAYOUT_PACKED", layout);
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess)
        err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess)
        return cuda_fail(err, "device query");
    const size_t limit = muca::sweep_smem_limit();
    int64_t best = 0;
    int32_t best_wpb = 0;
    for (int wpb = 32; wpb <= 256; wpb += 32) {
        if (std::max(muca::sweep_smem_bytes(L, wpb, true), muca::full_smem_bytes(L, wpb, true)) > limit)
            continue;
        const int64_t per_sm = (int64_t)muca::resident_blocks(L, layout, wpb) * wpb;
        if (per_sm > best || (per_sm == best && per_sm > 0)) {
            best = per_sm;
            best_wpb = wpb;
        }
    }
    if (best == 0)
        return fail(MUCA_EINVAL, "no block size fits L = %d", L);
    *n_walkers = best * sms;
    if (walkers_per_block)
        *walkers_per_block = best_wpb;
    return MUCA_OK;
}

int muca_create_ex(const muca_options *opt, muca_t *out)
{
    if (!opt || !out)
        return fail(MUCA_EINVAL, "NULL argument");
    *out = nullptr;
    const int32_t L = opt->L;
    if (L < 4 || L > 64 || L % 4 != 0)
        return fail(MUCA_EINVAL, "L = %d: must be a multiple of 4 in [4, 64]", L);
    if (opt->n_walkers == MUCA_WALKERS_OPTIMAL) {
        muca_options o = *opt;
        int32_t wpb = 0;
        const int rc = muca_optimal_walkers(L, opt->layout == MUCA_LAYOUT_PACKED ? MUCA_LAYOUT_PACKED : MUCA_LAYOUT_INT8,
                                            &o.n_walkers, &wpb);
        if (rc != MUCA_OK)
            return rc;
        if (o.walkers_per_block == 0)
            o.walkers_per_block = wpb;
        return muca_create_ex(&o, out);
    }
    if (opt->n_walkers < 1 || opt->n_walkers > INT32_MAX)
        return fail(MUCA_EINVAL, "n_walkers = %lld out of range", (long long)opt->n_walkers);
    if (opt->first_walker < 0 || opt->first_walker > (int64_t)INT32_MAX - opt->n_walkers)
        return fail(MUCA_EINVAL, "first_walker = %lld: the walker indices must stay below 2^31",
                    (long long)opt->first_walker);
    if (opt->layout != MUCA_LAYOUT_INT8 && opt->layout != MUCA_LAYOUT_PACKED && opt->layout != MUCA_LAYOUT_AUTO)
        return fail(MUCA_EINVAL, "unknown layout %d", opt->layout);
    if (opt->layout == MUCA_LAYOUT_AUTO || opt->walkers_per_block == MUCA_WPB_TUNE) {
        muca_options tuned;
        int rc = tune_options(*opt, &tuned);
        if (rc != MUCA_OK)
            return rc;
        return muca_create_ex(&tuned, out);
    }
    int32_t wpb = opt->walkers_per_block;
    if (wpb == 0)
        wpb = default_walkers_per_block(L, opt->layout, opt->n_walkers);
    if (wpb < 32 || wpb > 256 || wpb % 32 != 0)
        return fail(MUCA_EINVAL, "walkers_per_block = %d: must be a multiple of 32 in [32, 256]", wpb);
    const size_t smem = std::max(muca::sweep_smem_bytes(L, wpb, true), muca::full_smem_bytes(L, wpb, true));
    if (smem > muca::sweep_smem_limit())
        return fail(MUCA_EINVAL, "L = %d with %d walkers per block needs %zu bytes of shared memory", L, wpb,
                    smem);

    muca_s *h = new (std::nothrow) muca_s;
    if (!h)
        return fail(MUCA_ENOMEM, "host allocation failed");
    h->L = L;
    h->N = L * L;
    h->W = opt->n_walkers;
    h->seed = opt->seed;
    h->walker0 = (uint32_t)opt->first_walker;
    h->layout = opt->layout;
    h->wpb = wpb;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        h->alloc = g_alloc;
    }
    const size_t nb = (size_t)h->N + 1;
    const size_t off_lat = 0;
    const size_t off_e = off_lat + align256(muca::lattice_bytes(L, h->layout, h->W));
    const size_t off_T = off_e + align256((size_t)h->W * sizeof(int32_t));
    const size_t off_H = off_T + align256(nb * 5 * sizeof(uint32_t));
    const size_t off_err = off_H + align256(nb * sizeof(unsigned long long));
    const size_t total = off_err + 256;

    auto cleanup = [&](int rc) {
        muca_destroy(h);
        return rc;
    };
    cudaError_t err = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
    if (err != cudaSuccess)
        return cleanup(cuda_fail(err, "stream create"));
    h->stream = h->own_stream;
    err = cudaEventCreateWithFlags(&h->table_copied, cudaEventDisableTiming);
    if (err != cudaSuccess)
        return cleanup(cuda_fail(err, "event create"));
    h->block = device_alloc(h->alloc, total);
    if (!h->block)
        return cleanup(fail(MUCA_ENOMEM, "device allocation of %zu bytes failed", total));
    char *base = static_cast<char *>(h->block);
    h->d_lattice = base + off_lat;
    h->d_energy = reinterpret_cast<int32_t *>(base + off_e);
    h->d_table = reinterpret_cast<uint32_t *>(base + off_T);
    h->d_hist = reinterpret_cast<unsigned long long *>(base + off_H);
    h->d_err = reinterpret_cast<uint32_t *>(base + off_err);
    err = cudaMallocHost(reinterpret_cast<void **>(&h->h_table), nb * 5 * sizeof(uint32_t));
    if (err != cudaSuccess)
        return cleanup(cuda_fail(err, "pinned table buffer"));
    err = cudaMallocHost(reinterpret_cast<void **>(&h->h_hist), nb * sizeof(unsigned long long));
    if (err != cudaSuccess)
        return cleanup(cuda_fail(err, "pinned histogram buffer"));
    err = cudaMallocHost(reinterpret_cast<void **>(&h->h_err), sizeof(uint32_t));
    if (err != cudaSuccess)
        return cleanup(cuda_fail(err, "pinned error word"));
    *h->h_err = 0;
    h->lnW.assign(nb, 0.0);
    err = cudaMemsetAsync(h->d_hist, 0, nb * sizeof(unsigned long long), h->stream);
    if (err == cudaSuccess)
        err = cudaMemsetAsync(h->d_err, 0, sizeof(uint32_t), h->stream);
    if (err != cudaSuccess)
        return cleanup(cuda_fail(err, "memset"));
    err = muca::launch_init(L, h->layout, h->W, h->seed, h->walker0, h->d_lattice, h->d_energy, h->stream);
    if (err != cudaSuccess)
        return cleanup(cuda_fail(err, "init launch"));
    int rc = upload_table(h);
    if (rc != MUCA_OK)
        return cleanup(rc);
    rc = sync_and_check(h);
    if (rc != MUCA_OK)
        return cleanup(rc);
    *out = h;
    return MUCA_OK;
}

int muca_destroy(muca_t h)
{
    if (!h)
        return MUCA_OK;
    if (h->stream)
        cudaStreamSynchronize(h->stream);
    device_free(h->alloc, h->block);
    device_free(h->alloc, h->iter_block);
    if (h->h_iter)
        cudaFreeHost(h->h_iter);
    if (h->h_table)
        cudaFreeHost(h->h_table);
    if (h->h_hist)
        cudaFreeHost(h->h_hist);
    if (h->h_err)
        cudaFreeHost(h->h_err);
    if (h->table_copied)
        cudaEventDestroy(h->table_copied);
    if (h->own_stream)
        cudaStreamDestroy(h->own_stream);
    delete h;
    return MUCA_OK;
}

int muca_measure_issue_rate(int32_t kind, double *per_second)
{
    if (!per_second)
        return fail(MUCA_EINVAL, "NULL argument");
    if (kind < MUCA_PROBE_XOR || kind > MUCA_PROBE_PHILOX)
        return fail(MUCA_EINVAL, "unknown probe kind %d", kind);
    MUCA_CUDA(muca::measure_issue_rate(kind, per_second), "issue-rate probe");
    return MUCA_OK;
}

int muca_set_histogram_reducer(muca_t h, muca_histogram_reducer fn, void *ctx, int64_t total_walkers)
{
    int rc = validate(h);
    if (rc)
        return rc;
    if (fn && total_walkers < h->W)
        return fail(MUCA_EINVAL, "total_walkers = %lld is below this instance's %lld walkers",
                    (long long)total_walkers, (long long)h->W);
    h->reducer = fn;
    h->reducer_ctx = fn ? ctx : nullptr;
    h->total_walkers = fn ? total_walkers : 0;
    return MUCA_OK;
}

int muca_set_iteration_observer(muca_t h, muca_iteration_observer fn, void *ctx)
{
    int rc = validate(h);
    if (rc)
        return rc;
    h->observer = fn;
    h->observer_ctx = fn ? ctx : nullptr;
    return MUCA_OK;
}

int muca_set_site_order(muca_t h, int32_t order)
{
    int rc = validate(h);
    if (rc)
        return rc;
    if (order != MUCA_ORDER_TYPEWRITER && order != MUCA_ORDER_RANDOM)
        return fail(MUCA_EINVAL, "unknown site order %d", order);
    h->order = order;
    return MUCA_OK;
}

int muca_get_site_order(muca_t h, int32_t *order)
{
    int rc = validate(h);
    if (rc)
        return rc;
    if (!order)
        return fail(MUCA_EINVAL, "NULL argument");
    *order = h->order;
    return MUCA_OK;
}

int muca_set_stream(muca_t h, void *cuda_stream)
{
    int rc = validate(h);
    if (rc)
        return rc;
    MUCA_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    h->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : h->own_stream;
    return MUCA_OK;
}

int muca_set_weights(muca_t h, const double *lnW, size_t n_bins)
{
    int rc = validate(h);
    if (rc)
        return rc;
    if (!lnW || n_bins != (size_t)h->N + 1)
        return fail(MUCA_EINVAL, "weights need %d bins", h->N + 1);
    for (size_t i = 0; i < n_bins; ++i)
        if (!std::isfinite(lnW[i]))
            return fail(MUCA_EINVAL, "ln W[%zu] is not finite", i);
    h->lnW.assign(lnW, lnW + n_bins);
    return upload_table(h);
}

int muca_get_weights(muca_t h, double *lnW_out, size_t n_bins)
{
    int rc = validate(h);
    if (rc)
        return rc;
    if (!lnW_out || n_bins != (size_t)h->N + 1)
        return fail(MUCA_EINVAL, "weights need %d bins", h->N + 1);
    std::copy(h->lnW.begin(), h->lnW.end(), lnW_out);
    return MUCA_OK;
}

int muca_get_table(muca_t h, uint32_t *T_out, size_t n)
{
    int rc = validate(h);
    if (rc)
        return rc;
    if (!T_out || n != ((size_t)h->N + 1) * 5)
        return fail(MUCA_EINVAL, "table has %d entries", (h->N + 1) * 5);
    MUCA_CUDA(cudaMemcpyAsync(T_out, h->d_table, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream),
              "table read");
    MUCA_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    return MUCA_OK;
}

int muca_sweep(muca_t h, uint64_t n_sweeps, int record)
{
    int rc = validate(h);
    if (rc)
        return rc;
    if (n_sweeps > UINT64_MAX / (uint64_t)h->N)
        return fail(MUCA_EINVAL, "n_sweeps too large");
    return run_attempts(h, n_sweeps * (uint64_t)h->N, record != 0);
}

int muca_attempts(muca_t h, uint64_t n_attempts, int record)
{
    int rc = validate(h);
    if (rc)
        return rc;
    return run_attempts(h, n_attempts, record != 0);
}

int muca_get_histogram(muca_t h, uint64_t *out, size_t n_bins)
{
    int rc = validate(h);
    if (rc)
        return rc;
    if (!out || n_bins != (size_t)h->N + 1)
        return fail(MUCA_EINVAL, "histogram has %d bins", h->N + 1);
    std::vector<uint64_t> H;
    rc = read_histogram(h, H);
    if (rc)
        return rc;
    std::copy(H.begin(), H.end(), out);
    return MUCA_OK;
}

int muca_reset_histogram(muca_t h)
{
    int rc = validate(h);
    if (rc)
        return rc;
    MUCA_CUDA(cudaMemsetAsync(h->d_hist, 0, ((size_t)h->N + 1) * sizeof(unsigned long long), h->stream),
              "histogram reset");
    return MUCA_OK;
}

int muca_iterate_until_flat(muca_t h, const muca_params *p_in, muca_stats *stats)
{
    int rc = validate(h);
    if (rc)
        return rc;
    muca_params p;
    if (p_in)
        p = *p_in;
    else
        muca_default_params(&p);
    if (p.schedule != MUCA_SCHEDULE_SWEEPS && p.schedule != MUCA_SCHEDULE_PAPER)
        return fail(MUCA_EINVAL, "unknown schedule %d", p.schedule);
    if (p.stop_rule < MUCA_STOP_MIN_MEAN || p.stop_rule > MUCA_STOP_CHEBYSHEV)
        return fail(MUCA_EINVAL, "unknown stop rule %d", p.stop_rule);
    if (p.max_iterations < 1)
        return fail(MUCA_EINVAL, "max_iterations must be positive");
    if (p.resume != 0 && p.resume != 1)
        return fail(MUCA_EINVAL, "resume must be 0 or 1");
    const auto start = std::chrono::steady_clock::now();
    const int32_t N = h->N;
    std::vector<uint64_t> H;
    const IterSchedule s0 = p.resume ? h->sched : IterSchedule{};
    int32_t prev_width = s0.prev_width, prev_lo = s0.prev_lo, prev_hi = s0.prev_hi;
    bool full = s0.full != 0;
    uint64_t upd_prev = s0.upd_prev, spent = 0;
    int32_t n = 0;
    bool flat = false, timed_out = false;
    double metric = 0.0;
    while (n < p.max_iterations) {
        uint64_t n_therm, n_upd;
        if (p.schedule == MUCA_SCHEDULE_SWEEPS) {
            n_therm = p.therm_sweeps * (uint64_t)N;
            n_upd = p.sweeps_per_iter * (uint64_t)N;
        } else {
            // Sec. 3: w = max(w', 10) with w' the extent covered in the previous
            // iteration; N_therm = f_therm w; Eq. (7) until the whole range was covered,
            // then growth by 1.1 per iteration; both truncated and increased by one.
            const int32_t w = std::max(prev_width, 10);
            n_therm = (uint64_t)(p.f_therm * (double)w);
            if (full) {
                n_upd = (uint64_t)std::floor(p.growth * (double)upd_prev) + 1u;
            } else {
                const double walkers = (double)(h->total_walkers > 0 ? h->total_walkers : h->W);
                n_upd = (uint64_t)std::floor(p.factor * std::pow((double)w, p.z) / walkers) + 1u;
                full = prev_width == N + 1;
            }
        }
        rc = upload_table(h);
        if (rc)
            return rc;
        rc = run_attempts(h, n_therm, false);
        if (rc)
            return rc;
        rc = muca_reset_histogram(h);
        if (rc)
            return rc;
        rc = run_attempts(h, n_upd, true);
        if (rc)
            return rc;
        rc = read_reduced_histogram(h, H);
        if (rc)
            return rc;
        spent += n_therm + n_upd;
        ++n;
        if (p.stop_rule == MUCA_STOP_MIN_MEAN)
            metric = min_over_mean(N, H);
        else if (p.stop_rule == MUCA_STOP_KL)
            metric = kullback_leibler(N, H, (double)kl_support(N, prev_lo, prev_hi, H));
        else
            metric = chebyshev(N, H);
        flat = p.stop_rule == MUCA_STOP_MIN_MEAN ? metric >= p.flat_threshold : metric < p.flat_threshold;
        if (h->observer)
            h->observer(n, H.data(), H.size(), metric, n_therm, n_upd, h->observer_ctx);
        if (flat)
            break;
        // Eq. (4) in logarithms: ln W <- ln W - ln H on visited energies.
        for (int32_t e = 0; e <= N; ++e)
            if (H[(size_t)e])
                h->lnW[(size_t)e] -= muca::fp64::log((double)H[(size_t)e]);
        int32_t lo, hi;
        if (visited_range(N, H, lo, hi)) {
            prev_width = hi - lo + 1;
            prev_lo = lo;
            prev_hi = hi;
        } else {
            prev_width = 0;
            prev_lo = prev_hi = -1;
        }
        upd_prev = n_upd;
        h->sched.prev_width = prev_width;
        h->sched.prev_lo = prev_lo;
        h->sched.prev_hi = prev_hi;
        h->sched.full = full ? 1 : 0;
        h->sched.upd_prev = upd_prev;
        if (p.deadline_s > 0.0) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - start).count();
            if (el > p.deadline_s) {
                timed_out = true;
                break;
            }
        }
    }
    // keep the device table consistent with the weights held on the host
    rc = upload_table(h);
    if (rc)
        return rc;
    if (stats) {
        stats->iterations = n;
        stats->converged = flat ? 1 : 0;
        stats->last_metric = metric;
        stats->attempts_per_walker = spent;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - start).count();
    }
    if (flat)
        return MUCA_OK;
    if (timed_out)
        return fail(MUCA_ETIMEOUT, "deadline of %.3f s passed after %d iterations", p.deadline_s, n);
    return fail(MUCA_ENOTCONVERGED, "histogram not flat after %d iterations (metric %g)", n, metric);
}

int muca_build_table(int32_t L, const double *lnW, size_t n_bins, uint32_t *T_out)
{
    if (L < 4 || L > 64 || L % 4 != 0)
        return fail(MUCA_EINVAL, "L = %d: must be a multiple of 4 in [4, 64]", L);
    if (!lnW || !T_out || n_bins != (size_t)L * L + 1)
        return fail(MUCA_EINVAL, "need %d weights and a table buffer", L * L + 1);
    for (size_t e = 0; e < n_bins; ++e)
        if (!std::isfinite(lnW[e]))
            return fail(MUCA_EINVAL, "ln W[%zu] is not finite", e);
    build_table(L, std::vector<double>(lnW, lnW + n_bins), T_out);
    return MUCA_OK;
}

int muca_update_weights(int32_t L, double *lnW, const uint64_t *H, size_t n_bins)
{
    if (L < 4 || L > 64 || L % 4 != 0)
        return fail(MUCA_EINVAL, "L = %d: must be a multiple of 4 in [4, 64]", L);
    if (!lnW || !H || n_bins != (size_t)L * L + 1)
        return fail(MUCA_EINVAL, "need %d weights and histogram counts", L * L + 1);
    for (size_t e = 0; e < n_bins; ++e)
        if (H[e])
            lnW[e] -= muca::fp64::log((double)H[e]);
    return MUCA_OK;
}

int muca_iterate_device(muca_t h, const muca_params *p_in, int32_t iterations_per_sync, muca_stats *stats)
{
    int rc = validate(h);
    if (rc)
        return rc;
    muca_params p;
    if (p_in)
        p = *p_in;
    else
        muca_default_params(&p);
    if (p.schedule != MUCA_SCHEDULE_SWEEPS)
        return fail(MUCA_EINVAL, "muca_iterate_device runs the fixed-sweep schedule only");
    if (p.resume != 0 && p.resume != 1)
        return fail(MUCA_EINVAL, "resume must be 0 or 1");
    if (h->reducer)
        return fail(MUCA_EINVAL, "muca_iterate_device cannot reduce histograms over instances");
    if (p.stop_rule < MUCA_STOP_MIN_MEAN || p.stop_rule > MUCA_STOP_CHEBYSHEV)
        return fail(MUCA_EINVAL, "unknown stop rule %d", p.stop_rule);
    if (p.max_iterations < 1)
        return fail(MUCA_EINVAL, "max_iterations must be positive");
    if (iterations_per_sync < 1)
        return fail(MUCA_EINVAL, "iterations_per_sync must be positive");
    const auto start = std::chrono::steady_clock::now();
    const int32_t N = h->N;
    const size_t nb = (size_t)N + 1;
    if (!h->iter_block) {
        const size_t off_state = align256(nb * sizeof(double));
        h->iter_block = device_alloc(h->alloc, off_state + align256(sizeof(muca::IterState)));
        if (!h->iter_block)
            return fail(MUCA_ENOMEM, "device allocation for the iteration state failed");
        h->d_lnW = static_cast<double *>(h->iter_block);
        h->d_iter = reinterpret_cast<muca::IterState *>(static_cast<char *>(h->iter_block) + off_state);
        MUCA_CUDA(cudaMallocHost(reinterpret_cast<void **>(&h->h_iter), sizeof(muca::IterState)),
                  "pinned iteration state");
        MUCA_CUDA(muca::configure_iter_metric(N), "metric kernel shared memory");
    }
    const uint64_t n_therm = p.therm_sweeps * (uint64_t)N, n_upd = p.sweeps_per_iter * (uint64_t)N;
    const uint64_t t_start = h->t;
    // the first table and the weights from the host; the state zeroed
    MUCA_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    std::memset(h->h_iter, 0, sizeof(muca::IterState));
    h->h_iter->prev_lo = p.resume ? h->sched.prev_lo : -1;
    h->h_iter->prev_hi = p.resume ? h->sched.prev_hi : -1;
    MUCA_CUDA(cudaMemcpyAsync(h->d_iter, h->h_iter, sizeof(muca::IterState), cudaMemcpyHostToDevice, h->stream),
              "iteration state upload");
    MUCA_CUDA(cudaMemcpyAsync(h->d_lnW, h->lnW.data(), nb * sizeof(double), cudaMemcpyHostToDevice, h->stream),
              "weights upload");
    rc = upload_table(h);
    if (rc)
        return rc;
    const uint32_t *done = &h->d_iter->done;
    int32_t enqueued = 0;
    bool timed_out = false;
    for (;;) {
        const int32_t batch = std::min(iterations_per_sync, p.max_iterations - enqueued);
        for (int32_t i = 0; i < batch; ++i) {
            if ((rc = run_attempts(h, n_therm, false, done)) != MUCA_OK)
                return rc;
            MUCA_CUDA(muca::launch_iter_reset_hist(h->d_hist, (int32_t)nb, h->d_iter, h->stream), "histogram reset");
            if ((rc = run_attempts(h, n_upd, true, done)) != MUCA_OK)
                return rc;
            MUCA_CUDA(muca::launch_iter_metric(h->d_iter, N, h->d_hist, p.stop_rule, p.flat_threshold,
                                               p.max_iterations, h->stream),
                      "metric launch");
            MUCA_CUDA(muca::launch_iter_recursion(h->d_iter, N, h->d_lnW, h->d_hist, h->stream), "recursion launch");
            MUCA_CUDA(muca::launch_iter_table(h->d_iter, N, h->d_lnW, h->d_table, h->stream), "table launch");
        }
        enqueued += batch;
        MUCA_CUDA(cudaMemcpyAsync(h->h_iter, h->d_iter, sizeof(muca::IterState), cudaMemcpyDeviceToHost, h->stream),
                  "iteration state read");
        if ((rc = sync_and_check(h)) != MUCA_OK)
            return rc;
        if (h->h_iter->done || enqueued >= p.max_iterations)
            break;
        if (p.deadline_s > 0.0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - start).count() > p.deadline_s) {
            timed_out = true;
            break;
        }
    }
    const muca::IterState st = *h->h_iter;
    // launches after the last tested iteration did nothing: the counter covers the rest
    h->t = t_start + (uint64_t)st.iterations * (n_therm + n_upd);
    MUCA_CUDA(cudaMemcpyAsync(h->lnW.data(), h->d_lnW, nb * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
              "weights read");
    MUCA_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    const bool flat = st.done == 1u;
    if (st.iterations > (flat ? 1 : 0)) {   // at least one weight update: the state the host loop keeps
        h->sched.prev_lo = st.prev_lo;
        h->sched.prev_hi = st.prev_hi;
        h->sched.prev_width = st.prev_lo >= 0 ? st.prev_hi - st.prev_lo + 1 : 0;
        h->sched.upd_prev = n_upd;
    }
    if (stats) {
        stats->iterations = st.iterations;
        stats->converged = flat ? 1 : 0;
        stats->last_metric = st.metric;
        stats->attempts_per_walker = (uint64_t)st.iterations * (n_therm + n_upd);
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - start).count();
    }
    if (flat)
        return MUCA_OK;
    if (timed_out)
        return fail(MUCA_ETIMEOUT, "deadline of %.3f s passed after %d iterations", p.deadline_s, st.iterations);
    return fail(MUCA_ENOTCONVERGED, "histogram not flat after %d iterations (metric %g)", st.iterations, st.metric);
}

int muca_production(muca_t h, uint64_t therm_sweeps, uint64_t n_sweeps, uint64_t *H_out, double *ln_g_out,
                    size_t n_bins)
{
    int rc = validate(h);
    if (rc)
        return rc;
    const int32_t N = h->N;
    if (!ln_g_out || n_bins != (size_t)N + 1)
        return fail(MUCA_EINVAL, "ln g needs %d bins", N + 1);
    rc = upload_table(h);
    if (rc)
        return rc;
    rc = muca_sweep(h, therm_sweeps, 0);
    if (rc)
        return rc;
    rc = muca_reset_histogram(h);
    if (rc)
        return rc;
    rc = muca_sweep(h, n_sweeps, 1);
    if (rc)
        return rc;
    std::vector<uint64_t> H;
    rc = read_reduced_histogram(h, H);
    if (rc)
        return rc;
    // Sec. 3.3: ln g = ln H - ln W on visited energies, normalised to 2^N states.
    ln_dos_from_histogram(N, h->lnW, H.data(), ln_g_out);
    if (H_out)
        std::copy(H.begin(), H.end(), H_out);
    return MUCA_OK;
}

int muca_get_energies(muca_t h, int32_t *e_out, size_t n)
{
    int rc = validate(h);
    if (rc)
        return rc;
    if (!e_out || n != (size_t)h->W)
        return fail(MUCA_EINVAL, "energies have %lld entries", (long long)h->W);
    MUCA_CUDA(cudaMemcpyAsync(e_out, h->d_energy, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream),
              "energy read");
    return sync_and_check(h);
}

int muca_get_lattice(muca_t h, int8_t *out, size_t n)
{
    int rc = validate(h);
    if (rc)
        return rc;
    const size_t total = (size_t)h->W * (size_t)h->N;
    if (!out || n != total)
        return fail(MUCA_EINVAL, "lattice has %zu entries", total);
    int8_t *tmp = static_cast<int8_t *>(device_alloc(h->alloc, total));
    if (!tmp)
        return fail(MUCA_ENOMEM, "device allocation of %zu bytes failed", total);
    cudaError_t err = muca::launch_unpack(h->L, h->layout, h->W, h->d_lattice, tmp, h->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(out, tmp, total, cudaMemcpyDeviceToHost, h->stream);
    // the buffer goes back to the allocator only after every use of it has finished
    const cudaError_t sync = cudaStreamSynchronize(h->stream);
    if (err == cudaSuccess)
        err = sync;
    device_free(h->alloc, tmp);
    if (err != cudaSuccess)
        return cuda_fail(err, "lattice read");
    return sync_and_check(h);
}

int muca_set_lattice(muca_t h, const int8_t *spins, size_t n)
{
    int rc = validate(h);
    if (rc)
        return rc;
    const size_t total = (size_t)h->W * (size_t)h->N;
    if (!spins || n != total)
        return fail(MUCA_EINVAL, "lattice has %zu entries", total);
    for (size_t i = 0; i < total; ++i)
        if (spins[i] != 1 && spins[i] != -1)
            return fail(MUCA_EINVAL, "spin %zu is %d, not +1 or -1", i, (int)spins[i]);
    int8_t *tmp = static_cast<int8_t *>(device_alloc(h->alloc, total));
    if (!tmp)
        return fail(MUCA_ENOMEM, "device allocation of %zu bytes failed", total);
    cudaError_t err = cudaMemcpyAsync(tmp, spins, total, cudaMemcpyHostToDevice, h->stream);
    if (err == cudaSuccess)
        err = muca::launch_pack(h->L, h->layout, h->W, tmp, h->d_lattice, h->d_energy, h->stream);
    const cudaError_t sync = cudaStreamSynchronize(h->stream);
    if (err == cudaSuccess)
        err = sync;
    device_free(h->alloc, tmp);
    if (err != cudaSuccess)
        return cuda_fail(err, "lattice upload");
    return sync_and_check(h);
}

int muca_set_attempt_counter(muca_t h, uint64_t t)
{
    int rc = validate(h);
    if (rc)
        return rc;
    h->t = t;
    return MUCA_OK;
}

int muca_save(muca_t h, const char *path)
{
    int rc = validate(h);
    if (rc)
        return rc;
    if (!path)
        return fail(MUCA_EINVAL, "NULL path");
    const size_t N = (size_t)h->N, W = (size_t)h->W, nb = N + 1, row = (N + 7) / 8;
    std::vector<uint64_t> H;
    if ((rc = read_histogram(h, H)) != MUCA_OK)
        return rc;
    std::vector<int32_t> e(W);
    if ((rc = muca_get_energies(h, e.data(), W)) != MUCA_OK)
        return rc;
    std::vector<int8_t> spins(W * N);
    if ((rc = muca_get_lattice(h, spins.data(), spins.size())) != MUCA_OK)
        return rc;
    std::vector<uint8_t> bits(W * row, 0);
    for (size_t w = 0; w < W; ++w)
        for (size_t i = 0; i < N; ++i)
            if (spins[w * N + i] < 0)
                bits[w * row + i / 8] |= (uint8_t)(1u << (i % 8));
    FileCloser fc{std::fopen(path, "wb")};
    if (!fc.f)
        return fail(MUCA_EIO, "cannot open %s for writing", path);
    const int32_t L = h->L, layout = h->layout, wpb = h->wpb, order = h->order;
    const int64_t nw = h->W, first = h->walker0;
    const uint64_t seed = h->seed, t = h->t;
    const int32_t sched[4] = {h->sched.prev_width, h->sched.prev_lo, h->sched.prev_hi, h->sched.full};
    const bool ok = put(fc.f, kCheckpointMagic, 8) && put(fc.f, &L, 1) && put(fc.f, &layout, 1) &&
                    put(fc.f, &nw, 1) && put(fc.f, &seed, 1) && put(fc.f, &wpb, 1) && put(fc.f, &order, 1) &&
                    put(fc.f, &t, 1) && put(fc.f, &first, 1) && put(fc.f, sched, 4) &&
                    put(fc.f, &h->sched.upd_prev, 1) && put(fc.f, h->lnW.data(), nb) && put(fc.f, H.data(), nb) &&
                    put(fc.f, e.data(), W) && put(fc.f, bits.data(), bits.size());
    if (!ok || std::fflush(fc.f) != 0)
        return fail(MUCA_EIO, "writing %s failed", path);
    return MUCA_OK;
}

int muca_load(const char *path, muca_t *out)
{
    if (!path || !out)
        return fail(MUCA_EINVAL, "NULL argument");
    *out = nullptr;
    FileCloser fc{std::fopen(path, "rb")};
    if (!fc.f)
        return fail(MUCA_EIO, "cannot open %s", path);
    char magic[8];
    muca_options o;
    std::memset(&o, 0, sizeof o);
    int32_t order = 0;
    uint64_t t = 0;
    if (!get(fc.f, magic, 8) ||
        (std::memcmp(magic, kCheckpointMagic, 8) != 0 && std::memcmp(magic, kCheckpointMagicV1, 8) != 0))
        return fail(MUCA_EIO, "%s is not a checkpoint of this library", path);
    const bool has_sched = std::memcmp(magic, kCheckpointMagic, 8) == 0;
    IterSchedule sched;
    int32_t sched_words[4] = {0, -1, -1, 0};
    if (!get(fc.f, &o.L, 1) || !get(fc.f, &o.layout, 1) || !get(fc.f, &o.n_walkers, 1) || !get(fc.f, &o.seed, 1) ||
        !get(fc.f, &o.walkers_per_block, 1) || !get(fc.f, &order, 1) || !get(fc.f, &t, 1) ||
        !get(fc.f, &o.first_walker, 1) ||
        (has_sched && (!get(fc.f, sched_words, 4) || !get(fc.f, &sched.upd_prev, 1))))
        return fail(MUCA_EIO, "%s: truncated header", path);
    sched.prev_width = sched_words[0];
    sched.prev_lo = sched_words[1];
    sched.prev_hi = sched_words[2];
    sched.full = sched_words[3];
    if (o.L < 4 || o.L > 64 || o.L % 4 != 0 || o.n_walkers < 1 || o.n_walkers > INT32_MAX ||
        o.first_walker < 0 || o.first_walker > (int64_t)INT32_MAX - o.n_walkers ||
        (o.layout != MUCA_LAYOUT_INT8 && o.layout != MUCA_LAYOUT_PACKED))
        return fail(MUCA_EIO, "%s: invalid header", path);
    {
        const int32_t nbins = o.L * o.L + 1;
        const bool no_range = sched.prev_lo == -1 && sched.prev_hi == -1 && sched.prev_width == 0;
        const bool range_ok = sched.prev_lo >= 0 && sched.prev_lo <= sched.prev_hi && sched.prev_hi < nbins &&
                              sched.prev_width == sched.prev_hi - sched.prev_lo + 1;
        if ((!no_range && !range_ok) || (sched.full != 0 && sched.full != 1))
            return fail(MUCA_EIO, "%s: invalid iteration state", path);
    }
    const size_t N = (size_t)o.L * o.L, W = (size_t)o.n_walkers, nb = N + 1, row = (N + 7) / 8;
    std::vector<double> lnW(nb);
    std::vector<uint64_t> H(nb);
    std::vector<int32_t> e(W);
    std::vector<uint8_t> bits(W * row);
    if (!get(fc.f, lnW.data(), nb) || !get(fc.f, H.data(), nb) || !get(fc.f, e.data(), W) ||
        !get(fc.f, bits.data(), bits.size()))
        return fail(MUCA_EIO, "%s: truncated", path);
    std::vector<int8_t> spins(W * N);
    for (size_t w = 0; w < W; ++w)
        for (size_t i = 0; i < N; ++i)
            spins[w * N + i] = ((bits[w * row + i / 8] >> (i % 8)) & 1u) ? (int8_t)-1 : (int8_t)1;
    muca_t h = nullptr;
    int rc = muca_create_ex(&o, &h);
    if (rc)
        return rc;
    auto cleanup = [&](int code) {
        muca_destroy(h);
        return code;
    };
    if ((rc = muca_set_site_order(h, order)) != MUCA_OK || (rc = muca_set_weights(h, lnW.data(), nb)) != MUCA_OK ||
        (rc = muca_set_lattice(h, spins.data(), spins.size())) != MUCA_OK)
        return cleanup(rc);
    std::vector<int32_t> e_now(W);
    if ((rc = muca_get_energies(h, e_now.data(), W)) != MUCA_OK)
        return cleanup(rc);
    if (e_now != e)
        return cleanup(fail(MUCA_EIO, "%s: stored energies do not match the stored lattices", path));
    std::copy(H.begin(), H.end(), h->h_hist);
    cudaError_t err = cudaMemcpyAsync(h->d_hist, h->h_hist, nb * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                                      h->stream);
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(h->stream);
    if (err != cudaSuccess)
        return cleanup(cuda_fail(err, "histogram upload"));
    h->t = t;
    h->sched = sched;
    *out = h;
    return MUCA_OK;
}

int muca_get_info(muca_t h, int32_t *L, int64_t *n_walkers, uint64_t *attempt_counter, int32_t *layout,
                  int32_t *walkers_per_block)
{
    int rc = validate(h);
    if (rc)
        return rc;
    if (L)
        *L = h->L;
    if (n_walkers)
        *n_walkers = h->W;
    if (attempt_counter)
        *attempt_counter = h->t;
    if (layout)
        *layout = h->layout;
    if (walkers_per_block)
        *walkers_per_block = h->wpb;
    return MUCA_OK;
}

int muca_synchronize(muca_t h)
{
    int rc = validate(h);
    if (rc)
        return rc;
    return sync_and_check(h);
}

int muca_synchronize_timeout(muca_t h, double seconds)
{
    int rc = validate(h);
    if (rc)
        return rc;
    if (!(seconds >= 0.0))
        return fail(MUCA_EINVAL, "negative time limit");
    cudaEvent_t ev = nullptr;
    MUCA_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event create");
    cudaError_t err = cudaEventRecord(ev, h->stream);
    const auto start = std::chrono::steady_clock::now();
    bool done = false;
    while (err == cudaSuccess) {
        err = cudaEventQuery(ev);
        if (err == cudaSuccess) {
            done = true;
            break;
        }
        if (err != cudaErrorNotReady)
            break;
        err = cudaSuccess;
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - start).count() > seconds)
            break;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    cudaEventDestroy(ev);
    if (err != cudaSuccess)
        return cuda_fail(err, "stream wait");
    if (!done)
        return fail(MUCA_ETIMEOUT, "the queued work did not finish within %.3f s", seconds);
    return sync_and_check(h);
}

int muca_philox(const uint32_t *ctr, const uint32_t key[2], size_t n, uint32_t *out)
{
    if (!ctr || !key || !out)
        return fail(MUCA_EINVAL, "NULL argument");
    if (n == 0)
        return MUCA_OK;
    uint32_t *d = nullptr;
    MUCA_CUDA(cudaMalloc(&d, n * 8 * sizeof(uint32_t)), "philox buffers");
    cudaError_t err = cudaMemcpy(d, ctr, n * 4 * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = muca::launch_philox(d, key[0], key[1], n, d + 4 * n, nullptr);
    if (err == cudaSuccess)
        err = cudaMemcpy(out, d + 4 * n, n * 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (err != cudaSuccess)
        return cuda_fail(err, "philox evaluation");
    return MUCA_OK;
}


int muca_batch_create(const muca_t *instances, int32_t n, muca_batch_t *out)
{
    if (!instances || n < 1 || !out)
        return fail(MUCA_EINVAL, "batch needs at least one instance");
    *out = nullptr;
    for (int32_t i = 0; i < n; ++i) {
        if (!instances[i])
            return fail(MUCA_EINVAL, "instance %d is NULL", i);
        if (!batchable_L(instances[i]->L))
            return fail(MUCA_EINVAL, "instance %d: L = %d has no whole-sweep kernel (8, 16, 24, 32, 48, 64)", i,
                        instances[i]->L);
        if (instances[i]->order != MUCA_ORDER_TYPEWRITER)
            return fail(MUCA_EINVAL, "instance %d: the batched kernel runs typewriter order only", i);
        if (instances[i]->reducer)
            return fail(MUCA_EINVAL, "instance %d has a histogram reducer: batches iterate instances alone", i);
        for (int32_t j = 0; j < i; ++j)
            if (instances[j] == instances[i])
                return fail(MUCA_EINVAL, "instance %d appears twice", i);
    }
    muca_batch_s *b = new (std::nothrow) muca_batch_s;
    if (!b)
        return fail(MUCA_ENOMEM, "host allocation failed");
    b->inst.assign(instances, instances + n);
    {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        b->alloc = g_alloc;
    }
    auto cleanup = [&](int rc) {
        muca_batch_destroy(b);
        return rc;
    };
    const size_t limit = muca::sweep_smem_limit() - 1024;
    size_t items = 0;
    for (muca_t h : b->inst) {
        int32_t wpb = 256;
        while (wpb > 32 && muca::full_smem_bytes(h->L, wpb, true) > limit)
            wpb -= 32;
        b->item_wpb.push_back(wpb);
        b->smem = std::max(b->smem, muca::full_smem_bytes(h->L, wpb, true));
        items += (size_t)((h->W + wpb - 1) / wpb);
    }
    b->items_capacity = items;
    cudaError_t err = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (err == cudaSuccess)
        err = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
    if (err == cudaSuccess)
        err = muca::configure_batch(b->smem);
    if (err != cudaSuccess)
        return cleanup(cuda_fail(err, "batch set-up"));
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int occ = muca::batch_resident_blocks(b->smem);
    if (occ < 1)
        return cleanup(fail(MUCA_EINVAL, "batched kernel does not fit an SM with %zu bytes of shared memory", b->smem));
    b->grid = sms * occ;
    const size_t off_items = align256(sizeof(muca::SweepArgs) * 2 * (size_t)n);
    const size_t off_counter = off_items + align256(sizeof(muca::BatchItem) * items);
    b->block = device_alloc(b->alloc, off_counter + 256);
    if (!b->block)
        return cleanup(fail(MUCA_ENOMEM, "batch device allocation failed"));
    b->d_args = static_cast<muca::SweepArgs *>(b->block);
    b->d_items = reinterpret_cast<muca::BatchItem *>(static_cast<char *>(b->block) + off_items);
    b->d_counter = reinterpret_cast<uint32_t *>(static_cast<char *>(b->block) + off_counter);
    err = cudaMallocHost(reinterpret_cast<void **>(&b->h_args), sizeof(muca::SweepArgs) * 2 * (size_t)n);
    if (err == cudaSuccess)
        err = cudaMallocHost(reinterpret_cast<void **>(&b->h_items), sizeof(muca::BatchItem) * items);
    if (err != cudaSuccess)
        return cleanup(cuda_fail(err, "batch pinned buffers"));
    // from now on every call on a member instance is ordered with the batch's work
    for (muca_t h : b->inst) {
        err = cudaStreamSynchronize(h->stream);
        if (err != cudaSuccess)
            return cleanup(cuda_fail(err, "instance synchronize"));
        b->saved_streams.push_back(h->stream);
        h->stream = b->stream;
    }
    *out = b;
    return MUCA_OK;
}

int muca_batch_destroy(muca_batch_t b)
{
    if (!b)
        return MUCA_OK;
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    for (size_t i = 0; i < b->saved_streams.size(); ++i)
        b->inst[i]->stream = b->saved_streams[i];
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    device_free(b->alloc, b->block);
    if (b->h_args)
        cudaFreeHost(b->h_args);
    if (b->h_items)
        cudaFreeHost(b->h_items);
    if (b->staged)
        cudaEventDestroy(b->staged);
    if (b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
    return MUCA_OK;
}

int muca_batch_info(muca_batch_t b, int32_t *n_instances, int32_t *grid, size_t *smem_bytes)
{
    if (!b)
        return fail(MUCA_EINVAL, "NULL batch");
    if (n_instances)
        *n_instances = (int32_t)b->inst.size();
    if (grid)
        *grid = b->grid;
    if (smem_bytes)
        *smem_bytes = b->smem;
    return MUCA_OK;
}

int muca_batch_sweep(muca_batch_t b, uint64_t n_sweeps, int record)
{
    if (!b)
        return fail(MUCA_EINVAL, "NULL batch");
    if (n_sweeps == 0)
        return MUCA_OK;
    for (muca_t h : b->inst)
        if (h->t % (uint64_t)h->N != 0)
            return fail(MUCA_EINVAL, "batched launches need every member at a sweep boundary");
    // every work item is one block: its 32-bit shared counts take 256 walkers x attempts
    uint64_t max_n = UINT64_MAX;
    for (muca_t h : b->inst)
        max_n = std::min<uint64_t>(max_n, (record ? 0xFFFFFFFFull / 256ull : UINT64_MAX) / (uint64_t)h->N);
    std::vector<int32_t> all(b->inst.size());
    for (size_t i = 0; i < all.size(); ++i)
        all[i] = (int32_t)i;
    int rc = stage_wait(b);
    if (rc)
        return rc;
    if (b->members != all) {
        build_items(b, all);
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
    }
    rc = upload_items(b);
    if (rc)
        return rc;
    while (n_sweeps > 0) {
        const uint64_t chunk = std::min(n_sweeps, max_n);
        rc = stage_wait(b);
        if (rc)
            return rc;
        for (size_t j = 0; j < b->inst.size(); ++j) {
            muca_t h = b->inst[j];
            b->h_args[j] = make_args(h, h->t, chunk * (uint64_t)h->N);
            h->t += chunk * (uint64_t)h->N;
        }
        MUCA_CUDA(cudaMemcpyAsync(b->d_args, b->h_args, sizeof(muca::SweepArgs) * b->inst.size(),
                                  cudaMemcpyHostToDevice, b->stream),
                  "batch descriptor upload");
        MUCA_CUDA(cudaEventRecord(b->staged, b->stream), "batch upload event");
        MUCA_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(uint32_t), b->stream), "work counter reset");
        MUCA_CUDA(muca::launch_batch(b->d_args, b->d_items, b->n_items, b->d_counter, b->grid, b->smem, record != 0,
                                     b->stream),
                  "batched launch");
        n_sweeps -= chunk;
    }
    return MUCA_OK;
}

int muca_batch_iterate(muca_batch_t b, const muca_params *p_in, muca_stats *stats)
{
    if (!b)
        return fail(MUCA_EINVAL, "NULL batch");
    muca_params p;
    if (p_in)
        p = *p_in;
    else
        muca_default_params(&p);
    const size_t n = b->inst.size();
    for (muca_t h : b->inst) {
        int rc = check_iteration_params(p, h);
        if (rc)
            return rc;
    }
    const auto start = std::chrono::steady_clock::now();
    std::vector<muca_stats> st(n);
    std::memset(st.data(), 0, sizeof(muca_stats) * n);
    for (muca_t h : b->inst) {
        h->kl_lo = p.resume ? h->sched.prev_lo : -1;
        h->kl_hi = p.resume ? h->sched.prev_hi : -1;
    }
    std::vector<int32_t> active(n);
    for (size_t i = 0; i < n; ++i)
        active[i] = (int32_t)i;
    bool timed_out = false;
    while (!active.empty()) {
        std::vector<uint64_t> therm(active.size(), p.therm_sweeps), rec(active.size(), p.sweeps_per_iter);
        int rc = batch_run_iteration(b, active, therm, rec);
        if (rc)
            return rc;
        const double now = std::chrono::duration<double>(std::chrono::steady_clock::now() - start).count();
        std::vector<int32_t> next;
        for (int32_t i : active) {
            muca_stats &s = st[(size_t)i];
            s.seconds = now;
            if (!member_update(b->inst[(size_t)i], p, s))
                next.push_back(i);
        }
        active.swap(next);
        if (p.deadline_s > 0.0 && now > p.deadline_s && !active.empty()) {
            timed_out = true;
            break;
        }
    }
    // device tables follow the host weights again
    for (muca_t h : b->inst) {
        int rc = upload_table(h);
        if (rc)
            return rc;
    }
    MUCA_CUDA(cudaStreamSynchronize(b->stream), "batch synchronize");
    bool all = true;
    for (size_t i = 0; i < n; ++i) {
        all = all && st[i].converged;
        if (stats)
            stats[i] = st[i];
    }
    if (all)
        return MUCA_OK;
    if (timed_out)
        return fail(MUCA_ETIMEOUT, "deadline of %.3f s passed", p.deadline_s);
    return fail(MUCA_ENOTCONVERGED, "not every instance became flat");
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Serving: requests for whole weight iterations arrive over time; they are admitted
// while their device memory fits the budget, their state stays resident, and every
// step advances all admitted requests by one batched iteration.  Finished requests
// free their memory for the next ones (continuous batching).
// ---------------------------------------------------------------------------------
struct ServerRequest {
    muca_request req;
    double t_arrival = 0.0, t_admit = -1.0, t_done = -1.0;
    int32_t state = MUCA_REQ_QUEUED;
    int32_t code = MUCA_OK;
    size_t bytes = 0;
    muca_t h = nullptr;
    muca_stats st{};
    std::vector<double> lnW;
};

struct muca_server_s {
    size_t budget = 0, used = 0;
    std::vector<ServerRequest> reqs;
    std::vector<int64_t> queue;       // queued ids in arrival order
    std::vector<int64_t> active;      // admitted ids
    muca_batch_t batch = nullptr;
    std::vector<int64_t> batch_ids;   // members of `batch`, in order
    std::chrono::steady_clock::time_point t0;
    uint64_t attempts = 0;            // walker-attempts run by the server
    int32_t steps = 0;
};

extern "C" {
int muca_batch_sweep_noalloc(const muca_raw_instance *instances, int32_t n, uint64_t n_sweeps, int record,
                             void *cuda_stream)
{
    if (!instances || n < 1)
        return fail(MUCA_EINVAL, "no instances given");
    if (n > MUCA_NOALLOC_MAX_INSTANCES)
        return fail(MUCA_EINVAL, "%d instances exceed the allocation-free limit of %d", n, MUCA_NOALLOC_MAX_INSTANCES);
    if (n_sweeps == 0)
        return MUCA_OK;
    const size_t limit = muca::sweep_smem_limit() - 1024;
    muca::SweepArgs descs[MUCA_NOALLOC_MAX_INSTANCES];
    int32_t wpbs[MUCA_NOALLOC_MAX_INSTANCES];
    size_t smem = 0;
    for (int32_t i = 0; i < n; ++i) {
        const muca_raw_instance &r = instances[i];
        if (!batchable_L(r.L))
            return fail(MUCA_EINVAL, "instance %d: L = %d not in {8, 16, 24, 32, 48, 64}", i, r.L);
        if (r.layout != MUCA_LAYOUT_INT8 && r.layout != MUCA_LAYOUT_PACKED)
            return fail(MUCA_EINVAL, "instance %d: unknown layout %d", i, r.layout);
        if (r.n_walkers < 1 || r.n_walkers > INT32_MAX)
            return fail(MUCA_EINVAL, "instance %d: n_walkers = %lld out of range", i, (long long)r.n_walkers);
        if (!r.lattice || !r.energy || !r.table || !r.hist || !r.err)
            return fail(MUCA_EINVAL, "instance %d: NULL device buffer", i);
        const uint64_t N = (uint64_t)r.L * (uint64_t)r.L;
        if (r.t0 % N != 0)
            return fail(MUCA_EINVAL, "instance %d: t0 is not at a sweep boundary", i);
        if (n_sweeps > UINT64_MAX / N || (record && n_sweeps * N > 0xFFFFFFFFull / 256ull))
            return fail(MUCA_EINVAL, "instance %d: %llu sweeps exceed one launch (at most %llu recorded attempts per walker)",
                        i, (unsigned long long)n_sweeps, (unsigned long long)(0xFFFFFFFFull / 256ull));
        int32_t wpb = 256;
        while (wpb > 32 && muca::full_smem_bytes(r.L, wpb, true) > limit)
            wpb -= 32;
        wpbs[i] = wpb;
        smem = std::max(smem, muca::full_smem_bytes(r.L, wpb, true));
        muca::SweepArgs &d = descs[i];
        d.L = r.L;
        d.layout = r.layout;
        d.W = r.n_walkers;
        d.seed = r.seed;
        d.t0 = r.t0;
        d.n = n_sweeps * N;
        d.lattice = r.lattice;
        d.energy = r.energy;
        d.table = r.table;
        d.hist = r.hist;
        d.err = r.err;
    }
    MUCA_CUDA(muca::launch_batch_noalloc(descs, wpbs, n, smem, record != 0, static_cast<cudaStream_t>(cuda_stream)),
              "allocation-free batched sweep");
    return MUCA_OK;
}


static double server_now(muca_server_t s)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

int muca_server_create(size_t hbm_budget_bytes, muca_server_t *out)
{
    if (!out || hbm_budget_bytes == 0)
        return fail(MUCA_EINVAL, "server needs a memory budget");
    muca_server_s *s = new (std::nothrow) muca_server_s;
    if (!s)
        return fail(MUCA_ENOMEM, "host allocation failed");
    s->budget = hbm_budget_bytes;
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return MUCA_OK;
}

int muca_server_destroy(muca_server_t s)
{
    if (!s)
        return MUCA_OK;
    muca_batch_destroy(s->batch);
    for (ServerRequest &r : s->reqs)
        muca_destroy(r.h);
    delete s;
    return MUCA_OK;
}

int muca_server_submit(muca_server_t s, const muca_request *r, int64_t *id)
{
    if (!s || !r || !id)
        return fail(MUCA_EINVAL, "NULL argument");
    if (!batchable_L(r->L))
        return fail(MUCA_EINVAL, "L = %d not in {8, 16, 24, 32, 48, 64}", r->L);
    if (r->n_walkers < 1 || r->n_walkers > INT32_MAX)
        return fail(MUCA_EINVAL, "n_walkers out of range");
    if (r->layout == MUCA_LAYOUT_AUTO || r->walkers_per_block == MUCA_WPB_TUNE)
        return fail(MUCA_EINVAL, "requests take an explicit layout and block size (0 = default)");
    if (r->params.schedule != MUCA_SCHEDULE_SWEEPS || r->params.max_iterations < 1 || r->params.resume ||
        r->params.stop_rule < MUCA_STOP_MIN_MEAN || r->params.stop_rule > MUCA_STOP_CHEBYSHEV ||
        r->params.sweeps_per_iter * (uint64_t)r->L * (uint64_t)r->L > 0xFFFFFFFFull / 256ull)
        return fail(MUCA_EINVAL, "request parameters: fixed-sweep schedule, valid stop rule and sweeps");
    ServerRequest q;
    q.req = *r;
    q.t_arrival = server_now(s);
    q.bytes = instance_device_bytes(r->L, r->layout, r->n_walkers);
    if (q.bytes > s->budget)
        return fail(MUCA_ENOMEM, "request needs %zu bytes, more than the whole budget", q.bytes);
    *id = (int64_t)s->reqs.size();
    s->reqs.push_back(std::move(q));
    s->queue.push_back(*id);
    return MUCA_OK;
}

int muca_server_step(muca_server_t s, int32_t *n_active, int32_t *n_queued)
{
    if (!s)
        return fail(MUCA_EINVAL, "NULL server");
    // admission: every queued request that fits the remaining budget, in arrival order
    std::vector<int64_t> still;
    for (int64_t id : s->queue) {
        ServerRequest &q = s->reqs[(size_t)id];
        if (s->used + q.bytes > s->budget) {
            still.push_back(id);
            continue;
        }
        muca_options o;
        std::memset(&o, 0, sizeof o);
        o.L = q.req.L;
        o.n_walkers = q.req.n_walkers;
        o.seed = q.req.seed;
        o.layout = q.req.layout;
        o.walkers_per_block = q.req.walkers_per_block;
        int rc = muca_create_ex(&o, &q.h);
        if (rc == MUCA_ENOMEM) {
            still.push_back(id);
            continue;
        }
        if (rc != MUCA_OK) {
            q.state = MUCA_REQ_DONE;
            q.code = rc;
            q.t_done = server_now(s);
            continue;
        }
        q.state = MUCA_REQ_ACTIVE;
        q.t_admit = server_now(s);
        s->used += q.bytes;
        s->active.push_back(id);
    }
    s->queue.swap(still);
    if (!s->active.empty()) {
        if (s->active != s->batch_ids) {
            muca_batch_destroy(s->batch);
            s->batch = nullptr;
            std::vector<muca_t> hs;
            for (int64_t id : s->active)
                hs.push_back(s->reqs[(size_t)id].h);
            int rc = muca_batch_create(hs.data(), (int32_t)hs.size(), &s->batch);
            if (rc)
                return rc;
            s->batch_ids = s->active;
        }
        const size_t na = s->active.size();
        std::vector<int32_t> members(na);
        std::vector<uint64_t> therm(na), rec(na);
        for (size_t j = 0; j < na; ++j) {
            const ServerRequest &q = s->reqs[(size_t)s->active[j]];
            members[j] = (int32_t)j;
            therm[j] = q.req.params.therm_sweeps;
            rec[j] = q.req.params.sweeps_per_iter;
        }
        int rc = batch_run_iteration(s->batch, members, therm, rec);
        if (rc)
            return rc;
        s->steps += 1;
        const double now = server_now(s);
        std::vector<int64_t> next;
        for (size_t j = 0; j < na; ++j) {
            ServerRequest &q = s->reqs[(size_t)s->active[j]];
            s->attempts += (therm[j] + rec[j]) * (uint64_t)q.h->N * (uint64_t)q.h->W;
            q.st.seconds = now - q.t_admit;
            if (!member_update(q.h, q.req.params, q.st)) {
                next.push_back(s->active[j]);
                continue;
            }
            q.state = MUCA_REQ_DONE;
            q.code = q.st.converged ? MUCA_OK : MUCA_ENOTCONVERGED;
            q.t_done = now;
            q.lnW = q.h->lnW;
        }
        if (next.size() != s->active.size()) {
            // finished requests leave: drop the batch first, then free their memory
            muca_batch_destroy(s->batch);
            s->batch = nullptr;
            s->batch_ids.clear();
            for (int64_t id : s->active) {
                ServerRequest &q = s->reqs[(size_t)id];
                if (q.state == MUCA_REQ_DONE) {
                    muca_destroy(q.h);
                    q.h = nullptr;
                    s->used -= q.bytes;
                }
            }
            s->active.swap(next);
        }
    }
    if (n_active)
        *n_active = (int32_t)s->active.size();
    if (n_queued)
        *n_queued = (int32_t)s->queue.size();
    return MUCA_OK;
}

int muca_server_status(muca_server_t s, int64_t id, muca_request_status *out)
{
    if (!s || !out || id < 0 || id >= (int64_t)s->reqs.size())
        return fail(MUCA_EINVAL, "unknown request");
    const ServerRequest &q = s->reqs[(size_t)id];
    out->state = q.state;
    out->code = q.code;
    out->stats = q.st;
    const double now = server_now(s);
    out->seconds_queued = (q.t_admit >= 0.0 ? q.t_admit : now) - q.t_arrival;
    out->seconds_total = (q.t_done >= 0.0 ? q.t_done : now) - q.t_arrival;
    return MUCA_OK;
}

int muca_server_weights(muca_server_t s, int64_t id, double *lnW_out, size_t n_bins)
{
    if (!s || !lnW_out || id < 0 || id >= (int64_t)s->reqs.size())
        return fail(MUCA_EINVAL, "unknown request");
    const ServerRequest &q = s->reqs[(size_t)id];
    if (q.state != MUCA_REQ_DONE || q.lnW.empty())
        return fail(MUCA_EINVAL, "request %lld has no final weights", (long long)id);
    if (n_bins != q.lnW.size())
        return fail(MUCA_EINVAL, "weights have %zu bins", q.lnW.size());
    std::copy(q.lnW.begin(), q.lnW.end(), lnW_out);
    return MUCA_OK;
}

int muca_server_totals(muca_server_t s, uint64_t *walker_attempts, double *seconds, int32_t *steps, size_t *bytes_in_use)
{
    if (!s)
        return fail(MUCA_EINVAL, "NULL server");
    if (walker_attempts)
        *walker_attempts = s->attempts;
    if (seconds)
        *seconds = server_now(s);
    if (steps)
        *steps = s->steps;
    if (bytes_in_use)
        *bytes_in_use = s->used;
    return MUCA_OK;
}


int muca_production_jackknife(muca_t h, uint64_t therm_sweeps, int32_t n_chunks, uint64_t sweeps_per_chunk,
                              uint64_t *H_chunks_out, double *ln_g_out, double *ln_g_err_out, size_t n_bins)
{
    int rc = validate(h);
    if (rc)
        return rc;
    const int32_t N = h->N;
    const size_t B = (size_t)N + 1;
    if (!ln_g_out || !ln_g_err_out || n_bins != B)
        return fail(MUCA_EINVAL, "ln g and its error need %d bins", N + 1);
    if (n_chunks < 2 || sweeps_per_chunk == 0)
        return fail(MUCA_EINVAL, "a jackknife needs at least two non-empty chunks");
    rc = upload_table(h);
    if (rc)
        return rc;
    rc = muca_sweep(h, therm_sweeps, 0);
    if (rc)
        return rc;
    std::vector<uint64_t> chunks((size_t)n_chunks * B), total(B, 0), H;
    for (int32_t c = 0; c < n_chunks; ++c) {
        rc = muca_reset_histogram(h);
        if (rc)
            return rc;
        rc = muca_sweep(h, sweeps_per_chunk, 1);
        if (rc)
            return rc;
        rc = read_reduced_histogram(h, H);
        if (rc)
            return rc;
        for (size_t e = 0; e < B; ++e) {
            chunks[(size_t)c * B + e] = H[e];
            total[e] += H[e];
        }
    }
    // Sec. 3.3: leave-one-chunk-out estimates, error sqrt((n-1)/n sum (x_c - mean)^2)
    ln_dos_from_histogram(N, h->lnW, total.data(), ln_g_out);
    std::vector<double> loo((size_t)n_chunks * B);
    std::vector<uint64_t> rest(B);
    for (int32_t c = 0; c < n_chunks; ++c) {
        for (size_t e = 0; e < B; ++e)
            rest[e] = total[e] - chunks[(size_t)c * B + e];
        ln_dos_from_histogram(N, h->lnW, rest.data(), loo.data() + (size_t)c * B);
    }
    for (size_t e = 0; e < B; ++e) {
        if (!total[e]) {
            ln_g_err_out[e] = NAN;
            continue;
        }
        double mean = 0.0;
        bool missing = false;
        for (int32_t c = 0; c < n_chunks; ++c) {
            const double v = loo[(size_t)c * B + e];
            missing = missing || v == -INFINITY;
            mean += v;
        }
        if (missing) {
            ln_g_err_out[e] = INFINITY;
            continue;
        }
        mean /= (double)n_chunks;
        double ss = 0.0;
        for (int32_t c = 0; c < n_chunks; ++c) {
            const double d = loo[(size_t)c * B + e] - mean;
            ss += d * d;
        }
        ln_g_err_out[e] = std::sqrt((double)(n_chunks - 1) / (double)n_chunks * ss);
    }
    if (H_chunks_out)
        std::copy(chunks.begin(), chunks.end(), H_chunks_out);
    return MUCA_OK;
}

int muca_reweight(int32_t L, const double *ln_g, size_t n_bins, const double *betas, size_t n_betas,
                  double *energy_per_spin, double *specific_heat_per_spin)
{
    if (L < 2 || !ln_g || n_bins != (size_t)L * L + 1 || (n_betas && (!betas || !energy_per_spin)))
        return fail(MUCA_EINVAL, "reweighting needs L*L+1 values of ln g and output arrays");
    const int32_t N = L * L;
    for (size_t b = 0; b < n_betas; ++b) {
        const double beta = betas[b];
        // Eq. (1): P(E) ~ g(E) exp(-beta E) on E = -2N + 4e, summed in log space
        double top = -INFINITY;
        for (int32_t e = 0; e <= N; ++e)
            if (ln_g[e] != -INFINITY)
                top = std::max(top, ln_g[e] - beta * (-2.0 * N + 4.0 * e));
        if (top == -INFINITY)
            return fail(MUCA_EINVAL, "ln g has no finite entry");
        double z = 0.0, m1 = 0.0, m2 = 0.0;
        for (int32_t e = 0; e <= N; ++e) {
            if (ln_g[e] == -INFINITY)
                continue;
            const double E = -2.0 * N + 4.0 * e;
            const double p = std::exp(ln_g[e] - beta * E - top);
            z += p;
            m1 += p * E;
            m2 += p * E * E;
        }
        const double mean = m1 / z;
        energy_per_spin[b] = mean / (double)N;
        if (specific_heat_per_spin)
            specific_heat_per_spin[b] = beta * beta * (m2 / z - mean * mean) / (double)N;
    }
    return MUCA_OK;
}

const char *muca_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
