// muca_api_batch.cu - many instances in one launch of the batched persistent kernel
// (one CUDA graph per weight iteration), the allocation-free batched sweep, and the
// request server that admits simulations by device memory and advances them together.
#include "muca_host.h"

using namespace muca_host;

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
    muca::SweepArgs *d_args = nullptr;    // [2 n]: thermalization, recording (with n_therm: both)
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
// descriptors, zeroed histograms, one launch that runs every member's thermalization and
// then its recorded attempts (the recording descriptors carry n_therm), histogram and
// error-word reads.  The host refills the pinned buffers before every replay.
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

int check_iteration_params(const muca_params &p)
{
    if (p.schedule != MUCA_SCHEDULE_SWEEPS && p.schedule != MUCA_SCHEDULE_PAPER)
        return fail(MUCA_EINVAL, "unknown schedule %d", p.schedule);
    if (p.stop_rule < MUCA_STOP_MIN_MEAN || p.stop_rule > MUCA_STOP_CHEBYSHEV || p.max_iterations < 1)
        return fail(MUCA_EINVAL, "bad stop rule or max_iterations");
    if (p.resume != 0 && p.resume != 1)
        return fail(MUCA_EINVAL, "resume must be 0 or 1");
    return MUCA_OK;
}

// Attempts per walker of member h's next iteration under p, from the member's iteration
// state, as muca_iterate_until_flat forms them (Sec. 3: N_therm = f_therm w with
// w = max(w', 10); Eq. (7) until an iteration has started at the full width, growth by
// `growth` after it).  full_after is the full-coverage flag the member keeps if the
// iteration is not its last.
void iteration_counts(muca_t h, const muca_params &p, uint64_t &n_therm, uint64_t &n_upd, bool &full_after)
{
    full_after = h->sched.full != 0;
    if (p.schedule == MUCA_SCHEDULE_SWEEPS) {
        n_therm = p.therm_sweeps * (uint64_t)h->N;
        n_upd = p.sweeps_per_iter * (uint64_t)h->N;
        return;
    }
    const int32_t w = std::max(h->sched.prev_width, 10);
    n_therm = (uint64_t)(p.f_therm * (double)w);
    if (full_after) {
        n_upd = (uint64_t)std::floor(p.growth * (double)h->sched.upd_prev) + 1u;
    } else {
        const double walkers = (double)(h->total_walkers > 0 ? h->total_walkers : h->W);
        n_upd = (uint64_t)std::floor(p.factor * std::pow((double)w, p.z) / walkers) + 1u;
        full_after = h->sched.prev_width == h->N + 1;
    }
}

// Reads the members' histograms and error words into their pinned buffers and waits.
int read_back(muca_batch_t b, const std::vector<int32_t> &active)
{
    for (int32_t j : active) {
        const muca_t h = b->inst[(size_t)j];
        MUCA_CUDA(cudaMemcpyAsync(h->h_hist, h->d_hist, sizeof(unsigned long long) * ((size_t)h->N + 1),
                                  cudaMemcpyDeviceToHost, b->stream),
                  "histogram read");
        MUCA_CUDA(cudaMemcpyAsync(h->h_err, h->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->stream),
                  "error word read");
    }
    MUCA_CUDA(cudaStreamSynchronize(b->stream), "batch synchronize");
    return MUCA_OK;
}

// One weight iteration of the members `active` (indices into b->inst): member j
// thermalizes therm[j] attempts per walker and records rec[j], all members in one
// replay of the iteration graph (one launch for both phases), or, when some member
// records more attempts than one launch's 32-bit shared counts take, as a thermalization
// launch and several recording launches issued directly.  Afterwards each member's
// histogram is in its pinned buffer and its attempt counter is advanced.
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
    const uint64_t cap = max_recorded_attempts(256);
    bool chunked = false;
    for (size_t j = 0; j < nm; ++j)
        chunked = chunked || rec[j] > cap;
    for (size_t j = 0; j < nm; ++j) {
        muca_t h = b->inst[(size_t)active[j]];
        // the member's own last upload (muca_set_weights) may still read its staging buffer
        MUCA_CUDA(cudaEventSynchronize(h->table_copied), "waiting for the member's weights upload");
        build_table(h->L, h->lnW, h->h_table);
        b->h_args[j] = make_args(h, h->t, therm[j]);
        if (chunked) {   // a thermalization launch, then recording launches of at most cap attempts
            b->h_args[nm + j] = make_args(h, h->t + therm[j], std::min(rec[j], cap));
        } else {         // one launch: the thermalization in front of the recorded attempts
            b->h_args[nm + j] = make_args(h, h->t, rec[j]);
            b->h_args[nm + j].n_therm = therm[j];
        }
    }
    if (!chunked) {
        MUCA_CUDA(cudaGraphLaunch(b->exec, b->stream), "batch iteration launch");
        MUCA_CUDA(cudaStreamSynchronize(b->stream), "batch synchronize");
    } else {
        for (int32_t j : active) {
            const muca_t h = b->inst[(size_t)j];
            MUCA_CUDA(cudaMemcpyAsync(h->d_table, h->h_table, sizeof(uint32_t) * 5 * ((size_t)h->N + 1),
                                      cudaMemcpyHostToDevice, b->stream),
                      "table upload");
        }
        MUCA_CUDA(cudaMemcpyAsync(b->d_args, b->h_args, sizeof(muca::SweepArgs) * 2 * nm, cudaMemcpyHostToDevice,
                                  b->stream),
                  "batch descriptor upload");
        MUCA_CUDA(cudaMemsetAsync(b->d_counter, 0, 2 * sizeof(uint32_t), b->stream), "work counter reset");
        MUCA_CUDA(muca::launch_batch(b->d_args, b->d_items, b->n_items, b->d_counter, b->grid, b->smem, false,
                                     b->stream),
                  "batched thermalization");
        for (int32_t j : active) {
            const muca_t h = b->inst[(size_t)j];
            MUCA_CUDA(cudaMemsetAsync(h->d_hist, 0, sizeof(unsigned long long) * ((size_t)h->N + 1), b->stream),
                      "histogram reset");
        }
        for (uint64_t done = 0;;) {
            MUCA_CUDA(muca::launch_batch(b->d_args + nm, b->d_items, b->n_items, b->d_counter + 1, b->grid, b->smem,
                                         true, b->stream),
                      "batched recording");
            done += cap;
            bool more = false;
            for (size_t j = 0; j < nm; ++j)
                more = more || rec[j] > done;
            if (!more)
                break;
            // the next chunk: members that have finished record nothing
            MUCA_CUDA(cudaStreamSynchronize(b->stream), "batch synchronize");
            for (size_t j = 0; j < nm; ++j) {
                const muca_t h = b->inst[(size_t)active[j]];
                const uint64_t left = rec[j] > done ? rec[j] - done : 0u;
                b->h_args[nm + j] = make_args(h, h->t + therm[j] + std::min(rec[j], done), std::min(left, cap));
            }
            MUCA_CUDA(cudaMemcpyAsync(b->d_args + nm, b->h_args + nm, sizeof(muca::SweepArgs) * nm,
                                      cudaMemcpyHostToDevice, b->stream),
                      "batch descriptor upload");
            MUCA_CUDA(cudaMemsetAsync(b->d_counter + 1, 0, sizeof(uint32_t), b->stream), "work counter reset");
        }
        rc = read_back(b, active);
        if (rc)
            return rc;
    }
    for (size_t j = 0; j < nm; ++j)
        b->inst[(size_t)active[j]]->t += therm[j] + rec[j];
    return check_members(b);
}

// Host half of one iteration for a member whose histogram is in its pinned buffer:
// stop metric, flatness, Eq. (4) recursion and the member's iteration state (n_therm,
// n_upd and full_after as iteration_counts gave them).  Returns true when the member is
// finished (flat, or max_iterations reached).
bool member_update(muca_t h, const muca_params &p, muca_stats &s, uint64_t n_therm, uint64_t n_upd, bool full_after)
{
    const int32_t N = h->N;
    std::vector<uint64_t> H(h->h_hist, h->h_hist + N + 1);
    s.iterations += 1;
    s.attempts_per_walker += n_therm + n_upd;
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
    h->sched.full = full_after ? 1 : 0;
    h->sched.upd_prev = n_upd;
    return s.iterations >= p.max_iterations;
}

size_t instance_device_bytes(int32_t L, int32_t layout, int64_t W)
{
    const size_t nb = (size_t)L * L + 1;
    return align256(muca::lattice_bytes(L, layout == MUCA_LAYOUT_PACKED ? MUCA_LAYOUT_PACKED : MUCA_LAYOUT_INT8, W)) +
           align256((size_t)W * sizeof(int32_t)) + align256(nb * 5 * sizeof(uint32_t)) +
           align256(nb * sizeof(unsigned long long)) + 256 + align256(nb * sizeof(double));
}

}  // namespace

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
        const int stride = muca::batch_table_stride(h->L);
        while (wpb > 32 && muca::full_smem_bytes(h->L, wpb, true, false, stride) > limit)
            wpb -= 32;
        b->item_wpb.push_back(wpb);
        b->smem = std::max(b->smem, muca::full_smem_bytes(h->L, wpb, true, false, stride));
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
    int dev = 0, sms = 0;
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess)
        err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess)
        return cleanup(cuda_fail(err, "multiprocessor count"));
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
    int rc = check_iteration_params(p);
    if (rc)
        return rc;
    const auto start = std::chrono::steady_clock::now();
    std::vector<muca_stats> st(n);
    std::memset(st.data(), 0, sizeof(muca_stats) * n);
    for (muca_t h : b->inst) {
        if (!p.resume)
            h->sched = IterSchedule{};
        h->kl_lo = h->sched.prev_lo;
        h->kl_hi = h->sched.prev_hi;
    }
    std::vector<int32_t> active(n);
    for (size_t i = 0; i < n; ++i)
        active[i] = (int32_t)i;
    bool timed_out = false;
    while (!active.empty()) {
        const size_t na = active.size();
        std::vector<uint64_t> therm(na), rec(na);
        std::vector<char> full(na);
        for (size_t j = 0; j < na; ++j) {
            bool f;
            iteration_counts(b->inst[(size_t)active[j]], p, therm[j], rec[j], f);
            full[j] = f;
        }
        rc = batch_run_iteration(b, active, therm, rec);
        if (rc)
            return rc;
        const double now = std::chrono::duration<double>(std::chrono::steady_clock::now() - start).count();
        std::vector<int32_t> next;
        for (size_t j = 0; j < na; ++j) {
            const int32_t i = active[j];
            muca_stats &s = st[(size_t)i];
            s.seconds = now;
            if (!member_update(b->inst[(size_t)i], p, s, therm[j], rec[j], full[j] != 0))
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

// Whether the byte ranges [a, a + na) and [b, b + nb) intersect.
static bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
    return pa < pb + nb && pb < pa + na;
}

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
    int32_t prefix[MUCA_NOALLOC_MAX_INSTANCES + 1];
    prefix[0] = 0;
    int64_t items = 0;
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
        while (wpb > 32 && muca::full_smem_bytes(r.L, wpb, true, true) > limit)
            wpb -= 32;
        wpbs[i] = wpb;
        smem = std::max(smem, muca::full_smem_bytes(r.L, wpb, true, true));
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
        // work items before instance i + 1, summed in 64 bits
        items += (r.n_walkers + wpb - 1) / wpb;
        if (items > INT32_MAX)
            return fail(MUCA_EINVAL, "more than %d work items of up to 256 walkers in one call", INT32_MAX);
        prefix[i + 1] = (int32_t)items;
    }
    // every instance updates its lattices and energies in place: no two may share them
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j) {
            const muca_raw_instance &a = instances[i], &b = instances[j];
            if (overlaps(a.lattice, muca::lattice_bytes(a.L, a.layout, a.n_walkers), b.lattice,
                         muca::lattice_bytes(b.L, b.layout, b.n_walkers)) ||
                overlaps(a.energy, sizeof(int32_t) * (size_t)a.n_walkers, b.energy,
                         sizeof(int32_t) * (size_t)b.n_walkers))
                return fail(MUCA_EINVAL, "instances %d and %d share lattice or energy memory", i, j);
        }
    MUCA_CUDA(muca::launch_batch_noalloc(descs, wpbs, prefix, n, smem, record != 0,
                                         static_cast<cudaStream_t>(cuda_stream)),
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
    if (check_iteration_params(r->params) != MUCA_OK || r->params.resume)
        return fail(MUCA_EINVAL, "request parameters: a schedule, a stop rule, max_iterations >= 1, no resume");
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
        std::vector<char> full(na);
        for (size_t j = 0; j < na; ++j) {
            const ServerRequest &q = s->reqs[(size_t)s->active[j]];
            members[j] = (int32_t)j;
            bool f;
            iteration_counts(q.h, q.req.params, therm[j], rec[j], f);
            full[j] = f;
        }
        int rc = batch_run_iteration(s->batch, members, therm, rec);
        if (rc)
            return rc;
        s->steps += 1;
        const double now = server_now(s);
        std::vector<int64_t> next;
        for (size_t j = 0; j < na; ++j) {
            ServerRequest &q = s->reqs[(size_t)s->active[j]];
            s->attempts += (therm[j] + rec[j]) * (uint64_t)q.h->W;
            q.st.seconds = now - q.t_admit;
            if (!member_update(q.h, q.req.params, q.st, therm[j], rec[j], full[j] != 0)) {
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

}  // extern "C"
