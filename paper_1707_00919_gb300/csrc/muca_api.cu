// muca_api.cu - host side of the C ABI declared in include/muca.h: instances (creation,
// block-size choice, streams, allocator hook), weights and the threshold table built from
// ln W (Sec. 2.3, integer form), sweeps, histogram, lattice and energy transfers, state
// and checkpoints.  The weight iteration (Eq. 4, the stop rules, the schedule of Eq. 7)
// is in muca_api_iterate.cu, batches and serving in muca_api_batch.cu; everything per
// attempt runs in the kernels.
#include "muca_host.h"

using namespace muca_host;

namespace muca_host {

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

// ln W to the device (staged through the pinned table buffer, which holds 20 bytes per
// energy), then the thresholds built there by the same arithmetic as build_table.
int upload_table(muca_t h)
{
    MUCA_CUDA(cudaEventSynchronize(h->table_copied), "waiting for the previous table upload");
    double *stage = reinterpret_cast<double *>(h->h_table);
    std::copy(h->lnW.begin(), h->lnW.end(), stage);
    MUCA_CUDA(cudaMemcpyAsync(h->d_lnW, stage, h->lnW.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream),
              "weights upload");
    MUCA_CUDA(cudaEventRecord(h->table_copied, h->stream), "weights upload event");
    MUCA_CUDA(muca::launch_table(h->N, h->d_lnW, h->d_table, h->stream), "table build");
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

static muca::SweepArgs sweep_args(muca_t h, uint64_t n, const uint32_t *skip)
{
    muca::SweepArgs a;
    a.L = h->L;
    a.layout = h->layout;
    a.W = h->W;
    a.seed = h->seed;
    a.t0 = h->t;
    a.n = n;
    a.lattice = h->d_lattice;
    a.energy = h->d_energy;
    a.table = h->d_table;
    a.hist = h->d_hist;
    a.err = h->d_err;
    a.skip = skip;
    a.walker0 = h->walker0;
    return a;
}

int run_attempts(muca_t h, uint64_t n, bool record, const uint32_t *skip)
{
    const uint64_t cap = record ? max_recorded_attempts(h->wpb) : UINT64_MAX;
    while (n > 0) {
        const uint64_t chunk = std::min(n, cap);
        const muca::SweepArgs a = sweep_args(h, chunk, skip);
        if (h->order == MUCA_ORDER_RANDOM)
            MUCA_CUDA(muca::launch_random_sweep(a, h->wpb, record, h->stream), "random-order sweep launch");
        else
            MUCA_CUDA(muca::launch_sweep(a, h->wpb, record, h->stream), "sweep launch");
        h->t += chunk;
        n -= chunk;
    }
    return MUCA_OK;
}

int run_therm_record(muca_t h, uint64_t n_therm, uint64_t n_record, const uint32_t *skip)
{
    if (h->order == MUCA_ORDER_RANDOM || n_therm == 0 || n_record == 0 || n_record > max_recorded_attempts(h->wpb) ||
        n_therm > UINT64_MAX - n_record) {
        const int rc = run_attempts(h, n_therm, false, skip);
        return rc != MUCA_OK ? rc : run_attempts(h, n_record, true, skip);
    }
    muca::SweepArgs a = sweep_args(h, n_record, skip);
    a.n_therm = n_therm;
    MUCA_CUDA(muca::launch_sweep_fused(a, h->wpb, h->stream), "sweep launch");
    h->t += n_therm + n_record;
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

int validate(muca_t h)
{
    if (!h)
        return fail(MUCA_EINVAL, "NULL instance");
    return MUCA_OK;
}

}  // namespace muca_host

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

// Block size for L, layout and W by occupancy: the makespan of a launch is set by the
// most loaded SM sub-partition (one walker per thread, one warp per 32 walkers), so the
// cost of a block size is waves x warps per sub-partition in a full wave; ties go to
// the larger block.
int default_walkers_per_block(int32_t L, int32_t layout, int64_t W)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || sms < 1)
        sms = 1;   // no device answer: size as for one SM (the launch itself reports the error)
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
    const size_t off_W = off_err + 256;
    const size_t total = off_W + align256(nb * sizeof(double));

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
    h->d_lnW = reinterpret_cast<double *>(base + off_W);
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
    if (kind < MUCA_PROBE_XOR || kind > MUCA_PROBE_MIXED_ONE_WARP)
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

int muca_thermalize_and_record(muca_t h, uint64_t n_therm, uint64_t n_record)
{
    int rc = muca_reset_histogram(h);
    if (rc)
        return rc;
    return run_therm_record(h, n_therm, n_record);
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

const char *muca_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
