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
#include <vector>

#include <cuda_runtime.h>

#include "../../include/muca.h"
#include "muca_internal.h"

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
    uint64_t t = 0;                  // attempt counter (tag 0 stream)
};

namespace {

// Acceptance thresholds from ln W (Sec. 2.3, integer form): see muca.h.
void build_table(int32_t L, const std::vector<double> &lnW, uint32_t *T)
{
    const int32_t N = L * L;
    for (int32_t e = 0; e <= N; ++e)
        for (int32_t k = 0; k <= 4; ++k) {
            const int32_t to = e + 2 - k;
            uint32_t v = 0u;
            if (to >= 0 && to <= N) {
                const double dw = lnW[(size_t)to] - lnW[(size_t)e];
                if (dw >= 0.0) {
                    v = 0xFFFFFFFFu;
                } else {
                    const double scaled = std::floor(std::exp(dw) * 4294967296.0);
                    v = scaled >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)scaled;
                }
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

int run_attempts(muca_t h, uint64_t n, bool record)
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
            d += p * std::log(p * q);
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

int validate(muca_t h)
{
    if (!h)
        return fail(MUCA_EINVAL, "NULL instance");
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

int muca_create_ex(const muca_options *opt, muca_t *out)
{
    if (!opt || !out)
        return fail(MUCA_EINVAL, "NULL argument");
    *out = nullptr;
    const int32_t L = opt->L;
    if (L < 4 || L > 64 || L % 4 != 0)
        return fail(MUCA_EINVAL, "L = %d: must be a multiple of 4 in [4, 64]", L);
    if (opt->n_walkers < 1 || opt->n_walkers > INT32_MAX)
        return fail(MUCA_EINVAL, "n_walkers = %lld out of range", (long long)opt->n_walkers);
    if (opt->layout != MUCA_LAYOUT_INT8 && opt->layout != MUCA_LAYOUT_PACKED)
        return fail(MUCA_EINVAL, "unknown layout %d", opt->layout);
    int32_t wpb = opt->walkers_per_block;
    if (wpb == 0)
        wpb = 64;
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
    err = muca::launch_init(L, h->layout, h->W, h->seed, h->d_lattice, h->d_energy, h->stream);
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
    const auto start = std::chrono::steady_clock::now();
    const int32_t N = h->N;
    std::vector<uint64_t> H;
    int32_t prev_width = 0, prev_accessible = 0;
    bool full = false;
    uint64_t upd_prev = 0, spent = 0;
    int32_t n = 0;
    bool flat = false, timed_out = false;
    double metric = 0.0;
    while (n < p.max_iterations) {
        uint64_t n_therm, n_upd;
        double q;
        if (p.schedule == MUCA_SCHEDULE_SWEEPS) {
            n_therm = p.therm_sweeps * (uint64_t)N;
            n_upd = p.sweeps_per_iter * (uint64_t)N;
            q = (double)(N - 1);
        } else {
            // Sec. 3: w = max(w', 10) with w' the extent covered in the previous
            // iteration; N_therm = f_therm w; Eq. (7) until the whole range was covered,
            // then growth by 1.1 per iteration; both truncated and increased by one.
            const int32_t w = std::max(prev_width, 10);
            n_therm = (uint64_t)(p.f_therm * (double)w);
            if (full) {
                n_upd = (uint64_t)std::floor(p.growth * (double)upd_prev) + 1u;
            } else {
                n_upd = (uint64_t)std::floor(p.factor * std::pow((double)w, p.z) / (double)h->W) + 1u;
                full = prev_width == N + 1;
            }
            q = (double)std::max(prev_accessible, 10);
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
        rc = read_histogram(h, H);
        if (rc)
            return rc;
        spent += n_therm + n_upd;
        ++n;
        if (p.stop_rule == MUCA_STOP_MIN_MEAN)
            metric = min_over_mean(N, H);
        else if (p.stop_rule == MUCA_STOP_KL)
            metric = kullback_leibler(N, H, q);
        else
            metric = chebyshev(N, H);
        flat = p.stop_rule == MUCA_STOP_MIN_MEAN ? metric >= p.flat_threshold : metric < p.flat_threshold;
        if (flat)
            break;
        // Eq. (4) in logarithms: ln W <- ln W - ln H on visited energies.
        for (int32_t e = 0; e <= N; ++e)
            if (H[(size_t)e])
                h->lnW[(size_t)e] -= std::log((double)H[(size_t)e]);
        int32_t lo, hi;
        if (visited_range(N, H, lo, hi)) {
            prev_width = hi - lo + 1;
            prev_accessible = 0;
            for (int32_t e = lo; e <= hi; ++e)
                prev_accessible += accessible(N, e) ? 1 : 0;
        } else {
            prev_width = prev_accessible = 0;
        }
        upd_prev = n_upd;
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
    rc = read_histogram(h, H);
    if (rc)
        return rc;
    // Sec. 3.3: ln g = ln H - ln W on visited energies, normalised to 2^N states.
    double top = -INFINITY;
    for (int32_t e = 0; e <= N; ++e) {
        ln_g_out[e] = H[(size_t)e] ? std::log((double)H[(size_t)e]) - h->lnW[(size_t)e] : -INFINITY;
        top = std::max(top, ln_g_out[e]);
    }
    if (top > -INFINITY) {
        double s = 0.0;
        for (int32_t e = 0; e <= N; ++e)
            if (H[(size_t)e])
                s += std::exp(ln_g_out[e] - top);
        const double shift = (double)N * std::log(2.0) - (top + std::log(s));
        for (int32_t e = 0; e <= N; ++e)
            if (H[(size_t)e])
                ln_g_out[e] += shift;
    }
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
    if (err == cudaSuccess)
        err = cudaStreamSynchronize(h->stream);
    device_free(h->alloc, tmp);
    if (err != cudaSuccess)
        return cuda_fail(err, "lattice read");
    return sync_and_check(h);
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
