// muca_api_iterate.cu - the weight iteration on the host and on the device (Eq. 4, the
// stop rules of Sec. 3 and Eq. (6) / (A.1), the schedule of Eq. (7)), the production
// estimate of ln g with its jackknife errors (Sec. 3.3) and canonical reweighting (Eq. 1).
#include "muca_host.h"

using namespace muca_host;

namespace muca_host {

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

}  // namespace muca_host

extern "C" {

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
        rc = muca_reset_histogram(h);
        if (rc)
            return rc;
        rc = run_therm_record(h, n_therm, n_upd);
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

int muca_flatness(int32_t L, const uint64_t *H, size_t n_bins, int32_t prev_lo, int32_t prev_hi,
                  double *min_over_mean_out, double *kl_out, double *chebyshev_out, int32_t *lo_out, int32_t *hi_out)
{
    if (L < 4 || L > 64 || L % 4 != 0)
        return fail(MUCA_EINVAL, "L = %d: must be a multiple of 4 in [4, 64]", L);
    const int32_t N = L * L;
    if (!H || n_bins != (size_t)N + 1)
        return fail(MUCA_EINVAL, "need a histogram of %d bins", N + 1);
    if (prev_lo >= 0 && (prev_hi < prev_lo || prev_hi > N))
        return fail(MUCA_EINVAL, "previous range [%d, %d] is not inside [0, %d]", prev_lo, prev_hi, N);
    const std::vector<uint64_t> h(H, H + n_bins);
    const int32_t plo = prev_lo >= 0 ? prev_lo : -1, phi = prev_lo >= 0 ? prev_hi : -1;
    if (min_over_mean_out)
        *min_over_mean_out = min_over_mean(N, h);
    if (kl_out)
        *kl_out = kullback_leibler(N, h, (double)kl_support(N, plo, phi, h));
    if (chebyshev_out)
        *chebyshev_out = chebyshev(N, h);
    int32_t lo, hi;
    visited_range(N, h, lo, hi);
    if (lo_out)
        *lo_out = lo;
    if (hi_out)
        *hi_out = hi;
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
        h->iter_block = device_alloc(h->alloc, align256(sizeof(muca::IterState)));
        if (!h->iter_block)
            return fail(MUCA_ENOMEM, "device allocation for the iteration state failed");
        h->d_iter = static_cast<muca::IterState *>(h->iter_block);
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
    rc = upload_table(h);   // the weights to the device and the first table
    if (rc)
        return rc;
    const uint32_t *done = &h->d_iter->done;
    int32_t enqueued = 0;
    bool timed_out = false;
    for (;;) {
        const int32_t batch = std::min(iterations_per_sync, p.max_iterations - enqueued);
        for (int32_t i = 0; i < batch; ++i) {
            MUCA_CUDA(muca::launch_iter_reset_hist(h->d_hist, (int32_t)nb, h->d_iter, h->stream), "histogram reset");
            if ((rc = run_therm_record(h, n_therm, n_upd, done)) != MUCA_OK)
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
    if (therm_sweeps > UINT64_MAX / (uint64_t)N || n_sweeps > UINT64_MAX / (uint64_t)N)
        return fail(MUCA_EINVAL, "sweep count too large");
    rc = muca_thermalize_and_record(h, therm_sweeps * (uint64_t)N, n_sweeps * (uint64_t)N);
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
    if (therm_sweeps > UINT64_MAX / (uint64_t)N || sweeps_per_chunk > UINT64_MAX / (uint64_t)N)
        return fail(MUCA_EINVAL, "sweep count too large");
    std::vector<uint64_t> chunks((size_t)n_chunks * B), total(B, 0), H;
    for (int32_t c = 0; c < n_chunks; ++c) {
        // the thermalization runs with the first chunk
        rc = muca_thermalize_and_record(h, c == 0 ? therm_sweeps * (uint64_t)N : 0u, sweeps_per_chunk * (uint64_t)N);
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

}  // extern "C"
