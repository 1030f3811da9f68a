// Regularisation-parameter search and continuation (Sec. 3, "Parameter
// identification"): a host-side driver of warm-started claire_register
// solves.  See include/claire.h for the schedule.
#include "internal.h"

#include <chrono>
#include <cmath>
#include <cstring>

#define SEARCH_TRY(expr)                 \
    do {                                 \
        const claire_status s_ = (expr); \
        if (s_ < 0) return s_;           \
    } while (0)

namespace claire {
namespace {

struct SearchRun {
    claire_ctx* c;
    claire_search_opts o;
    claire_search_report* R;
    float* valid = nullptr;  // last accepted velocity (device, 3N)
    float* trial = nullptr;  // velocity of the running solve
    size_t n3 = 0;
    bool have_valid = false;
    claire_report last_valid{};

    ~SearchRun()
    {
        if (valid) cudaFree(valid);
        if (trial) cudaFree(trial);
    }

    bool budget() const { return R->solves < o.max_solves && R->solves < CLAIRE_MAX_SEARCH_SOLVES; }

    // one registration at (bv, bw) from `start`; *ok = valid by the bounds
    claire_status solve(double bv, double bw, const float* start, bool check, bool* ok)
    {
        SEARCH_TRY(claire_set_beta(c, bv, bw));
        if (cudaMemcpyAsync(trial, start, n3 * sizeof(float), cudaMemcpyDefault, ctx_stream(c)) != cudaSuccess)
            return ctx_fail(c, CLAIRE_ECUDA, "search: copy of the start velocity");
        claire_report rep;
        const claire_status st = claire_register(c, trial, &rep);
        if (st < 0 && st != CLAIRE_ELINESEARCH && st != CLAIRE_ETIMEOUT) return st;
        const int k = R->solves++;
        const bool in_bounds = rep.detj_min >= o.jmin && rep.detj_max <= 1.0 / o.jmin;
        *ok = st >= 0 && (!check || in_bounds);
        R->trace_beta_v[k] = bv;
        R->trace_beta_w[k] = bw;
        R->trace_detj_min[k] = rep.detj_min;
        R->trace_detj_max[k] = rep.detj_max;
        R->trace_valid[k] = *ok ? 1 : 0;
        R->trace_gn_iters[k] = rep.gn_iters;
        if (*ok) {
            std::swap(valid, trial);
            have_valid = true;
            last_valid = rep;
        }
        return CLAIRE_OK;
    }
};

claire_status setup(SearchRun& S, claire_ctx* c, const float* v_in, const claire_search_opts* opts,
                    claire_search_report* rep)
{
    S.c = c;
    if (opts) {
        S.o = *opts;
    } else {
        claire_default_search_opts(&S.o);
    }
    const claire_search_opts& o = S.o;
    if (!(o.beta_v_max > 0) || !(o.beta_v_min > 0) || o.beta_v_min > o.beta_v_max || !(o.beta_w_max >= 0) ||
        !(o.beta_w_min >= 0) || !(o.jmin > 0 && o.jmin < 1) || !(o.bisect_rtol > 0) || o.max_solves < 1)
        return ctx_fail(c, CLAIRE_EINVAL, "invalid search options");
    std::memset(rep, 0, sizeof(*rep));
    S.R = rep;
    S.n3 = 3 * ctx_points(c);
    if (cudaMalloc(&S.valid, S.n3 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&S.trial, S.n3 * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(c, CLAIRE_ENOMEM, "search: velocity buffers");
    }
    if (cudaMemcpyAsync(S.valid, v_in, S.n3 * sizeof(float), cudaMemcpyDefault, ctx_stream(c)) != cudaSuccess)
        return ctx_fail(c, CLAIRE_ECUDA, "search: copy of the initial velocity");
    return CLAIRE_OK;
}

claire_status finish(SearchRun& S, float* v_inout, double bv, double bw, claire_status st)
{
    SEARCH_TRY(claire_set_beta(S.c, bv, bw));
    S.R->beta_v = bv;
    S.R->beta_w = bw;
    S.R->last = S.last_valid;
    const float* src = S.have_valid ? S.valid : S.trial;
    if (cudaMemcpyAsync(v_inout, src, S.n3 * sizeof(float), cudaMemcpyDefault, ctx_stream(S.c)) != cudaSuccess ||
        cudaStreamSynchronize(ctx_stream(S.c)) != cudaSuccess)
        return ctx_fail(S.c, CLAIRE_ECUDA, "search: copy of the result");
    return st;
}

}  // namespace
}  // namespace claire

using namespace claire;

extern "C" claire_status claire_default_search_opts(claire_search_opts* o)
{
    if (!o) return CLAIRE_EINVAL;
    o->beta_v_max = 1.0;
    o->beta_v_min = 1e-5;
    o->beta_w_max = 1e-5;
    o->beta_w_min = 1e-7;
    o->jmin = 0.1;
    o->bisect_rtol = 0.1;
    o->max_solves = 40;
    return CLAIRE_OK;
}

extern "C" claire_status claire_param_search(claire_ctx* c, float* v_inout, const claire_search_opts* opts,
                                             claire_search_report* rep)
{
    if (!c || !v_inout || !rep) return CLAIRE_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    SearchRun S;
    SEARCH_TRY(setup(S, c, v_inout, opts, rep));
    const claire_search_opts& o = S.o;
    // (i) beta_v by factors of 10 from beta_v_max, then bisection
    double bw = o.beta_w_max, bv = o.beta_v_max;
    double hi = -1.0, lo = -1.0;  // smallest valid / largest breaching beta_v
    while (S.budget()) {
        bool ok = false;
        SEARCH_TRY(S.solve(bv, bw, S.valid, true, &ok));
        if (!ok) {
            lo = bv;
            break;
        }
        hi = bv;
        if (bv / 10.0 < o.beta_v_min) break;
        bv /= 10.0;
    }
    if (hi < 0) {  // even beta_v_max breaches: return that solve
        rep->t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return finish(S, v_inout, o.beta_v_max, bw, CLAIRE_ENOTCONVERGED);
    }
    if (lo > 0) {
        while (S.budget() && (hi - lo) > o.bisect_rtol * hi) {
            const double mid = 0.5 * (hi + lo);
            bool ok = false;
            SEARCH_TRY(S.solve(mid, bw, S.valid, true, &ok));
            if (ok)
                hi = mid;
            else
                lo = mid;
        }
    }
    const double bv_star = hi;
    // (ii) beta_w by factors of 10 while valid.  The accepted velocity of (i)
    // belongs to beta_v* (the last accepted solve is always at the current hi).
    double bw_star = bw;
    while (S.budget() && bw_star / 10.0 >= o.beta_w_min && bw_star > 0) {
        bool ok = false;
        SEARCH_TRY(S.solve(bv_star, bw_star / 10.0, S.valid, true, &ok));
        if (!ok) break;
        bw_star /= 10.0;
    }
    rep->t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return finish(S, v_inout, bv_star, bw_star, static_cast<claire_status>(S.last_valid.status));
}

extern "C" claire_status claire_param_continuation(claire_ctx* c, float* v_inout, double target_v, double target_w,
                                                   const claire_search_opts* opts, claire_search_report* rep)
{
    if (!c || !v_inout || !rep) return CLAIRE_EINVAL;
    if (!(target_v > 0) || !(target_w >= 0)) return ctx_fail(c, CLAIRE_EINVAL, "invalid target weights");
    const auto t0 = std::chrono::steady_clock::now();
    SearchRun S;
    SEARCH_TRY(setup(S, c, v_inout, opts, rep));
    const claire_search_opts& o = S.o;
    const double bw0 = o.beta_w_max > target_w ? o.beta_w_max : target_w;
    // stage 1: beta_v = beta_v_max, /10, ..., 10^ceil(log10 target_v), then target_v
    const double stop = std::pow(10.0, std::ceil(std::log10(target_v)));
    for (double bv = o.beta_v_max; bv >= stop * (1.0 - 1e-12) && S.budget(); bv /= 10.0) {
        bool ok = false;
        SEARCH_TRY(S.solve(bv, bw0, S.valid, false, &ok));
    }
    if (S.budget() && std::fabs(stop - target_v) > 1e-12 * target_v) {
        bool ok = false;
        SEARCH_TRY(S.solve(target_v, bw0, S.valid, false, &ok));
    }
    // stage 2: beta_w from beta_w_max down to target_w in factors of 10
    for (double bw = bw0 / 10.0; bw >= target_w * (1.0 - 1e-12) && S.budget(); bw /= 10.0) {
        bool ok = false;
        SEARCH_TRY(S.solve(target_v, bw, S.valid, false, &ok));
    }
    rep->t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return finish(S, v_inout, target_v, target_w, static_cast<claire_status>(S.last_valid.status));
}
