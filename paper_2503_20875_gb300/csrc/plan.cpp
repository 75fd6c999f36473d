// Host planner: geometry of the resampled grid and the t0 grid (Sec. 2.1.1,
// Sec. 2.1.3), the resampled template (Sec. 2.1.2) and the per-duration window
// tables that the linear kernel stages in shared memory.
//
// Index decisions (grid bins, window membership, nearest template sample) are
// taken in IEEE FP64 with one rounding per operation in a fixed order. This
// translation unit is compiled with -ffp-contract=off so that no multiply-add
// is fused. The t0 step is realised as s = c p / q (1 <= q <= 64) and every
// position is measured in integer ticks of c / q: grid point n is at tick n q,
// t0 point i at tick i p. A window therefore depends on i only through
// i mod q, which is what lets one table serve every t0 of a phase class.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace {

bool usable(double t, float f, float e) {
    return std::isfinite(t) && std::isfinite(f) && std::isfinite(e) && e > 0.0f;
}

// Realise s / c as p / q: the smallest q <= 64 whose rounded p / q is within
// 1e-9 (relative) of s / c, otherwise the q with the least relative error
// (earliest q on ties); p >= 1.
void realise_step(double ratio, int64_t *p_out, int64_t *q_out) {
    int64_t bp = 1, bq = 1;
    double berr = INFINITY;
    for (int64_t q = 1; q <= 64; ++q) {
        int64_t p = (int64_t)std::floor(ratio * (double)q + 0.5);
        if (p < 1) p = 1;
        double err = std::fabs((double)p / (double)q - ratio) / ratio;
        if (err <= 1e-9) {
            bp = p;
            bq = q;
            break;
        }
        if (err < berr) {
            berr = err;
            bp = p;
            bq = q;
        }
    }
    *p_out = bp;
    *q_out = bq;
}

// Fraction of the window of a t0 point covered at tick offset d = n q - i p:
// x = (d + Dt / 2) / Dt, Dt = D q / c (duration in ticks).
inline double window_pos(int64_t d, double Dt) {
    double num = (double)d + 0.5 * Dt;
    return num / Dt;
}

}  // namespace

int plan_build(cetra_ctx *ctx, const cetra_params *params, const double *time, const float *flux,
               const float *flux_err, int64_t n_points, const double *durations, int n_dur,
               const float *tmpl, int tmpl_len, cetra_plan *plan, bool with_tables) {
    if (!params || !time || !flux || !flux_err || !durations || (with_tables && !tmpl))
        return set_error(ctx, CETRA_EINVAL, "plan: NULL input pointer");
    if (n_points < 1) return set_error(ctx, CETRA_EINVAL, "plan: n_points < 1");
    if (n_dur < 1) return set_error(ctx, CETRA_EINVAL, "plan: n_dur < 1");
    if (with_tables && tmpl_len < 1) return set_error(ctx, CETRA_EINVAL, "plan: tmpl_len < 1");
    const int L = params->template_samples > 0 ? params->template_samples : 1024;
    if (L < 2) return set_error(ctx, CETRA_EINVAL, "plan: template_samples < 2");

    // --- clean inputs, reference time (Sec. 2: times relative to the start)
    double t_ref = INFINITY, t_max = -INFINITY;
    int64_t kept = 0;
    for (int64_t k = 0; k < n_points; ++k) {
        if (!usable(time[k], flux[k], flux_err[k])) continue;
        ++kept;
        t_ref = std::min(t_ref, time[k]);
        t_max = std::max(t_max, time[k]);
    }
    if (kept < 1) return set_error(ctx, CETRA_EINVAL, "plan: no finite point with sigma > 0");
    double dmin = INFINITY, dmax = 0.0;
    for (int j = 0; j < n_dur; ++j) {
        double D = durations[j];
        if (!(D > 0.0) || !std::isfinite(D))
            return set_error(ctx, CETRA_EINVAL, "plan: durations must be finite and > 0");
        dmin = std::min(dmin, D);
        dmax = std::max(dmax, D);
    }

    // --- cadence: given, or the median of the positive gaps between sorted
    //     relative times (Sec. 2.1.1 default)
    double c = params->cadence;
    if (!(c > 0.0)) {
        std::vector<double> tau;
        tau.reserve((size_t)kept);
        for (int64_t k = 0; k < n_points; ++k)
            if (usable(time[k], flux[k], flux_err[k])) tau.push_back(time[k] - t_ref);
        std::sort(tau.begin(), tau.end());
        std::vector<double> gaps;
        gaps.reserve(tau.size());
        for (size_t k = 1; k < tau.size(); ++k) {
            double g = tau[k] - tau[k - 1];
            if (g > 0.0) gaps.push_back(g);
        }
        if (gaps.empty())
            return set_error(ctx, CETRA_EINVAL, "plan: cadence undefined (fewer than 2 times)");
        size_t h = gaps.size() / 2;
        std::nth_element(gaps.begin(), gaps.begin() + h, gaps.end());
        double hi = gaps[h];
        if (gaps.size() % 2) {
            c = hi;
        } else {
            double lo = *std::max_element(gaps.begin(), gaps.begin() + h);
            c = 0.5 * (lo + hi);
        }
    }
    double s = params->t0_step;
    if (!(s > 0.0)) s = 0.01 * dmin;  // Sec. 2.1.3 default: 1 % of the shortest duration
    if (!std::isfinite(c) || !std::isfinite(s))
        return set_error(ctx, CETRA_EINVAL, "plan: cadence or t0 step not finite");
    int64_t p, q;
    realise_step(s / c, &p, &q);
    if (p > 64)
        return set_error(ctx, CETRA_EINVAL,
                         "plan: t0 step longer than 64 cadences is not supported");

    plan->t_ref = t_ref;
    plan->cadence = c;
    plan->p = p;
    plan->q = q;
    plan->t0_step = (c * (double)p) / (double)q;
    plan->tau_max = t_max - t_ref;
    // Sec. 2.1.1: pad by half the longest duration at both ends
    plan->n_pad = (int64_t)std::ceil((0.5 * dmax) / c);
    plan->n_grid = 2 * plan->n_pad + (int64_t)std::floor(plan->tau_max / c + 0.5) + 1;
    // Sec. 2.1.3: t0 grid from the padded origin over the padded grid
    plan->n_t0 = ((plan->n_grid - 1) * q) / p + 1;
    plan->n_kept = kept;
    plan->J = n_dur;
    plan->L = L;
    plan->flux_is_offset = params->flux_is_offset ? 1 : 0;
    plan->precision = params->precision;
    plan->durations.assign(durations, durations + n_dur);
    if (plan->n_grid > (int64_t)INT32_MAX / 2 || plan->n_t0 > (int64_t)INT32_MAX / 2 ||
        plan->n_t0 * (int64_t)n_dur > (int64_t)UINT32_MAX)
        return set_error(ctx, CETRA_EINVAL, "plan: grid too large (n_dur * n_t0 must fit 32 bits)");
    plan->ab_ld = ((plan->n_t0 + FOLD_PAD) + 1) & ~(int64_t)1;
    if (!with_tables) return CETRA_OK;

    // --- template (Sec. 2.1.2): linear interpolation to L samples over
    //     x in [0, 1], divided by the largest absolute value
    plan->T.assign((size_t)L, 0.0);
    for (int l = 0; l < L; ++l) {
        if (tmpl_len == 1) {
            plan->T[l] = (double)tmpl[0];
            continue;
        }
        double pos = (double)((int64_t)l * (tmpl_len - 1)) / (double)(L - 1);
        int64_t i0 = std::min<int64_t>((int64_t)std::floor(pos), tmpl_len - 2);
        double fr = pos - (double)i0;
        double a = (double)tmpl[i0], b = (double)tmpl[i0 + 1];
        plan->T[l] = a * (1.0 - fr) + b * fr;
    }
    double mx = 0.0;
    for (double v : plan->T) mx = std::max(mx, std::fabs(v));
    if (!(mx > 0.0) || !std::isfinite(mx))
        return set_error(ctx, CETRA_EINVAL, "plan: template is zero or not finite");
    for (double &v : plan->T) v /= mx;

    // --- window tables per (duration j, phase class r)
    const int64_t nclass = q;
    plan->win_a.assign((size_t)n_dur * nclass, 0);
    plan->win_len.assign((size_t)n_dur * nclass, 0);
    plan->win_padlen.assign((size_t)n_dur * nclass, 0);
    plan->win_off.assign((size_t)n_dur * nclass, 0);
    plan->tables.clear();
    const int64_t pad_to = p * LIN_RB;
    int32_t max_padlen = 0;
    for (int j = 0; j < n_dur; ++j) {
        const double Dt = (durations[j] * (double)q) / c;
        for (int64_t r = 0; r < nclass; ++r) {
            // ticks of grid point n relative to t0 point r: d = n q - r p
            int64_t lo = (int64_t)std::floor(((double)(r * p) - 0.5 * Dt) / (double)q) - 2;
            int64_t hi = (int64_t)std::ceil(((double)(r * p) + 0.5 * Dt) / (double)q) + 2;
            int64_t first = 0, count = 0;
            std::vector<float2> row;
            for (int64_t n = lo; n <= hi; ++n) {
                double x = window_pos(n * q - r * p, Dt);
                if (!(x >= 0.0 && x <= 1.0)) continue;
                if (count == 0) first = n;
                int64_t l = (int64_t)std::floor(x * (double)(L - 1) + 0.5);
                double m = plan->T[(size_t)l];
                row.push_back(make_float2((float)m, (float)(m * m)));
                ++count;
            }
            if (count > (int64_t)INT32_MAX / 4)
                return set_error(ctx, CETRA_EINVAL, "plan: window longer than 2^29 points");
            int64_t padlen = ((count + pad_to - 1) / pad_to) * pad_to;
            row.resize((size_t)padlen, make_float2(0.f, 0.f));
            size_t idx = (size_t)j * nclass + (size_t)r;
            plan->win_a[idx] = (int32_t)first;
            plan->win_len[idx] = (int32_t)count;
            plan->win_padlen[idx] = (int32_t)padlen;
            plan->win_off[idx] = (int64_t)plan->tables.size();
            plan->tables.insert(plan->tables.end(), row.begin(), row.end());
            max_padlen = std::max<int32_t>(max_padlen, (int32_t)padlen);
        }
    }
    plan->max_padlen = max_padlen;
    return CETRA_OK;
}

namespace {
template <typename T>
int upload(cetra_ctx *ctx, T **dst, const T *src, size_t n) {
    *dst = nullptr;
    if (n == 0) return CETRA_OK;
    cudaError_t e = cudaMalloc((void **)dst, n * sizeof(T));
    if (e != cudaSuccess) {
        *dst = nullptr;
        return set_error(ctx, CETRA_ENOMEM, std::string("plan upload: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_error(ctx, CETRA_ECUDA, cudaGetErrorString(e));
    return CETRA_OK;
}
}  // namespace

int plan_upload(cetra_ctx *ctx, cetra_plan *plan) {
    int rc;
    if ((rc = upload(ctx, &plan->d_durations, plan->durations.data(), plan->durations.size())))
        return rc;
    if ((rc = upload(ctx, &plan->d_win_a, plan->win_a.data(), plan->win_a.size()))) return rc;
    if ((rc = upload(ctx, &plan->d_win_len, plan->win_len.data(), plan->win_len.size()))) return rc;
    if ((rc = upload(ctx, &plan->d_win_padlen, plan->win_padlen.data(), plan->win_padlen.size())))
        return rc;
    if ((rc = upload(ctx, &plan->d_win_off, plan->win_off.data(), plan->win_off.size()))) return rc;
    plan->lin_order.resize(plan->win_padlen.size());
    for (size_t x = 0; x < plan->lin_order.size(); ++x) plan->lin_order[x] = (int32_t)x;
    std::stable_sort(plan->lin_order.begin(), plan->lin_order.end(), [&](int32_t a, int32_t b) {
        return plan->win_padlen[(size_t)a] > plan->win_padlen[(size_t)b];
    });
    if ((rc = upload(ctx, &plan->d_lin_order, plan->lin_order.data(), plan->lin_order.size())))
        return rc;
    if ((rc = upload(ctx, &plan->d_tables, plan->tables.data(), plan->tables.size()))) return rc;
    cudaError_t e = linear_configure(plan, ctx);
    if (e != cudaSuccess) return set_error(ctx, CETRA_ECUDA, cudaGetErrorString(e));
    return CETRA_OK;
}

void plan_free_device(cetra_plan *plan) {
    cudaFree(plan->d_durations);
    cudaFree(plan->d_win_a);
    cudaFree(plan->d_win_len);
    cudaFree(plan->d_win_padlen);
    cudaFree(plan->d_win_off);
    cudaFree(plan->d_lin_order);
    cudaFree(plan->d_tables);
    plan->d_durations = nullptr;
    plan->d_win_a = plan->d_win_len = plan->d_win_padlen = nullptr;
    plan->d_win_off = nullptr;
    plan->d_lin_order = nullptr;
    plan->d_tables = nullptr;
}

ws_layout workspace_layout(const cetra_plan *plan, int n_periods) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    ws_layout L{};
    size_t ng = (size_t)plan->n_grid;
    size_t off = 0;
    L.grid = off;  // interleaved (W y, W) per resampled cell
    off = up(off + ng * sizeof(float2));
    L.lin_status = off;  // bounded-wait status of the linear stage
    off = up(off + sizeof(int));
    L.ab = off;
    off = up(off + (size_t)plan->J * (size_t)plan->ab_ld * sizeof(float2));
    L.logl0 = off;
    off = up(off + sizeof(double));
    L.status = off;
    off = up(off + sizeof(int));
    L.keys = off;
    off = up(off + (size_t)std::max(n_periods, 0) * sizeof(unsigned long long));
    L.total = off;
    return L;
}
