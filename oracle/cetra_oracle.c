/*
 * CETRA oracle: a plain, slow, FP64 CPU restatement of the transit search of
 * Smith et al. 2025 (CETRA), Sec. 2.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check of the build
 * entry point and the CPU-baseline leg of the benchmark load this library. The
 * product path (the CUDA library) never links, imports or calls it, and this
 * file shares no code, header, helper or table with it.
 *
 * Every step follows the paper in its own order and notation:
 *   Sec. 2.1.1  resampling onto a regular grid, null padding
 *   Sec. 2.1.2  template resampling by linear interpolation, nearest-neighbour lookup
 *   Sec. 2.1.3  duration / t0 / period grids
 *   Sec. 2.2    linear search: two passes per window (Eq. 1 and Eq. 2)
 *   Sec. 2.3    periodic search: common depth (Eq. 3, Eq. 4) and per-period max
 *
 * Readings of points the paper leaves open (each is stated where it is used):
 *   R1  t_i is the window mid-time; the window is [t_i - D/2, t_i + D/2]
 *       (Sec. 2.1.3 calls t_i the transit mid-point).
 *   R2  "nearest" means floor(x + 1/2) (ties round up) for the resample bin,
 *       the template sample and the epoch cell.
 *   R3  Template samples sit at x_l = l/(L-1); sample 0 is first contact,
 *       sample L-1 last contact. The resampled template is divided by its
 *       largest absolute value.
 *   R4  Window edges are inclusive at both ends (the ceil/floor of Sec. 2.1.1).
 *   R5  The t0 grid starts at the padded grid origin and spans the padded grid.
 *   R6  Phases per period: i < ceil(P/s).
 *   R7  The t0 step is realised as s = c*p/q with integers p >= 1 and
 *       1 <= q <= 64: the smallest q whose p/q is within 1e-9 (relative) of
 *       s/c, else the p/q with the least relative error (ties: smaller q).
 *       Index arithmetic then runs on integer "ticks" of length c/q: grid
 *       point n sits at tick n*q, t0 point i at tick i*p.
 *   R8  Index decisions are taken in IEEE FP64, one rounding per operation,
 *       in the order written here (no fused multiply-add).
 *   R9  Non-finite t/f/sigma and sigma <= 0 are dropped. Flux is normalised
 *       to a baseline of 1 unless flagged as an offset; y = 1 - f (Sec. 2).
 *   R10 A cell is null when no in-window point has W > 0 and m != 0.
 *       Null cells are skipped by the fold; a period with no valid cell is null.
 *   R11 Ties in the per-period maximum go to the smallest duration index j,
 *       then the smallest t0 index i.
 *   R12 A period shorter than one t0 step (P/s < 1) has no distinct phase and
 *       would fold one window onto itself; such a period (and a non-finite
 *       one) is null.
 *   R17 Masking a detected signal (Sec. 4.2: before each new search the flux in
 *       and around the previous search's best signal is nulled) acts on
 *       the resampled grid: cell k, at g_k = t_ref + (k - n_pad) c, is nulled
 *       when |g_k - (t0 + n P)| < h for the nearest epoch n = floor(d/P + 1/2),
 *       d = g_k - t0; h is half the masked width (a multiple of the duration,
 *       chosen by the caller).
 *   R18 Single-transit (monotransit) events from the linear search (Sec. 1,
 *       Sec. 5): greedily, the window with the largest LR among windows with a
 *       positive depth whose mid-time is not within an earlier event's
 *       duration of that event's mid-time (|i - i_e| < D_e q / (c p), FP64);
 *       ties go to the smallest j, then the smallest i.
 *
 * Parity unpinned: R1, R3, R5, R6 and R7 are conventions that no external fact
 * fixes (the GPU path takes the same ones); every computation around them is
 * pinned by the CPU tests against closed forms, brute force and invariants.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (R8 needs
 * -ffp-contract=off: aarch64 compilers contract a*b+c into fma by default).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

#define ORACLE_QMAX 64

typedef struct {
    double t_ref;     /* min of the kept times (absolute days) */
    double cadence;   /* c: resample cadence (days) */
    double t0_step;   /* s = c*p/q, realised t0 step (days) */
    int64_t p, q;     /* s/c = p/q (R7) */
    int64_t n_pad;    /* null points padded at each end */
    int64_t n_grid;   /* N_g */
    int64_t n_t0;     /* I */
    int64_t n_kept;   /* input points kept after cleaning (R9) */
    double tau_max;   /* largest kept time relative to t_ref */
} oracle_geom;

static int keep_point(double t, double f, double e) {
    return isfinite(t) && isfinite(f) && isfinite(e) && e > 0.0;
}

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * R7: realise s/c as p/q.
 */
static void rational_step(double ratio, int64_t *p_out, int64_t *q_out) {
    int64_t best_p = 1, best_q = 1;
    double best_err = INFINITY;
    for (int64_t q = 1; q <= ORACLE_QMAX; q++) {
        double pq = ratio * (double)q;
        int64_t p = (int64_t)floor(pq + 0.5);
        if (p < 1) p = 1;
        double err = fabs((double)p / (double)q - ratio) / ratio;
        if (err <= 1e-9) { best_p = p; best_q = q; break; }
        if (err < best_err) { best_err = err; best_p = p; best_q = q; }
    }
    *p_out = best_p;
    *q_out = best_q;
}

/*
 * Sec. 2.1.1 (resampling) and Sec. 2.1.3 (grids): the geometry of the
 * resampled light curve and of the t0 grid.
 *   c     = cadence if > 0, else the median of the positive differences of the
 *           sorted relative times (Sec. 2.1.1: default is the median cadence).
 *   s     = t0_step if > 0, else 0.01 * min(D) (Sec. 2.1.3 default), then R7.
 *   n_pad = ceil((max D / 2) / c)  (Sec. 2.1.1: pad by half the max duration)
 *   N_g   = 2 n_pad + floor(tau_max / c + 1/2) + 1
 *   I     = floor((N_g - 1) q / p) + 1   (R5: t_i spans the padded grid)
 */
int oracle_geometry(const double *time, const float *flux, const float *flux_err, int64_t n,
                    double cadence, double t0_step, const double *durations, int n_dur,
                    oracle_geom *g) {
    if (n < 1 || n_dur < 1 || !g) return ORACLE_EINVAL;
    memset(g, 0, sizeof(*g));
    double t_ref = INFINITY, t_max = -INFINITY;
    int64_t kept = 0;
    for (int64_t k = 0; k < n; k++) {
        if (!keep_point(time[k], flux[k], flux_err[k])) continue;
        kept++;
        if (time[k] < t_ref) t_ref = time[k];
        if (time[k] > t_max) t_max = time[k];
    }
    if (kept < 1) return ORACLE_EINVAL;
    double dmin = INFINITY, dmax = 0.0;
    for (int j = 0; j < n_dur; j++) {
        if (!(durations[j] > 0.0) || !isfinite(durations[j])) return ORACLE_EINVAL;
        if (durations[j] < dmin) dmin = durations[j];
        if (durations[j] > dmax) dmax = durations[j];
    }
    double c = cadence;
    if (!(c > 0.0)) {
        /* median of the positive diffs of the sorted relative times */
        double *tau = (double *)malloc(sizeof(double) * (size_t)kept);
        if (!tau) return ORACLE_ENOMEM;
        int64_t m = 0;
        for (int64_t k = 0; k < n; k++)
            if (keep_point(time[k], flux[k], flux_err[k])) tau[m++] = time[k] - t_ref;
        qsort(tau, (size_t)m, sizeof(double), cmp_double);
        int64_t nd = 0;
        for (int64_t k = 1; k < m; k++) {
            double d = tau[k] - tau[k - 1];
            if (d > 0.0) tau[nd++] = d; /* reuse the buffer (nd <= k - 1 < k) */
        }
        if (nd == 0) { free(tau); return ORACLE_EINVAL; }
        qsort(tau, (size_t)nd, sizeof(double), cmp_double);
        c = (nd % 2) ? tau[nd / 2] : 0.5 * (tau[nd / 2 - 1] + tau[nd / 2]);
        free(tau);
    }
    double s = t0_step;
    if (!(s > 0.0)) s = 0.01 * dmin;
    if (!isfinite(c) || !isfinite(s)) return ORACLE_EINVAL;
    int64_t p, q;
    rational_step(s / c, &p, &q);

    g->t_ref = t_ref;
    g->cadence = c;
    g->p = p;
    g->q = q;
    g->t0_step = (c * (double)p) / (double)q;
    g->n_pad = (int64_t)ceil((0.5 * dmax) / c);
    g->tau_max = t_max - t_ref;
    g->n_grid = 2 * g->n_pad + (int64_t)floor(g->tau_max / c + 0.5) + 1;
    g->n_t0 = ((g->n_grid - 1) * q) / p + 1;
    g->n_kept = kept;
    return ORACLE_OK;
}

/*
 * Sec. 2.1.1: each observation goes to the nearest grid point,
 *   k = n_pad + floor(tau / c + 1/2)  (R2),
 * and the points of one grid cell combine as an inverse-variance weighted
 * mean with formally propagated variance:
 *   W_k = sum 1/sigma^2,  y_k = sum(y/sigma^2) / W_k,  sigma_k^2 = 1/W_k.
 * Empty cells are null: W_k = 0 (infinite error), y_k = 0.
 */
int oracle_resample(const double *time, const float *flux, const float *flux_err, int64_t n,
                    int flux_is_offset, const oracle_geom *g, double *y_grid, double *w_grid) {
    double *wy = (double *)calloc((size_t)g->n_grid, sizeof(double));
    if (!wy) return ORACLE_ENOMEM;
    for (int64_t k = 0; k < g->n_grid; k++) w_grid[k] = 0.0;
    for (int64_t k = 0; k < n; k++) {
        if (!keep_point(time[k], flux[k], flux_err[k])) continue;
        double tau = time[k] - g->t_ref;
        int64_t bin = g->n_pad + (int64_t)floor(tau / g->cadence + 0.5);
        double f = (double)flux[k];
        double y = flux_is_offset ? f : 1.0 - f;
        double sig = (double)flux_err[k];
        double w = 1.0 / (sig * sig);
        w_grid[bin] += w;
        wy[bin] += w * y;
    }
    for (int64_t k = 0; k < g->n_grid; k++)
        y_grid[k] = (w_grid[k] > 0.0) ? wy[k] / w_grid[k] : 0.0;
    free(wy);
    return ORACLE_OK;
}

/*
 * Sec. 2.1.2: the supplied model (tmpl_len samples from first to last
 * contact) is resampled to L samples by linear interpolation, then divided
 * by its largest absolute value (R3).
 */
int oracle_template(const float *tmpl, int tmpl_len, int L, double *out) {
    if (tmpl_len < 1 || L < 2) return ORACLE_EINVAL;
    for (int l = 0; l < L; l++) {
        if (tmpl_len == 1) { out[l] = (double)tmpl[0]; continue; }
        double pos = (double)((int64_t)l * (tmpl_len - 1)) / (double)(L - 1);
        int64_t i0 = (int64_t)floor(pos);
        if (i0 > tmpl_len - 2) i0 = tmpl_len - 2;
        double frac = pos - (double)i0;
        out[l] = (double)tmpl[i0] * (1.0 - frac) + (double)tmpl[i0 + 1] * frac;
    }
    double mx = 0.0;
    for (int l = 0; l < L; l++) if (fabs(out[l]) > mx) mx = fabs(out[l]);
    if (!(mx > 0.0) || !isfinite(mx)) return ORACLE_EINVAL;
    for (int l = 0; l < L; l++) out[l] /= mx;
    return ORACLE_OK;
}

/*
 * Position of grid point n inside the window of (t_i, D_j), as a fraction of
 * the duration (0 = window start, 1 = window end), in ticks of c/q (R7, R8):
 *   x = ((n q - i p) + Dt/2) / Dt,   Dt = (D q) / c.
 * This is (g_n - (t_i - D/2)) / D of Sec. 2.1.1 written in ticks.
 */
static double window_x(int64_t n, int64_t i, int64_t p, int64_t q, double Dt) {
    double d = (double)(n * q - i * p);
    double num = d + 0.5 * Dt;
    return num / Dt;
}

/*
 * Sec. 2.2, linear search, for every (t_i, D_j):
 *  window:  grid points n with 0 <= x_n <= 1 (R1, R4)
 *  model:   m_n = T[floor(x_n (L-1) + 1/2)]  (nearest template sample, R2)
 *  pass 1:  over points with W_n > 0 and m_n != 0,
 *             Delta_n = y_n / m_n,  weight_n = m_n^2 W_n   (sigma_Delta_n = sigma_n / m_n)
 *             Delta_ij = sum(weight Delta_n) / sum(weight),  var_ij = 1 / sum(weight)
 *  pass 2:  LR_ij = sum_n W_n [ -1/2 (Delta_ij m_n - y_n)^2 + 1/2 y_n^2 ]   (Eq. 2)
 *  null:    sum(weight) == 0  -> NaN in all three outputs (R10, Sec. 2.2 last para.)
 * Outputs are [J][I] row-major (t0 contiguous). kappa (nullable) receives
 * sum_n |m_n W_n y_n| over the window, the condition number of A = sum m W y
 * used to bound FP32 cancellation in the tests.
 */
static void linear_cell(const oracle_geom *g, const double *y_grid, const double *w_grid,
                        double D, const double *T, int L, int64_t i,
                        double *depth, double *depth_var, double *lr, double *kappa) {
    const int64_t Ng = g->n_grid, p = g->p, q = g->q;
    double Dt = (D * (double)q) / g->cadence;
    /* candidate grid points (a superset of the window; membership is decided by x) */
    int64_t lo = (int64_t)floor(((double)(i * p) - 0.5 * Dt) / (double)q) - 1;
    int64_t hi = (int64_t)ceil(((double)(i * p) + 0.5 * Dt) / (double)q) + 1;
    if (lo < 0) lo = 0;
    if (hi > Ng - 1) hi = Ng - 1;
    double sw = 0.0, swd = 0.0, kap = 0.0;
    for (int64_t n = lo; n <= hi; n++) {
        double x = window_x(n, i, p, q, Dt);
        if (!(x >= 0.0 && x <= 1.0) || !(w_grid[n] > 0.0)) continue;
        int64_t l = (int64_t)floor(x * (double)(L - 1) + 0.5);
        double m = T[l];
        kap += fabs(m * w_grid[n] * y_grid[n]);
        if (m == 0.0) continue;
        double dn = y_grid[n] / m;
        double wt = m * m * w_grid[n];
        sw += wt;
        swd += wt * dn;
    }
    if (kappa) *kappa = kap;
    if (!(sw > 0.0)) {
        *depth = NAN; *depth_var = NAN; *lr = NAN;
        return;
    }
    double dep = swd / sw;
    double r = 0.0;
    for (int64_t n = lo; n <= hi; n++) {
        double x = window_x(n, i, p, q, Dt);
        if (!(x >= 0.0 && x <= 1.0) || !(w_grid[n] > 0.0)) continue;
        int64_t l = (int64_t)floor(x * (double)(L - 1) + 0.5);
        double m = T[l];
        double res = dep * m - y_grid[n];
        r += w_grid[n] * (-0.5 * res * res + 0.5 * y_grid[n] * y_grid[n]);
    }
    *depth = dep;
    *depth_var = 1.0 / sw;
    *lr = r;
}

int oracle_linear(const oracle_geom *g, const double *y_grid, const double *w_grid,
                  const double *durations, int n_dur, const double *T, int L,
                  double *depth, double *depth_var, double *lr, double *kappa) {
    const int64_t I = g->n_t0;
    const int64_t total = (int64_t)n_dur * I;
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t ji = 0; ji < total; ji++) {
        int j = (int)(ji / I);
        int64_t i = ji % I;
        linear_cell(g, y_grid, w_grid, durations[j], T, L, i, &depth[ji], &depth_var[ji],
                    &lr[ji], kappa ? &kappa[ji] : NULL);
    }
    return ORACLE_OK;
}

/* The same linear search evaluated only at the n_cells cells (j[c], i[c]). */
int oracle_linear_cells(const oracle_geom *g, const double *y_grid, const double *w_grid,
                        const double *durations, int n_dur, const double *T, int L,
                        int64_t n_cells, const int32_t *j, const int64_t *i,
                        double *depth, double *depth_var, double *lr, double *kappa) {
    for (int64_t c = 0; c < n_cells; c++)
        if (j[c] < 0 || j[c] >= n_dur || i[c] < 0 || i[c] >= g->n_t0) return ORACLE_EINVAL;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < n_cells; c++)
        linear_cell(g, y_grid, w_grid, durations[j[c]], T, L, i[c], &depth[c], &depth_var[c],
                    &lr[c], kappa ? &kappa[c] : NULL);
    return ORACLE_OK;
}

/*
 * Sec. 2.3, periodic search, for every period P_k:
 *  P in t0 steps:  Ps = (P q) / (c p)                      (R7, R8)
 *  phases:         i < min(I, ceil(Ps))                    (R6)
 *  durations:      D_j < P_k (Sec. 2.3: windows must not overlap), and
 *                  mask[k][j] != 0 when a mask is given
 *  epoch cells:    i + o_e,  o_e = floor(e Ps + 1/2), e = 0, 1, ... while < I
 *                  (nearest-neighbour epoch cell, R2); null cells skipped
 *  common depth:   Z = sum(Delta_e / var_e) / sum(1 / var_e),  var_Z = 1 / sum(1 / var_e)
 *  likelihood:     LR_ijk = sum_e [ LR_e - 1/2 (Delta_e - Z)^2 / var_e ]   (Eq. 4 summed)
 *  reduction:      max over (j, i); ties -> smallest j, then smallest i (R11)
 * Outputs per period: LR, t0 (absolute days, mid-time), D, Z, var_Z and the
 * winning (i, j); NaN and -1 for a period with no valid cell.
 */
/* Eq. 3 / Eq. 4 at one (t_i, D_j, P_k); returns 0 when no epoch cell is valid. */
static int fold_cell(int64_t I, const double *dep, const double *var, const double *lrj,
                     double Ps, int64_t i, double *lr_out, double *z_out, double *zvar_out) {
    double sw = 0.0, swd = 0.0;
    int any = 0;
    for (int64_t e = 0;; e++) {
        int64_t cell = i + (int64_t)floor((double)e * Ps + 0.5);
        if (cell >= I) break;
        if (isnan(lrj[cell])) continue;
        sw += 1.0 / var[cell];
        swd += dep[cell] / var[cell];
        any = 1;
    }
    if (!any) return 0;
    double Z = swd / sw;
    double L = 0.0;
    for (int64_t e = 0;; e++) {
        int64_t cell = i + (int64_t)floor((double)e * Ps + 0.5);
        if (cell >= I) break;
        if (isnan(lrj[cell])) continue;
        double dz = dep[cell] - Z;
        L += lrj[cell] - 0.5 * dz * dz / var[cell];
    }
    *lr_out = L;
    *z_out = Z;
    *zvar_out = 1.0 / sw;
    return 1;
}

static double period_steps(const oracle_geom *g, double P) {
    return (P * (double)g->q) / (g->cadence * (double)g->p);
}

int oracle_periodic(const oracle_geom *g, const double *durations, int n_dur,
                    const double *depth, const double *depth_var, const double *lr,
                    const double *periods, int n_per, const uint8_t *mask,
                    double *lr_out, double *t0_out, double *dur_out, double *z_out,
                    double *zvar_out, int64_t *i_out, int32_t *j_out) {
    const int64_t I = g->n_t0, p = g->p, q = g->q;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < n_per; k++) {
        double P = periods[k];
        double Ps = period_steps(g, P);
        double cph = ceil(Ps);
        int64_t nph = (cph < (double)I) ? (int64_t)cph : I;
        double best = -INFINITY, best_z = NAN, best_v = NAN;
        int64_t best_i = -1;
        int best_j = -1;
        int valid = Ps >= 1.0 && isfinite(Ps); /* R12 */
        for (int j = 0; valid && j < n_dur; j++) {
            if (!(durations[j] < P)) continue;
            if (mask && !mask[(int64_t)k * n_dur + j]) continue;
            const double *dep = depth + (int64_t)j * I;
            const double *var = depth_var + (int64_t)j * I;
            const double *lrj = lr + (int64_t)j * I;
            for (int64_t i = 0; i < nph; i++) {
                double L, Z, V;
                if (!fold_cell(I, dep, var, lrj, Ps, i, &L, &Z, &V)) continue;
                if (L > best) {
                    best = L; best_z = Z; best_v = V; best_i = i; best_j = j;
                }
            }
        }
        if (best_j < 0) {
            lr_out[k] = NAN; t0_out[k] = NAN; dur_out[k] = NAN; z_out[k] = NAN;
            zvar_out[k] = NAN; i_out[k] = -1; j_out[k] = -1;
        } else {
            lr_out[k] = best;
            /* t_i = g_0 + i s = t_ref + (i p - n_pad q) c / q */
            t0_out[k] = g->t_ref + ((double)(best_i * p - g->n_pad * q) * g->cadence) / (double)q;
            dur_out[k] = durations[best_j];
            z_out[k] = best_z;
            zvar_out[k] = best_v;
            i_out[k] = best_i;
            j_out[k] = best_j;
        }
    }
    return ORACLE_OK;
}

/* The periodic likelihood of Eq. 4 at the given (i[k], j[k]) of each period k
 * (NaN where no epoch cell is valid or the cell is out of range). */
int oracle_periodic_at(const oracle_geom *g, int n_dur, const double *depth,
                       const double *depth_var, const double *lr, const double *periods,
                       int n_per, const int64_t *i_at, const int32_t *j_at,
                       double *lr_out, double *z_out, double *zvar_out) {
    const int64_t I = g->n_t0;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < n_per; k++) {
        lr_out[k] = NAN; z_out[k] = NAN; zvar_out[k] = NAN;
        if (j_at[k] < 0 || j_at[k] >= n_dur || i_at[k] < 0 || i_at[k] >= I) continue;
        double Ps = period_steps(g, periods[k]);
        if (!(Ps >= 1.0) || !isfinite(Ps)) continue;
        int64_t o = (int64_t)j_at[k] * I;
        double L, Z, V;
        if (fold_cell(I, depth + o, depth_var + o, lr + o, Ps, i_at[k], &L, &Z, &V)) {
            lr_out[k] = L; z_out[k] = Z; zvar_out[k] = V;
        }
    }
    return ORACLE_OK;
}

/*
 * Period grid of a batched search: P_k = pmin * ratio^k for k = 0, 1, ... while
 * P_k <= pmax, with ratio^k by least-significant-bit-first square-and-multiply in
 * FP64 (x = 1, b = ratio; for each bit of k: if set, x = x * b; then b = b * b).
 * Writes at most `cap` periods and returns how many the grid has (or -1 on bad input).
 */
int64_t oracle_period_grid(double pmin, double ratio, double pmax, int64_t cap, double *out) {
    if (!(pmin > 0.0) || !(ratio > 1.0) || !isfinite(pmax) || !isfinite(ratio)) return -1;
    int64_t n = 0;
    for (int64_t k = 0;; k++) {
        double x = 1.0, b = ratio;
        for (int64_t m = k; m; m >>= 1) {
            if (m & 1) x = x * b;
            b = b * b;
        }
        double P = pmin * x;
        if (!(P <= pmax)) break;
        if (n < cap) out[n] = P;
        n++;
    }
    return n;
}

/*
 * Sec. 2.2 (last paragraph): the constant-flux log-likelihood, Eq. 1 at
 * Delta = 0 over the non-null grid points:
 *   logL0 = sum_{W_k > 0} [ -1/2 y_k^2 W_k - 1/2 ln(2 pi / W_k) ].
 * Adding it to any LR gives the whole-curve log-likelihood.
 */
double oracle_logl0(const oracle_geom *g, const double *y_grid, const double *w_grid) {
    double s = 0.0;
    for (int64_t k = 0; k < g->n_grid; k++) {
        if (!(w_grid[k] > 0.0)) continue;
        s += -0.5 * y_grid[k] * y_grid[k] * w_grid[k] - 0.5 * log(2.0 * M_PI / w_grid[k]);
    }
    return s;
}

/*
 * R17: null the resampled cells within h (days) of any mid-time t0 + n P of a
 * detected signal: W_k = 0 and y_k = 0 (the cell then carries no information).
 * Returns the number of cells nulled by this call.
 */
int64_t oracle_mask_transits(const oracle_geom *g, double *y_grid, double *w_grid, double P,
                             double t0, double h) {
    int64_t n_masked = 0;
    if (!(P > 0.0) || !isfinite(P) || !(h > 0.0)) return 0;
    for (int64_t k = 0; k < g->n_grid; k++) {
        double gk = g->t_ref + (double)(k - g->n_pad) * g->cadence;
        double d = gk - t0;
        double n = floor(d / P + 0.5);
        double r = fabs(d - n * P);
        if (r < h) {
            if (w_grid[k] > 0.0) n_masked++;
            w_grid[k] = 0.0;
            y_grid[k] = 0.0;
        }
    }
    return n_masked;
}

/*
 * R18: up to max_events single-transit events from the linear-search arrays
 * ([J][I] depth and LR; NaN marks a null window). Writes each event's (i, j) and
 * returns how many were found.
 */
int oracle_monotransits(const oracle_geom *g, const double *durations, int n_dur,
                        const double *depth, const double *lr, int max_events,
                        int64_t *ev_i, int32_t *ev_j) {
    const int64_t I = g->n_t0;
    double *half = (double *)malloc(sizeof(double) * (size_t)(max_events > 0 ? max_events : 1));
    if (!half) return -1;
    int n = 0;
    for (; n < max_events; n++) {
        double best = 0.0;
        int64_t bi = -1;
        int bj = -1;
        for (int j = 0; j < n_dur; j++) {
            for (int64_t i = 0; i < I; i++) {
                double v = lr[(int64_t)j * I + i];
                if (isnan(v) || !(depth[(int64_t)j * I + i] > 0.0)) continue;
                int hidden = 0;
                for (int e = 0; e < n && !hidden; e++)
                    hidden = (double)llabs(i - ev_i[e]) < half[e];
                if (hidden) continue;
                if (bj < 0 || v > best) {  /* first in (j, i) order wins ties */
                    best = v; bi = i; bj = j;
                }
            }
        }
        if (bj < 0) break;
        ev_i[n] = bi;
        ev_j[n] = bj;
        half[n] = (durations[bj] * (double)g->q) / (g->cadence * (double)g->p);
    }
    free(half);
    return n;
}
