// Internal declarations shared by the host planner (plan.cpp), the C ABI
// (capi.cpp) and the kernels (kernels.cu). Not installed, not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "cetra.h"

// Kernels the library launches, for per-kernel event timing.
enum kernel_id { KID_RESAMPLE = 0, KID_LINEAR, KID_FOLD, KID_FINALIZE, KID_LOGL0, KID_COUNT };
extern const char *const kernel_names[KID_COUNT];

// Makes `dev` the calling thread's current device for the guard's scope and restores the
// caller's device afterwards; `status` is the result of switching.
struct device_guard {
    int prev = -1;
    cudaError_t status = cudaSuccess;
    explicit device_guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) status = cudaSetDevice(dev);
    }
    ~device_guard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
    device_guard(const device_guard &) = delete;
    device_guard &operator=(const device_guard &) = delete;
};

struct cetra_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    int64_t launches = 0;
    int num_sms = 0;
    size_t max_smem_optin = 0;
    // event timing (cetra_profile_enable): one start/stop pair per launch
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[KID_COUNT];
    std::vector<cudaEvent_t> event_pool;
};

// Record a start (begin = true) or stop event around a launch when profiling.
void prof_mark(cetra_ctx *ctx, kernel_id id, bool begin);

// Geometry and window tables (Sec. 2.1). Built on the host in FP64, the tables
// uploaded once. Window tables: for every duration j and t0 phase class
// r = i mod q, the grid points of the window of t0 index i = r + q u are
// n = a[j][r] + p u + k, k = 0 .. len[j][r]-1, with template samples tab[k].
struct cetra_plan {
    int device = 0;
    double t_ref = 0, cadence = 0, t0_step = 0, tau_max = 0;
    int64_t p = 1, q = 1, n_pad = 0, n_grid = 0, n_t0 = 0, n_kept = 0;
    int J = 0, L = 0;
    int flux_is_offset = 0, precision = 0;
    std::vector<double> durations;
    std::vector<double> T;             // resampled template (FP64)
    std::vector<int32_t> win_a;        // [J*q] first grid point (class base, may be < 0)
    std::vector<int32_t> win_len;      // [J*q] window length
    std::vector<int32_t> win_padlen;   // [J*q] length padded to the kernel's multiple
    std::vector<int64_t> win_off;      // [J*q] offset into the table array
    std::vector<float2> tables;        // (m, m^2) per window point
    int32_t max_padlen = 0;
    int64_t ab_ld = 0;  // row stride (cells) of the (A, B) grid: n_t0 + zero padding, even
    // linear kernel launch shape, chosen from p and the table lengths
    int lin_threads = 128, lin_kc = 0;
    size_t lin_smem = 0;
    // device copies (owned)
    double *d_durations = nullptr;
    int32_t *d_win_a = nullptr, *d_win_len = nullptr, *d_win_padlen = nullptr;
    // linear-stage rows (duration, phase class) by decreasing window length: the kernel takes
    // its longest blocks first, so the last wave holds the shortest ones
    std::vector<int32_t> lin_order;
    int32_t *d_lin_order = nullptr;
    int64_t *d_win_off = nullptr;
    float2 *d_tables = nullptr;
};

struct cetra_linear_grid {
    cetra_ctx *ctx = nullptr;
    cetra_plan *plan = nullptr;
    void *d_work = nullptr;
    size_t work_bytes = 0;
};

// Register block of the linear kernel: outputs per thread. Odd, so that the
// stride-RB shared-memory reads of a warp fall in distinct banks.
#ifndef LIN_RB_OUTPUTS
#define LIN_RB_OUTPUTS 9
#endif
constexpr int LIN_RB = LIN_RB_OUTPUTS;
#ifndef LIN_MIN_BLOCKS
#define LIN_MIN_BLOCKS 4  // resident linear blocks per SM the register allocation must allow
#endif
constexpr int LIN_SUB = 16;  // register blocks per partial sum of the linear kernel
// Fold kernel shape (fold.cu, compile-time). A block is FT_THREADS consumer threads, each
// folding FT_R phases of every period of a group of up to FT_G periods, plus one producer warp
// that issues the bulk copies of the staged strips.
#ifndef FT_R
#define FT_R 4            // phases per consumer thread
#endif
#ifndef FT_STRIP
#define FT_STRIP 2048     // cells per staged strip at most (a tile plus the offsets' spread)
#endif
#ifndef FT_KAHAN_GROUP
#define FT_KAHAN_GROUP 2  // epochs summed plainly before each compensated step
#endif
#ifndef FT_NSTAGE
#define FT_NSTAGE 8       // strips in flight per block at most (as many as the ring holds)
#endif
#ifndef FT_RING_BYTES
#define FT_RING_BYTES (56 * 1024)  // strip ring: FT_RING_BYTES / strip bytes stages, <= FT_NSTAGE
#endif
#ifndef FT_MIN_BLOCKS
#define FT_MIN_BLOCKS 2
#endif
#ifndef FT_TAB_BYTES
#define FT_TAB_BYTES (40 * 1024)  // epoch table: u16 offsets + two int32 per epoch
#endif
#ifndef FT_ITEMS_PER_SLOT
#define FT_ITEMS_PER_SLOT 2  // single-curve launches: work items per block slot at least (a
#endif                       // launch of fewer groups splits its durations into chunks)
#ifndef FT_CWARPS
#define FT_CWARPS 7       // consumer warps per block (+ the producer warp: 8 warps, 128 registers)
#endif
constexpr int FT_THREADS = FT_CWARPS * 32;           // consumer threads
constexpr int FT_BLOCK = FT_THREADS + 32;            // + the producer warp
constexpr int FT_T = FT_THREADS * FT_R;              // phases per tile
constexpr int FT_G = 8;                              // periods per group
constexpr int FT_PACK_MAXJ = 64;                     // durations a duration-packed item may hold
constexpr long long FT_WAIT_CYCLES = 2000000000ll;  // ~1 s of SM clocks before a wait gives up
constexpr uint32_t FT_SUSPEND_NS = 20000;            // suspend hint of one barrier try
constexpr int FOLD_PAD = FT_STRIP + 16;  // zero cells after each grid row
// (A, B) grids larger than this are folded one duration per work item, so that the blocks
// running at the same time read one row and the L2 holds it
constexpr size_t FT_L2_GRID_BYTES = (size_t)64 << 20;
size_t fold_smem_bytes();
// Opt the fold kernels in to their dynamic shared memory (fold.cu).
cudaError_t fold_configure();
// The same for the batched fold kernels (fold_batch.cu; called by fold_configure).
cudaError_t batch_fold_configure();

// Device view of one light curve of a batch (cetra_batch_*).
struct batch_curve {
    double t_ref;         // smallest kept time
    double pmin, ratio;   // period grid P_k = pmin * ratio^k (square-and-multiply), k < n_periods
    int64_t pt_off;       // first input point
    int64_t grid_off;     // first resampled cell
    int64_t ab_off;       // first (A, B) cell
    int64_t ld;           // (A, B) row stride (cells)
    int64_t per_off;      // first period (index into the batch's per-period keys)
    int32_t n_grid, I;    // resampled cells, t0 points (0: curve without usable points)
    int32_t n_periods;
    int32_t pad_;
};

// Period k of a batch curve: pmin * ratio^k with ratio^k by LSB-first square-and-multiply
// in FP64 (one rounding per multiplication): the batch's period-grid definition.
double batch_period_host(double pmin, double ratio, int64_t k);

// Workspace layout (byte offsets, 256-aligned).
struct ws_layout {
    size_t grid, lin_status, ab, keys, logl0, status, total;
};
ws_layout workspace_layout(const cetra_plan *plan, int n_periods);

// Host planner (plan.cpp)
int plan_build(cetra_ctx *ctx, const cetra_params *params, const double *time, const float *flux,
               const float *flux_err, int64_t n_points, const double *durations, int n_dur,
               const float *tmpl, int tmpl_len, cetra_plan *plan, bool with_tables);
int plan_upload(cetra_ctx *ctx, cetra_plan *plan);
void plan_free_device(cetra_plan *plan);

// Kernel launchers (kernels.cu). Return cudaSuccess or the launch error.
// The resampled grid is one interleaved (W y, W) pair per cell.
cudaError_t launch_resample(cetra_ctx *ctx, const cetra_plan *plan, const double *time,
                            const float *flux, const float *err, int64_t n, float2 *grid);
// status: set to CETRA_ETIMEOUT if a staging copy's bounded wait gave up (outputs NaN).
cudaError_t launch_linear(cetra_ctx *ctx, const cetra_plan *plan, const float2 *grid, float2 *ab,
                          float *depth, float *var, float *dlogl, int *status);
// Dynamic shared memory of the linear kernel: the table chunk and the grid span, each with
// two spare cells (a one-cell shift lines global 16-byte units up with shared ones).
inline size_t linear_smem_bytes(int p, int threads, int kc) {
    return ((size_t)((kc + 3) & ~1) + (size_t)p * threads * LIN_RB + (size_t)kc + 2) *
           sizeof(float) * 2;
}
cudaError_t launch_fold(cetra_ctx *ctx, const cetra_plan *plan, const float2 *ab,
                        const double *periods, int K, const uint8_t *mask,
                        unsigned long long *keys, int *status);
cudaError_t launch_finalize(cetra_ctx *ctx, const cetra_plan *plan, const float2 *ab,
                            const double *periods, int K, const unsigned long long *keys,
                            const int *status, double *dlogl, double *t0, double *dur, double *depth, double *var,
                            int64_t *oi, int32_t *oj);
cudaError_t launch_logl0(cetra_ctx *ctx, const cetra_plan *plan, const float2 *grid,
                         double *out);
cudaError_t linear_configure(cetra_plan *plan, const cetra_ctx *ctx);

// Batched form (kernels.cu). `stream` is the batch's own stream (capturable).
cudaError_t launch_batch_resample(cudaStream_t stream, int num_sms, const cetra_plan *plan,
                                  const double *time, const float *flux, const float *err,
                                  int64_t n_points, const int64_t *pt_offsets, int n_curves,
                                  const batch_curve *curves, float2 *grid);
cudaError_t launch_batch_linear(cudaStream_t stream, const cetra_plan *plan, int threads,
                                const int64_t *tile_off, int n_curves, int64_t n_tiles,
                                const batch_curve *curves, const float2 *grid, float2 *ab,
                                int *status);
cudaError_t launch_batch_fold(cudaStream_t stream, int blocks, int variant, const cetra_plan *plan,
                              const float2 *ab, const batch_curve *curves,
                              const int64_t *group_off, int n_curves, int64_t n_items,
                              int *queue, unsigned long long *period_keys,
                              unsigned long long *curve_keys, int *status,
                              const int64_t *item_list, const unsigned long long *n_items_dev,
                              const int64_t *order_off, const int32_t *order_curve);
// Self-test of the bounded barrier wait (kernels.cu): d_out[0] = 1 if the wait gave up,
// d_out[1] its duration in units of 2^20 SM clocks (d_out may be NULL); a wait that gave up
// also stores CETRA_ETIMEOUT in *d_status, as the fold does (d_status may be NULL).
cudaError_t launch_wait_timeout_selftest(cudaStream_t stream, int *d_out, int *d_status = nullptr);
// Roofline microbenchmarks: one full wave of blocks (peak_grid), PEAK_THREADS threads each;
// *work = flop (FMA) or bytes loaded (shared memory) of one launch.
constexpr int PEAK_THREADS = 256;
int peak_grid(int num_sms, bool smem);
cudaError_t launch_peak(cudaStream_t stream, bool smem, int blocks, int iters, float *d_out,
                        double *work);
// Method neighbours (neighbours.cu): masking a detected signal, single-transit events.
cudaError_t launch_mask(cetra_ctx *ctx, const cetra_plan *plan, float2 *grid, double P,
                        double t0, double h, unsigned long long *counts);
size_t mono_scratch_words(const cetra_plan *plan, int max_events);
cudaError_t launch_monotransits(cetra_ctx *ctx, const cetra_plan *plan, const float2 *ab,
                                unsigned long long *scratch, int max_events,
                                cetra_event *events, int *n_events);
// Learned-proposal selection: per curve, the fold work items of its best period intervals
// (SEL_MAX_INTERVALS intervals at most).
constexpr int SEL_MAX_INTERVALS = 1024;
cudaError_t launch_batch_select(cudaStream_t stream, const batch_curve *curves,
                                const int64_t *group_off, int n_curves, const float *scores,
                                int n_int, double p_lo, double p_hi, double top_frac,
                                unsigned char *flags, int64_t *items, unsigned long long *counts);
cudaError_t launch_batch_features(cudaStream_t stream, int num_sms, const cetra_plan *plan,
                                  const float2 *ab, const batch_curve *curves, int n_curves,
                                  int n_bins, float *out);
cudaError_t launch_batch_finalize(cudaStream_t stream, const cetra_plan *plan, const float2 *ab,
                                  const batch_curve *curves, int n_curves,
                                  const unsigned long long *period_keys,
                                  const unsigned long long *curve_keys, const int *status,
                                  cetra_best *best);
cudaError_t batch_configure(const cetra_plan *plan);
int batch_fold_variants();
int batch_fold_blocks_per_sm(int variant);

int set_error(cetra_ctx *ctx, int code, const std::string &msg);
