// Learned period-interval proposal (not in the paper; a deployment aid for the periodic
// search of Sec. 2.3): a 1-D CNN reads the max-pooled linear-search likelihood ratios of a
// curve ([durations][bins]) and marks the bins that hold transits; a comb over that map
// scores log-spaced period intervals, and the fold then evaluates the best intervals first.
//
// Network: log1p(features) -> conv(Cin -> 32, k 9) ReLU -> conv(32 -> 32) ReLU ->
// conv(32 -> 32) ReLU -> conv(32 -> 1) -> logit per bin. Weights are kept in FP32 (the
// training copy) and used in BF16 (rounded to nearest even) by every kernel; sums are FP32.
// Training: binary cross-entropy with logits against per-bin transit labels (positive
// weight w+), Adam. All kernels are written here; nothing calls a library.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "internal.h"

namespace {

constexpr int CNN_K = 9;           // kernel width
constexpr int CNN_HALF = CNN_K / 2;
constexpr int CNN_C = 32;          // hidden channels
constexpr int CNN_LAYERS = 4;
constexpr int CONV_TT = 256;       // time bins per block
constexpr int CONV_RT = 8;         // time bins per thread
constexpr int CONV_RC = 8;         // output channels per thread
constexpr int CONV_THREADS = (CONV_TT / CONV_RT) * (CNN_C / CONV_RC);  // 128
constexpr size_t kCombSmemMax = 96 * 1024;  // maps up to 24,576 bins are staged in shared memory

// ------------------------------------------------------------------------------- kernels

// x0 = log1p(max(f, 0))
__global__ void cnn_prep_kernel(const float *__restrict__ f, float *__restrict__ x, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        x[i] = log1pf(fmaxf(f[i], 0.0f));
}

// y[b][co][t] = act(bias[co] + sum_ci sum_k w[co][ci][k] x[b][ci][t + k - 4]), zero padding.
// One block: all output channels (cout <= 32) of CONV_TT bins of one curve. Thread:
// CONV_RT consecutive bins x CONV_RC channels; the input window slides through registers
// and each (ci, k) weight is one broadcast shared load for CONV_RT FMAs.
__global__ void __launch_bounds__(CONV_THREADS)
cnn_conv_kernel(const float *__restrict__ x, const __nv_bfloat16 *__restrict__ w,
                const float *__restrict__ bias, float *__restrict__ y, int cin, int cout, int T,
                int relu) {
    extern __shared__ float cs[];
    float *ws = cs;                                // [cout][cin][9]
    float *xs = cs + cout * cin * CNN_K;           // [cin][CONV_TT + 8]
    const int b = blockIdx.y;
    const int t0 = blockIdx.x * CONV_TT;
    const int tid = threadIdx.x;
    for (int i = tid; i < cout * cin * CNN_K; i += blockDim.x) ws[i] = __bfloat162float(w[i]);
    const int span = CONV_TT + CNN_K - 1;
    const float *xb = x + (int64_t)b * cin * T;
    for (int i = tid; i < cin * span; i += blockDim.x) {
        const int ci = i / span, u = i % span;
        const int t = t0 + u - CNN_HALF;
        xs[i] = (t >= 0 && t < T) ? xb[(int64_t)ci * T + t] : 0.0f;
    }
    __syncthreads();
    const int tt = (tid % (CONV_TT / CONV_RT)) * CONV_RT;  // first bin of this thread
    const int cg = tid / (CONV_TT / CONV_RT);               // channel group
    float acc[CONV_RC][CONV_RT];
#pragma unroll
    for (int c = 0; c < CONV_RC; ++c)
#pragma unroll
        for (int r = 0; r < CONV_RT; ++r) acc[c][r] = 0.0f;
    const int co0 = cg * CONV_RC;
    for (int ci = 0; ci < cin; ++ci) {
        float xv[CONV_RT + CNN_K - 1];
#pragma unroll
        for (int u = 0; u < CONV_RT + CNN_K - 1; ++u) xv[u] = xs[ci * span + tt + u];
#pragma unroll
        for (int c = 0; c < CONV_RC; ++c) {
            if (co0 + c >= cout) break;
            const float *wr = ws + ((co0 + c) * cin + ci) * CNN_K;
#pragma unroll
            for (int k = 0; k < CNN_K; ++k) {
                const float wk = wr[k];
#pragma unroll
                for (int r = 0; r < CONV_RT; ++r) acc[c][r] = fmaf(wk, xv[r + k], acc[c][r]);
            }
        }
    }
    float *yb = y + (int64_t)b * cout * T;
#pragma unroll
    for (int c = 0; c < CONV_RC; ++c) {
        const int co = co0 + c;
        if (co >= cout) break;
        const float bb = bias ? bias[co] : 0.0f;
#pragma unroll
        for (int r = 0; r < CONV_RT; ++r) {
            float v = acc[c][r] + bb;
            if (relu) v = fmaxf(v, 0.0f);
            yb[(int64_t)co * T + t0 + tt + r] = v;
        }
    }
}

// Weight and bias gradients of one conv layer:
// dW[co][ci][k] += sum_{b,t} g[b][co][t] x[b][ci][t + k - 4],  db[co] += sum_{b,t} g[b][co][t].
// One block per (curve, CONV_TT bins): thread (ci, group of 4 co) slides a 9-wide input
// window along the tile; partial sums are added to the global gradient with atomics.
__global__ void __launch_bounds__(256)
cnn_wgrad_kernel(const float *__restrict__ x, const float *__restrict__ g,
                 float *__restrict__ dw, float *__restrict__ db, int cin, int cout, int T) {
    extern __shared__ float cs[];
    const int span = CONV_TT + CNN_K - 1;
    float *xs = cs;                 // [cin][span]
    float *gs = cs + cin * span;    // [cout][CONV_TT]
    const int b = blockIdx.y, t0 = blockIdx.x * CONV_TT, tid = threadIdx.x;
    const float *xb = x + (int64_t)b * cin * T;
    const float *gb = g + (int64_t)b * cout * T;
    for (int i = tid; i < cin * span; i += blockDim.x) {
        const int ci = i / span, u = i % span;
        const int t = t0 + u - CNN_HALF;
        xs[i] = (t >= 0 && t < T) ? xb[(int64_t)ci * T + t] : 0.0f;
    }
    for (int i = tid; i < cout * CONV_TT; i += blockDim.x)
        gs[i] = gb[(int64_t)(i / CONV_TT) * T + t0 + i % CONV_TT];
    __syncthreads();
    const int ci = tid % 32, cg = tid / 32;  // 32 input channels x 8 groups of 4 outputs
    if (ci < cin && cg * 4 < cout) {
        float acc[4][CNN_K];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int k = 0; k < CNN_K; ++k) acc[c][k] = 0.0f;
        float win[CNN_K];
#pragma unroll
        for (int k = 0; k < CNN_K; ++k) win[k] = xs[ci * span + k];
        for (int t = 0; t < CONV_TT; ++t) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int co = cg * 4 + c;
                const float gv = co < cout ? gs[co * CONV_TT + t] : 0.0f;
#pragma unroll
                for (int k = 0; k < CNN_K; ++k) acc[c][k] = fmaf(gv, win[k], acc[c][k]);
            }
#pragma unroll
            for (int k = 0; k < CNN_K - 1; ++k) win[k] = win[k + 1];
            win[CNN_K - 1] = xs[ci * span + min(t + CNN_K, span - 1)];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int co = cg * 4 + c;
            if (co >= cout) break;
#pragma unroll
            for (int k = 0; k < CNN_K; ++k) atomicAdd(&dw[(co * cin + ci) * CNN_K + k], acc[c][k]);
        }
    }
    if (tid < cout) {
        float s = 0.0f;
        for (int t = 0; t < CONV_TT; ++t) s += gs[tid * CONV_TT + t];
        atomicAdd(&db[tid], s);
    }
}

// wt[ci][co][k] = w[co][ci][8 - k]: the input gradient is a conv of g with these weights.
__global__ void cnn_transpose_kernel(const __nv_bfloat16 *__restrict__ w,
                                     __nv_bfloat16 *__restrict__ wt, int cin, int cout) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cin * cout * CNN_K) return;
    const int k = i % CNN_K, co = (i / CNN_K) % cout, ci = i / (CNN_K * cout);
    wt[i] = w[(co * cin + ci) * CNN_K + (CNN_K - 1 - k)];
}

// g *= (a > 0): back through ReLU.
__global__ void cnn_relu_back_kernel(float *__restrict__ g, const float *__restrict__ a,
                                     int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        if (!(a[i] > 0.0f)) g[i] = 0.0f;
}

// Weighted binary cross-entropy with logits, mean over bins:
// l = w+ y softplus(-z) + (1 - y) softplus(z);  dl/dz = (sigmoid(z) (w+ y + 1 - y) - w+ y) / n.
__global__ void cnn_bce_kernel(const float *__restrict__ z, const float *__restrict__ y,
                               float *__restrict__ g, int64_t n, float wpos,
                               double *__restrict__ loss) {
    __shared__ double red[32];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float inv = 1.0f / (float)n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float zi = z[i], yi = y[i];
        const float sp_pos = fmaxf(zi, 0.0f) + log1pf(expf(-fabsf(zi)));  // softplus(z)
        const float sp_neg = sp_pos - zi;                                 // softplus(-z)
        acc += (double)(wpos * yi * sp_neg + (1.0f - yi) * sp_pos);
        const float s = 1.0f / (1.0f + expf(-zi));
        g[i] = (s * (wpos * yi + 1.0f - yi) - wpos * yi) * inv;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) atomicAdd(loss, acc / (double)n);
    }
}

__global__ void cnn_sigmoid_kernel(const float *__restrict__ z, float *__restrict__ p, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        p[i] = 1.0f / (1.0f + expf(-z[i]));
}

__global__ void cnn_round_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb,
                                 int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

// Adam on the FP32 training copy.
__global__ void cnn_adam_kernel(float *__restrict__ w, const float *__restrict__ g,
                                float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                                float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Proposal map: m[b][t] = p[b][t] max_j max(f[b][j][t], 0), the network's transit
// probability times the best window LR of the bin (Sec. 2.2). (Measured against p times the
// window SNR and p^2 times the SNR: this weighting recovers the most injected planets.)
__global__ void cnn_map_kernel(const float *__restrict__ prob, const float *__restrict__ f,
                               int J, int T, int64_t n, float *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const int64_t b = x / T, t = x % T;
        const float *fb = f + b * J * T + t;
        float m = 0.0f;
        for (int j = 0; j < J; ++j) m = fmaxf(m, fb[(int64_t)j * T]);
        out[x] = prob[x] * m;
    }
}

// Period comb over per-bin maps p[b][t]: curve b has V = n_valid[b] valid bins of bw[b] days.
// Interval q has log-spaced edges lo = p_lo (p_hi / p_lo)^(q / n_int), hi = the same at q + 1
// (days), or blo, bhi in bins. Its trial periods are Pb_m = blo + (bhi - blo)(m + 1/2) / nP,
// m < nP = max(1, ceil((bhi - blo) V / blo)), so that the phase of the last epoch drifts by at
// most about one bin between neighbouring trials; trials below 1 bin or above V / 2 are
// skipped. Epochs run in 32.32 fixed point: F = floor(Pb 2^32 + 1/2), and for each phase
// ph < ceil(Pb) the epochs are t_e = (ph 2^32 + e F + 2^31) >> 32 < V; the score is
// sum_e p[t_e] / sqrt(E). The interval's score is the best of those, and 0 if none is positive.
// One block per (interval, curve); the curve's map is staged in shared memory when it fits.
// The trials' FP64 arithmetic (Pb, F, phase count) is done once per trial into shared memory,
// COMB_CHUNK trials at a time; the block's threads then share the (trial, phase) pairs of the
// chunk (consecutive lanes take consecutive phases of one trial) with 32-bit index arithmetic
// and a 64-bit fixed-point epoch loop.
constexpr int COMB_CHUNK = 256;
template <bool SMEM>
__global__ void cnn_comb_kernel(const float *__restrict__ p, const double *__restrict__ bw,
                                const int *__restrict__ n_valid, int T, double p_lo,
                                double p_hi, int n_int, float *__restrict__ scores) {
    extern __shared__ float cmap[];
    __shared__ unsigned long long trial_F[COMB_CHUNK];
    __shared__ uint32_t trial_nph[COMB_CHUNK];
    const int b = blockIdx.y, q = blockIdx.x;
    const int V = n_valid ? min(max(n_valid[b], 0), T) : T;
    const float *pb = p + (int64_t)b * T;
    if (SMEM) {
        for (int t = threadIdx.x; t < V; t += blockDim.x) cmap[t] = pb[t];
        __syncthreads();
    }
    const float *src = SMEM ? cmap : pb;
    const double lo = p_lo * pow(p_hi / p_lo, (double)q / n_int);
    const double hi = p_lo * pow(p_hi / p_lo, (double)(q + 1) / n_int);
    const double w = bw[b];
    float best = 0.0f;
    const double blo = w > 0.0 ? lo / w : 0.0, bhi = w > 0.0 ? hi / w : 0.0;  // in bins
    if (w > 0.0 && V > 0 && bhi >= 1.0 && blo <= 0.5 * (double)V) {  // uniform over the block
        const int64_t nP = max((int64_t)1, (int64_t)ceil((bhi - blo) * (double)V / blo));
        // phases of the longest trial (<= V / 2 < 2^30)
        const uint32_t nph = (uint32_t)ceil(fmin(bhi, 0.5 * (double)V));
        const uint64_t end = (uint64_t)V << 32;
        const int64_t per_chunk = min((int64_t)COMB_CHUNK, (int64_t)(0xFFFFFFFFu / nph));
        for (int64_t m0 = 0; m0 < nP; m0 += per_chunk) {
            const int cnt = (int)min(per_chunk, nP - m0);
            __syncthreads();  // the previous chunk's trials are no longer read
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                const double Pb = blo + (bhi - blo) * ((double)(m0 + i) + 0.5) / (double)nP;
                const bool ok = Pb >= 1.0 && Pb <= 0.5 * (double)V;
                trial_F[i] = ok ? (unsigned long long)floor(Pb * 4294967296.0 + 0.5) : 0ull;
                trial_nph[i] = ok ? (uint32_t)ceil(Pb) : 0u;
            }
            __syncthreads();
            const uint32_t pairs = (uint32_t)cnt * nph;
            for (uint32_t x = threadIdx.x; x < pairs; x += blockDim.x) {
                const uint32_t m = x / nph, ph = x - m * nph;
                if (ph >= trial_nph[m]) continue;
                const unsigned long long F = trial_F[m];
                float s = 0.0f;
                int E = 0;
                for (uint64_t acc = ((uint64_t)ph << 32) + (1ull << 31); acc < end; acc += F) {
                    s += src[acc >> 32];
                    ++E;
                }
                best = fmaxf(best, s / sqrtf((float)E));  // E >= 1: ph < ceil(Pb) <= V/2
            }
        }
    }
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_down_sync(0xFFFFFFFFu, best, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mx = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mx = fmaxf(mx, red[i]);
        scores[(int64_t)b * n_int + q] = mx;
    }
}

unsigned grid_for(int64_t n, int threads, int num_sms) {
    int64_t blocks = (n + threads - 1) / threads;
    if (blocks > (int64_t)num_sms * 32) blocks = (int64_t)num_sms * 32;
    return (unsigned)std::max<int64_t>(blocks, 1);
}

}  // namespace

// ------------------------------------------------------------------------------- host side

struct cetra_cnn {
    int device = 0;
    int cin = 0, T = 0, max_batch = 0;
    int ch_in[CNN_LAYERS], ch_out[CNN_LAYERS];
    int64_t w_off[CNN_LAYERS], b_off[CNN_LAYERS], n_params = 0;
    float *d_params = nullptr, *d_grads = nullptr, *d_m = nullptr, *d_v = nullptr;
    __nv_bfloat16 *d_wb = nullptr, *d_wt = nullptr;  // BF16 weights, transposed scratch
    float *d_act[CNN_LAYERS + 1] = {};  // act[0] = log1p(features), act[l + 1] = layer l output
    float *d_g = nullptr, *d_g2 = nullptr;  // gradient buffers [max_batch][32][T]
    double *d_loss = nullptr;
    void *d_mem = nullptr;
    int adam_step = 0;
};

namespace {

int cnn_fail(cetra_ctx *ctx, cudaError_t e, const char *what) {
    return set_error(ctx, CETRA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t conv_smem(int cin, int cout) {
    return ((size_t)cout * cin * CNN_K + (size_t)cin * (CONV_TT + CNN_K - 1)) * sizeof(float);
}
size_t wgrad_smem(int cin, int cout) {
    return ((size_t)cin * (CONV_TT + CNN_K - 1) + (size_t)cout * CONV_TT) * sizeof(float);
}

cudaError_t conv(cetra_ctx *ctx, const float *x, const __nv_bfloat16 *w, const float *bias,
                 float *y, int cin, int cout, int T, int B, int relu) {
    dim3 grid((unsigned)(T / CONV_TT), (unsigned)B);
    cnn_conv_kernel<<<grid, CONV_THREADS, conv_smem(cin, cout), ctx->stream>>>(x, w, bias, y, cin,
                                                                             cout, T, relu);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t forward(cetra_ctx *ctx, cetra_cnn *n, const float *features, int B) {
    const int64_t nin = (int64_t)B * n->cin * n->T;
    cnn_prep_kernel<<<grid_for(nin, 256, ctx->num_sms), 256, 0, ctx->stream>>>(features,
                                                                                n->d_act[0], nin);
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        e = conv(ctx, n->d_act[l], n->d_wb + n->w_off[l], n->d_params + n->b_off[l],
                 n->d_act[l + 1], n->ch_in[l], n->ch_out[l], n->T, B, l < CNN_LAYERS - 1);
        if (e) return e;
    }
    return cudaSuccess;
}

cudaError_t round_weights(cetra_ctx *ctx, cetra_cnn *n) {
    cnn_round_kernel<<<(unsigned)((n->n_params + 255) / 256), 256, 0, ctx->stream>>>(
        n->d_params, n->d_wb, n->n_params);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int cetra_cnn_create(cetra_ctx *ctx, int in_channels, int n_bins, int max_batch, uint64_t seed,
                     cetra_cnn **out) {
    if (!ctx || !out) return set_error(ctx, CETRA_EINVAL, "cnn_create: NULL argument");
    *out = nullptr;
    if (in_channels < 1 || in_channels > CNN_C || n_bins < CONV_TT || n_bins % CONV_TT ||
        max_batch < 1)
        return set_error(ctx, CETRA_EINVAL,
                         "cnn_create: need 1 <= in_channels <= 32, n_bins a multiple of 256, max_batch >= 1");
    cetra_cnn *n = new (std::nothrow) cetra_cnn;
    if (!n) return set_error(ctx, CETRA_ENOMEM, "cnn_create: host allocation");
    n->device = ctx->device;
    n->cin = in_channels;
    n->T = n_bins;
    n->max_batch = max_batch;
    int64_t off = 0;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        n->ch_in[l] = l == 0 ? in_channels : CNN_C;
        n->ch_out[l] = l == CNN_LAYERS - 1 ? 1 : CNN_C;
        n->w_off[l] = off;
        off += (int64_t)n->ch_out[l] * n->ch_in[l] * CNN_K;
        n->b_off[l] = off;
        off += n->ch_out[l];
    }
    n->n_params = off;
    // He-normal weights, zero biases, from a seeded generator
    std::vector<float> init((size_t)off, 0.0f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.0f, 1.0f);
    for (int l = 0; l < CNN_LAYERS; ++l) {
        const float sd = std::sqrt(2.0f / (float)(n->ch_in[l] * CNN_K));
        for (int64_t i = 0; i < (int64_t)n->ch_out[l] * n->ch_in[l] * CNN_K; ++i)
            init[(size_t)(n->w_off[l] + i)] = sd * nd(rng);
    }
    const size_t P = (size_t)off;
    const size_t act = (size_t)max_batch * CNN_C * n_bins;
    const size_t bytes = P * sizeof(float) * 4 + P * sizeof(__nv_bfloat16) * 2 + 256 * 8 +
                         act * sizeof(float) * (CNN_LAYERS + 1 + 2) + 1024;
    device_guard dguard(ctx->device);
    cudaError_t e = dguard.status;
    if (!e) e = cudaMalloc(&n->d_mem, bytes);
    if (e) {
        delete n;
        return set_error(ctx, CETRA_ENOMEM, "cnn_create: device allocation");
    }
    char *p = static_cast<char *>(n->d_mem);
    auto take = [&](size_t nb) {
        char *r = p;
        p += (nb + 255) & ~(size_t)255;
        return r;
    };
    n->d_params = reinterpret_cast<float *>(take(P * 4));
    n->d_grads = reinterpret_cast<float *>(take(P * 4));
    n->d_m = reinterpret_cast<float *>(take(P * 4));
    n->d_v = reinterpret_cast<float *>(take(P * 4));
    n->d_wb = reinterpret_cast<__nv_bfloat16 *>(take(P * 2));
    n->d_wt = reinterpret_cast<__nv_bfloat16 *>(take(P * 2));
    n->d_loss = reinterpret_cast<double *>(take(8));
    for (int l = 0; l <= CNN_LAYERS; ++l) n->d_act[l] = reinterpret_cast<float *>(take(act * 4));
    n->d_g = reinterpret_cast<float *>(take(act * 4));
    n->d_g2 = reinterpret_cast<float *>(take(act * 4));
    e = cudaMemcpy(n->d_params, init.data(), P * 4, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(n->d_m, 0, P * 4);
    if (!e) e = cudaMemset(n->d_v, 0, P * 4);
    if (!e)
        e = cudaFuncSetAttribute(cnn_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)conv_smem(CNN_C, CNN_C));
    if (!e)
        e = cudaFuncSetAttribute(cnn_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)wgrad_smem(CNN_C, CNN_C));
    if (!e) e = round_weights(ctx, n);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    if (e) {
        cudaFree(n->d_mem);
        delete n;
        return cnn_fail(ctx, e, "cnn_create");
    }
    *out = n;
    return CETRA_OK;
}

void cetra_cnn_destroy(cetra_cnn *n) {
    if (!n) return;
    device_guard dguard(n->device);
    cudaFree(n->d_mem);
    delete n;
}

int64_t cetra_cnn_param_count(const cetra_cnn *n) { return n ? n->n_params : 0; }

int cetra_cnn_shape(const cetra_cnn *n, int *in_channels, int *n_bins, int *max_batch) {
    if (!n) return CETRA_EINVAL;
    if (in_channels) *in_channels = n->cin;
    if (n_bins) *n_bins = n->T;
    if (max_batch) *max_batch = n->max_batch;
    return CETRA_OK;
}

int cetra_cnn_get_params(cetra_ctx *ctx, const cetra_cnn *n, float *host) {
    if (!ctx || !n || !host) return set_error(ctx, CETRA_EINVAL, "cnn_get_params: NULL argument");
    device_guard dguard(ctx->device);
    cudaError_t e = dguard.status;
    if (!e) e = cudaMemcpyAsync(host, n->d_params, (size_t)n->n_params * 4,
                                    cudaMemcpyDeviceToHost, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    return e ? cnn_fail(ctx, e, "cnn_get_params") : CETRA_OK;
}

int cetra_cnn_set_params(cetra_ctx *ctx, cetra_cnn *n, const float *host) {
    if (!ctx || !n || !host) return set_error(ctx, CETRA_EINVAL, "cnn_set_params: NULL argument");
    device_guard dguard(ctx->device);
    cudaError_t e = dguard.status;
    if (!e) e = cudaMemcpyAsync(n->d_params, host, (size_t)n->n_params * 4,
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (!e) e = round_weights(ctx, n);
    // new parameters start a new optimisation: clear Adam's moments and step count
    if (!e) e = cudaMemsetAsync(n->d_m, 0, (size_t)n->n_params * 4, ctx->stream);
    if (!e) e = cudaMemsetAsync(n->d_v, 0, (size_t)n->n_params * 4, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    n->adam_step = 0;
    return e ? cnn_fail(ctx, e, "cnn_set_params") : CETRA_OK;
}

int cetra_cnn_forward(cetra_ctx *ctx, cetra_cnn *n, const float *d_features, int B,
                      float *d_prob) {
    if (!ctx || !n || !d_features || !d_prob || B < 1 || B > n->max_batch)
        return set_error(ctx, CETRA_EINVAL, "cnn_forward: bad argument");
    device_guard dguard(ctx->device);
    cudaError_t e = dguard.status;
    if (!e) e = forward(ctx, n, d_features, B);
    if (!e) {
        const int64_t m = (int64_t)B * n->T;
        cnn_sigmoid_kernel<<<grid_for(m, 256, ctx->num_sms), 256, 0, ctx->stream>>>(
            n->d_act[CNN_LAYERS], d_prob, m);
        ctx->launches++;
        e = cudaGetLastError();
    }
    return e ? cnn_fail(ctx, e, "cnn_forward") : CETRA_OK;
}

int cetra_cnn_backward(cetra_ctx *ctx, cetra_cnn *n, const float *d_features,
                       const float *d_labels, int B, float pos_weight, double *loss,
                       float *host_grads) {
    if (!ctx || !n || !d_features || !d_labels || B < 1 || B > n->max_batch)
        return set_error(ctx, CETRA_EINVAL, "cnn_backward: bad argument");
    const int T = n->T;
    device_guard dguard(ctx->device);
    cudaError_t e = dguard.status;
    if (!e) e = forward(ctx, n, d_features, B);
    if (!e) e = cudaMemsetAsync(n->d_grads, 0, (size_t)n->n_params * 4, ctx->stream);
    if (!e) e = cudaMemsetAsync(n->d_loss, 0, sizeof(double), ctx->stream);
    const int64_t m = (int64_t)B * T;
    if (!e) {
        cnn_bce_kernel<<<grid_for(m, 256, ctx->num_sms), 256, 0, ctx->stream>>>(
            n->d_act[CNN_LAYERS], d_labels, n->d_g, m, pos_weight, n->d_loss);
        ctx->launches++;
        e = cudaGetLastError();
    }
    float *g = n->d_g, *g_next = n->d_g2;
    for (int l = CNN_LAYERS - 1; l >= 0 && !e; --l) {
        const int cin = n->ch_in[l], cout = n->ch_out[l];
        if (l < CNN_LAYERS - 1) {  // back through this layer's ReLU
            const int64_t cnt = (int64_t)B * cout * T;
            cnn_relu_back_kernel<<<grid_for(cnt, 256, ctx->num_sms), 256, 0, ctx->stream>>>(
                g, n->d_act[l + 1], cnt);
            ctx->launches++;
            if ((e = cudaGetLastError())) break;
        }
        dim3 grid((unsigned)(T / CONV_TT), (unsigned)B);
        cnn_wgrad_kernel<<<grid, 256, wgrad_smem(cin, cout), ctx->stream>>>(
            n->d_act[l], g, n->d_grads + n->w_off[l], n->d_grads + n->b_off[l], cin, cout, T);
        ctx->launches++;
        if ((e = cudaGetLastError())) break;
        if (l > 0) {  // gradient of the layer input: conv of g with the flipped, transposed weights
            const int nw = cin * cout * CNN_K;
            cnn_transpose_kernel<<<(nw + 255) / 256, 256, 0, ctx->stream>>>(
                n->d_wb + n->w_off[l], n->d_wt, cin, cout);
            ctx->launches++;
            if ((e = cudaGetLastError())) break;
            if ((e = conv(ctx, g, n->d_wt, nullptr, g_next, cout, cin, T, B, 0))) break;
            std::swap(g, g_next);
        }
    }
    if (!e && loss) e = cudaMemcpyAsync(loss, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (!e && host_grads)
        e = cudaMemcpyAsync(host_grads, n->d_grads, (size_t)n->n_params * 4,
                            cudaMemcpyDeviceToHost, ctx->stream);
    if (!e && (loss || host_grads)) e = cudaStreamSynchronize(ctx->stream);
    return e ? cnn_fail(ctx, e, "cnn_backward") : CETRA_OK;
}

int cetra_cnn_adam(cetra_ctx *ctx, cetra_cnn *n, float lr, float beta1, float beta2, float eps) {
    if (!ctx || !n) return set_error(ctx, CETRA_EINVAL, "cnn_adam: NULL argument");
    device_guard dguard(ctx->device);
    if (dguard.status) return cnn_fail(ctx, dguard.status, "cnn_adam");
    n->adam_step++;
    const float c1 = 1.0f - std::pow(beta1, (float)n->adam_step);
    const float c2 = 1.0f - std::pow(beta2, (float)n->adam_step);
    cnn_adam_kernel<<<(unsigned)((n->n_params + 255) / 256), 256, 0, ctx->stream>>>(
        n->d_params, n->d_grads, n->d_m, n->d_v, n->n_params, lr, beta1, beta2, eps, c1, c2);
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (!e) e = round_weights(ctx, n);
    return e ? cnn_fail(ctx, e, "cnn_adam") : CETRA_OK;
}

int cetra_cnn_map(cetra_ctx *ctx, const float *d_prob, const float *d_features, int B,
                  int n_dur, int n_bins, float *d_map) {
    if (!ctx || !d_prob || !d_features || !d_map || B < 1 || n_dur < 1 || n_bins < 1)
        return set_error(ctx, CETRA_EINVAL, "cnn_map: bad argument");
    device_guard dguard(ctx->device);
    if (dguard.status) return cnn_fail(ctx, dguard.status, "cnn_map");
    const int64_t n = (int64_t)B * n_bins;
    cnn_map_kernel<<<grid_for(n, 256, ctx->num_sms), 256, 0, ctx->stream>>>(d_prob, d_features,
                                                                           n_dur, n_bins, n, d_map);
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    return e ? cnn_fail(ctx, e, "cnn_map") : CETRA_OK;
}

int cetra_cnn_comb(cetra_ctx *ctx, const float *d_prob, int B, int n_bins,
                   const double *d_bin_days, const int *d_n_valid, double p_lo, double p_hi,
                   int n_intervals, float *d_scores) {
    if (!ctx || !d_prob || !d_bin_days || !d_scores || B < 1 || B > 65535 || n_bins < 1 ||
        n_bins > (1 << 30) || n_intervals < 1 || !(p_lo > 0.0) || !(p_hi > p_lo))
        return set_error(ctx, CETRA_EINVAL, "cnn_comb: bad argument");
    device_guard dguard(ctx->device);
    if (dguard.status) return cnn_fail(ctx, dguard.status, "cnn_comb");
    dim3 grid((unsigned)n_intervals, (unsigned)B);
    const size_t smem = (size_t)n_bins * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (smem <= kCombSmemMax) {
        e = cudaFuncSetAttribute(cnn_comb_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (!e)
            cnn_comb_kernel<true><<<grid, 256, smem, ctx->stream>>>(
                d_prob, d_bin_days, d_n_valid, n_bins, p_lo, p_hi, n_intervals, d_scores);
    } else {
        cnn_comb_kernel<false><<<grid, 256, 0, ctx->stream>>>(
            d_prob, d_bin_days, d_n_valid, n_bins, p_lo, p_hi, n_intervals, d_scores);
    }
    ctx->launches++;
    if (!e) e = cudaGetLastError();
    return e ? cnn_fail(ctx, e, "cnn_comb") : CETRA_OK;
}

}  // extern "C"
