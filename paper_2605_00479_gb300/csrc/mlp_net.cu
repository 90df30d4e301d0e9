// mlp_net.cu -- the telegraph surrogate network on the tensor cores.
//
// A multilayer perceptron maps 4 standardised log-parameters of the
// telegraph model (log kon, log koff, log km, log gamma; zero-padded to 16)
// through three hidden layers of 256 GELU units to 128 logits; a softmax over
// them is the predicted law of the mRNA count (bins 0..127, the last one
// holding >= 127).  Training minimises the cross-entropy against histograms
// that the SSA engine produces, with AdamW on fp32 master weights.
//
// Every matrix product is the tcgen05 GEMM of mlp_tc.cu, with bf16 operands
// and fp32 accumulation.  The epilogue of each GEMM writes the next GEMM's
// operands directly in the packed core-matrix layout (and, for the weight
// gradients, the transposed copy), so no separate re-layout pass exists.
//
// Parameter vector (fp32), in this order: W1 [256][16] (input columns 4..15
// are padding and stay zero), b1 [256], W2 [256][256], b2, W3 [256][256], b3,
// W4 [128][256], b4 [128].
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "../../include/ssa.h"
#include "mlp_tc.cuh"

namespace {

constexpr int kIn[4] = {16, 256, 256, 256};
constexpr int kOut[4] = {256, 256, 256, 128};
constexpr int64_t kOffW[4] = {0, 4352, 70144, 135936};
constexpr int64_t kOffB[4] = {4096, 69888, 135680, 168704};
constexpr int64_t kParams = 168832;
constexpr int kBins = 128;

__device__ __forceinline__ uint16_t f2bf(float x)
{
    uint16_t h;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
    return h;
}

// features [B][4] -> X0 packed [Bpad][16] and its transpose [16][Bpad]
__global__ void pack_features_kernel(const float *feat, int B, int Bpad, uint8_t *x_pk, uint8_t *xT_pk)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Bpad) return;
    uint16_t h[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) h[c] = (r < B && c < 4) ? f2bf(feat[(int64_t)r * 4 + c]) : (uint16_t)0;
    uint4 lo, hi;
    lo.x = h[0] | (h[1] << 16); lo.y = h[2] | (h[3] << 16); lo.z = h[4] | (h[5] << 16); lo.w = h[6] | (h[7] << 16);
    hi.x = h[8] | (h[9] << 16); hi.y = h[10] | (h[11] << 16); hi.z = h[12] | (h[13] << 16); hi.w = h[14] | (h[15] << 16);
    *reinterpret_cast<uint4 *>(x_pk + mlp::packed_offset(r, 0, 16)) = lo;
    *reinterpret_cast<uint4 *>(x_pk + mlp::packed_offset(r, 8, 16)) = hi;
    if (xT_pk) {
#pragma unroll
        for (int c = 0; c < 16; ++c) *reinterpret_cast<uint16_t *>(xT_pk + mlp::packed_offset(c, r, Bpad)) = h[c];
    }
}

// bf16 copies of one weight matrix W [out][in]: packed W (rows out, C = in)
// and packed W^T (rows in, C = out).
__global__ void refresh_weights_kernel(const float *W, int out, int in, uint8_t *w_pk, uint8_t *wT_pk)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)out * in) return;
    const int n = (int)(i / in), k = (int)(i % in);
    const uint16_t h = f2bf(W[i]);
    *reinterpret_cast<uint16_t *>(w_pk + mlp::packed_offset(n, k, in)) = h;
    *reinterpret_cast<uint16_t *>(wT_pk + mlp::packed_offset(k, n, out)) = h;
}

// One warp per row: softmax of 128 logits; with targets, the cross-entropy,
// d loss / d logits = (q - p) / B (bf16, packed and transposed) and the
// output-bias gradient; without, the probabilities.
__global__ void softmax_ce_kernel(const float *logits, const float *targets, int B, int Bpad, float *probs,
                                  uint8_t *dz_pk, uint8_t *dzT_pk, float *bias_grad, float *loss)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= Bpad) return;
    const int r = warp;
    const bool valid = r < B;
    float z[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) z[i] = valid ? logits[(int64_t)r * kBins + lane * 4 + i] : 0.0f;
    float mx = fmaxf(fmaxf(z[0], z[1]), fmaxf(z[2], z[3]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    float e[4], sum = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        e[i] = expf(z[i] - mx);
        sum += e[i];
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    const float lse = logf(sum);
    if (!targets) {
        if (valid) {
#pragma unroll
            for (int i = 0; i < 4; ++i) probs[(int64_t)r * kBins + lane * 4 + i] = e[i] / sum;
        }
        return;
    }
    uint16_t h[4];
    float ce = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float d = 0.0f;
        if (valid) {
            const float p = targets[(int64_t)r * kBins + lane * 4 + i];
            const float q = e[i] / sum;
            d = (q - p) / (float)B;
            ce -= p * (z[i] - mx - lse);
            atomicAdd(&bias_grad[lane * 4 + i], d);
        }
        h[i] = f2bf(d);
    }
    uint2 v;
    v.x = h[0] | (h[1] << 16);
    v.y = h[2] | (h[3] << 16);
    *reinterpret_cast<uint2 *>(dz_pk + mlp::packed_offset(r, lane * 4, kBins)) = v;
#pragma unroll
    for (int i = 0; i < 4; ++i) *reinterpret_cast<uint16_t *>(dzT_pk + mlp::packed_offset(lane * 4 + i, r, Bpad)) = h[i];
    for (int o = 16; o > 0; o >>= 1) ce += __shfl_xor_sync(0xFFFFFFFFu, ce, o);
    if (lane == 0 && valid) atomicAdd(loss, ce / (float)B);
}

// AdamW on the fp32 master parameters (weight decay on weights only; the
// padding columns of W1 stay zero).
__device__ __forceinline__ void adamw_update(int64_t i, float *theta, const float *grad, float *m, float *v, float lr,
                                             float beta1, float beta2, float eps, float wd, float bc1, float bc2)
{
    constexpr int64_t b0 = kOffB[0], w1 = kOffW[1], b1 = kOffB[1], w2 = kOffW[2], b2 = kOffB[2], w3 = kOffW[3],
                      b3 = kOffB[3];
    if (i < b0 && (i % 16) >= 4) return;   // W1 padding
    const bool is_bias = (i >= b0 && i < w1) || (i >= b1 && i < w2) || (i >= b2 && i < w3) || i >= b3;
    const float g = grad[i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * g;
    const float vi = beta2 * v[i] + (1.0f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mhat = mi / bc1, vhat = vi / bc2;
    float t = theta[i];
    if (!is_bias) t -= lr * wd * t;
    t -= lr * mhat / (sqrtf(vhat) + eps);
    theta[i] = t;
}

__global__ void adamw_kernel(float *theta, const float *grad, float *m, float *v, int64_t n, float lr, float beta1,
                             float beta2, float eps, float wd, float bc1, float bc2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) adamw_update(i, theta, grad, m, v, lr, beta1, beta2, eps, wd, bc1, bc2);
}

// Schedule of a device-driven training run: the step counters and this
// step's learning rate and bias corrections live in device memory, so one
// captured step replays unchanged.
struct TrainSched {
    long long adam_step;   // AdamW steps taken so far (all runs)
    long long local;       // step index within this run
    float lr, bc1, bc2;
};

constexpr float kBeta1 = 0.9f, kBeta2 = 0.999f, kEps = 1e-8f;

// Same values as the host computes for one train step: the cosine schedule in
// binary64 rounded to binary32, and 1 - beta^t in binary64 (beta widened from
// binary32) rounded once.
__global__ void schedule_kernel(TrainSched *sc, long long n_steps, float lr_max, float lr_min)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const long long k = sc->local;
    const double frac = n_steps > 1 ? (double)k / (double)(n_steps - 1) : 0.0;
    sc->lr = (float)((double)lr_min + 0.5 * ((double)lr_max - (double)lr_min) * (1.0 + cos(3.141592653589793 * frac)));
    const long long t = sc->adam_step + 1;
    sc->bc1 = (float)(1.0 - pow((double)kBeta1, (double)t));
    sc->bc2 = (float)(1.0 - pow((double)kBeta2, (double)t));
    sc->adam_step = t;
}

__global__ void adamw_sched_kernel(float *theta, const float *grad, float *m, float *v, int64_t n,
                                   const TrainSched *sc, float wd)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) adamw_update(i, theta, grad, m, v, sc->lr, kBeta1, kBeta2, kEps, wd, sc->bc1, sc->bc2);
}

// Minibatch of step `local`: rows (local * B + j) mod n_rows, one block per row.
__global__ void gather_batch_kernel(const float *features, const float *targets, int64_t n_rows, int B,
                                    const TrainSched *sc, float *feat_b, float *targ_b)
{
    const int j = blockIdx.x;
    if (j >= B) return;
    const int64_t row = (int64_t)((sc->local * (long long)B + j) % n_rows);
    for (int c = threadIdx.x; c < kBins; c += blockDim.x) targ_b[(int64_t)j * kBins + c] = targets[row * kBins + c];
    if (threadIdx.x < 4) feat_b[(int64_t)j * 4 + threadIdx.x] = features[row * 4 + threadIdx.x];
}

// End of a step: record its loss every `every` steps, advance the step index.
__global__ void finish_step_kernel(const float *loss, TrainSched *sc, long long every, float *trace)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const long long k = sc->local;
    if (trace && k % every == 0) trace[k / every] = *loss;
    sc->local = k + 1;
}

// Normalised histogram of one species' counts per parameter set:
// hist[s][b] = #{trajectories of set s with min(count, bins-1) = b} / traj_per_set.
__global__ void histogram_kernel(const int32_t *counts, int64_t traj_per_set, int bins, float *hist)
{
    extern __shared__ unsigned int hcount[];
    const int64_t s = blockIdx.x;
    for (int b = threadIdx.x; b < bins; b += blockDim.x) hcount[b] = 0;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < traj_per_set; t += blockDim.x) {
        int c = counts[s * traj_per_set + t];
        c = c < 0 ? 0 : (c >= bins ? bins - 1 : c);
        atomicAdd(&hcount[c], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < bins; b += blockDim.x) hist[s * bins + b] = (float)hcount[b] / (float)traj_per_set;
}

// W1 between two histograms per row: sum_b |CDF_p(b) - CDF_q(b)| (one warp per row).
__global__ void hist_w1_kernel(const float *p, const float *q, int64_t rows, int bins, float *w1)
{
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    float carry = 0.0f, acc = 0.0f;
    for (int b0 = 0; b0 < bins; b0 += 32) {
        const int b = b0 + lane;
        float d = b < bins ? p[r * bins + b] - q[r * bins + b] : 0.0f;
        // inclusive prefix sum over the warp
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(0xFFFFFFFFu, d, o);
            if (lane >= o) d += y;
        }
        const float cdf = carry + d;
        acc += b < bins ? fabsf(cdf) : 0.0f;
        carry = __shfl_sync(0xFFFFFFFFu, cdf, 31);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0) w1[r] = acc;
}

// Expected W1 between a law p and the empirical histogram of n draws from it,
// per row: sum_b E|F_n(b) - F(b)| with n F_n(b) binomial(n, F(b)), each term
// by its normal approximation sqrt(2 F (1 - F) / (pi n)) (one warp per row).
// 1 - F is taken as the remaining mass T - F (T the row total, summed in the
// same order), so bins past the last nonzero probability contribute exactly 0.
__global__ void hist_w1_noise_kernel(const float *p, int64_t rows, int bins, float n, float *out)
{
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const float scale = 2.0f / (3.14159265358979f * n);
    // inclusive prefix sums of the row, 32 bins at a time
    auto prefix = [&](int b0, float carry) {
        const int b = b0 + lane;
        float d = b < bins ? p[r * bins + b] : 0.0f;
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(0xFFFFFFFFu, d, o);
            if (lane >= o) d += y;
        }
        return carry + d;
    };
    float total = 0.0f;
    for (int b0 = 0; b0 < bins; b0 += 32) total = __shfl_sync(0xFFFFFFFFu, prefix(b0, total), 31);
    float carry = 0.0f, acc = 0.0f;
    for (int b0 = 0; b0 < bins; b0 += 32) {
        const int b = b0 + lane;
        const float F = prefix(b0, carry);
        const float rest = fmaxf(total - F, 0.0f);
        acc += b < bins - 1 ? sqrtf(scale * fmaxf(F, 0.0f) * rest) : 0.0f;
        carry = __shfl_sync(0xFFFFFFFFu, F, 31);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0) out[r] = acc;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Deterministic He-normal initialisation on the host (splitmix64 + Box-Muller).
uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

struct ssa_surrogate {
    int max_batch, bpad_max;
    float *theta, *m, *v, *grad;
    uint8_t *w_pk[4], *wT_pk[4];
    uint8_t *x_pk, *xT_pk;
    float *z[3];
    uint8_t *y_pk[3], *yT_pk[3];
    float *logits;
    uint8_t *dz4_pk, *dz4T_pk;
    uint8_t *dz_pk[3], *dzT_pk[3];
    float *loss;
    int *error;
    int64_t step;
    float *feat_b, *targ_b;   // minibatch of a device-driven training run
    void *sched;              // its TrainSched
    char *arena;
};

namespace {

cudaError_t refresh_all(ssa_surrogate *s, cudaStream_t st)
{
    for (int l = 0; l < 4; ++l) {
        const int64_t n = (int64_t)kOut[l] * kIn[l];
        refresh_weights_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->theta + kOffW[l], kOut[l], kIn[l],
                                                                          s->w_pk[l], s->wT_pk[l]);
    }
    return cudaGetLastError();
}

mlp::GemmArgs gemm_args(ssa_surrogate *s)
{
    mlp::GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.error = s->error;
    return g;
}

// forward pass; with_transposes writes the copies the backward pass needs
cudaError_t forward(ssa_surrogate *s, int B, int Bpad, const float *features, bool with_transposes, cudaStream_t st)
{
    pack_features_kernel<<<(Bpad + 127) / 128, 128, 0, st>>>(features, B, Bpad, s->x_pk,
                                                              with_transposes ? s->xT_pk : nullptr);
    cudaError_t e = cudaGetLastError();
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
        mlp::GemmArgs g = gemm_args(s);
        g.A = l == 0 ? s->x_pk : s->y_pk[l - 1];
        g.lda_cols = kIn[l];
        g.B = s->w_pk[l];
        g.ldb_cols = kIn[l];
        g.M = Bpad;
        g.m_valid = B;
        g.N = kOut[l];
        g.K = kIn[l];
        g.kchunk = kIn[l];
        g.bias = s->theta + kOffB[l];
        if (l < 3) {
            g.epi = mlp::EPI_HIDDEN_FWD;
            g.fout = s->z[l];
            g.ld_fout = 256;
            g.pk_out = s->y_pk[l];
            g.pkT_out = with_transposes ? s->yT_pk[l] : nullptr;
            g.pkT_cols = Bpad;
        } else {
            g.epi = mlp::EPI_LOGITS;
            g.fout = s->logits;
            g.ld_fout = kBins;
        }
        e = mlp::launch_gemm(g, st);
    }
    return e;
}

cudaError_t backward(ssa_surrogate *s, int B, int Bpad, const float *targets, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(s->grad, 0, sizeof(float) * kParams, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->loss, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    softmax_ce_kernel<<<(Bpad * 32 + 255) / 256, 256, 0, st>>>(s->logits, targets, B, Bpad, nullptr, s->dz4_pk,
                                                               s->dz4T_pk, s->grad + kOffB[3], s->loss);
    e = cudaGetLastError();
    // layer l = 3..0: weight gradient, then (l > 0) the gradient of the layer below
    for (int l = 3; l >= 0 && e == cudaSuccess; --l) {
        const uint8_t *dzT = l == 3 ? s->dz4T_pk : s->dzT_pk[l];
        const uint8_t *dz = l == 3 ? s->dz4_pk : s->dz_pk[l];
        mlp::GemmArgs g = gemm_args(s);   // dW_l = dZ_l^T X_l  (reduction over the batch)
        g.A = dzT;
        g.lda_cols = Bpad;
        g.B = l == 0 ? s->xT_pk : s->yT_pk[l - 1];
        g.ldb_cols = Bpad;
        g.M = kOut[l];
        g.m_valid = kOut[l];
        g.N = kIn[l];
        g.K = Bpad;
        g.kchunk = Bpad < 256 ? Bpad : 256;
        g.epi = mlp::EPI_STORE_F32;
        g.fout = s->grad + kOffW[l];
        g.ld_fout = kIn[l];
        e = mlp::launch_gemm(g, st);
        if (l == 0 || e != cudaSuccess) break;
        mlp::GemmArgs d = gemm_args(s);   // dZ_{l-1} = (dZ_l W_l) * gelu'(Z_{l-1})
        d.A = dz;
        d.lda_cols = kOut[l];
        d.B = s->wT_pk[l];
        d.ldb_cols = kOut[l];
        d.M = Bpad;
        d.m_valid = B;
        d.N = kIn[l];
        d.K = kOut[l];
        d.kchunk = kOut[l];
        d.epi = mlp::EPI_HIDDEN_BWD;
        d.zin = s->z[l - 1];
        d.pk_out = s->dz_pk[l - 1];
        d.pkT_out = s->dzT_pk[l - 1];
        d.pkT_cols = Bpad;
        d.bias_grad = s->grad + kOffB[l - 1];
        e = mlp::launch_gemm(d, st);
    }
    return e;
}

int check_batch(const ssa_surrogate *s, int B)
{
    if (!s) return SSA_EINVAL;
    if (B < 1 || B > s->max_batch) return SSA_EINVAL;
    return SSA_OK;
}

int bpad_of(int B) { return (B + 255) / 256 * 256; }

}  // namespace

extern "C" {

int64_t ssa_surrogate_param_count(void) { return kParams; }

int ssa_surrogate_create(int max_batch, uint64_t seed, ssa_surrogate **out)
{
    if (!out || max_batch < 1 || max_batch > (1 << 20)) return SSA_EINVAL;
    *out = nullptr;
    ssa_surrogate *s = new (std::nothrow) ssa_surrogate;
    if (!s) return SSA_ENOMEM;
    std::memset(s, 0, sizeof(*s));
    s->max_batch = max_batch;
    const int Bp = bpad_of(max_batch);
    s->bpad_max = Bp;
    size_t sizes[64];
    int n = 0;
    for (int q = 0; q < 4; ++q) sizes[n++] = align256(sizeof(float) * kParams);        // theta m v grad
    for (int l = 0; l < 4; ++l) sizes[n++] = align256((size_t)kOut[l] * kIn[l] * 2);  // w_pk
    for (int l = 0; l < 4; ++l) sizes[n++] = align256((size_t)kOut[l] * kIn[l] * 2);  // wT_pk
    sizes[n++] = align256((size_t)Bp * 16 * 2);                                        // x_pk
    sizes[n++] = align256((size_t)Bp * 16 * 2);                                        // xT_pk
    for (int l = 0; l < 3; ++l) sizes[n++] = align256((size_t)Bp * 256 * 4);           // z
    for (int l = 0; l < 3; ++l) sizes[n++] = align256((size_t)Bp * 256 * 2);           // y_pk
    for (int l = 0; l < 3; ++l) sizes[n++] = align256((size_t)Bp * 256 * 2);           // yT_pk
    sizes[n++] = align256((size_t)Bp * kBins * 4);                                     // logits
    sizes[n++] = align256((size_t)Bp * kBins * 2);                                     // dz4_pk
    sizes[n++] = align256((size_t)Bp * kBins * 2);                                     // dz4T_pk
    for (int l = 0; l < 3; ++l) sizes[n++] = align256((size_t)Bp * 256 * 2);           // dz_pk
    for (int l = 0; l < 3; ++l) sizes[n++] = align256((size_t)Bp * 256 * 2);           // dzT_pk
    sizes[n++] = 256;                                                                  // loss + error
    sizes[n++] = align256((size_t)max_batch * 4 * 4);                                  // feat_b
    sizes[n++] = align256((size_t)max_batch * kBins * 4);                              // targ_b
    sizes[n++] = align256(sizeof(TrainSched));                                         // sched
    size_t total = 0;
    for (int i = 0; i < n; ++i) total += sizes[i];
    if (cudaMalloc(reinterpret_cast<void **>(&s->arena), total) != cudaSuccess) {
        delete s;
        return SSA_ENOMEM;
    }
    if (cudaMemset(s->arena, 0, total) != cudaSuccess) {
        cudaFree(s->arena);
        delete s;
        return SSA_ECUDA;
    }
    char *p = s->arena;
    int i = 0;
    auto take = [&](void *dst) {
        *reinterpret_cast<char **>(dst) = p;
        p += sizes[i++];
    };
    take(&s->theta); take(&s->m); take(&s->v); take(&s->grad);
    for (int l = 0; l < 4; ++l) take(&s->w_pk[l]);
    for (int l = 0; l < 4; ++l) take(&s->wT_pk[l]);
    take(&s->x_pk); take(&s->xT_pk);
    for (int l = 0; l < 3; ++l) take(&s->z[l]);
    for (int l = 0; l < 3; ++l) take(&s->y_pk[l]);
    for (int l = 0; l < 3; ++l) take(&s->yT_pk[l]);
    take(&s->logits); take(&s->dz4_pk); take(&s->dz4T_pk);
    for (int l = 0; l < 3; ++l) take(&s->dz_pk[l]);
    for (int l = 0; l < 3; ++l) take(&s->dzT_pk[l]);
    s->loss = reinterpret_cast<float *>(p);
    s->error = reinterpret_cast<int *>(p + 16);
    p += sizes[i++];
    take(&s->feat_b);
    take(&s->targ_b);
    take(&s->sched);

    // He-normal weights (std sqrt(2 / fan_in), fan_in = 4 for the first layer), zero biases
    float *h = new (std::nothrow) float[kParams];
    if (!h) {
        cudaFree(s->arena);
        delete s;
        return SSA_ENOMEM;
    }
    uint64_t st = seed;
    for (int64_t q = 0; q < kParams; ++q) h[q] = 0.0f;
    for (int l = 0; l < 4; ++l) {
        const double sd = std::sqrt(2.0 / (l == 0 ? 4.0 : (double)kIn[l]));
        for (int64_t q = 0; q < (int64_t)kOut[l] * kIn[l]; ++q) {
            if (l == 0 && (q % 16) >= 4) continue;
            const double u1 = ((double)(splitmix64(st) >> 11) + 1.0) * 0x1p-53;
            const double u2 = (double)(splitmix64(st) >> 11) * 0x1p-53;
            h[kOffW[l] + q] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    cudaError_t e = cudaMemcpy(s->theta, h, sizeof(float) * kParams, cudaMemcpyHostToDevice);
    delete[] h;
    if (e == cudaSuccess) e = refresh_all(s, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(s->arena);
        delete s;
        return SSA_ECUDA;
    }
    *out = s;
    return SSA_OK;
}

void ssa_surrogate_destroy(ssa_surrogate *s)
{
    if (!s) return;
    cudaFree(s->arena);
    delete s;
}

int ssa_surrogate_set_params(ssa_surrogate *s, const float *params)
{
    if (!s || !params) return SSA_EINVAL;
    cudaError_t e = cudaMemcpy(s->theta, params, sizeof(float) * kParams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(s->m, 0, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMemset(s->v, 0, sizeof(float) * kParams);
    if (e == cudaSuccess) e = refresh_all(s, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    s->step = 0;
    return e == cudaSuccess ? SSA_OK : SSA_ECUDA;
}

int ssa_surrogate_get_params(ssa_surrogate *s, float *params)
{
    if (!s || !params) return SSA_EINVAL;
    return cudaMemcpy(params, s->theta, sizeof(float) * kParams, cudaMemcpyDeviceToHost) == cudaSuccess ? SSA_OK
                                                                                                         : SSA_ECUDA;
}

int ssa_surrogate_get_state(ssa_surrogate *s, float *theta, float *m, float *v, float *grad, int64_t *adam_steps)
{
    if (!s) return SSA_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return SSA_ECUDA;
    const size_t bytes = sizeof(float) * kParams;
    cudaError_t e = cudaSuccess;
    if (theta) e = cudaMemcpy(theta, s->theta, bytes, cudaMemcpyDeviceToHost);
    if (m && e == cudaSuccess) e = cudaMemcpy(m, s->m, bytes, cudaMemcpyDeviceToHost);
    if (v && e == cudaSuccess) e = cudaMemcpy(v, s->v, bytes, cudaMemcpyDeviceToHost);
    if (grad && e == cudaSuccess) e = cudaMemcpy(grad, s->grad, bytes, cudaMemcpyDeviceToHost);
    if (adam_steps) *adam_steps = s->step;
    return e == cudaSuccess ? SSA_OK : SSA_ECUDA;
}

int ssa_surrogate_predict(ssa_surrogate *s, int B, const float *features, float *probs, void *stream)
{
    if (check_batch(s, B) != SSA_OK || !features || !probs) return SSA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int Bpad = bpad_of(B);
    cudaError_t e = forward(s, B, Bpad, features, false, st);
    if (e == cudaSuccess) {
        softmax_ce_kernel<<<(Bpad * 32 + 255) / 256, 256, 0, st>>>(s->logits, nullptr, B, Bpad, probs, nullptr,
                                                                   nullptr, nullptr, nullptr);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? SSA_OK : SSA_ECUDA;
}

int ssa_surrogate_train_step(ssa_surrogate *s, int B, const float *features, const float *targets, float lr,
                             float weight_decay, float *loss_out, void *stream)
{
    if (check_batch(s, B) != SSA_OK || !features || !targets || !(lr >= 0.0f)) return SSA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int Bpad = bpad_of(B);
    cudaError_t e = forward(s, B, Bpad, features, true, st);
    if (e == cudaSuccess) e = backward(s, B, Bpad, targets, st);
    if (e != cudaSuccess) return SSA_ECUDA;
    s->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    // 1 - beta^t in binary64, rounded once: subtracting a rounded beta^t from
    // 1 in binary32 would cancel (about 250 ulp off for beta2 at t = 4)
    const float bc1 = (float)(1.0 - std::pow((double)b1, (double)s->step));
    const float bc2 = (float)(1.0 - std::pow((double)b2, (double)s->step));
    adamw_kernel<<<(unsigned)((kParams + 255) / 256), 256, 0, st>>>(s->theta, s->grad, s->m, s->v, kParams, lr, b1, b2,
                                                                   1e-8f, weight_decay, bc1, bc2);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = refresh_all(s, st);
    if (e == cudaSuccess && loss_out)
        e = cudaMemcpyAsync(loss_out, s->loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? SSA_OK : SSA_ECUDA;
}

}  // extern "C"

namespace {

// One training step of a device-driven run (all its inputs in device memory).
cudaError_t scheduled_step(ssa_surrogate *s, int64_t n_steps, int64_t n_rows, const float *features,
                           const float *targets, int B, float lr_max, float lr_min, float wd, int64_t every,
                           float *trace, cudaStream_t st)
{
    TrainSched *sc = static_cast<TrainSched *>(s->sched);
    const int Bpad = bpad_of(B);
    schedule_kernel<<<1, 32, 0, st>>>(sc, (long long)n_steps, lr_max, lr_min);
    gather_batch_kernel<<<(unsigned)B, 128, 0, st>>>(features, targets, n_rows, B, sc, s->feat_b, s->targ_b);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = forward(s, B, Bpad, s->feat_b, true, st);
    if (e == cudaSuccess) e = backward(s, B, Bpad, s->targ_b, st);
    if (e != cudaSuccess) return e;
    adamw_sched_kernel<<<(unsigned)((kParams + 255) / 256), 256, 0, st>>>(s->theta, s->grad, s->m, s->v, kParams, sc,
                                                                          wd);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = refresh_all(s, st);
    if (e == cudaSuccess) {
        finish_step_kernel<<<1, 32, 0, st>>>(s->loss, sc, (long long)every, trace);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

extern "C" {

int ssa_surrogate_train(ssa_surrogate *s, int64_t n_steps, int64_t n_rows, const float *features,
                        const float *targets, int batch, float lr_max, float lr_min, float weight_decay,
                        int64_t loss_every, float *loss_trace, void *stream)
{
    if (check_batch(s, batch) != SSA_OK || n_steps < 0 || n_rows < 1 || !features || !targets ||
        !(lr_max >= 0.0f) || !(lr_min >= 0.0f) || loss_every < 1)
        return SSA_EINVAL;
    if (n_steps == 0) return SSA_OK;
    // a capturable stream: the caller's, or a private one ordered after the
    // legacy stream (the call synchronises before it returns)
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t ev = nullptr;
    const bool own = st == nullptr;
    cudaError_t e = cudaSuccess;
    if (own) {
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, nullptr);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
    }
    TrainSched init;   // copied from pageable memory: staged before the call returns
    init.adam_step = (long long)s->step;
    init.local = 0;
    init.lr = init.bc1 = init.bc2 = 0.0f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->sched, &init, sizeof(init), cudaMemcpyHostToDevice, st);
    // step 0 runs directly (it also sets the kernels' attributes); the rest
    // replay one captured step
    if (e == cudaSuccess)
        e = scheduled_step(s, n_steps, n_rows, features, targets, batch, lr_max, lr_min, weight_decay, loss_every,
                           loss_trace, st);
    int64_t done = 1;
    if (e == cudaSuccess && n_steps > 1) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaError_t eg = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (eg == cudaSuccess) {
            const cudaError_t ec = scheduled_step(s, n_steps, n_rows, features, targets, batch, lr_max, lr_min,
                                                  weight_decay, loss_every, loss_trace, st);
            eg = cudaStreamEndCapture(st, &graph);
            if (eg == cudaSuccess) eg = ec;
        }
        if (eg == cudaSuccess) eg = cudaGraphInstantiate(&exec, graph, 0);
        while (done < n_steps && eg == cudaSuccess) {
            eg = cudaGraphLaunch(exec, st);
            if (eg == cudaSuccess) ++done;
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (eg != cudaSuccess) cudaGetLastError();   // a step that did not capture runs directly below
    }
    for (; done < n_steps && e == cudaSuccess; ++done)
        e = scheduled_step(s, n_steps, n_rows, features, targets, batch, lr_max, lr_min, weight_decay, loss_every,
                           loss_trace, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    if (ev) cudaEventDestroy(ev);
    if (own && st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return SSA_ECUDA;
    s->step += n_steps;
    return SSA_OK;
}

int ssa_surrogate_gradients(ssa_surrogate *s, int B, const float *features, const float *targets, float *grads,
                            float *loss)
{
    if (check_batch(s, B) != SSA_OK || !features || !targets || !grads) return SSA_EINVAL;
    const int Bpad = bpad_of(B);
    cudaError_t e = forward(s, B, Bpad, features, true, nullptr);
    if (e == cudaSuccess) e = backward(s, B, Bpad, targets, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(grads, s->grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && loss) e = cudaMemcpy(loss, s->loss, sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SSA_OK : SSA_ECUDA;
}

int ssa_surrogate_status(ssa_surrogate *s)
{
    if (!s) return SSA_EINVAL;
    int h = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return SSA_ECUDA;
    if (cudaMemcpy(&h, s->error, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SSA_ECUDA;
    return h ? SSA_ETIMEDOUT : SSA_OK;
}

int ssa_mlp_softmax_xent(int B, const float *logits, const float *targets, float *probs, uint16_t *dz,
                         float *bias_grad, float *loss, void *stream)
{
    if (B < 1 || B > (1 << 20) || !logits) return SSA_EINVAL;
    if (!targets && !probs) return SSA_EINVAL;
    if (targets && (!dz || !bias_grad || !loss)) return SSA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int Bpad = bpad_of(B);
    uint8_t *pk = nullptr;
    const size_t half = (size_t)Bpad * kBins * 2;
    if (targets && cudaMallocAsync(reinterpret_cast<void **>(&pk), 2 * half, st) != cudaSuccess) return SSA_ENOMEM;
    softmax_ce_kernel<<<(Bpad * 32 + 255) / 256, 256, 0, st>>>(logits, targets, B, Bpad, probs, pk,
                                                               pk ? pk + half : nullptr, bias_grad, loss);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && targets) {
        const int64_t n = (int64_t)B * kBins;
        mlp::unpack_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pk, B, kBins, dz);
        e = cudaGetLastError();
    }
    if (pk) cudaFreeAsync(pk, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? SSA_OK : SSA_ECUDA;
}

int ssa_histogram(const int32_t *counts, int64_t n_sets, int64_t traj_per_set, int bins, float *hist, void *stream)
{
    if (!counts || !hist || n_sets < 1 || traj_per_set < 1 || bins < 1 || bins > 4096) return SSA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    histogram_kernel<<<(unsigned)n_sets, 256, (size_t)bins * sizeof(unsigned int), st>>>(counts, traj_per_set, bins,
                                                                                          hist);
    return cudaGetLastError() == cudaSuccess ? SSA_OK : SSA_ECUDA;
}

int ssa_hist_w1_noise(const float *p, int64_t rows, int bins, double n_draws, float *out, void *stream)
{
    if (!p || !out || rows < 1 || bins < 1 || !(n_draws >= 1.0)) return SSA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    hist_w1_noise_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(p, rows, bins, (float)n_draws, out);
    return cudaGetLastError() == cudaSuccess ? SSA_OK : SSA_ECUDA;
}

int ssa_hist_w1(const float *p, const float *q, int64_t rows, int bins, float *w1, void *stream)
{
    if (!p || !q || !w1 || rows < 1 || bins < 1) return SSA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    hist_w1_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(p, q, rows, bins, w1);
    return cudaGetLastError() == cudaSuccess ? SSA_OK : SSA_ECUDA;
}

}  // extern "C"
