// tau_device.cuh -- mixed-precision tau-leaping on the GPU.
//
// Explicit tau-leaping (the approximate family of the paper's Table 1; its
// combination with reduced precision is untested there, Sec. 5, and named as
// future work, Sec. 6): with a fixed leap tau, each leap fires k_j ~ Poisson(a_j tau)
// of every channel at once, x += sum_j nu_j k_j.  Contract (shared with the
// oracle, written independently):
//  * leap n covers [n tau, (n+1) tau), L = ceil(t_end / tau) leaps; the leap
//    grid is exact binary64; before leap n every sample s_k < (n+1) tau
//    receives the current state, after the last leap the rest the final one;
//  * a_j by the direct method's propensity contract; lambda_j = a_j * tau in
//    the accumulator type, or rnd16(a_j * rnd16(tau)) in uniform modes (SR
//    slot sr_ops + j); SR slots of leap n come from stream 1 blocks [nB, (n+1)B);
//  * k_j from the Poisson sampler below (binary64 in FP64 mode, binary32
//    otherwise): Knuth's multiplication method for lambda < 10, Hoermann's
//    transformed rejection (PTRS) at 10 and above, uniforms from Philox with
//    counter (word block, leap n, trajectory id, 2 + j);
//  * x += sum_j nu_j k_j in 64-bit integers, negative counts set to 0 with
//    status TAU_CLAMPED (16); the event count is sum_j k_j.
#pragma once

#include <type_traits>

#include "ssa_device.cuh"

namespace ssa {

constexpr uint32_t ST_TAU_CLAMPED = 16;

// e^x for x in [-30, 0]: x = k ln2 + r (Cody-Waite), Taylor series of e^r
// (r^7 in binary32, r^13 in binary64), times 2^k built from its bits.
__device__ __forceinline__ float exp_f32(float x)
{
    const float kLn2Hi = 0x1.62e400p-1f;
    const float kLn2Lo = 0x1.7f7d1cp-20f;
    const float kInvLn2 = 0x1.715476p+0f;
    float kf = x * kInvLn2;
    kf = kf + 0.5f;
    int k = (int)kf;
    if ((float)k > kf) k -= 1;
    const float fk = (float)k;
    float r = x - fk * kLn2Hi;
    r = r - fk * kLn2Lo;
    float p = 1.0f / 5040.0f;
    p = p * r + 1.0f / 720.0f;
    p = p * r + 1.0f / 120.0f;
    p = p * r + 1.0f / 24.0f;
    p = p * r + 1.0f / 6.0f;
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    return p * __uint_as_float((uint32_t)(k + 127) << 23);
}

__device__ __forceinline__ double exp_f64(double x)
{
    const double kLn2Hi = 0x1.62e42fee00000p-1;
    const double kLn2Lo = 0x1.a39ef35793c76p-33;
    const double kInvLn2 = 0x1.71547652b82fep+0;
    double kf = x * kInvLn2;
    kf = kf + 0.5;
    int k = (int)kf;
    if ((double)k > kf) k -= 1;
    const double fk = (double)k;
    double r = x - fk * kLn2Hi;
    r = r - fk * kLn2Lo;
    double p = 1.0 / 6227020800.0;
    p = p * r + 1.0 / 479001600.0;
    p = p * r + 1.0 / 39916800.0;
    p = p * r + 1.0 / 3628800.0;
    p = p * r + 1.0 / 362880.0;
    p = p * r + 1.0 / 40320.0;
    p = p * r + 1.0 / 5040.0;
    p = p * r + 1.0 / 720.0;
    p = p * r + 1.0 / 120.0;
    p = p * r + 1.0 / 24.0;
    p = p * r + 1.0 / 6.0;
    p = p * r + 0.5;
    p = p * r + 1.0;
    p = p * r + 1.0;
    return p * __longlong_as_double((long long)((uint64_t)(k + 1023) << 52));
}

// log k!: summed logarithms below 10, Stirling's series at 10 and above.
__device__ __forceinline__ float logfact_f32(float k)
{
    if (k < 10.0f) {
        float s = 0.0f;
        for (int i = 2; (float)i <= k; ++i) s = s + log_f32((float)i);
        return s;
    }
    const float kHalfLn2Pi = 0x1.d67f1cp-1f;
    const float x = k + 1.0f;
    const float lx = log_f32(x);
    float s = (x - 0.5f) * lx;
    s = s - x;
    s = s + kHalfLn2Pi;
    s = s + (1.0f / 12.0f) / x;
    s = s - (1.0f / 360.0f) / (x * x * x);
    return s;
}

__device__ __forceinline__ double logfact_f64(double k)
{
    if (k < 10.0) {
        double s = 0.0;
        for (int i = 2; (double)i <= k; ++i) s = s + log_f64((double)i);
        return s;
    }
    const double kHalfLn2Pi = 0x1.d67f1c864beb5p-1;
    const double x = k + 1.0;
    const double lx = log_f64(x);
    double s = (x - 0.5) * lx;
    s = s - x;
    s = s + kHalfLn2Pi;
    s = s + (1.0 / 12.0) / x;
    s = s - (1.0 / 360.0) / (x * x * x);
    s = s + (1.0 / 1260.0) / (x * x * x * x * x);
    return s;
}

// Words of one (leap, channel) sampler stream.
struct SamplerWords {
    uint32_t k0, k1, leap, traj, stream, w;
    uint4 blk;
    __device__ __forceinline__ uint32_t next()
    {
        if ((w & 3u) == 0u) blk = philox4x32_10(make_uint4(w >> 2, leap, traj, stream), k0, k1);
        const uint32_t i = w & 3u;
        w += 1;
        return i == 0 ? blk.x : (i == 1 ? blk.y : (i == 2 ? blk.z : blk.w));
    }
};

__device__ inline int64_t poisson_f32(float lam, SamplerWords &s)
{
    if (!(lam > 0.0f)) return 0;
    if (lam < 10.0f) {
        const float L = exp_f32(-lam);
        float p = 1.0f;
        int64_t k = -1;
        for (int it = 0; it < 1000; ++it) {
            const float v = (float)((s.next() >> 8) + 1u) * 0x1p-24f;
            k += 1;
            p = p * v;
            if (!(p > L)) return k;
        }
        return k;
    }
    const float slam = sqrtf(lam);
    const float loglam = log_f32(lam);
    const float b = 0.931f + 2.53f * slam;
    const float a = -0.059f + 0.02483f * b;
    const float invalpha = 1.1239f + 1.1328f / (b - 3.4f);
    const float vr = 0.9277f - 3.6224f / (b - 2.0f);
    const float log_invalpha = log_f32(invalpha);
    const float kmax = lam + 64.0f * slam + 64.0f;
    for (int it = 0; it < 100; ++it) {
        const float U = (float)(s.next() >> 8) * 0x1p-24f - 0.5f;
        const float V = (float)((s.next() >> 8) + 1u) * 0x1p-24f;
        const float aU = U < 0.0f ? -U : U;
        const float us = 0.5f - aU;
        if (!(us > 0.0f)) continue;
        float kf = (2.0f * a / us + b) * U;
        kf = kf + lam;
        kf = kf + 0.43f;
        kf = floorf(kf);
        if (us >= 0.07f && V <= vr) return (int64_t)kf;
        if (kf < 0.0f || (us < 0.013f && V > us)) continue;
        if (kf > kmax) continue;
        float lhs = log_f32(V) + log_invalpha;
        lhs = lhs - log_f32(a / (us * us) + b);
        float rhs = -lam + kf * loglam;
        rhs = rhs - logfact_f32(kf);
        if (lhs <= rhs) return (int64_t)kf;
    }
    return (int64_t)floorf(lam);
}

__device__ inline int64_t poisson_f64(double lam, SamplerWords &s)
{
    if (!(lam > 0.0)) return 0;
    if (lam < 10.0) {
        const double L = exp_f64(-lam);
        double p = 1.0;
        int64_t k = -1;
        for (int it = 0; it < 1000; ++it) {
            const double v = ((double)s.next() + 1.0) * 0x1p-32;
            k += 1;
            p = p * v;
            if (!(p > L)) return k;
        }
        return k;
    }
    const double slam = sqrt(lam);
    const double loglam = log_f64(lam);
    const double b = 0.931 + 2.53 * slam;
    const double a = -0.059 + 0.02483 * b;
    const double invalpha = 1.1239 + 1.1328 / (b - 3.4);
    const double vr = 0.9277 - 3.6224 / (b - 2.0);
    const double log_invalpha = log_f64(invalpha);
    const double kmax = lam + 64.0 * slam + 64.0;
    for (int it = 0; it < 100; ++it) {
        const double U = (double)s.next() * 0x1p-32 - 0.5;
        const double V = ((double)s.next() + 1.0) * 0x1p-32;
        const double aU = U < 0.0 ? -U : U;
        const double us = 0.5 - aU;
        if (!(us > 0.0)) continue;
        double kf = (2.0 * a / us + b) * U;
        kf = kf + lam;
        kf = kf + 0.43;
        kf = floor(kf);
        if (us >= 0.07 && V <= vr) return (int64_t)kf;
        if (kf < 0.0 || (us < 0.013 && V > us)) continue;
        if (kf > kmax) continue;
        double lhs = log_f64(V) + log_invalpha;
        lhs = lhs - log_f64(a / (us * us) + b);
        double rhs = -lam + kf * loglam;
        rhs = rhs - logfact_f64(kf);
        if (lhs <= rhs) return (int64_t)kf;
    }
    return (int64_t)floor(lam);
}

template <class Model, int PREC>
__device__ void tau_finish(const RunArgs &a, Lane<Model, PREC> &L)
{
    while (L.k < a.K) {
        store_state<Model>(a, L.k, L.item, L.x, L.status);
        L.k += 1;
    }
    a.status[L.item] = L.status;
    if (a.n_events) a.n_events[L.item] = L.ev;
    if (a.t_final) a.t_final[L.item] = L.n > 0 ? (double)L.n * a.tau : 0.0;
    L.active = false;
}

// Propensities of a compiled structure: the direct method's chain (the same
// operations and rounding slots as general_propensities), unrolled.
template <class Model, int PREC, int SR>
__device__ __forceinline__ void static_propensities(const RunArgs &a, const Lane<Model, PREC> &L,
                                                    Rounder<PREC, SR> &R, typename ModeTraits<PREC>::P *prop)
{
    using P = typename ModeTraits<PREC>::P;
    unroll<Model::M>([&](auto J) {
        constexpr int j = decltype(J)::value;
        int op = Model::template chain_start<j>(a);
        if (Model::template law<j>(a) == 1) {
            const int reg = Model::template hill_reg<j>(a);
            int xr = 0;
            unroll<Model::N>([&](auto I) {
                constexpr int i = decltype(I)::value;
                if (i == reg) xr = L.x[i];
            });
            const P Pv = R.rnd((P)xr, op++);
            P q = Pv;
            const int h = Model::template hill_h<j>(a);
            for (int m = 1; m < h; ++m) q = R.rnd(q * Pv, op++);
            const P d = R.rnd(P(1) + q, op++);
            const P f = R.rnd(L.h1[j] / d, op++);
            prop[j] = R.rnd(L.h0[j] + f, op++);
        } else {
            P av = L.c[j];
            bool zero = false;
            unroll<Model::N>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const int rr = Model::template order<j, i>(a);
                if (rr > 0 && !Model::template folded<j, i>(a)) {
                    zero = zero || (L.x[i] < rr);
                    for (int m = 0; m < rr; ++m) {
                        const P f = R.rnd((P)(L.x[i] - m), op++);
                        av = R.rnd(av * f, op++);
                    }
                }
            });
            prop[j] = zero ? P(0) : av;
        }
    });
}

// Out-of-line sampler call for the unrolled channel loop of compiled
// structures (one copy of the sampler instead of one per channel).
template <int PREC>
__device__ __noinline__ int64_t poisson_call(typename ModeTraits<PREC>::P lam, SamplerWords &s)
{
    if constexpr (ModeTraits<PREC>::kF64) return poisson_f64(lam, s);
    else return poisson_f32(lam, s);
}

// Smallest m >= 0 with fl(m * tau) > s in binary64.  Since fl(m * tau) does
// not decrease with m, "s < fl((n + 1) * tau)" (snapshot s is written before
// leap n) is "n + 1 >= m": the leap loop then needs no binary64 operation.
__device__ inline int64_t first_leap_after(double s, double tau)
{
    const double g = floor(s / tau);
    int64_t m = g < 0.0 ? 0 : (g > 4.0e18 ? (int64_t)4.0e18 : (int64_t)g);
    for (int i = 0; i < 64 && !((double)m * tau > s); ++i) ++m;
    for (int i = 0; i < 64 && m > 0 && (double)(m - 1) * tau > s; ++i) --m;
    return m;
}

// One leap n = L.n of an active lane.  m_first[k]: first_leap_after(sample
// k, tau); tau32: tau rounded to binary32.
template <class Model, int PREC, int SR>
__device__ __noinline__ void tau_leap(const RunArgs &a, Lane<Model, PREC> &L, const int64_t *m_first, float tau32)
{
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    constexpr bool kGeneral = std::is_same<Model, GeneralModel>::value;
    const int64_t n = L.n;
    while (L.k < a.K && n + 1 >= m_first[L.k]) {
        store_state<Model>(a, L.k, L.item, L.x, L.status);
        L.k += 1;
    }
    Rounder<PREC, SR> R;
    if constexpr (Tr::k16 && SR) {
        const int sr_total = Model::total_chain_ops(a) + (Tr::kUniform ? Model::last(a) + 1 : 0);
        R.bits.base = (uint64_t)n * (uint64_t)((sr_total + 7) >> 3);
        R.bits.traj = L.traj;
        R.bits.k0 = a.key0;
        R.bits.k1 = a.key1;
        R.bits.cur = -1;
    }
    float tau16 = tau32;
    if constexpr (Tr::k16) tau16 = rn16<Tr::kFmt>(tau32);
    const int lam_op = Model::total_chain_ops(a);   // SR slot of lambda_0 (uniform modes)
    auto lambda_of = [&](P prop, int j) -> P {
        if constexpr (Tr::kF64) return prop * a.tau;
        else if constexpr (Tr::kUniform) return R.rnd(prop * tau16, lam_op + j);
        else return prop * tau32;
    };
    P prop[Model::M];
    P lam[Model::M];
    uint32_t bad = 0;
    if constexpr (kGeneral) {
        general_propensities<PREC, SR>(a, L, R, prop);
#pragma unroll 1
        for (int j = 0; j < a.M; ++j) {
            const P v = lambda_of(prop[j], j);
            lam[j] = v;
            if (v != v) bad |= ST_NAN;
            else if (v == P(__int_as_float(0x7F800000))) bad |= ST_OVERFLOW;
        }
    } else {
        static_propensities<Model, PREC, SR>(a, L, R, prop);
        unroll<Model::M>([&](auto J) {
            constexpr int j = decltype(J)::value;
            const P v = lambda_of(prop[j], j);
            lam[j] = v;
            if (v != v) bad |= ST_NAN;
            else if (v == P(__int_as_float(0x7F800000))) bad |= ST_OVERFLOW;
        });
    }
    if (bad) {
        L.status |= bad;
        tau_finish<Model, PREC>(a, L);
        return;
    }
    int64_t dx[Model::N];
#pragma unroll
    for (int i = 0; i < Model::N; ++i) dx[i] = 0;
    SamplerWords sw;
    sw.k0 = a.key0;
    sw.k1 = a.key1;
    sw.leap = (uint32_t)n;
    sw.traj = L.traj;
    if constexpr (kGeneral) {
#pragma unroll 1
        for (int j = 0; j < a.M; ++j) {
            sw.stream = 2u + (uint32_t)j;
            sw.w = 0;
            int64_t kj;
            if constexpr (Tr::kF64) kj = poisson_f64(lam[j], sw);
            else kj = poisson_f32(lam[j], sw);
            L.ev += kj;
#pragma unroll 1
            for (int i = 0; i < a.N; ++i) dx[i] += kj * (int64_t)a.stoich[j][i];
        }
    } else {
        unroll<Model::M>([&](auto J) {
            constexpr int j = decltype(J)::value;
            sw.stream = 2u + (uint32_t)j;
            sw.w = 0;
            const int64_t kj = poisson_call<PREC>(lam[j], sw);
            L.ev += kj;
            unroll<Model::N>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const int nu = Model::template nu<j, i>(a);
                if (nu != 0) dx[i] += kj * (int64_t)nu;
            });
        });
    }
    if constexpr (kGeneral) {
#pragma unroll 1
        for (int i = 0; i < a.N; ++i) {
            int64_t v = (int64_t)L.x[i] + dx[i];
            if (v < 0) {
                v = 0;
                L.status |= ST_TAU_CLAMPED;
            }
            if (v > 2147483647) v = 2147483647;
            L.x[i] = (int)v;
        }
    } else {
        unroll<Model::N>([&](auto I) {
            constexpr int i = decltype(I)::value;
            int64_t v = (int64_t)L.x[i] + dx[i];
            if (v < 0) {
                v = 0;
                L.status |= ST_TAU_CLAMPED;
            }
            if (v > 2147483647) v = 2147483647;
            L.x[i] = (int)v;
        });
    }
    L.n = n + 1;
    if (L.n >= a.n_leaps) tau_finish<Model, PREC>(a, L);
}
// Persistent tau-leaping kernel: lanes refill from the work queue as in the
// direct method; each loop iteration runs one leap.  Model is a compiled
// structure (StaticModel) or the runtime-table GeneralModel.
template <class Model, int PREC, int SR>
__global__ void __launch_bounds__(256) tau_kernel(const __grid_constant__ RunArgs a)
{
    using P = typename ModeTraits<PREC>::P;
    __shared__ int64_t m_first[kMaxK];
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) m_first[k] = first_leap_after(a.samples[k], a.tau);
    __syncthreads();
    const float tau32 = (float)a.tau;
    const unsigned lane = threadIdx.x & 31u;
    const P no_samples[1] = {P(0)};
    Lane<Model, PREC> L;
    L.active = false;
    bool drained = false;
    for (;;) {
        const unsigned need = __ballot_sync(0xFFFFFFFFu, !L.active && !drained);
        if (need) {
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(a.queue_head, (unsigned long long)__popc(need));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (!L.active && !drained) {
                const unsigned long long item = base + (unsigned long long)__popc(need & ((1u << lane) - 1u));
                if (item < (unsigned long long)a.n_work) {
                    init_lane<Model, PREC>(a, L, (int64_t)item, no_samples);
                    L.ev = 0;
                    if (a.n_leaps <= 0) tau_finish<Model, PREC>(a, L);
                } else {
                    drained = true;
                }
            }
        }
        if (__ballot_sync(0xFFFFFFFFu, L.active) == 0u) break;
        if (L.active) tau_leap<Model, PREC, SR>(a, L, m_first, tau32);
    }
}

// Launch of one structure's kernel for (precision, rounding); the grid is
// sized from occupancy (persistent), capped by the work.
template <class Model>
cudaError_t tau_launch_model(const RunArgs &a, int prec, int sr, int block, int blocks_per_sm, cudaStream_t stream,
                             int *grid_out)
{
    using K = void (*)(const RunArgs);
    K k = nullptr;
    switch (prec) {
    case FP64: k = tau_kernel<Model, FP64, 0>; break;
    case FP32: k = tau_kernel<Model, FP32, 0>; break;
    case MIXED_F16: k = sr ? tau_kernel<Model, MIXED_F16, 1> : tau_kernel<Model, MIXED_F16, 0>; break;
    case MIXED_BF16: k = sr ? tau_kernel<Model, MIXED_BF16, 1> : tau_kernel<Model, MIXED_BF16, 0>; break;
    case UNIFORM_F16: k = sr ? tau_kernel<Model, UNIFORM_F16, 1> : tau_kernel<Model, UNIFORM_F16, 0>; break;
    case UNIFORM_BF16: k = sr ? tau_kernel<Model, UNIFORM_BF16, 1> : tau_kernel<Model, UNIFORM_BF16, 0>; break;
    default: return cudaErrorInvalidValue;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    long long grid = (long long)sms * per_sm;
    const long long need = (a.n_work + block - 1) / block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    *grid_out = (int)grid;
    k<<<(unsigned)grid, (unsigned)block, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace ssa
