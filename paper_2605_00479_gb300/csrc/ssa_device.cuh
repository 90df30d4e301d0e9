// ssa_device.cuh -- device side of the GB300 ensemble engine for the
// reduced-precision Gillespie direct method.
//
// One GPU lane runs one trajectory at a time; a lane whose trajectory has
// finished takes the next one from a device work queue (warp-aggregated
// atomicAdd), so warps stay full while trajectories of very different
// lengths retire.  State, propensities and partial sums live in registers;
// the model structure is either compiled in (structure-specialised kernels)
// or read from kernel parameters (the general kernel).
//
// Arithmetic contract (the paper's Sec. 2 direct method, Sec. 3.2 precision
// partition, Sec. 3.3 stochastic rounding; readings where it is silent):
//  * c'_j is rounded to the propensity type once, by RN (binary64 ->
//    binary32 -> 16-bit).
//  * Mass action: a = c'; for species i ascending, m = 0..r-1:
//    f = rnd(x_i - m); a = rnd(a * f).  a = +0 when some x_i < r_ij.
//    Hill: P = rnd(x_reg); q = P; (h-1) times q = rnd(q * P);
//    d = rnd(1 + q); f = rnd(alpha / d); a = rnd(alpha0 + f).
//  * A 16-bit operation is the binary32 operation on the widened operands
//    followed by one rounding (RN: cvt.rn; SR: cvt.rs with 16 random bits of
//    which binary16 uses the low 13, bfloat16 all 16).
//  * Random numbers: Philox4x32-10, key = seed, counter = (block lo,
//    block hi, trajectory id, stream).  Stream 0: step n uses words 2n and
//    2n+1 (u1 in (0,1], u2 in [0,1)).  Stream 1 (SR bits): step n owns blocks
//    [n*B, (n+1)*B), B = ceil(S/8) for S rounding operations per step; SR
//    operation i uses the low (even i) / high (odd i) half of word i/2.
//  * Uniform mode rounds, in this order: propensity chains, partial sums
//    S_1..S_{M-1}, E = rnd(-log u1), U2 = rnd(u2), tau = rnd(E / a0),
//    target = rnd(U2 * a0), t_new = rnd(t + tau).  Selective SR (uniform
//    modes) rounds only S_1..S_{M-1} and t_new stochastically, with SR slots
//    0..M-1, and everything else to nearest.
//  * log: ln x = e ln2 + 2 atanh(s), s = (m-1)/(m+1), m in [sqrt(1/2),
//    sqrt(2)], odd series to s^9 (binary32) / s^23 (binary64), ln2 split into
//    a 16-bit (binary32) or 32-bit (binary64) head and a tail.
// This file is compiled with -fmad=false: no multiply-add is contracted, so
// each operation is one IEEE-754 operation in round-to-nearest-even.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

namespace ssa {

constexpr int kMaxN = 8;
constexpr int kMaxM = 16;
constexpr int kMaxK = 1024;

// Minimum resident 256-thread blocks per SM requested from the register
// allocator for the single-model kernels (1 = no register cap below 255).
#ifndef SSA_MIN_BLOCKS
#define SSA_MIN_BLOCKS 1
#endif

// Per kernel: a register budget, as 256-thread blocks per SM, where it was
// measured to pay (the A/B against uncapped builds, GB300).  The one-species
// birth-death structure's round-to-nearest kernels (not fp64) fit 48
// registers without spilling: five blocks (40 warps) instead of four, +16%.
// For Schloegl, telegraph and dimer the same budget costs about 8% more
// instructions and is slower; 64 registers for mixed stochastic rounding and
// fp64 (-2%, -4%) and 80 for uniform stochastic rounding (0..+2%) did not pay
// either.  Every other kernel keeps the compiler's choice.
#ifndef SSA_KERNEL_BUDGETS
#define SSA_KERNEL_BUDGETS 1   // 0: every kernel at SSA_MIN_BLOCKS (for comparisons)
#endif

template <class Model, int PREC, int SR>
struct KernelMinBlocks {
    static constexpr int value = (SSA_KERNEL_BUDGETS && Model::N == 1 && SR == 0 && PREC != 0) ? 5 : SSA_MIN_BLOCKS;
};

enum Precision { FP64 = 0, FP32 = 1, MIXED_F16 = 2, MIXED_BF16 = 3, UNIFORM_F16 = 4, UNIFORM_BF16 = 5 };
enum TrajStatus { ST_OVERFLOW = 1, ST_MAX_EVENTS = 2, ST_STATE_RANGE = 4, ST_NAN = 8 };

// Kernel arguments.  Passed by value as a __grid_constant__ parameter (about
// 10 KB): the model structure for the general kernel, the rate constants of
// the first parameter set and the sample times ride in parameter space.
struct RunArgs {
    // structure (read only by the general kernel)
    int N, M, K;
    int sr_ops;                        // rounding operations per step (SR modes)
    int8_t order[kMaxM][kMaxN];
    int32_t stoich[kMaxM][kMaxN];      // constant species already zeroed
    int8_t folded[kMaxM][kMaxN];       // factor folded into c' (normalise)
    int8_t law[kMaxM];
    int8_t hill_h[kMaxM];
    int8_t hill_reg[kMaxM];
    int16_t chain_start[kMaxM];        // first SR operation of each chain
    // work
    int64_t n_traj;                    // work items (output column count)
    int64_t n_work;                    // items to simulate (n_traj, or fewer while tuning)
    int slice_pairs;                   // step pairs between refill checks (>= 1)
    uint32_t traj_offset;              // global id of item 0
    int n_sets;                        // parameter sets
    int64_t traj_per_set;              // item r uses set r / traj_per_set
    double cprime[kMaxM];              // set 0: c'_j in binary64 (after folding)
    double hill_a0[kMaxM];
    double hill_a[kMaxM];
    int32_t x0[kMaxN];
    const double *cprime_tab;          // [n_sets][M] when n_sets > 1
    const double *hill_tab;            // [n_sets][M][2] (alpha0, alpha) or null
    const int32_t *x0_tab;             // [n_sets][N] or null (then x0 above)
    double t_end;
    double tau;                        // tau-leaping: leap size (0 for the direct method)
    int64_t n_leaps;                   // tau-leaping: ceil(t_end / tau)
    double samples[kMaxK];
    uint32_t key0, key1;
    int64_t max_events;
    // outputs
    void *out;                         // [K][out_N][n_traj] int32 or int16
    int state_bytes;
    uint32_t out_mask;                 // bit i: species i is stored (ascending order)
    int out_N;                         // stored species (popcount of out_mask)
    uint32_t *status;
    int64_t *n_events;
    double *t_final;
    unsigned long long *queue_head;    // zero before launch
    unsigned long long *tail_stats;    // [moved, lock waits given up, resumed at block end]; null: no tail compaction
    int lock_spins;                    // bound on one hand-off lock wait (0: kPoolLockSpins)
    // Longest-first scheduling: two launches of the same kernel.  Launch 1
    // (parked set) runs every trajectory up to max_events events, here the
    // parking point, and parks those still unfinished there (state, clock,
    // next snapshot); launch 2 (resume_order set) resumes the parked
    // trajectories in the order the ordering kernels chose (largest
    // predicted remaining work first).
    int64_t cap_events;                // launch 1: the caller's event cap
    double *park_t;                    // [n_work] clock at parking
    int32_t *park_k;                   // [n_work] next snapshot
    uint32_t *park_status;             // [n_work]
    int32_t *park_x;                   // [N][n_work] state
    uint8_t *parked;                   // [n_work] set to 1 when parked (zero before launch 1); null: no parking
    const int64_t *resume_order;       // launch 2: items to resume, largest key first; null: items 0 .. n_work-1
    const unsigned long long *resume_count;   // launch 2: entries of resume_order
    int64_t resume_events;             // launch 2: events every parked trajectory has fired
};

// ------------------------------------------------------------------ Philox
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// --------------------------------------------------------------------- log
__device__ __forceinline__ float log_f32(float x)
{
    const float kLn2Hi = 0x1.62e400p-1f;       // leading 16 bits of ln 2
    const float kLn2Lo = 0x1.7f7d1cp-20f;      // ln 2 - kLn2Hi, rounded
    uint32_t u = __float_as_uint(x);
    int e = (int)(u >> 23) - 127;
    uint32_t mb = (u & 0x7FFFFFu) | 0x3F800000u;
    if (mb > 0x3FB504F3u) {                     // mantissa above sqrt(2)
        mb -= 0x00800000u;
        e += 1;
    }
    const float m = __uint_as_float(mb);
    const float f = m - 1.0f;
    const float d = m + 1.0f;
    const float s = f / d;
    const float z = s * s;
    float p = 2.0f / 9.0f;
    p = z * p; p = (2.0f / 7.0f) + p;
    p = z * p; p = (2.0f / 5.0f) + p;
    p = z * p; p = (2.0f / 3.0f) + p;
    float r = s * z;
    r = r * p;
    const float two_s = s + s;
    r = two_s + r;
    const float ef = (float)e;
    float lo = ef * kLn2Lo;
    lo = lo + r;
    const float hi = ef * kLn2Hi;
    return hi + lo;
}

__device__ __forceinline__ double log_f64(double x)
{
    const double kLn2Hi = 0x1.62e42fee00000p-1;   // leading 32 bits of ln 2
    const double kLn2Lo = 0x1.a39ef35793c76p-33;
    uint64_t u = (uint64_t)__double_as_longlong(x);
    int e = (int)(u >> 52) - 1023;
    uint64_t mb = (u & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    if (mb > 0x3FF6A09E667F3BCCull) {
        mb -= 0x0010000000000000ull;
        e += 1;
    }
    const double m = __longlong_as_double((long long)mb);
    const double f = m - 1.0;
    const double d = m + 1.0;
    const double s = f / d;
    const double z = s * s;
    double p = 2.0 / 23.0;
    p = z * p; p = (2.0 / 21.0) + p;
    p = z * p; p = (2.0 / 19.0) + p;
    p = z * p; p = (2.0 / 17.0) + p;
    p = z * p; p = (2.0 / 15.0) + p;
    p = z * p; p = (2.0 / 13.0) + p;
    p = z * p; p = (2.0 / 11.0) + p;
    p = z * p; p = (2.0 / 9.0) + p;
    p = z * p; p = (2.0 / 7.0) + p;
    p = z * p; p = (2.0 / 5.0) + p;
    p = z * p; p = (2.0 / 3.0) + p;
    double r = s * z;
    r = r * p;
    const double two_s = s + s;
    r = two_s + r;
    const double ef = (double)e;
    double lo = ef * kLn2Lo;
    lo = lo + r;
    const double hi = ef * kLn2Hi;
    return hi + lo;
}

// --------------------------------------------------------- 16-bit rounding
// FMT 0: binary16, FMT 1: bfloat16.  Values are carried widened in binary32
// registers; widening is exact.
template <int FMT>
__device__ __forceinline__ float widen16(uint16_t h)
{
    if constexpr (FMT == 0) {
        float y;
        asm("cvt.f32.f16 %0, %1;" : "=f"(y) : "h"(h));
        return y;
    } else {
        return __uint_as_float((uint32_t)h << 16);
    }
}

template <int FMT>
__device__ __forceinline__ float rn16(float x)
{
    uint16_t h;
    if constexpr (FMT == 0) {
        asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(x));
    } else {
        asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
    }
    return widen16<FMT>(h);
}

// Stochastic rounding with the hardware's paired conversion: the low half of
// the result rounds operand b with rbits[15:0], the high half operand a with
// rbits[31:16].  Both operands are x; `hi` picks the half.
template <int FMT>
__device__ __forceinline__ float sr16(float x, uint32_t rbits, bool hi)
{
    uint32_t d;
    if constexpr (FMT == 0) {
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(x), "f"(x), "r"(rbits));
    } else {
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(x), "f"(x), "r"(rbits));
    }
    return widen16<FMT>((uint16_t)(hi ? (d >> 16) : (d & 0xFFFFu)));
}

// Native round-to-nearest 16-bit arithmetic on bit patterns.  For +, -, *
// and / the binary32 result rounded once to binary16 or bfloat16 equals the
// correctly rounded 16-bit result (binary32 has at least 2p+2 significand
// bits for both formats), so these give exactly the contract's RN values.
template <int FMT>
struct Native16 {
    __device__ static __forceinline__ uint16_t from_int(int v)
    {
        uint16_t h;
        if constexpr (FMT == 0) {
            asm("cvt.rn.f16.s32 %0, %1;" : "=h"(h) : "r"(v));
        } else {
            const float f = (float)v;   // exact below 2^24; rounded as the contract says above
            asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(f));
        }
        return h;
    }
    __device__ static __forceinline__ uint16_t from_f32(float v)
    {
        uint16_t h;
        if constexpr (FMT == 0) asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(v));
        else asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(v));
        return h;
    }
    __device__ static __forceinline__ float to_f32(uint16_t h) { return widen16<FMT>(h); }
    __device__ static __forceinline__ uint16_t mul(uint16_t a, uint16_t b)
    {
        uint16_t d;
        if constexpr (FMT == 0) asm("mul.rn.f16 %0, %1, %2;" : "=h"(d) : "h"(a), "h"(b));
        else asm("mul.rn.bf16 %0, %1, %2;" : "=h"(d) : "h"(a), "h"(b));
        return d;
    }
    __device__ static __forceinline__ uint16_t add(uint16_t a, uint16_t b)
    {
        uint16_t d;
        if constexpr (FMT == 0) asm("add.rn.f16 %0, %1, %2;" : "=h"(d) : "h"(a), "h"(b));
        else asm("add.rn.bf16 %0, %1, %2;" : "=h"(d) : "h"(a), "h"(b));
        return d;
    }
};

// ------------------------------------------------------------ mode traits
template <int PREC>
struct ModeTraits {
    static constexpr bool kF64 = PREC == FP64;
    static constexpr bool kF32 = PREC == FP32;
    static constexpr bool kMixed = PREC == MIXED_F16 || PREC == MIXED_BF16;
    static constexpr bool kUniform = PREC == UNIFORM_F16 || PREC == UNIFORM_BF16;
    static constexpr bool k16 = kMixed || kUniform;
    static constexpr int kFmt = (PREC == MIXED_BF16 || PREC == UNIFORM_BF16) ? 1 : 0;
    using P = typename std::conditional<kF64, double, float>::type;   // propensity / sum / time
};

// Lazily generated SR-stream blocks of the current step.  With operation
// indices known at compile time the block checks fold away.
struct SRBits {
    uint64_t base;     // first block of this step: n * B
    uint32_t traj, k0, k1;
    int cur;
    uint4 blk;
    __device__ __forceinline__ uint32_t word(int op)
    {
        const int b = op >> 3;
        if (b != cur) {
            const uint64_t g = base + (uint64_t)b;
            blk = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), traj, 1u), k0, k1);
            cur = b;
        }
        const int w = (op >> 1) & 3;
        return w == 0 ? blk.x : (w == 1 ? blk.y : (w == 2 ? blk.z : blk.w));
    }
};

// Rounding of one operation result to the propensity / uniform type.
// SR = 0: round to nearest; 1: stochastic rounding after every operation;
// 2: stochastic rounding only at the accumulation points (partial sums and
// the clock), round to nearest elsewhere.
template <int PREC, int SR>
struct Rounder {
    using T = ModeTraits<PREC>;
    SRBits bits;
    __device__ __forceinline__ typename T::P rnd(typename T::P x, int op)
    {
        if constexpr (T::k16) {
            if constexpr (SR == 1) return sr16<T::kFmt>(x, bits.word(op), (op & 1) != 0);
            else return rn16<T::kFmt>(x);
        } else {
            return x;
        }
    }
    __device__ __forceinline__ typename T::P rnd_acc(typename T::P x, int op)
    {
        if constexpr (T::k16) {
            if constexpr (SR != 0) return sr16<T::kFmt>(x, bits.word(op), (op & 1) != 0);
            else return rn16<T::kFmt>(x);
        } else {
            return x;
        }
    }
};

// ---------------------------------------------------------- compile-time loops
template <int... Is, class F>
__device__ __forceinline__ void unroll_impl(std::integer_sequence<int, Is...>, F &&f)
{
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void unroll(F &&f)
{
    unroll_impl(std::make_integer_sequence<int, N>{}, static_cast<F &&>(f));
}

// ------------------------------------------------------------- model policies
// A structure description S provides N, M and constexpr tables ord, nu, lw,
// hh (Hill exponent), hreg (regulator) and cs (constant species).  Every
// accessor is forced to a compile-time constant through integral_constant.
template <class S, bool NORM>
struct StaticCounts {
    __host__ __device__ static constexpr int chain_ops(int j)
    {
        if (S::lw[j] == 1) return S::hh[j] + 3;
        int ops = 0;
        for (int i = 0; i < S::N; ++i)
            if (!(NORM && S::cs[i] && S::ord[j][i] > 0)) ops += 2 * S::ord[j][i];
        return ops;
    }
    __host__ __device__ static constexpr int chain_start(int j)
    {
        int s = 0;
        for (int q = 0; q < j; ++q) s += chain_ops(q);
        return s;
    }
};

template <class S, bool NORM>
struct StaticModel {
    using C = StaticCounts<S, NORM>;
    static constexpr int N = S::N;
    static constexpr int M = S::M;
    template <int J> __device__ static constexpr bool active(const RunArgs &) { return true; }
    template <int J, int I> __device__ static constexpr int order(const RunArgs &)
    {
        return std::integral_constant<int, S::ord[J][I]>::value;
    }
    template <int J, int I> __device__ static constexpr int nu(const RunArgs &)
    {
        return std::integral_constant<int, S::cs[I] ? 0 : S::nu[J][I]>::value;
    }
    template <int J, int I> __device__ static constexpr bool folded(const RunArgs &)
    {
        return std::integral_constant<bool, (NORM && S::cs[I] && S::ord[J][I] > 0)>::value;
    }
    template <int J> __device__ static constexpr int law(const RunArgs &) { return std::integral_constant<int, S::lw[J]>::value; }
    template <int J> __device__ static constexpr int hill_h(const RunArgs &) { return std::integral_constant<int, S::hh[J]>::value; }
    template <int J> __device__ static constexpr int hill_reg(const RunArgs &) { return std::integral_constant<int, S::hreg[J]>::value; }
    template <int J> __device__ static constexpr int chain_start(const RunArgs &)
    {
        return std::integral_constant<int, C::chain_start(J)>::value;
    }
    __device__ static constexpr int total_chain_ops(const RunArgs &)
    {
        return std::integral_constant<int, C::chain_start(M)>::value;
    }
    __device__ static constexpr int last(const RunArgs &) { return M - 1; }
};

// General kernel: structure from the kernel arguments, bounded by kMaxN/kMaxM.
struct GeneralModel {
    static constexpr int N = kMaxN;
    static constexpr int M = kMaxM;
    template <int J> __device__ static bool active(const RunArgs &a) { return J < a.M; }
    template <int J, int I> __device__ static int order(const RunArgs &a) { return a.order[J][I]; }
    template <int J, int I> __device__ static int nu(const RunArgs &a) { return a.stoich[J][I]; }
    template <int J, int I> __device__ static bool folded(const RunArgs &a) { return a.folded[J][I] != 0; }
    template <int J> __device__ static int law(const RunArgs &a) { return a.law[J]; }
    template <int J> __device__ static int hill_h(const RunArgs &a) { return a.hill_h[J]; }
    template <int J> __device__ static int hill_reg(const RunArgs &a) { return a.hill_reg[J]; }
    template <int J> __device__ static int chain_start(const RunArgs &a) { return a.chain_start[J]; }
    __device__ static int total_chain_ops(const RunArgs &a) { return a.sr_ops; }
    __device__ static int last(const RunArgs &a) { return a.M - 1; }
};

// --------------------------------------------------------------- lane state
template <class Model, int PREC>
struct Lane {
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    int x[Model::N];
    P c[Model::M];       // c'_j in the propensity type
    P h0[Model::M];      // alpha0 (Hill rows)
    P h1[Model::M];      // alpha  (Hill rows)
    uint16_t c16[Model::M], h016[Model::M], h116[Model::M];   // bit patterns (RN 16-bit modes)
    P t;
    P s_next;            // next sample time (or +inf)
    int64_t n;           // events fired (direct method) / leaps done (tau-leaping)
    int64_t ev;          // reactions fired (tau-leaping)
    int64_t item;        // work item
    uint32_t traj;       // global trajectory id
    int k;               // next snapshot
    uint32_t status;
    bool active;
};

template <int PREC>
__device__ __forceinline__ typename ModeTraits<PREC>::P to_time(double v)
{
    using Tr = ModeTraits<PREC>;
    if constexpr (Tr::kF64) return v;
    else if constexpr (Tr::kUniform) return rn16<Tr::kFmt>((float)v);
    else return (float)v;
}

template <int PREC>
__device__ __forceinline__ typename ModeTraits<PREC>::P to_prop(double v)
{
    using Tr = ModeTraits<PREC>;
    if constexpr (Tr::kF64) return v;
    else if constexpr (Tr::k16) return rn16<Tr::kFmt>((float)v);
    else return (float)v;
}

template <int PREC>
__device__ __forceinline__ bool is_nan(typename ModeTraits<PREC>::P v) { return v != v; }

// --------------------------------------------------------------- snapshots
template <class Model>
__device__ __forceinline__ void store_state(const RunArgs &a, int k, int64_t item, const int *x, uint32_t &status)
{
    const int64_t col = item;
    const int64_t stride = a.n_traj;
    unroll<Model::N>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (i < a.N && ((a.out_mask >> i) & 1u)) {
            const int j = __popc(a.out_mask & ((1u << i) - 1u));   // position among the stored species
            const int64_t idx = ((int64_t)k * a.out_N + j) * stride + col;
            int v = x[i];
            if (a.state_bytes == 2) {
                if (v > 32767) { v = 32767; status |= ST_STATE_RANGE; }
                if (v < -32768) { v = -32768; status |= ST_STATE_RANGE; }
                static_cast<int16_t *>(a.out)[idx] = (int16_t)v;
            } else {
                static_cast<int32_t *>(a.out)[idx] = v;
            }
        }
    });
}

template <class Model, int PREC>
__device__ void finish(const RunArgs &a, Lane<Model, PREC> &L)
{
    while (L.k < a.K) {
        store_state<Model>(a, L.k, L.item, L.x, L.status);
        L.k += 1;
    }
    a.status[L.item] = L.status;
    if (a.n_events) a.n_events[L.item] = L.n;
    if (a.t_final) a.t_final[L.item] = (double)L.t;
    L.active = false;
}

// ------------------------------------------------------------ lane refill
template <class Model, int PREC>
__device__ void init_lane(const RunArgs &a, Lane<Model, PREC> &L, int64_t item, const typename ModeTraits<PREC>::P *smp)
{
    using P = typename ModeTraits<PREC>::P;
    L.item = item;
    L.traj = a.traj_offset + (uint32_t)item;
    const int set = a.n_sets > 1 ? (int)(item / a.traj_per_set) : 0;
    unroll<Model::N>([&](auto I) {
        constexpr int i = decltype(I)::value;
        L.x[i] = a.x0_tab ? a.x0_tab[(int64_t)set * a.N + i] : a.x0[i];
    });
    unroll<Model::M>([&](auto J) {
        constexpr int j = decltype(J)::value;
        if (Model::template active<j>(a)) {
            const double c = a.n_sets > 1 ? a.cprime_tab[(int64_t)set * a.M + j] : a.cprime[j];
            L.c[j] = to_prop<PREC>(c);
            if (Model::template law<j>(a) == 1) {
                const double g0 = (a.n_sets > 1 && a.hill_tab) ? a.hill_tab[((int64_t)set * a.M + j) * 2 + 0] : a.hill_a0[j];
                const double g1 = (a.n_sets > 1 && a.hill_tab) ? a.hill_tab[((int64_t)set * a.M + j) * 2 + 1] : a.hill_a[j];
                L.h0[j] = to_prop<PREC>(g0);
                L.h1[j] = to_prop<PREC>(g1);
            } else {
                L.h0[j] = P(0);
                L.h1[j] = P(0);
            }
        } else {
            L.c[j] = P(0);
            L.h0[j] = P(0);
            L.h1[j] = P(0);
        }
    });
    if constexpr (ModeTraits<PREC>::k16) {
        unroll<Model::M>([&](auto J) {
            constexpr int j = decltype(J)::value;
            L.c16[j] = Native16<ModeTraits<PREC>::kFmt>::from_f32(L.c[j]);
            L.h016[j] = Native16<ModeTraits<PREC>::kFmt>::from_f32(L.h0[j]);
            L.h116[j] = Native16<ModeTraits<PREC>::kFmt>::from_f32(L.h1[j]);
        });
    }
    L.t = P(0);
    L.n = 0;
    L.k = 0;
    L.status = 0;
    L.s_next = a.K > 0 ? smp[0] : P(__int_as_float(0x7F800000));
    L.active = true;
}

// Longest-first scheduling, launch 1: park an unfinished trajectory at the
// parking point (between step pairs: L.n is even).  Its priority is computed
// by the ordering kernels from the parked state.  The stores sit out of line,
// with the state passed by value, so the step keeps its registers.
static __device__ __noinline__ void park_store(const RunArgs &a, int64_t it, double t, int k, uint32_t status,
                                               int x0, int x1, int x2, int x3, int x4, int x5, int x6, int x7)
{
    const int x[kMaxN] = {x0, x1, x2, x3, x4, x5, x6, x7};
    a.parked[it] = 1u;
    a.park_t[it] = t;
    a.park_k[it] = k;
    a.park_status[it] = status;
#pragma unroll
    for (int i = 0; i < kMaxN; ++i)
        if (i < a.N) a.park_x[(int64_t)i * a.n_work + it] = x[i];
}

template <class Model, int PREC>
__device__ __forceinline__ void park(const RunArgs &a, Lane<Model, PREC> &L)
{
    static_assert(kMaxN == 8, "park_store takes eight species");
    int v[kMaxN];
    unroll<kMaxN>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if constexpr (i < Model::N) v[i] = L.x[i];
        else v[i] = 0;
    });
    park_store(a, L.item, (double)L.t, L.k, L.status, v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]);
    L.active = false;
}

// Longest-first scheduling, launch 2: continue a parked trajectory.  Every
// quantity a lane holds besides (x, t, n, k, status) is a function of the
// item, and random numbers are keyed by (trajectory id, n), so the resumed
// trajectory is the same one an unparked run produces.
template <class Model, int PREC>
__device__ __forceinline__ void resume_lane(const RunArgs &a, Lane<Model, PREC> &L, int64_t item,
                                            const typename ModeTraits<PREC>::P *smp)
{
    using P = typename ModeTraits<PREC>::P;
    init_lane<Model, PREC>(a, L, item, smp);
    L.n = a.resume_events;
    L.t = (P)a.park_t[item];
    L.k = a.park_k[item];
    L.status = a.park_status[item];
    unroll<Model::N>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (i < a.N) L.x[i] = a.park_x[(int64_t)i * a.n_work + item];
    });
    L.s_next = L.k < a.K ? smp[L.k] : P(__int_as_float(0x7F800000));
}

// ------------------------------------------------------------ one SSA step
// Executes step n = L.n with uniform words (w0, w1).  Returns with L.active
// cleared when the trajectory has finished (results written).
template <class Model, int PREC, int SR>
__device__ __forceinline__ void ssa_step(const RunArgs &a, Lane<Model, PREC> &L, uint32_t w0, uint32_t w1,
                                         const typename ModeTraits<PREC>::P *smp, typename ModeTraits<PREC>::P t_end)
{
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    constexpr int M = Model::M;

    if (L.n >= a.max_events) {
        if (a.parked && L.n < a.cap_events) {
            park<Model, PREC>(a, L);
            return;
        }
        L.status |= ST_MAX_EVENTS;
        finish<Model, PREC>(a, L);
        return;
    }

    Rounder<PREC, SR> R;
    int sr_total = 0;
    if constexpr (Tr::k16 && SR) {
        sr_total = SR == 2 ? Model::last(a) + 1
                           : Model::total_chain_ops(a) + (Tr::kUniform ? (Model::last(a) + 5) : 0);
        const int B = (sr_total + 7) >> 3;
        R.bits.base = (uint64_t)L.n * (uint64_t)B;
        R.bits.traj = L.traj;
        R.bits.k0 = a.key0;
        R.bits.k1 = a.key1;
        R.bits.cur = -1;
    }

    // 1. propensities a_j (Sec. 2 step 1), in the propensity type
    P prop[M];
    if constexpr (Tr::k16 && SR != 1) {
        using H = Native16<Tr::kFmt>;
        unroll<M>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if (Model::template law<j>(a) == 1) {
                const int reg = Model::template hill_reg<j>(a);
                int xr = 0;
                unroll<Model::N>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    if (i == reg) xr = L.x[i];
                });
                const uint16_t Pv = H::from_int(xr);
                uint16_t q = Pv;
                const int h = Model::template hill_h<j>(a);
                for (int m = 1; m < h; ++m) q = H::mul(q, Pv);
                const uint16_t d = H::add(H::from_f32(1.0f), q);
                const uint16_t f = H::from_f32(H::to_f32(L.h116[j]) / H::to_f32(d));
                prop[j] = H::to_f32(H::add(L.h016[j], f));
            } else {
                uint16_t av = L.c16[j];
                bool zero = false;
                unroll<Model::N>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    const int r = Model::template order<j, i>(a);
                    if (r > 0 && !Model::template folded<j, i>(a)) {
                        zero = zero || (L.x[i] < r);
                        for (int m = 0; m < r; ++m) av = H::mul(av, H::from_int(L.x[i] - m));
                    }
                });
                prop[j] = zero ? P(0) : H::to_f32(av);
            }
        });
    } else unroll<M>([&](auto J) {
        constexpr int j = decltype(J)::value;
        prop[j] = P(0);
        if (!Model::template active<j>(a)) return;
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
                const int r = Model::template order<j, i>(a);
                if (r > 0 && !Model::template folded<j, i>(a)) {
                    zero = zero || (L.x[i] < r);
                    for (int m = 0; m < r; ++m) {
                        const P f = R.rnd((P)(L.x[i] - m), op++);
                        av = R.rnd(av * f, op++);
                    }
                }
            });
            prop[j] = zero ? P(0) : av;
        }
    });

    // 2. partial sums S_j and a0 (Sec. 2 step 1; sensitive operation 1)
    P S[M];
    P a0 = P(0);
    {
        int op = SR == 2 ? 0 : Model::total_chain_ops(a);
        unroll<M>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if (!Model::template active<j>(a)) { S[j] = a0; return; }
            if constexpr (j == 0) {
                S[0] = prop[0];
            } else {
                if constexpr (Tr::kUniform) S[j] = R.rnd_acc(S[j - 1] + prop[j], op++);
                else S[j] = S[j - 1] + prop[j];
            }
            a0 = S[j];
        });
    }

    // degenerate states (readings for a0 = NaN, inf, 0)
    if (is_nan<PREC>(a0)) { L.status |= ST_NAN; finish<Model, PREC>(a, L); return; }
    if (a0 == P(__int_as_float(0x7F800000))) { L.status |= ST_OVERFLOW; finish<Model, PREC>(a, L); return; }
    if (a0 == P(0)) { finish<Model, PREC>(a, L); return; }

    // 3. waiting time and selection target (Sec. 2 steps 2-3)
    P tau, target, t_new;
    if constexpr (Tr::kF64) {
        const double u1 = ((double)w0 + 1.0) * 0x1p-32;
        const double u2 = (double)w1 * 0x1p-32;
        const double E = -log_f64(u1);
        tau = E / a0;
        target = u2 * a0;
        t_new = L.t + tau;
    } else {
        const float u1 = (float)((w0 >> 8) + 1u) * 0x1p-24f;
        const float u2 = (float)(w1 >> 8) * 0x1p-24f;
        if constexpr (Tr::kUniform) {
            int op = Model::total_chain_ops(a) + Model::last(a);
            const float E = R.rnd(-log_f32(u1), op++);
            const float U2 = R.rnd(u2, op++);
            tau = R.rnd(E / a0, op++);
            target = R.rnd(U2 * a0, op++);
            t_new = R.rnd_acc(L.t + tau, SR == 2 ? Model::last(a) : op);
        } else {
            const float E = -log_f32(u1);
            tau = E / a0;
            target = u2 * a0;
            t_new = L.t + tau;
        }
    }

    // 4a. snapshots strictly before the event time
    while (L.s_next < t_new) {
        store_state<Model>(a, L.k, L.item, L.x, L.status);
        L.k += 1;
        L.s_next = L.k < a.K ? smp[L.k] : P(__int_as_float(0x7F800000));
    }
    if (t_new > t_end) { finish<Model, PREC>(a, L); return; }

    // 4b. selection: smallest mu with S_mu > target; else last a_j > 0
    int mu = -1;
    unroll<M>([&](auto J) {
        constexpr int j = M - 1 - decltype(J)::value;
        if (Model::template active<j>(a) && S[j] > target) mu = j;
    });
    if (mu < 0) {
        unroll<M>([&](auto J) {
            constexpr int j = decltype(J)::value;
            if (Model::template active<j>(a) && prop[j] > P(0)) mu = j;
        });
    }

    // 4c. integer state update x += nu_mu, clock t = t_new
    bool negative = false;
    unroll<Model::N>([&](auto I) {       // branch-free: d_i = nu[mu][i] by selects
        constexpr int i = decltype(I)::value;
        int d = 0;
        bool moves = false;
        unroll<M>([&](auto J) {
            constexpr int j = decltype(J)::value;
            const int v = Model::template nu<j, i>(a);
            if (v != 0) {
                d = (mu == j) ? v : d;
                moves = true;
            }
        });
        if (moves) {
            L.x[i] += d;
            negative = negative || (L.x[i] < 0);
        }
    });
    L.t = t_new;
    L.n += 1;
    if (negative) {
        L.status |= ST_STATE_RANGE;
        finish<Model, PREC>(a, L);
    }
}

// Propensities of the general model (runtime structure), reading R3.
template <int PREC, int SR>
__device__ __forceinline__ void general_propensities(const RunArgs &a, const Lane<GeneralModel, PREC> &L,
                                                     Rounder<PREC, SR> &R, typename ModeTraits<PREC>::P *prop)
{
    using P = typename ModeTraits<PREC>::P;
#pragma unroll 1
    for (int j = 0; j < a.M; ++j) {
        int op = a.chain_start[j];
        if (a.law[j] == 1) {
            const P Pv = R.rnd((P)L.x[a.hill_reg[j]], op++);
            P q = Pv;
            for (int m = 1; m < a.hill_h[j]; ++m) q = R.rnd(q * Pv, op++);
            const P d = R.rnd(P(1) + q, op++);
            const P f = R.rnd(L.h1[j] / d, op++);
            prop[j] = R.rnd(L.h0[j] + f, op++);
        } else {
            P av = L.c[j];
            bool zero = false;
#pragma unroll 1
            for (int i = 0; i < a.N; ++i) {
                const int r = a.order[j][i];
                if (r == 0 || a.folded[j][i]) continue;
                zero = zero || (L.x[i] < r);
                for (int m = 0; m < r; ++m) {
                    const P f = R.rnd((P)(L.x[i] - m), op++);
                    av = R.rnd(av * f, op++);
                }
            }
            prop[j] = zero ? P(0) : av;
        }
    }
}

// ------------------------------------------------- one step, general model
// Same contract as ssa_step, with the structure read from the kernel
// arguments in runtime loops (state and tables in local memory).  Used for
// networks that match no compiled structure.
template <int PREC, int SR>
__device__ __noinline__ void ssa_step_general(const RunArgs &a, Lane<GeneralModel, PREC> &L, uint32_t w0, uint32_t w1,
                                              const typename ModeTraits<PREC>::P *smp,
                                              typename ModeTraits<PREC>::P t_end)
{
    using Tr = ModeTraits<PREC>;
    using P = typename Tr::P;
    const P kInf = P(__int_as_float(0x7F800000));

    if (L.n >= a.max_events) {
        if (a.parked && L.n < a.cap_events) {
            park<GeneralModel, PREC>(a, L);
            return;
        }
        L.status |= ST_MAX_EVENTS;
        finish<GeneralModel, PREC>(a, L);
        return;
    }
    Rounder<PREC, SR> R;
    if constexpr (Tr::k16 && SR) {
        const int sr_total = SR == 2 ? a.M : a.sr_ops + (Tr::kUniform ? (a.M - 1 + 5) : 0);
        R.bits.base = (uint64_t)L.n * (uint64_t)((sr_total + 7) >> 3);
        R.bits.traj = L.traj;
        R.bits.k0 = a.key0;
        R.bits.k1 = a.key1;
        R.bits.cur = -1;
    }

    // propensities
    P prop[kMaxM];
    general_propensities<PREC, SR>(a, L, R, prop);
    // partial sums
    P S[kMaxM];
    S[0] = prop[0];
    {
        int op = SR == 2 ? 0 : a.sr_ops;
#pragma unroll 1
        for (int j = 1; j < a.M; ++j) {
            if constexpr (Tr::kUniform) S[j] = R.rnd_acc(S[j - 1] + prop[j], op++);
            else S[j] = S[j - 1] + prop[j];
        }
    }
    const P a0 = S[a.M - 1];
    if (is_nan<PREC>(a0)) { L.status |= ST_NAN; finish<GeneralModel, PREC>(a, L); return; }
    if (a0 == kInf) { L.status |= ST_OVERFLOW; finish<GeneralModel, PREC>(a, L); return; }
    if (a0 == P(0)) { finish<GeneralModel, PREC>(a, L); return; }

    P tau, target, t_new;
    if constexpr (Tr::kF64) {
        const double u1 = ((double)w0 + 1.0) * 0x1p-32;
        const double u2 = (double)w1 * 0x1p-32;
        const double E = -log_f64(u1);
        tau = E / a0;
        target = u2 * a0;
        t_new = L.t + tau;
    } else {
        const float u1 = (float)((w0 >> 8) + 1u) * 0x1p-24f;
        const float u2 = (float)(w1 >> 8) * 0x1p-24f;
        if constexpr (Tr::kUniform) {
            int op = a.sr_ops + a.M - 1;
            const float E = R.rnd(-log_f32(u1), op++);
            const float U2 = R.rnd(u2, op++);
            tau = R.rnd(E / a0, op++);
            target = R.rnd(U2 * a0, op++);
            t_new = R.rnd_acc(L.t + tau, SR == 2 ? a.M - 1 : op);
        } else {
            const float E = -log_f32(u1);
            tau = E / a0;
            target = u2 * a0;
            t_new = L.t + tau;
        }
    }
    while (L.s_next < t_new) {
        store_state<GeneralModel>(a, L.k, L.item, L.x, L.status);
        L.k += 1;
        L.s_next = L.k < a.K ? smp[L.k] : kInf;
    }
    if (t_new > t_end) { finish<GeneralModel, PREC>(a, L); return; }

    int mu = -1;
#pragma unroll 1
    for (int j = 0; j < a.M; ++j)
        if (S[j] > target) { mu = j; break; }
    if (mu < 0) {
#pragma unroll 1
        for (int j = a.M - 1; j >= 0; --j)
            if (prop[j] > P(0)) { mu = j; break; }
    }
    bool negative = false;
#pragma unroll 1
    for (int i = 0; i < a.N; ++i) {
        L.x[i] += a.stoich[mu][i];
        negative = negative || (L.x[i] < 0);
    }
    L.t = t_new;
    L.n += 1;
    if (negative) {
        L.status |= ST_STATE_RANGE;
        finish<GeneralModel, PREC>(a, L);
    }
}

// ------------------------------------------------------- tail compaction
// Once the work queue has drained, lanes whose trajectories end stay idle
// until every lane of their warp is done, and an issue-bound SM spends the
// same issue slots on a warp with one busy lane as on a full one.  So a warp
// whose unfinished trajectories fit into the idle lanes of the other warps of
// its block hands them over through shared memory and leaves the work loop;
// the block's remaining trajectories then run on fewer, fuller warps.
// Between two step pairs a trajectory's whole state is (x, t, n, k, status,
// item): everything else a lane holds is a function of the item (constants,
// trajectory id, next sample time; random numbers are keyed by (id, n)), so
// a move is exact and results do not depend on it.
//
// Protocol (one lock per block, taken by lane 0 of a warp; every wait on it
// is bounded):
//  * `live` has bit w set while warp w is in the loop.  A warp gives its
//    trajectories away only while another warp is live and their idle lanes
//    (as last reported in `act`) can take them; it then clears its bit.
//  * A live warp leaves with no work only when the pool is empty (checked
//    under the lock).  Hence whenever the pool holds records some live warp
//    remains, and it takes them into idle lanes at its next refill check.
//  * Each warp leaves once, so a trajectory moves at most warps - 1 times.
//  * A lock wait that gives up (counted) decides nothing: a busy warp runs
//    on, an idle one leaves with its `live` bit still set, so records given
//    to the pool afterwards may find no taker.  Therefore, once every warp
//    of the block has left the loop, warp 0 checks the pool and resumes
//    whatever it still holds (counted), as the only live warp (so it never
//    gives work away), and no trajectory is ever left unfinished: results
//    never depend on give-ups.
constexpr int kPoolCap = 96;              // records held at once
constexpr int kPoolWarps = 8;             // warps per block (blockDim <= 256)
constexpr int kPoolLockSpins = 1 << 22;   // bound on the lock wait (under a second)

template <class Model, int PREC>
struct TailPool {
    using P = typename ModeTraits<PREC>::P;
    int lock;
    int count;                  // records held, in slots 0 .. count-1
    unsigned live;              // bit w: warp w still in the work loop
    int act[kPoolWarps];        // busy lanes of warp w at its last check
    int64_t item[kPoolCap];
    int64_t n[kPoolCap];
    P t[kPoolCap];
    int k[kPoolCap];
    uint32_t status[kPoolCap];
    int x[Model::N][kPoolCap];
};

template <class Model, int PREC>
__device__ __forceinline__ void pool_init(TailPool<Model, PREC> *p)
{
    if (threadIdx.x == 0) {
        const int nw = (int)((blockDim.x + 31u) >> 5);
        p->lock = 0;
        p->count = 0;
        p->live = (1u << nw) - 1u;
        for (int w = 0; w < kPoolWarps; ++w) p->act[w] = 32;
    }
}

__device__ __forceinline__ bool pool_acquire(int *lock, int spins)
{
    for (int i = 0; i < spins; ++i) {
        if (atomicCAS(lock, 0, 1) == 0) {
            __threadfence_block();
            return true;
        }
        __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void pool_release(int *lock)
{
    __threadfence_block();
    atomicExch(lock, 0);
}

// Lane 0's decision at a pool visit (kept out of line: it runs only after the
// queue has drained).  Returns (timeout << 31) | (op << 24) | (base << 12) | num.
static __device__ __noinline__ unsigned pool_decide(int *lock, int *count_p, unsigned *live_p, int *act, int w, int nb,
                                             unsigned long long *stats, int spins)
{
    volatile int *vcount = count_p;
    volatile unsigned *vlive = live_p;
    volatile int *vact = act;
    int cnt = *vcount;
    unsigned live = *vlive;
    int room = -cnt;
    for (int v = 0; v < kPoolWarps; ++v)
        if (v != w && ((live >> v) & 1u)) room += 32 - vact[v];
    const bool maybe = nb == 0 || (cnt > 0 && nb < 32) || (nb <= room && cnt + nb <= kPoolCap);
    vact[w] = nb;
    if (!maybe) return 0u;
    if (!pool_acquire(lock, spins)) {
        atomicAdd(&stats[1], 1ull);
        return 1u << 31;
    }
    cnt = *vcount;
    live = *vlive;
    room = -cnt;
    for (int v = 0; v < kPoolWarps; ++v)
        if (v != w && ((live >> v) & 1u)) room += 32 - vact[v];
    unsigned op = 0, base = 0, num = 0;
    if (cnt > 0 && nb < 32) {
        op = 1;
        num = (unsigned)min(cnt, 32 - nb);
        base = (unsigned)cnt - num;
        *vcount = (int)base;
        vact[w] = nb + (int)num;
    } else if (nb == 0) {
        op = 3;
        *vlive = live & ~(1u << w);
    } else if (nb <= room && cnt + nb <= kPoolCap && (live & ~(1u << w)) != 0u) {
        op = 2;
        num = (unsigned)nb;
        base = (unsigned)cnt;
        *vcount = cnt + nb;
        *vlive = live & ~(1u << w);
    }
    if (op == 0) pool_release(lock);
    return (op << 24) | (base << 12) | num;
}

// One visit of a warp to its block's pool at a refill check (whole warp).
// Takes records into idle lanes, or gives the warp's trajectories away.
// Returns true when the warp leaves the work loop.
template <class Model, int PREC>
__device__ __forceinline__ bool pool_visit(const RunArgs &a, TailPool<Model, PREC> *p, Lane<Model, PREC> &L,
                                           const typename ModeTraits<PREC>::P *smp)
{
    using P = typename ModeTraits<PREC>::P;
    const unsigned lane = threadIdx.x & 31u;
    const int w = (int)(threadIdx.x >> 5);
    const unsigned busy = __ballot_sync(0xFFFFFFFFu, L.active);
    const int nb = __popc(busy);
    // 0 nothing, 1 take records, 2 give trajectories away, 3 leave (idle, pool empty)
    int op = 0, base = 0, num = 0, ok = 1;
    if (lane == 0) {
        const unsigned r = pool_decide(&p->lock, &p->count, &p->live, p->act, w, nb, a.tail_stats,
                                       a.lock_spins > 0 ? a.lock_spins : kPoolLockSpins);
        ok = (int)(r >> 31) ^ 1;
        op = (int)((r >> 24) & 0x7Fu);
        base = (int)((r >> 12) & 0xFFFu);
        num = (int)(r & 0xFFFu);
    }
    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
    if (!ok) return nb == 0;   // lock wait gave up (counted): leave only if idle (records: block-end resume)
    op = __shfl_sync(0xFFFFFFFFu, op, 0);
    if (op == 0) return false;
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    num = __shfl_sync(0xFFFFFFFFu, num, 0);
    __syncwarp();
    __threadfence_block();   // lane 0 holds the lock: the records are ours to read or write
    const unsigned below = (1u << lane) - 1u;
    if (op == 1 && !L.active) {
        const int r = __popc(~busy & below);
        if (r < num) {
            const int s = base + r;
            init_lane<Model, PREC>(a, L, p->item[s], smp);
            L.n = p->n[s];
            L.t = p->t[s];
            L.k = p->k[s];
            L.status = p->status[s];
            unroll<Model::N>([&](auto I) {
                constexpr int i = decltype(I)::value;
                L.x[i] = p->x[i][s];
            });
            L.s_next = L.k < a.K ? smp[L.k] : P(__int_as_float(0x7F800000));
        }
    } else if (op == 2 && L.active) {
        const int s = base + __popc(busy & below);
        p->item[s] = L.item;
        p->n[s] = L.n;
        p->t[s] = L.t;
        p->k[s] = L.k;
        p->status[s] = L.status;
        unroll<Model::N>([&](auto I) {
            constexpr int i = decltype(I)::value;
            p->x[i][s] = L.x[i];
        });
        L.active = false;
    }
    __syncwarp();
    if (lane == 0) {
        pool_release(&p->lock);
        if (op == 2) atomicAdd(&a.tail_stats[0], (unsigned long long)num);
    }
    return op >= 2;
}

// ---------------------------------------------------------- the work loop
// Persistent loop of one warp over one work queue: lanes that are idle take
// the next items (one atomicAdd per warp), then every lane runs `slice_pairs`
// pairs of steps (one Philox block of stream 0 per pair) before the next
// refill check.  With a pool (single-queue kernel), warps of a block hand
// trajectories to each other once the queue has drained (tail compaction,
// above).  Returns once the warp has no more work, so the caller may move the
// whole warp to another queue.
template <class Model, int PREC, int SR>
__device__ __forceinline__ void run_queue(const RunArgs &a, const typename ModeTraits<PREC>::P *smp,
                                          typename ModeTraits<PREC>::P t_end,
                                          TailPool<Model, PREC> *pool = nullptr)
{
    const unsigned lane = threadIdx.x & 31u;
    Lane<Model, PREC> L;
    L.active = false;
    bool drained = false;
    const int slice = a.slice_pairs > 0 ? a.slice_pairs : 1;
    for (;;) {
        const unsigned need = __ballot_sync(0xFFFFFFFFu, !L.active && !drained);
        if (need) {
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(a.queue_head, (unsigned long long)__popc(need));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (!L.active && !drained) {
                const unsigned long long item = base + (unsigned long long)__popc(need & ((1u << lane) - 1u));
                if (a.resume_order) {
                    if (item < *a.resume_count) resume_lane<Model, PREC>(a, L, a.resume_order[item], smp);
                    else drained = true;
                } else if (item < (unsigned long long)a.n_work) {
                    init_lane<Model, PREC>(a, L, (int64_t)item, smp);
                } else {
                    drained = true;
                }
            }
        }
        // the pool's count may change between lanes' reads: decide by ballot, warp-uniformly
        if (pool && __any_sync(0xFFFFFFFFu, drained || *(volatile int *)&pool->count > 0)) {
            if (pool_visit<Model, PREC>(a, pool, L, smp)) break;
        }
        if (__ballot_sync(0xFFFFFFFFu, L.active) == 0u) break;
        for (int s = 0; s < slice; ++s) {
            // L.n is even for every active lane here: block n/2 holds steps n, n+1
            const uint64_t blk = (uint64_t)(L.n >> 1);
            const uint4 u = philox4x32_10(make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), L.traj, 0u), a.key0, a.key1);
            if constexpr (std::is_same<Model, GeneralModel>::value) {
                if (L.active) ssa_step_general<PREC, SR>(a, L, u.x, u.y, smp, t_end);
                if (L.active) ssa_step_general<PREC, SR>(a, L, u.z, u.w, smp, t_end);
            } else {
                if (L.active) ssa_step<Model, PREC, SR>(a, L, u.x, u.y, smp, t_end);
                if (L.active) ssa_step<Model, PREC, SR>(a, L, u.z, u.w, smp, t_end);
            }
            if (s + 1 < slice && __ballot_sync(0xFFFFFFFFu, L.active) == 0u) break;
        }
    }
}

template <int PREC>
__device__ __forceinline__ void load_samples(const double *samples, int K, typename ModeTraits<PREC>::P *smp)
{
    for (int k = threadIdx.x; k < K; k += blockDim.x) smp[k] = to_time<PREC>(samples[k]);
    __syncthreads();
}

// ------------------------------------------------------------- the kernels
// One model, one queue: arguments in parameter space.
template <class Model, int PREC, int SR>
__global__ void __launch_bounds__(256, (KernelMinBlocks<Model, PREC, SR>::value)) ssa_kernel(const __grid_constant__ RunArgs a)
{
    using P = typename ModeTraits<PREC>::P;
    __shared__ P smp[kMaxK];
    __shared__ TailPool<Model, PREC> pool;
    const bool pooled = a.tail_stats != nullptr;
    if (pooled) pool_init(&pool);
    load_samples<PREC>(a.samples, a.K, smp);   // ends with __syncthreads
    for (int pass = 0;; ++pass) {
        run_queue<Model, PREC, SR>(a, smp, to_time<PREC>(a.t_end), pooled ? &pool : nullptr);
        if (!pooled || pass > 0) break;
        // every warp has left the loop: records stranded by a lock wait that
        // gave up are resumed by warp 0 (the pool no longer changes)
        __syncthreads();
        if (pool.count == 0 || threadIdx.x >= 32) break;
        if (threadIdx.x == 0) {
            atomicAdd(&a.tail_stats[2], (unsigned long long)pool.count);
            // warp 0 is the only warp left: with stale `live` bits of warps
            // that left after a give-up, it could hand its work back to the
            // pool and leave; as the sole live warp it only takes records
            pool.live = 1u;
        }
        __syncwarp();
    }
}

// Several groups (heterogeneous structures and parameter sweeps), one queue
// per group, in one persistent launch.  Each warp drains the groups in order;
// a warp whose lanes have all finished group g moves on to g + 1 without
// waiting for other warps.  Group descriptors live in global memory.
constexpr int kMaxGroups = 16;

struct BatchArgs {
    int n_groups;
    int normalise;
    int K;
    double t_end;
    const RunArgs *groups;             // device [n_groups]
    int8_t family[kMaxGroups];         // 0 general, 1..5 compiled structures
    double samples[kMaxK];
};

}  // namespace ssa

#include "ssa_models.h"

namespace ssa {

template <int FAM, int PREC, int SR>
__device__ __forceinline__ void run_family(const RunArgs &a, int normalise, const typename ModeTraits<PREC>::P *smp,
                                           typename ModeTraits<PREC>::P t_end)
{
    if constexpr (FAM == 1) run_queue<StaticModel<models::BirthDeath, false>, PREC, SR>(a, smp, t_end);
    else if constexpr (FAM == 2) {
        if (normalise) run_queue<StaticModel<models::Schlogl, true>, PREC, SR>(a, smp, t_end);
        else run_queue<StaticModel<models::Schlogl, false>, PREC, SR>(a, smp, t_end);
    }
    else if constexpr (FAM == 3) run_queue<StaticModel<models::Telegraph, false>, PREC, SR>(a, smp, t_end);
    else if constexpr (FAM == 4) run_queue<StaticModel<models::Dimer, false>, PREC, SR>(a, smp, t_end);
    else if constexpr (FAM == 5) run_queue<StaticModel<models::Repressilator, false>, PREC, SR>(a, smp, t_end);
    else run_queue<GeneralModel, PREC, SR>(a, smp, t_end);
}

// FAMS lists the structure families compiled into this instantiation; a
// group whose family is not listed is skipped (the host never sends one).
template <int PREC, int SR, int... FAMS>
__global__ void __launch_bounds__(256) ssa_batch_kernel(const __grid_constant__ BatchArgs b)
{
    using P = typename ModeTraits<PREC>::P;
    __shared__ P smp[kMaxK];
    load_samples<PREC>(b.samples, b.K, smp);
    const P t_end = to_time<PREC>(b.t_end);
    for (int g = 0; g < b.n_groups; ++g) {
        const RunArgs &a = b.groups[g];
        const int fam = b.family[g];
        ((fam == FAMS ? (run_family<FAMS, PREC, SR>(a, b.normalise, smp, t_end), 0) : 0), ...);
    }
}

}  // namespace ssa
