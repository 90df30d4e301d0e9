/*
 * ssa_oracle.c -- reference implementation of the reduced-precision Gillespie
 * direct method (Kimpson, Flegg & Flegg, "Reduced-Precision Stochastic
 * Simulation for Mathematical Biology").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle: a plain, slow,
 * single-threaded CPU implementation written from the paper.  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table or constant generator with the CUDA engine in
 * paper_2605_00479_gb300/csrc; the two are written independently and agree
 * only because both follow the arithmetic contract spelled out below.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fno-fast-math -shared -fPIC.
 * No fused multiply-add is allowed: every operation below is one IEEE-754
 * binary32/binary64 operation in round-to-nearest-even.
 *
 * Paper passages followed (section / equation / table of the paper):
 *   - Direct method steps 1-4 (Sec. 2, "In the Direct Method formulation"):
 *       propensities and a0, tau = -ln(u1)/a0, smallest mu with
 *       sum_{j<=mu} a_j > u2*a0, x += nu_mu, t += tau.
 *   - Precision partition (Sec. 3.2 "Mixed-precision partitioning", Sec. 4
 *     mode list): FP64, FP32, mixed (16-bit propensities, fp32 sum and time,
 *     integer state), uniform (every operation in the 16-bit type).
 *   - Formats (Table "formats"): binary16 = 1/5/10 bits, bfloat16 = 1/8/7.
 *   - Stochastic rounding (Sec. 3.3, SR equation): round up with probability
 *     (x - x-)/(x+ - x-); applied after every arithmetic operation whose result
 *     type is the 16-bit type ("every-op" SR, Sec. 3.3).
 *   - Propensity forms: mass action with combinatorial factors (Sec. 4.2
 *     Schloegl k2 n(n-1)(n-2); Sec. 4.4 dimer kf nA(nA-1)/2) and Hill
 *     repression alpha0 + alpha/(1+P^h) (Sec. 4.5).
 *   - Propensity normalisation (Sec. 4.2, rescaled Schloegl): reservoir
 *     (constant) species are folded into the rate constant, k1*A and k3*B.
 *
 * Where the paper is silent the readings below are used (each one also listed
 * in the design notes):
 *   R1 rate constants are Gillespie c-constants; c'_j = c_j / prod_i r_ij!,
 *      computed in binary64, then (normalise) multiplied by the falling
 *      factorials of the constant species' counts, species ascending,
 *      factor m = 0..r-1 ascending.  c'_j is converted to the propensity type
 *      once, by round-to-nearest (binary64 -> binary32 -> 16-bit).
 *   R2 time in mixed mode is binary32 (Sec. 4 mode list).
 *   R3 propensity op order: a = c'; for each reactant species i ascending, for
 *      m = 0..r_ij-1: f = rnd(x_i - m); a = rnd(a * f).  Zero when any
 *      x_i < r_ij (no operations, but the step's random-bit schedule is fixed).
 *      Hill: P = rnd(x_reg); q = P; (h-1) times q = rnd(q*P); d = rnd(1 + q);
 *      f = rnd(alpha / d); a = rnd(alpha0 + f).
 *   R4 a 16-bit operation is the binary32 operation on the widened operands
 *      followed by one rounding to the 16-bit type.
 *   R5 SR rounding bits: each SR operation consumes one 16-bit random value.
 *      bfloat16: add the 16 bits to the 16 discarded bits of the binary32
 *      pattern and truncate.  binary16: add the low 13 bits, aligned with the
 *      most significant discarded bit, and truncate (13 bits of rounding
 *      resolution).  Overflow past the largest finite value gives infinity.
 *   R6 random numbers: Philox4x32-10 with key = (seed lo, seed hi) and
 *      counter = (block lo, block hi, trajectory id, stream).  Each trajectory
 *      reads two streams of 32-bit words (word w is lane w mod 4 of block w/4).
 *      Stream 0 holds the uniforms: step n takes words 2n and 2n+1,
 *      u1 = (w0 + 1) 2^-32 in (0,1] and u2 = w1 2^-32 in [0,1) in FP64 mode,
 *      u1 = ((w0 >> 8) + 1) 2^-24 and u2 = (w1 >> 8) 2^-24 otherwise, so every
 *      mode sees the same draws (common random numbers).  Stream 1 holds the
 *      SR bits: with S rounding operations per step and B = ceil(S/8), step n
 *      owns the whole blocks [n*B, (n+1)*B), i.e. words [4nB, 4nB + 4B), and
 *      operation i takes the low (even i) or high (odd i) half of word
 *      4nB + i/2; the unused tail of the last block is discarded.  RN modes
 *      never read stream 1.
 *   R7 uniform mode: E = rnd(-log(u1)) with log evaluated in binary32 on u1,
 *      U2 = rnd(u2), tau = rnd(E / a0), target = rnd(U2 * a0),
 *      t_new = rnd(t + tau).  SR operation order within a step: propensity
 *      chains (reaction order), partial sums S_1..S_{M-1}, E, U2, tau,
 *      target, t_new.
 *   R7b selective SR (rounding = 2, uniform modes only; the paper names the
 *      strategy, "SR applied only at accumulation points", without testing
 *      it): the partial sums S_1..S_{M-1} and t_new are rounded
 *      stochastically, every other operation by RN.  These M operations use
 *      SR slots 0..M-1 of the step (B = ceil(M/8) blocks).
 *   R8 log: own implementation, ln x = e ln2 + 2 atanh(s), s = (m-1)/(m+1),
 *      m in [sqrt(1/2), sqrt(2)], odd atanh series to s^9 (binary32) or s^23
 *      (binary64), Cody-Waite split of ln2, Horner order fixed below.
 *   R9 degenerate steps: a0 == 0 ends the trajectory (absorbing state);
 *      a0 = inf -> status OVERFLOW; a0 = NaN -> status NAN; n >= max_events
 *      -> status MAX_EVENTS; a negative count after an update -> status
 *      STATE_RANGE; remaining snapshots are filled with the current state.
 *      If no partial sum exceeds the target, the last reaction with a_j > 0
 *      fires.
 *   R10 snapshot k receives the state after every event with event time
 *      <= s_k: before an event at t_new is applied, all s_k < t_new are
 *      written.  Sample times and t_end are rounded to the time type by RN.
 */
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#include <math.h>   /* sqrt, sqrtf, floor, floorf, ceil (IEEE, exact) */

/* ------------------------------------------------------------------------ */
/* Bit access                                                                */
/* ------------------------------------------------------------------------ */
static uint32_t f2u(float x) { uint32_t u; memcpy(&u, &x, 4); return u; }
static float u2f(uint32_t u) { float x; memcpy(&x, &u, 4); return x; }
static uint64_t d2u(double x) { uint64_t u; memcpy(&u, &x, 8); return u; }
static double u2d(uint64_t u) { double x; memcpy(&x, &u, 8); return x; }

static int f32_is_nan(float x) { return (f2u(x) & 0x7FFFFFFFu) > 0x7F800000u; }
static int f32_is_inf(float x) { return (f2u(x) & 0x7FFFFFFFu) == 0x7F800000u; }
static int f64_is_nan(double x) { return (d2u(x) & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull; }
static int f64_is_inf(double x) { return (d2u(x) & 0x7FFFFFFFFFFFFFFFull) == 0x7FF0000000000000ull; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of the     */
/* multiply-xor bijection on a 128-bit counter with a 64-bit key that is      */
/* bumped by the Weyl constants between rounds.                               */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

typedef struct {
    uint32_t key[2];
    uint32_t traj;          /* global trajectory id */
    uint32_t stream;        /* 0: uniforms, 1: stochastic-rounding bits */
    uint64_t block;         /* index of the block held in buf */
    int have;
    uint32_t buf[4];
} word_stream;

static uint32_t stream_word(word_stream *s, uint64_t w)
{
    uint64_t b = w >> 2;
    if (!s->have || b != s->block) {
        uint32_t ctr[4];
        ctr[0] = (uint32_t)b;
        ctr[1] = (uint32_t)(b >> 32);
        ctr[2] = s->traj;
        ctr[3] = s->stream;
        oracle_philox4x32_10(ctr, s->key, s->buf);
        s->block = b;
        s->have = 1;
    }
    return s->buf[w & 3];
}

/* ------------------------------------------------------------------------ */
/* Natural logarithm (reading R8).  x = 2^e * m with m in [sqrt(1/2),sqrt(2)],*/
/* ln m = 2 atanh(s), s = (m - 1)/(m + 1), atanh s = s + s^3/3 + s^5/5 + ...  */
/* ln 2 = LN2_HI + LN2_LO with LN2_HI holding the leading 16 (binary32) or    */
/* 32 (binary64) bits of ln 2, so that e * LN2_HI is exact.                    */
/* Domain: positive normal numbers (the uniforms used are >= 2^-53).          */
/* ------------------------------------------------------------------------ */
float oracle_log_f32(float x)
{
    const float LN2_HI = 0x1.62e400p-1f;
    const float LN2_LO = 0x1.7f7d1cp-20f;
    uint32_t u = f2u(x);
    int e = (int)(u >> 23) - 127;
    uint32_t mb = (u & 0x7FFFFFu) | 0x3F800000u;      /* m in [1, 2) */
    if (mb > 0x3FB504F3u) {                             /* m > sqrt(2): halve it */
        mb -= 0x00800000u;
        e += 1;
    }
    float m = u2f(mb);
    float f = m - 1.0f;
    float d = m + 1.0f;
    float s = f / d;
    float z = s * s;
    /* 2 atanh(s) = 2s + s z (2/3 + z (2/5 + z (2/7 + z 2/9))) */
    float p = 2.0f / 9.0f;
    p = z * p;  p = (2.0f / 7.0f) + p;
    p = z * p;  p = (2.0f / 5.0f) + p;
    p = z * p;  p = (2.0f / 3.0f) + p;
    float r = s * z;
    r = r * p;
    float two_s = s + s;
    r = two_s + r;
    float ef = (float)e;
    float lo = ef * LN2_LO;
    lo = lo + r;
    float hi = ef * LN2_HI;
    return hi + lo;
}

double oracle_log_f64(double x)
{
    const double LN2_HI = 0x1.62e42fee00000p-1;
    const double LN2_LO = 0x1.a39ef35793c76p-33;
    uint64_t u = d2u(x);
    int e = (int)(u >> 52) - 1023;
    uint64_t mb = (u & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    if (mb > 0x3FF6A09E667F3BCCull) {                  /* m > sqrt(2) */
        mb -= 0x0010000000000000ull;
        e += 1;
    }
    double m = u2d(mb);
    double f = m - 1.0;
    double d = m + 1.0;
    double s = f / d;
    double z = s * s;
    /* coefficients 2/(2k+1), k = 1..11, evaluated by Horner from the top */
    double p = 2.0 / 23.0;
    p = z * p;  p = (2.0 / 21.0) + p;
    p = z * p;  p = (2.0 / 19.0) + p;
    p = z * p;  p = (2.0 / 17.0) + p;
    p = z * p;  p = (2.0 / 15.0) + p;
    p = z * p;  p = (2.0 / 13.0) + p;
    p = z * p;  p = (2.0 / 11.0) + p;
    p = z * p;  p = (2.0 / 9.0) + p;
    p = z * p;  p = (2.0 / 7.0) + p;
    p = z * p;  p = (2.0 / 5.0) + p;
    p = z * p;  p = (2.0 / 3.0) + p;
    double r = s * z;
    r = r * p;
    double two_s = s + s;
    r = two_s + r;
    double ef = (double)e;
    double lo = ef * LN2_LO;
    lo = lo + r;
    double hi = ef * LN2_HI;
    return hi + lo;
}

/* ------------------------------------------------------------------------ */
/* 16-bit formats.  binary16: 1 sign, 5 exponent (bias 15), 10 fraction bits, */
/* subnormal quantum 2^-24, largest finite 65504.  bfloat16: the upper 16     */
/* bits of a binary32 pattern.                                                 */
/* ------------------------------------------------------------------------ */
float oracle_f16_to_f32(uint16_t h)
{
    uint32_t sign = (uint32_t)(h >> 15) << 31;
    uint32_t e = (h >> 10) & 0x1Fu;
    uint32_t m = h & 0x3FFu;
    if (e == 31) return u2f(sign | 0x7F800000u | (m << 13));
    if (e == 0) {
        float v = (float)m * 0x1p-24f;                  /* exact */
        return (sign ? -v : v);
    }
    return u2f(sign | ((e - 15 + 127) << 23) | (m << 13));
}

float oracle_bf16_to_f32(uint16_t b) { return u2f((uint32_t)b << 16); }

/* binary32 -> binary16.  sr == 0: round to nearest, ties to even.
 * sr != 0: stochastic rounding with the low 13 bits of r (reading R5). */
uint16_t oracle_f32_to_f16(float x, int sr, uint32_t r)
{
    uint32_t u = f2u(x);
    uint16_t sign = (uint16_t)((u >> 16) & 0x8000u);
    uint32_t a = u & 0x7FFFFFFFu;
    if (a > 0x7F800000u) return sign | 0x7E00u;        /* NaN */
    if (a == 0x7F800000u) return sign | 0x7C00u;       /* infinity */
    if (a == 0) return sign;
    int be = (int)(a >> 23);
    uint64_t sig = (a & 0x7FFFFFu) | (be ? 0x800000u : 0u);
    int ex = be ? be - 150 : -149;                      /* |x| = sig * 2^ex */
    int E = be ? be - 127 : -126;
    if (E > 15) return sign | 0x7C00u;                  /* >= 2^16: beyond binary16 */
    int q = (E >= -14) ? E - 10 : -24;                  /* exponent of the binary16 quantum */
    int k = q - ex;                                     /* discarded bits, >= 13 */
    uint64_t n;
    if (!sr) {
        if (k > 40) {
            n = 0;                                       /* below half a quantum */
        } else {
            uint64_t one = 1;
            n = sig >> k;
            uint64_t rem = sig & ((one << k) - 1);
            uint64_t half = one << (k - 1);
            if (rem > half || (rem == half && (n & 1))) n += 1;
        }
    } else {
        if (k > 36) {
            n = 0;                                       /* sig + r13*2^(k-13) < 2^k */
        } else {
            uint64_t add = (uint64_t)(r & 0x1FFFu) << (k - 13);
            n = (sig + add) >> k;
        }
    }
    uint32_t hb;
    if (q == -24) hb = (uint32_t)n;                     /* n == 1024 encodes 2^-14 */
    else hb = ((uint32_t)(E + 15) << 10) + (uint32_t)(n - 1024);
    if (hb >= 0x7C00u) hb = 0x7C00u;
    return sign | (uint16_t)hb;
}

/* binary32 -> bfloat16.  sr == 0: round to nearest even.  sr != 0: add the
 * low 16 bits of r to the discarded half and truncate (reading R5). */
uint16_t oracle_f32_to_bf16(float x, int sr, uint32_t r)
{
    uint32_t u = f2u(x);
    uint16_t sign = (uint16_t)((u >> 16) & 0x8000u);
    uint32_t a = u & 0x7FFFFFFFu;
    if (a > 0x7F800000u) return sign | 0x7FC0u;
    if (a == 0x7F800000u) return sign | 0x7F80u;
    uint32_t n;
    if (!sr) {
        n = a >> 16;
        uint32_t rem = a & 0xFFFFu;
        if (rem > 0x8000u || (rem == 0x8000u && (n & 1u))) n += 1;
    } else {
        n = (a + (r & 0xFFFFu)) >> 16;
    }
    if (n >= 0x7F80u) n = 0x7F80u;
    return sign | (uint16_t)n;
}

/* ------------------------------------------------------------------------ */
/* Model and run parameters                                                  */
/* ------------------------------------------------------------------------ */
enum { P_FP64 = 0, P_FP32 = 1, P_MIXED_F16 = 2, P_MIXED_BF16 = 3, P_UNIFORM_F16 = 4, P_UNIFORM_BF16 = 5 };
enum { LAW_MASS_ACTION = 0, LAW_HILL = 1 };
enum { ST_OVERFLOW = 1, ST_MAX_EVENTS = 2, ST_STATE_RANGE = 4, ST_NAN = 8 };

#define OR_MAX_N 64
#define OR_MAX_M 64

typedef struct {
    int N, M;
    const int32_t *order;     /* [M][N] */
    const int32_t *stoich;    /* [M][N] */
    const int32_t *law;       /* [M] */
    const double *hill;       /* [M][4] alpha0, alpha, h, regulator */
    const uint8_t *constant;  /* [N] */
    int normalise;
    double cprime[OR_MAX_M];  /* R1, binary64 */
    int folded[OR_MAX_M][OR_MAX_N];  /* 1: factor moved into cprime */
} omodel;

/* ------------------------------------------------------------------------ */
/* Rounding context: which 16-bit format, RN or SR, and where this step's SR  */
/* values live in the trajectory's word stream.                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int bf16;          /* 0: binary16, 1: bfloat16 */
    int sr;
    word_stream *ws;
    uint64_t sr_base;  /* first SR word of the current step */
    int op;            /* SR operation index within the step */
} rounder;

/* Round a binary32 value to the 16-bit type; return it widened (exact). */
static float rnd16(rounder *R, float x)
{
    uint32_t r = 0;
    if (R->sr) {
        uint32_t w = stream_word(R->ws, R->sr_base + (uint64_t)(R->op >> 1));
        r = (R->op & 1) ? (w >> 16) : (w & 0xFFFFu);
    }
    R->op += 1;
    if (R->bf16) return oracle_bf16_to_f32(oracle_f32_to_bf16(x, R->sr, r));
    return oracle_f16_to_f32(oracle_f32_to_f16(x, R->sr, r));
}

/* round to the 16-bit type by RN without consuming an SR slot (constants) */
static float rn16(int bf16, float x)
{
    if (bf16) return oracle_bf16_to_f32(oracle_f32_to_bf16(x, 0, 0));
    return oracle_f16_to_f32(oracle_f32_to_f16(x, 0, 0));
}

static double factorial(int r)
{
    double f = 1.0;
    for (int i = 2; i <= r; ++i) f = f * (double)i;
    return f;
}

/* number of 16-bit rounding operations in the propensity chain of reaction j */
static int chain_ops(const omodel *md, int j)
{
    if (md->law[j] == LAW_HILL) return (int)md->hill[4 * j + 2] + 3;
    int ops = 0;
    for (int i = 0; i < md->N; ++i)
        if (!md->folded[j][i]) ops += 2 * md->order[j * md->N + i];
    return ops;
}

/* ------------------------------------------------------------------------ */
/* Propensities per precision family (reading R3)                            */
/* ------------------------------------------------------------------------ */
static int reactants_short(const omodel *md, int j, const int32_t *x)
{
    for (int i = 0; i < md->N; ++i) {
        int r = md->order[j * md->N + i];
        if (r > 0 && !md->folded[j][i] && x[i] < r) return 1;
    }
    return 0;
}

static double prop_f64(const omodel *md, int j, const int32_t *x, const double *cp, const double *h0, const double *h1)
{
    if (md->law[j] == LAW_HILL) {
        int hh = (int)md->hill[4 * j + 2];
        int reg = (int)md->hill[4 * j + 3];
        double P = (double)x[reg];
        double q = P;
        for (int m = 1; m < hh; ++m) q = q * P;
        double d = 1.0 + q;
        double f = h1[j] / d;
        return h0[j] + f;
    }
    if (reactants_short(md, j, x)) return 0.0;
    double a = cp[j];
    for (int i = 0; i < md->N; ++i) {
        if (md->folded[j][i]) continue;
        for (int m = 0; m < md->order[j * md->N + i]; ++m) a = a * (double)(x[i] - m);
    }
    return a;
}

static float prop_f32(const omodel *md, int j, const int32_t *x, const float *cp, const float *h0, const float *h1)
{
    if (md->law[j] == LAW_HILL) {
        int hh = (int)md->hill[4 * j + 2];
        int reg = (int)md->hill[4 * j + 3];
        float P = (float)x[reg];
        float q = P;
        for (int m = 1; m < hh; ++m) q = q * P;
        float d = 1.0f + q;
        float f = h1[j] / d;
        return h0[j] + f;
    }
    if (reactants_short(md, j, x)) return 0.0f;
    float a = cp[j];
    for (int i = 0; i < md->N; ++i) {
        if (md->folded[j][i]) continue;
        for (int m = 0; m < md->order[j * md->N + i]; ++m) a = a * (float)(x[i] - m);
    }
    return a;
}

/* 16-bit propensity; R->op must point at this reaction's first SR slot */
static float prop_16(const omodel *md, int j, const int32_t *x, const float *cp, const float *h0, const float *h1, rounder *R)
{
    int op_end = R->op + chain_ops(md, j);
    float a;
    if (md->law[j] == LAW_HILL) {
        int hh = (int)md->hill[4 * j + 2];
        int reg = (int)md->hill[4 * j + 3];
        float P = rnd16(R, (float)x[reg]);
        float q = P;
        for (int m = 1; m < hh; ++m) q = rnd16(R, q * P);
        float d = rnd16(R, 1.0f + q);
        float f = rnd16(R, h1[j] / d);
        a = rnd16(R, h0[j] + f);
    } else if (reactants_short(md, j, x)) {
        a = 0.0f;
    } else {
        a = cp[j];
        for (int i = 0; i < md->N; ++i) {
            if (md->folded[j][i]) continue;
            for (int m = 0; m < md->order[j * md->N + i]; ++m) {
                float f = rnd16(R, (float)(x[i] - m));
                a = rnd16(R, a * f);
            }
        }
    }
    R->op = op_end;  /* the schedule is fixed even when the chain was skipped */
    return a;
}

/* ------------------------------------------------------------------------ */
/* Output helpers                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    void *out;
    int state_bytes;
    int64_t n_traj;
    int64_t col;
    int K, N;
    uint32_t mask;   /* stored species (bit i: species i) */
    int outN;        /* number of stored species */
} sink;

/* Snapshot k of the stored species, in ascending species order. */
static void write_snapshot(const sink *S, int k, const int32_t *x, uint32_t *status)
{
    int j = 0;
    for (int i = 0; i < S->N; ++i) {
        if (!((S->mask >> i) & 1u)) continue;
        int64_t idx = ((int64_t)k * S->outN + j++) * S->n_traj + S->col;
        if (S->state_bytes == 2) {
            int32_t v = x[i];
            if (v > 32767) { v = 32767; *status |= ST_STATE_RANGE; }
            if (v < -32768) { v = -32768; *status |= ST_STATE_RANGE; }
            ((int16_t *)S->out)[idx] = (int16_t)v;
        } else {
            ((int32_t *)S->out)[idx] = x[i];
        }
    }
}

/* Returns 1 when a count went negative (the trajectory ends: R9).  The
 * STATE_RANGE bit alone does not end it: int16 snapshot storage sets the same
 * bit when it clamps, and storage never changes a trajectory. */
static int apply_event(const omodel *md, int mu, int32_t *x, uint32_t *status)
{
    int negative = 0;
    for (int i = 0; i < md->N; ++i) {
        if (md->constant && md->constant[i]) continue;
        x[i] += md->stoich[mu * md->N + i];
        if (x[i] < 0) negative = 1;
    }
    if (negative) *status |= ST_STATE_RANGE;
    return negative;
}

/* ------------------------------------------------------------------------ */
/* One trajectory per precision family                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    double t_end;
    int K;
    const double *samples;
    int64_t max_events;
} runp;

/* ------------------------------------------------------------------------ */
/* Step trace (test hook, single-threaded use): the inputs and intermediates  */
/* of step `g_trace_step` of the next trajectory simulated, so that a test    */
/* can recompute that one step independently.  Layout of the buffer:          */
/*   [0] 1 when recorded, [1] n, [2] t before the step, [3..3+N) x before,   */
/*   [16..16+M) propensities, [48..48+M) partial sums S_1..S_M, [80] a0,     */
/*   [81] u1, [82] u2, [83] E, [84] U2 (the u2 the target uses), [85] tau,   */
/*   [86] target, [87] t_new, [88] mu.  Values widened to binary64 (exact).  */
/* ------------------------------------------------------------------------ */
static double *g_trace = NULL;
static int64_t g_trace_step = -1;

void oracle_trace_step(double *buf, int64_t step)
{
    g_trace = buf;
    g_trace_step = step;
}

static void trace_record(const omodel *md, int64_t n, double t, const int32_t *x, const double *a,
                         const double *S, double u1, double u2, double E, double U2, double tau, double target,
                         double t_new, int mu)
{
    double *b = g_trace;
    g_trace = NULL;
    b[0] = 1.0;
    b[1] = (double)n;
    b[2] = t;
    for (int i = 0; i < md->N && i < 13; ++i) b[3 + i] = (double)x[i];
    for (int j = 0; j < md->M && j < 32; ++j) { b[16 + j] = a[j]; b[48 + j] = S[j]; }
    b[80] = S[md->M - 1];
    b[81] = u1; b[82] = u2; b[83] = E; b[84] = U2; b[85] = tau; b[86] = target; b[87] = t_new;
    b[88] = (double)mu;
}

static void trace_f32(const omodel *md, int64_t n, float t, const int32_t *x, const float *a, const float *S,
                      float u1, float u2, float E, float U2, float tau, float target, float t_new, int mu)
{
    double ad[OR_MAX_M], Sd[OR_MAX_M];
    for (int j = 0; j < md->M; ++j) { ad[j] = a[j]; Sd[j] = S[j]; }
    trace_record(md, n, t, x, ad, Sd, u1, u2, E, U2, tau, target, t_new, mu);
}

static void traj_f64(const omodel *md, const runp *rp, word_stream *ws, int32_t *x,
                     const sink *S, uint32_t *status, int64_t *n_events, double *t_final)
{
    const int M = md->M;
    double cp[OR_MAX_M], h0[OR_MAX_M], h1[OR_MAX_M], a[OR_MAX_M], Ssum[OR_MAX_M];
    for (int j = 0; j < M; ++j) {
        cp[j] = md->cprime[j];
        h0[j] = md->law[j] == LAW_HILL ? md->hill[4 * j] : 0.0;
        h1[j] = md->law[j] == LAW_HILL ? md->hill[4 * j + 1] : 0.0;
    }
    double t = 0.0;
    int64_t n = 0;
    int k = 0;
    for (;;) {
        if (n >= rp->max_events) { *status |= ST_MAX_EVENTS; break; }
        for (int j = 0; j < M; ++j) a[j] = prop_f64(md, j, x, cp, h0, h1);
        Ssum[0] = a[0];
        for (int j = 1; j < M; ++j) Ssum[j] = Ssum[j - 1] + a[j];
        double a0 = Ssum[M - 1];
        if (f64_is_nan(a0)) { *status |= ST_NAN; break; }
        if (f64_is_inf(a0)) { *status |= ST_OVERFLOW; break; }
        if (a0 == 0.0) break;
        uint64_t w = (uint64_t)n * 2u;
        uint32_t w0 = stream_word(ws, w), w1 = stream_word(ws, w + 1);
        double u1 = ((double)w0 + 1.0) * 0x1p-32;
        double u2 = (double)w1 * 0x1p-32;
        double E = -oracle_log_f64(u1);
        double tau = E / a0;
        double target = u2 * a0;
        double t_new = t + tau;
        while (k < rp->K && rp->samples[k] < t_new) write_snapshot(S, k++, x, status);
        if (t_new > rp->t_end) break;
        int mu = -1;
        for (int j = 0; j < M; ++j) if (Ssum[j] > target) { mu = j; break; }
        if (mu < 0) for (int j = M - 1; j >= 0; --j) if (a[j] > 0.0) { mu = j; break; }
        if (g_trace && n == g_trace_step) trace_record(md, n, t, x, a, Ssum, u1, u2, E, u2, tau, target, t_new, mu);
        const int negative = apply_event(md, mu, x, status);
        t = t_new;
        n += 1;
        if (negative) break;
    }
    while (k < rp->K) write_snapshot(S, k++, x, status);
    *n_events = n;
    *t_final = t;
}

/* FP32 mode (bf16 < 0) and mixed modes (bf16 = 0 binary16, 1 bfloat16) */
static void traj_f32_mixed(const omodel *md, const runp *rp, word_stream *ws, word_stream *wsr, int32_t *x,
                           const sink *S, uint32_t *status, int64_t *n_events, double *t_final,
                           int fmt, int sr)
{
    const int M = md->M;
    const int mixed = fmt >= 0;
    float cp[OR_MAX_M], h0[OR_MAX_M], h1[OR_MAX_M], a[OR_MAX_M], Ssum[OR_MAX_M];
    int nsr = 0;
    for (int j = 0; j < M; ++j) {
        float c = (float)md->cprime[j];
        float g0 = md->law[j] == LAW_HILL ? (float)md->hill[4 * j] : 0.0f;
        float g1 = md->law[j] == LAW_HILL ? (float)md->hill[4 * j + 1] : 0.0f;
        if (mixed) { c = rn16(fmt, c); g0 = rn16(fmt, g0); g1 = rn16(fmt, g1); }
        cp[j] = c; h0[j] = g0; h1[j] = g1;
        if (mixed && sr) nsr += chain_ops(md, j);
    }
    const uint64_t Ws = 4u * (uint64_t)((nsr + 7) / 8);   /* SR words per step: whole blocks */
    float t_end = (float)rp->t_end;
    float smp[1024];
    for (int kk = 0; kk < rp->K; ++kk) smp[kk] = (float)rp->samples[kk];
    rounder R;
    R.bf16 = fmt; R.sr = sr; R.ws = wsr; R.sr_base = 0; R.op = 0;
    float t = 0.0f;
    int64_t n = 0;
    int k = 0;
    for (;;) {
        if (n >= rp->max_events) { *status |= ST_MAX_EVENTS; break; }
        uint64_t w = (uint64_t)n * 2u;
        R.sr_base = (uint64_t)n * Ws;
        R.op = 0;
        for (int j = 0; j < M; ++j)
            a[j] = mixed ? prop_16(md, j, x, cp, h0, h1, &R) : prop_f32(md, j, x, cp, h0, h1);
        Ssum[0] = a[0];
        for (int j = 1; j < M; ++j) Ssum[j] = Ssum[j - 1] + a[j];
        float a0 = Ssum[M - 1];
        if (f32_is_nan(a0)) { *status |= ST_NAN; break; }
        if (f32_is_inf(a0)) { *status |= ST_OVERFLOW; break; }
        if (a0 == 0.0f) break;
        uint32_t w0 = stream_word(ws, w), w1 = stream_word(ws, w + 1);
        float u1 = (float)((w0 >> 8) + 1u) * 0x1p-24f;
        float u2 = (float)(w1 >> 8) * 0x1p-24f;
        float E = -oracle_log_f32(u1);
        float tau = E / a0;
        float target = u2 * a0;
        float t_new = t + tau;
        while (k < rp->K && smp[k] < t_new) write_snapshot(S, k++, x, status);
        if (t_new > t_end) break;
        int mu = -1;
        for (int j = 0; j < M; ++j) if (Ssum[j] > target) { mu = j; break; }
        if (mu < 0) for (int j = M - 1; j >= 0; --j) if (a[j] > 0.0f) { mu = j; break; }
        if (g_trace && n == g_trace_step) trace_f32(md, n, t, x, a, Ssum, u1, u2, E, u2, tau, target, t_new, mu);
        const int negative = apply_event(md, mu, x, status);
        t = t_new;
        n += 1;
        if (negative) break;
    }
    while (k < rp->K) write_snapshot(S, k++, x, status);
    *n_events = n;
    *t_final = (double)t;
}

/* Experiment switch for the readings the paper leaves silent in uniform mode
 * (how the random variates and the selection enter 16-bit arithmetic); 0 is
 * the contract (reading R7).  Bits: 1 round u1 to the 16-bit type (RN) before
 * the logarithm, as a 16-bit uniform draw would be; 2 keep u2 in binary32;
 * 4 keep the target U2 * a0 in binary32; 8 select over binary32 partial sums
 * (a0 and the clock still 16-bit).  Used only by the documented experiment
 * that compares these readings with the paper's rescaled Schloegl rows. */
static int g_uniform_variant = 0;

void oracle_set_uniform_variant(int v) { g_uniform_variant = v; }

static void traj_uniform(const omodel *md, const runp *rp, word_stream *ws, word_stream *wsr, int32_t *x,
                         const sink *S, uint32_t *status, int64_t *n_events, double *t_final,
                         int fmt, int sr)
{
    const int M = md->M;
    float cp[OR_MAX_M], h0[OR_MAX_M], h1[OR_MAX_M], a[OR_MAX_M], Ssum[OR_MAX_M];
    int nsr = 0;
    for (int j = 0; j < M; ++j) {
        cp[j] = rn16(fmt, (float)md->cprime[j]);
        h0[j] = md->law[j] == LAW_HILL ? rn16(fmt, (float)md->hill[4 * j]) : 0.0f;
        h1[j] = md->law[j] == LAW_HILL ? rn16(fmt, (float)md->hill[4 * j + 1]) : 0.0f;
        nsr += chain_ops(md, j);
    }
    nsr += (M - 1) + 5;   /* partial sums, E, U2, tau, target, t_new */
    if (sr == 2) nsr = M; /* selective SR: partial sums and t_new only */
    const uint64_t Ws = 4u * (uint64_t)((nsr + 7) / 8);   /* SR words per step: whole blocks */
    float t_end = rn16(fmt, (float)rp->t_end);
    float smp[1024];
    for (int kk = 0; kk < rp->K; ++kk) smp[kk] = rn16(fmt, (float)rp->samples[kk]);
    /* R rounds the propensity chains and the variates; A the accumulation
     * points (the same rounder unless SR is selective) */
    rounder R, Racc;
    R.bf16 = fmt; R.sr = sr == 1; R.ws = wsr; R.sr_base = 0; R.op = 0;
    Racc = R;
    Racc.sr = sr != 0;
    rounder *A = sr == 2 ? &Racc : &R;
    float t = 0.0f;
    int64_t n = 0;
    int k = 0;
    for (;;) {
        if (n >= rp->max_events) { *status |= ST_MAX_EVENTS; break; }
        uint64_t w = (uint64_t)n * 2u;
        R.sr_base = (uint64_t)n * Ws;
        R.op = 0;
        Racc.sr_base = R.sr_base;
        Racc.op = 0;
        for (int j = 0; j < M; ++j) a[j] = prop_16(md, j, x, cp, h0, h1, &R);
        Ssum[0] = a[0];
        for (int j = 1; j < M; ++j) Ssum[j] = rnd16(A, Ssum[j - 1] + a[j]);
        float a0 = Ssum[M - 1];
        float Sel[OR_MAX_M];   /* the sums the selection compares (variant 8: binary32) */
        Sel[0] = a[0];
        for (int j = 1; j < M; ++j) Sel[j] = (g_uniform_variant & 8) ? Sel[j - 1] + a[j] : Ssum[j];
        if (f32_is_nan(a0)) { *status |= ST_NAN; break; }
        if (f32_is_inf(a0)) { *status |= ST_OVERFLOW; break; }
        if (a0 == 0.0f) break;
        uint32_t w0 = stream_word(ws, w), w1 = stream_word(ws, w + 1);
        float u1 = (float)((w0 >> 8) + 1u) * 0x1p-24f;
        float u2 = (float)(w1 >> 8) * 0x1p-24f;
        if (g_uniform_variant & 1) u1 = rn16(fmt, u1);
        float E = rnd16(&R, -oracle_log_f32(u1));
        float U2 = rnd16(&R, u2);
        if (g_uniform_variant & 2) U2 = u2;
        float tau = rnd16(&R, E / a0);
        float target = rnd16(&R, U2 * a0);
        if (g_uniform_variant & 4) target = U2 * a0;
        float t_new = rnd16(A, t + tau);
        while (k < rp->K && smp[k] < t_new) write_snapshot(S, k++, x, status);
        if (t_new > t_end) break;
        int mu = -1;
        for (int j = 0; j < M; ++j) if (Sel[j] > target) { mu = j; break; }
        if (mu < 0) for (int j = M - 1; j >= 0; --j) if (a[j] > 0.0f) { mu = j; break; }
        if (g_trace && n == g_trace_step) trace_f32(md, n, t, x, a, Ssum, u1, u2, E, U2, tau, target, t_new, mu);
        const int negative = apply_event(md, mu, x, status);
        t = t_new;
        n += 1;
        if (negative) break;
    }
    while (k < rp->K) write_snapshot(S, k++, x, status);
    *n_events = n;
    *t_final = (double)t;
}

/* ------------------------------------------------------------------------ */
/* Public entry: simulate trajectories g0 .. g0+n_traj-1.  Returns 0 on        */
/* success, -1 on invalid arguments.                                           */
/* Snapshots: out[(k*Ns + j)*n_traj + r] for the j-th stored species (bit i of  */
/* out_species stores species i; 0 stores all), int32 or int16 per state_bytes. */
/* ------------------------------------------------------------------------ */
int oracle_run(int N, int M, const int32_t *order, const int32_t *stoich, const double *rate,
               const int32_t *law, const double *hill, const uint8_t *constant,
               const int32_t *x0, int64_t n_traj, uint64_t g0, double t_end,
               int K, const double *samples, int precision, int rounding, int normalise,
               uint64_t seed, int64_t max_events, int state_bytes, uint32_t out_species,
               void *out, uint32_t *status, int64_t *n_events, double *t_final)
{
    if (N < 1 || N > OR_MAX_N || M < 1 || M > OR_MAX_M || K < 0 || K > 1024) return -1;
    if (out_species >> N) return -1;
    if (precision < 0 || precision > 5 || rounding < 0 || rounding > 2) return -1;
    if (rounding == 1 && precision < 2) return -1;
    if (rounding == 2 && precision < 4) return -1;   /* selective SR: uniform modes only */
    if (state_bytes != 2 && state_bytes != 4) return -1;
    if (n_traj < 0 || g0 + (uint64_t)n_traj > 0x100000000ull) return -1;  /* 32-bit trajectory ids */
    omodel md;
    memset(&md, 0, sizeof(md));
    md.N = N; md.M = M; md.order = order; md.stoich = stoich; md.law = law;
    md.hill = hill; md.constant = constant; md.normalise = normalise;
    for (int j = 0; j < M; ++j) {
        if (law[j] == LAW_HILL) { md.cprime[j] = 0.0; continue; }
        double denom = 1.0;
        for (int i = 0; i < N; ++i) denom = denom * factorial(order[j * N + i]);
        double c = rate[j] / denom;
        if (normalise && constant) {
            for (int i = 0; i < N; ++i) {
                if (!constant[i] || order[j * N + i] == 0) continue;
                for (int m = 0; m < order[j * N + i]; ++m) c = c * (double)(x0[i] - m);
                md.folded[j][i] = 1;
            }
        }
        md.cprime[j] = c;
    }
    runp rp;
    rp.t_end = t_end; rp.K = K; rp.samples = samples; rp.max_events = max_events;
    for (int64_t r = 0; r < n_traj; ++r) {
        word_stream ws, wsr;
        memset(&ws, 0, sizeof(ws));
        ws.key[0] = (uint32_t)seed;
        ws.key[1] = (uint32_t)(seed >> 32);
        ws.traj = (uint32_t)(g0 + (uint64_t)r);
        ws.stream = 0;
        wsr = ws;
        wsr.stream = 1;
        int32_t x[OR_MAX_N];
        for (int i = 0; i < N; ++i) x[i] = x0[i];
        sink S;
        S.out = out; S.state_bytes = state_bytes; S.n_traj = n_traj; S.col = r; S.K = K; S.N = N;
        S.mask = out_species ? out_species : (uint32_t)((1u << N) - 1u);
        S.outN = 0;
        for (int i = 0; i < N; ++i) S.outN += (int)((S.mask >> i) & 1u);
        uint32_t st = 0;
        int64_t ne = 0;
        double tf = 0.0;
        switch (precision) {
        case P_FP64: traj_f64(&md, &rp, &ws, x, &S, &st, &ne, &tf); break;
        case P_FP32: traj_f32_mixed(&md, &rp, &ws, &wsr, x, &S, &st, &ne, &tf, -1, 0); break;
        case P_MIXED_F16: traj_f32_mixed(&md, &rp, &ws, &wsr, x, &S, &st, &ne, &tf, 0, rounding); break;
        case P_MIXED_BF16: traj_f32_mixed(&md, &rp, &ws, &wsr, x, &S, &st, &ne, &tf, 1, rounding); break;
        case P_UNIFORM_F16: traj_uniform(&md, &rp, &ws, &wsr, x, &S, &st, &ne, &tf, 0, rounding); break;
        default: traj_uniform(&md, &rp, &ws, &wsr, x, &S, &st, &ne, &tf, 1, rounding); break;
        }
        if (status) status[r] = st;
        if (n_events) n_events[r] = ne;
        if (t_final) t_final[r] = tf;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Array forms of the scalar primitives, for the pin tests.                   */
/* ------------------------------------------------------------------------ */
void oracle_f32_to_f16_array(const float *x, int64_t n, int sr, const uint32_t *r, uint16_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_f32_to_f16(x[i], sr, r ? r[i] : 0u);
}

void oracle_f32_to_bf16_array(const float *x, int64_t n, int sr, const uint32_t *r, uint16_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_f32_to_bf16(x[i], sr, r ? r[i] : 0u);
}

void oracle_f16_to_f32_array(const uint16_t *h, int64_t n, float *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_f16_to_f32(h[i]);
}

void oracle_log_f32_array(const float *x, int64_t n, float *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_log_f32(x[i]);
}

void oracle_log_f64_array(const double *x, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_log_f64(x[i]);
}

/* Philox blocks for counters (c0 + i, c1, c2, c3), i = 0..n-1 (no carry). */
void oracle_philox_array(const uint32_t ctr[4], const uint32_t key[2], int64_t n, uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t c[4];
        c[0] = ctr[0] + (uint32_t)i; c[1] = ctr[1]; c[2] = ctr[2]; c[3] = ctr[3];
        oracle_philox4x32_10(c, key, out + 4 * i);
    }
}

/* ======================================================================== */
/* Mixed-precision tau-leaping (the paper names the combination of reduced  */
/* precision with tau-leaping as future work, Sec. 5 and Sec. 6; explicit    */
/* tau-leaping is the approximate family of its Table 1).                   */
/*                                                                           */
/* Readings:                                                                 */
/*  T1 fixed leap size tau; leap n covers [n tau, (n+1) tau); L =            */
/*     ceil(t_end / tau) leaps; the leap grid is exact (binary64), precision */
/*     applies to propensities, lambda and the Poisson sampler.              */
/*  T2 a_j by reading R3 (RN/SR per mode; SR slots from stream 1, leap n     */
/*     owning blocks [nB, (n+1)B)); lambda_j = a_j tau in the accumulator    */
/*     type (binary64 / binary32), or rnd16(a_j * rnd16(tau)) in uniform     */
/*     mode (one SR slot per channel, after the chains).                     */
/*  T3 k_j ~ Poisson(lambda_j) by the sampler below in binary64 (FP64 mode)  */
/*     or binary32 (all other modes); its uniforms come from Philox with     */
/*     counter = (word block, leap n, trajectory id, 2 + j).                 */
/*  T4 x += sum_j nu_j k_j in 64-bit integers; a negative count is set to 0  */
/*     and flagged TAU_CLAMPED (16); events += sum_j k_j.                    */
/*  T5 snapshots: before leap n, every s_k < (n+1) tau receives the current  */
/*     state; after the last leap the remaining ones receive the final one. */
/* ======================================================================== */
enum { ST_TAU_CLAMPED = 16 };

/* exp by Cody-Waite reduction x = k ln2 + r, |r| <= ln2/2, Taylor series of  */
/* e^r (to r^7 in binary32, r^13 in binary64), scaled by 2^k.  Domain        */
/* [-30, 0] (the sampler needs exp(-lambda) for lambda < 10).               */
float oracle_exp_f32(float x)
{
    const float LN2_HI = 0x1.62e400p-1f;
    const float LN2_LO = 0x1.7f7d1cp-20f;
    const float INV_LN2 = 0x1.715476p+0f;
    float kf = x * INV_LN2;
    kf = kf + 0.5f;
    int k = (int)kf;
    if ((float)k > kf) k -= 1;                         /* floor */
    float fk = (float)k;
    float r = x - fk * LN2_HI;
    r = r - fk * LN2_LO;
    float p = 1.0f / 5040.0f;
    p = p * r + 1.0f / 720.0f;
    p = p * r + 1.0f / 120.0f;
    p = p * r + 1.0f / 24.0f;
    p = p * r + 1.0f / 6.0f;
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    return p * u2f((uint32_t)(k + 127) << 23);
}

double oracle_exp_f64(double x)
{
    const double LN2_HI = 0x1.62e42fee00000p-1;
    const double LN2_LO = 0x1.a39ef35793c76p-33;
    const double INV_LN2 = 0x1.71547652b82fep+0;
    double kf = x * INV_LN2;
    kf = kf + 0.5;
    int k = (int)kf;
    if ((double)k > kf) k -= 1;
    double fk = (double)k;
    double r = x - fk * LN2_HI;
    r = r - fk * LN2_LO;
    double p = 1.0 / 6227020800.0;                     /* 1/13! */
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
    return p * u2d((uint64_t)(k + 1023) << 52);
}

/* log k! : summed logarithms below 10, Stirling's series above. */
static float logfact_f32(float k)
{
    if (k < 10.0f) {
        float s = 0.0f;
        for (int i = 2; (float)i <= k; ++i) s = s + oracle_log_f32((float)i);
        return s;
    }
    const float HALF_LN_2PI = 0x1.d67f1cp-1f;           /* 0.5 ln(2 pi) */
    float x = k + 1.0f;
    float lx = oracle_log_f32(x);
    float s = (x - 0.5f) * lx;
    s = s - x;
    s = s + HALF_LN_2PI;
    s = s + (1.0f / 12.0f) / x;
    s = s - (1.0f / 360.0f) / (x * x * x);
    return s;
}

static double logfact_f64(double k)
{
    if (k < 10.0) {
        double s = 0.0;
        for (int i = 2; (double)i <= k; ++i) s = s + oracle_log_f64((double)i);
        return s;
    }
    const double HALF_LN_2PI = 0x1.d67f1c864beb5p-1;
    double x = k + 1.0;
    double lx = oracle_log_f64(x);
    double s = (x - 0.5) * lx;
    s = s - x;
    s = s + HALF_LN_2PI;
    s = s + (1.0 / 12.0) / x;
    s = s - (1.0 / 360.0) / (x * x * x);
    s = s + (1.0 / 1260.0) / (x * x * x * x * x);
    return s;
}

typedef struct {
    uint32_t key[2];
    uint32_t leap, traj, stream;
    uint32_t w;          /* next word */
    uint32_t buf[4];
    int have;
} sampler_words;

static uint32_t sampler_next(sampler_words *s)
{
    if ((s->w & 3u) == 0 || !s->have) {
        uint32_t ctr[4] = {s->w >> 2, s->leap, s->traj, s->stream};
        oracle_philox4x32_10(ctr, s->key, s->buf);
        s->have = 1;
    }
    return s->buf[s->w++ & 3u];
}

/* Poisson(lambda) in binary32: multiplication method below 10 (Knuth),     */
/* transformed rejection (Hoermann 1993, "PTRS") at 10 and above.           */
static int64_t poisson_f32(float lam, sampler_words *s)
{
    if (!(lam > 0.0f)) return 0;
    if (lam < 10.0f) {
        const float L = oracle_exp_f32(-lam);
        float p = 1.0f;
        int64_t k = -1;
        for (int it = 0; it < 1000; ++it) {
            const float v = (float)((sampler_next(s) >> 8) + 1u) * 0x1p-24f;
            k += 1;
            p = p * v;
            if (!(p > L)) return k;
        }
        return k;
    }
    const float slam = sqrtf(lam);
    const float loglam = oracle_log_f32(lam);
    const float b = 0.931f + 2.53f * slam;
    const float a = -0.059f + 0.02483f * b;
    const float invalpha = 1.1239f + 1.1328f / (b - 3.4f);
    const float vr = 0.9277f - 3.6224f / (b - 2.0f);
    const float log_invalpha = oracle_log_f32(invalpha);
    const float kmax = lam + 64.0f * slam + 64.0f;
    for (int it = 0; it < 100; ++it) {
        const float U = (float)(sampler_next(s) >> 8) * 0x1p-24f - 0.5f;
        const float V = (float)((sampler_next(s) >> 8) + 1u) * 0x1p-24f;
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
        float lhs = oracle_log_f32(V) + log_invalpha;
        lhs = lhs - oracle_log_f32(a / (us * us) + b);
        float rhs = -lam + kf * loglam;
        rhs = rhs - logfact_f32(kf);
        if (lhs <= rhs) return (int64_t)kf;
    }
    return (int64_t)floorf(lam);
}

static int64_t poisson_f64(double lam, sampler_words *s)
{
    if (!(lam > 0.0)) return 0;
    if (lam < 10.0) {
        const double L = oracle_exp_f64(-lam);
        double p = 1.0;
        int64_t k = -1;
        for (int it = 0; it < 1000; ++it) {
            const double v = ((double)sampler_next(s) + 1.0) * 0x1p-32;
            k += 1;
            p = p * v;
            if (!(p > L)) return k;
        }
        return k;
    }
    const double slam = sqrt(lam);
    const double loglam = oracle_log_f64(lam);
    const double b = 0.931 + 2.53 * slam;
    const double a = -0.059 + 0.02483 * b;
    const double invalpha = 1.1239 + 1.1328 / (b - 3.4);
    const double vr = 0.9277 - 3.6224 / (b - 2.0);
    const double log_invalpha = oracle_log_f64(invalpha);
    const double kmax = lam + 64.0 * slam + 64.0;
    for (int it = 0; it < 100; ++it) {
        const double U = (double)sampler_next(s) * 0x1p-32 - 0.5;
        const double V = ((double)sampler_next(s) + 1.0) * 0x1p-32;
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
        double lhs = oracle_log_f64(V) + log_invalpha;
        lhs = lhs - oracle_log_f64(a / (us * us) + b);
        double rhs = -lam + kf * loglam;
        rhs = rhs - logfact_f64(kf);
        if (lhs <= rhs) return (int64_t)kf;
    }
    return (int64_t)floor(lam);
}

/* one tau-leaping trajectory; prec as in oracle_run, sr 0/1 */
static void tau_traj(const omodel *md, int prec, int sr, double t_end, double tau, int K, const double *samples,
                     uint64_t seed, uint32_t traj, int32_t *x, const sink *S, uint32_t *status, int64_t *n_events,
                     double *t_final)
{
    const int M = md->M, N = md->N;
    const int fmt = (prec == P_MIXED_BF16 || prec == P_UNIFORM_BF16) ? 1 : 0;
    const int is16 = prec >= P_MIXED_F16, uniform = prec >= P_UNIFORM_F16;
    double cp64[OR_MAX_M], h064[OR_MAX_M], h164[OR_MAX_M];
    float cp[OR_MAX_M], h0[OR_MAX_M], h1[OR_MAX_M], a[OR_MAX_M];
    int nsr = 0;
    for (int j = 0; j < M; ++j) {
        cp64[j] = md->cprime[j];
        h064[j] = md->law[j] == LAW_HILL ? md->hill[4 * j] : 0.0;
        h164[j] = md->law[j] == LAW_HILL ? md->hill[4 * j + 1] : 0.0;
        cp[j] = (float)cp64[j];
        h0[j] = (float)h064[j];
        h1[j] = (float)h164[j];
        if (is16) { cp[j] = rn16(fmt, cp[j]); h0[j] = rn16(fmt, h0[j]); h1[j] = rn16(fmt, h1[j]); }
        nsr += chain_ops(md, j);
    }
    if (uniform) nsr += M;
    const uint64_t Ws = 4u * (uint64_t)((nsr + 7) / 8);
    const float tau32 = (float)tau;
    const float tau16 = is16 ? rn16(fmt, tau32) : tau32;
    word_stream wsr;
    memset(&wsr, 0, sizeof(wsr));
    wsr.key[0] = (uint32_t)seed; wsr.key[1] = (uint32_t)(seed >> 32); wsr.traj = traj; wsr.stream = 1;
    rounder R;
    R.bf16 = fmt; R.sr = sr; R.ws = &wsr; R.sr_base = 0; R.op = 0;
    const int64_t L = (int64_t)ceil(t_end / tau);
    int k = 0;
    int64_t events = 0;
    double t_last = 0.0;
    for (int64_t n = 0; n < L; ++n) {
        const double t_next = (double)(n + 1) * tau;
        while (k < K && samples[k] < t_next) write_snapshot(S, k++, x, status);
        double lam64[OR_MAX_M];
        float lam32[OR_MAX_M];
        R.sr_base = (uint64_t)n * Ws;
        R.op = 0;
        int bad = 0;
        for (int j = 0; j < M; ++j) {
            if (prec == P_FP64) {
                lam64[j] = prop_f64(md, j, x, cp64, h064, h164) * tau;
                if (f64_is_nan(lam64[j])) bad |= ST_NAN; else if (f64_is_inf(lam64[j])) bad |= ST_OVERFLOW;
            } else {
                a[j] = is16 ? prop_16(md, j, x, cp, h0, h1, &R) : prop_f32(md, j, x, cp, h0, h1);
            }
        }
        if (prec != P_FP64) {
            for (int j = 0; j < M; ++j) {
                lam32[j] = uniform ? rnd16(&R, a[j] * tau16) : a[j] * tau32;
                if (f32_is_nan(lam32[j])) bad |= ST_NAN; else if (f32_is_inf(lam32[j])) bad |= ST_OVERFLOW;
            }
        }
        if (bad) { *status |= (uint32_t)bad; break; }
        int64_t dx[OR_MAX_N];
        for (int i = 0; i < N; ++i) dx[i] = 0;
        for (int j = 0; j < M; ++j) {
            sampler_words sw;
            memset(&sw, 0, sizeof(sw));
            sw.key[0] = (uint32_t)seed; sw.key[1] = (uint32_t)(seed >> 32);
            sw.leap = (uint32_t)n; sw.traj = traj; sw.stream = 2u + (uint32_t)j;
            const int64_t kj = prec == P_FP64 ? poisson_f64(lam64[j], &sw) : poisson_f32(lam32[j], &sw);
            events += kj;
            for (int i = 0; i < N; ++i)
                if (!(md->constant && md->constant[i])) dx[i] += kj * (int64_t)md->stoich[j * N + i];
        }
        for (int i = 0; i < N; ++i) {
            int64_t v = (int64_t)x[i] + dx[i];
            if (v < 0) { v = 0; *status |= ST_TAU_CLAMPED; }
            if (v > 2147483647) v = 2147483647;
            x[i] = (int32_t)v;
        }
        t_last = t_next;
    }
    while (k < K) write_snapshot(S, k++, x, status);
    *n_events = events;
    *t_final = t_last;
}

int oracle_tau_run(int N, int M, const int32_t *order, const int32_t *stoich, const double *rate,
                   const int32_t *law, const double *hill, const uint8_t *constant,
                   const int32_t *x0, int64_t n_traj, uint64_t g0, double t_end, double tau,
                   int K, const double *samples, int precision, int rounding, int normalise,
                   uint64_t seed, int state_bytes, void *out, uint32_t *status, int64_t *n_events, double *t_final)
{
    if (N < 1 || N > OR_MAX_N || M < 1 || M > OR_MAX_M || K < 0 || K > 1024) return -1;
    if (precision < 0 || precision > 5 || rounding < 0 || rounding > 1) return -1;
    if (rounding == 1 && precision < 2) return -1;
    if (!(tau > 0.0) || !(t_end > 0.0) || t_end / tau > 2147483647.0) return -1;
    if (state_bytes != 2 && state_bytes != 4) return -1;
    if (n_traj < 0 || g0 + (uint64_t)n_traj > 0x100000000ull) return -1;
    omodel md;
    memset(&md, 0, sizeof(md));
    md.N = N; md.M = M; md.order = order; md.stoich = stoich; md.law = law;
    md.hill = hill; md.constant = constant; md.normalise = normalise;
    for (int j = 0; j < M; ++j) {
        if (law[j] == LAW_HILL) { md.cprime[j] = 0.0; continue; }
        double denom = 1.0;
        for (int i = 0; i < N; ++i) denom = denom * factorial(order[j * N + i]);
        double c = rate[j] / denom;
        if (normalise && constant) {
            for (int i = 0; i < N; ++i) {
                if (!constant[i] || order[j * N + i] == 0) continue;
                for (int m = 0; m < order[j * N + i]; ++m) c = c * (double)(x0[i] - m);
                md.folded[j][i] = 1;
            }
        }
        md.cprime[j] = c;
    }
    for (int64_t r = 0; r < n_traj; ++r) {
        int32_t x[OR_MAX_N];
        for (int i = 0; i < N; ++i) x[i] = x0[i];
        sink S;
        S.out = out; S.state_bytes = state_bytes; S.n_traj = n_traj; S.col = r; S.K = K; S.N = N;
        S.mask = (uint32_t)((1u << N) - 1u);
        S.outN = N;
        uint32_t st = 0;
        int64_t ne = 0;
        double tf = 0.0;
        tau_traj(&md, precision, rounding, t_end, tau, K, samples, seed, (uint32_t)(g0 + (uint64_t)r), x, &S, &st,
                 &ne, &tf);
        if (status) status[r] = st;
        if (n_events) n_events[r] = ne;
        if (t_final) t_final[r] = tf;
    }
    return 0;
}

/* Sampler checks: n Poisson(lambda) variates from (leap, traj, stream) word */
/* sequences leap = i, traj = 0, stream = 2; prec64 selects binary64.       */
void oracle_poisson_array(double lam, int prec64, uint64_t seed, int64_t n, int64_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        sampler_words sw;
        memset(&sw, 0, sizeof(sw));
        sw.key[0] = (uint32_t)seed; sw.key[1] = (uint32_t)(seed >> 32);
        sw.leap = (uint32_t)i; sw.traj = 0; sw.stream = 2;
        out[i] = prec64 ? poisson_f64(lam, &sw) : poisson_f32((float)lam, &sw);
    }
}

void oracle_exp_f32_array(const float *x, int64_t n, float *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_exp_f32(x[i]);
}

void oracle_exp_f64_array(const double *x, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_exp_f64(x[i]);
}

/* ======================================================================== */
/* Reaction-diffusion master equation (RDME) on a Cartesian lattice.  The    */
/* paper names the RDME -- well-mixed voxels whose reactions follow the SSA, */
/* coupled by stochastic hops between neighbours -- as the spatial setting   */
/* its question extends to (Sec. 1, Sec. 5, future work in Sec. 6); it gives */
/* no algorithm.  Readings (the CUDA engine implements the same contract):   */
/*  D1 lattice nx x ny x nz, voxel v = ix + nx (iy + ny iz); reflecting       */
/*     boundaries; hop directions in the order -x, +x, -y, +y, -z, +z.        */
/*  D2 channels of voxel v, in order: reactions j = 0..M-1 (the well-mixed   */
/*     propensity chain on x_v, reading R3), then for each species i with     */
/*     D_i > 0 (ascending) and each existing neighbour direction: the hop    */
/*     (i, dir), an order-1 channel of rate D_i: h = rnd(D_i' * rnd(x_vi)),   */
/*     zero when x_vi < 1; the two operations are computed once per species  */
/*     and the value repeats for each direction.  D_i' is D_i rounded once    */
/*     to the propensity type (RN), like c'_j.                                */
/*  D3 voxel total L_v = last partial sum S_C of its channels (S_1 = first   */
/*     channel value, S_c = S_{c-1} + value_c in the accumulator type).       */
/*  D4 sum tree: T = smallest power of two >= S leaves (padding leaves = 0), */
/*     heap order (node 1 the root, children 2q and 2q+1, leaf v at T + v);  */
/*     node q = left + right in the accumulator type; a0 = node 1.            */
/*  D5 event n: u1, u2, E, tau, target and t_new exactly as the well-mixed   */
/*     step (R6, R7); voxel by descent from the root with r = target: if      */
/*     left > r go left; else if right > 0 then r = r - left (accumulator     */
/*     type) and go right; else go left.  Channel within the voxel: smallest  */
/*     c with S_c > r, else the last channel with a positive value.          */
/*  D6 after an event the changed voxel(s) (one for a reaction, source and   */
/*     destination for a hop) are recomputed, then their ancestors, bottom-  */
/*     up, each node once.  Values are cached between events: a voxel's      */
/*     partial sums are recomputed for the selection from its state and the  */
/*     epoch at which it was last computed, which reproduces them exactly.   */
/*  D7 stochastic rounding bits (16-bit SR modes), 16 bits per operation as  */
/*     R5, from Philox counters (block lo, block hi, trajectory id, tag):     */
/*     voxel v computed at epoch e (0 = initial state, n + 1 = after event   */
/*     n): tag 0x80000000 | v, block = e * 2^32 + op / 8, operations in      */
/*     channel order (reaction chains, hop pairs, then the partial sums in   */
/*     uniform modes); tree node q at epoch e (uniform modes): tag            */
/*     0x40000000 | q, block e * 2^32, operation 0; event-level operations   */
/*     of event n (uniform modes): stream 1, B = ceil((5 + log2 T) / 8)      */
/*     blocks per event, slots E, U2, tau, target, t_new, then one slot per   */
/*     descent level.  Mixed modes round only the channel chains.             */
/*  D8 snapshots out[k][v][i][trajectory]; stops and status as R9; the       */
/*     event count includes hops.  With S = 1 the method is the well-mixed   */
/*     direct method operation for operation (RN modes and fp32/fp64).        */
/* ======================================================================== */
#define OR_MAX_S 4096
#define OR_MAX_CH (OR_MAX_M + 6 * OR_MAX_N)

typedef struct {
    int nx, ny, nz, S, T, depth;
    double D[OR_MAX_N];
} olattice;

static int lat_neighbour(const olattice *L, int v, int dir)
{
    int ix = v % L->nx, iy = (v / L->nx) % L->ny, iz = v / (L->nx * L->ny);
    switch (dir) {
    case 0: return ix > 0 ? v - 1 : -1;
    case 1: return ix < L->nx - 1 ? v + 1 : -1;
    case 2: return iy > 0 ? v - L->nx : -1;
    case 3: return iy < L->ny - 1 ? v + L->nx : -1;
    case 4: return iz > 0 ? v - L->nx * L->ny : -1;
    default: return iz < L->nz - 1 ? v + L->nx * L->ny : -1;
    }
}

typedef struct {
    void *out;
    int state_bytes;
    int64_t n_traj, col;
    int S, N;
} lsink;

static void write_lattice(const lsink *s, int k, const int32_t *x, uint32_t *status)
{
    for (int v = 0; v < s->S; ++v)
        for (int i = 0; i < s->N; ++i) {
            int64_t idx = (((int64_t)k * s->S + v) * s->N + i) * s->n_traj + s->col;
            int32_t val = x[v * s->N + i];
            if (s->state_bytes == 2) {
                if (val > 32767) { val = 32767; *status |= ST_STATE_RANGE; }
                if (val < -32768) { val = -32768; *status |= ST_STATE_RANGE; }
                ((int16_t *)s->out)[idx] = (int16_t)val;
            } else {
                ((int32_t *)s->out)[idx] = val;
            }
        }
}

/* Hop channel c >= M of voxel v: the species and the destination voxel. */
static void hop_channel(const omodel *md, const olattice *L, int v, int c, int *species, int *dest)
{
    int idx = c - md->M;
    for (int i = 0; i < md->N; ++i) {
        if (!(L->D[i] > 0.0)) continue;
        for (int dir = 0; dir < 6; ++dir) {
            int w = lat_neighbour(L, v, dir);
            if (w < 0) continue;
            if (idx == 0) { *species = i; *dest = w; return; }
            idx -= 1;
        }
    }
    *species = -1; *dest = -1;
}

static int n_neighbours(const olattice *L, int v)
{
    int c = 0;
    for (int dir = 0; dir < 6; ++dir) c += lat_neighbour(L, v, dir) >= 0;
    return c;
}

/* Voxel v in binary64 (D2, D3).  Returns L_v; when sel is not NULL, also   */
/* the selected channel for residual target r (D5).                        */
static double voxel_f64(const omodel *md, const olattice *L, const int32_t *xv, int v, const double *cp,
                        const double *h0, const double *h1, double r, int *sel)
{
    double val[OR_MAX_CH], Ssum[OR_MAX_CH];
    int C = 0;
    for (int j = 0; j < md->M; ++j) val[C++] = prop_f64(md, j, xv, cp, h0, h1);
    int nnb = n_neighbours(L, v);
    if (nnb > 0)
        for (int i = 0; i < md->N; ++i) {
            if (!(L->D[i] > 0.0)) continue;
            double h = xv[i] < 1 ? 0.0 : L->D[i] * (double)xv[i];
            for (int d = 0; d < nnb; ++d) val[C++] = h;
        }
    Ssum[0] = val[0];
    for (int c = 1; c < C; ++c) Ssum[c] = Ssum[c - 1] + val[c];
    if (sel) {
        int mu = -1;
        for (int c = 0; c < C; ++c) if (Ssum[c] > r) { mu = c; break; }
        if (mu < 0) for (int c = C - 1; c >= 0; --c) if (val[c] > 0.0) { mu = c; break; }
        *sel = mu;
    }
    return Ssum[C - 1];
}

/* Voxel v in binary32 arithmetic: kind 0 fp32, 1 mixed (16-bit channel      */
/* values), 2 uniform (16-bit values and sums).  R points at the voxel's SR  */
/* stream for this epoch (op = 0).                                            */
static float voxel_f32(const omodel *md, const olattice *L, const int32_t *xv, int v, const float *cp,
                       const float *h0, const float *h1, const float *Dp, int kind, rounder *R, float r, int *sel)
{
    float val[OR_MAX_CH], Ssum[OR_MAX_CH];
    int C = 0;
    for (int j = 0; j < md->M; ++j)
        val[C++] = kind == 0 ? prop_f32(md, j, xv, cp, h0, h1) : prop_16(md, j, xv, cp, h0, h1, R);
    int nnb = n_neighbours(L, v);
    if (nnb > 0)
        for (int i = 0; i < md->N; ++i) {
            if (!(L->D[i] > 0.0)) continue;
            float h;
            if (kind == 0) {
                h = xv[i] < 1 ? 0.0f : Dp[i] * (float)xv[i];
            } else if (xv[i] < 1) {
                h = 0.0f;
                R->op += 2;                 /* slots reserved, as for a short reactant */
            } else {
                float f = rnd16(R, (float)xv[i]);
                h = rnd16(R, Dp[i] * f);
            }
            for (int d = 0; d < nnb; ++d) val[C++] = h;
        }
    Ssum[0] = val[0];
    for (int c = 1; c < C; ++c) Ssum[c] = kind == 2 ? rnd16(R, Ssum[c - 1] + val[c]) : Ssum[c - 1] + val[c];
    if (sel) {
        int mu = -1;
        for (int c = 0; c < C; ++c) if (Ssum[c] > r) { mu = c; break; }
        if (mu < 0) for (int c = C - 1; c >= 0; --c) if (val[c] > 0.0f) { mu = c; break; }
        *sel = mu;
    }
    return Ssum[C - 1];
}

static void set_tag(word_stream *ws, uint32_t tag)
{
    ws->stream = tag;
    ws->have = 0;
}

/* Apply channel c of voxel v; returns the second changed voxel (hop) or -1.
 * *negative = 1 when a count went negative (the trajectory ends). */
static int rdme_apply(const omodel *md, const olattice *L, int v, int c, int32_t *x, uint32_t *status,
                      int *negative)
{
    const int N = md->N;
    *negative = 0;
    if (c < md->M) {
        *negative = apply_event(md, c, x + v * N, status);
        return -1;
    }
    int i, w;
    hop_channel(md, L, v, c, &i, &w);
    x[v * N + i] -= 1;
    x[w * N + i] += 1;
    if (x[v * N + i] < 0) {
        *status |= ST_STATE_RANGE;
        *negative = 1;
    }
    return w;
}

/* One RDME trajectory in binary64. */
static void rdme_traj_f64(const omodel *md, const olattice *L, const runp *rp, word_stream *ws, int32_t *x,
                          double *node, const lsink *snk, uint32_t *status, int64_t *n_events, double *t_final)
{
    const int N = md->N, S = L->S, T = L->T;
    double cp[OR_MAX_M], h0[OR_MAX_M], h1[OR_MAX_M];
    for (int j = 0; j < md->M; ++j) {
        cp[j] = md->cprime[j];
        h0[j] = md->law[j] == LAW_HILL ? md->hill[4 * j] : 0.0;
        h1[j] = md->law[j] == LAW_HILL ? md->hill[4 * j + 1] : 0.0;
    }
    for (int v = 0; v < T; ++v) node[T + v] = v < S ? voxel_f64(md, L, x + v * N, v, cp, h0, h1, 0.0, NULL) : 0.0;
    for (int q = T - 1; q >= 1; --q) node[q] = node[2 * q] + node[2 * q + 1];
    double t = 0.0;
    int64_t n = 0;
    int k = 0;
    for (;;) {
        if (n >= rp->max_events) { *status |= ST_MAX_EVENTS; break; }
        double a0 = node[1];
        if (f64_is_nan(a0)) { *status |= ST_NAN; break; }
        if (f64_is_inf(a0)) { *status |= ST_OVERFLOW; break; }
        if (a0 == 0.0) break;
        uint64_t w = (uint64_t)n * 2u;
        uint32_t w0 = stream_word(ws, w), w1 = stream_word(ws, w + 1);
        double u1 = ((double)w0 + 1.0) * 0x1p-32;
        double u2 = (double)w1 * 0x1p-32;
        double E = -oracle_log_f64(u1);
        double tau = E / a0;
        double target = u2 * a0;
        double t_new = t + tau;
        while (k < rp->K && rp->samples[k] < t_new) write_lattice(snk, k++, x, status);
        if (t_new > rp->t_end) break;
        int q = 1;
        double r = target;
        while (q < T) {
            double lf = node[2 * q], rt = node[2 * q + 1];
            if (lf > r) q = 2 * q;
            else if (rt > 0.0) { r = r - lf; q = 2 * q + 1; }
            else q = 2 * q;
        }
        int v = q - T, c = -1;
        voxel_f64(md, L, x + v * N, v, cp, h0, h1, r, &c);
        if (c < 0) { *status |= ST_NAN; break; }   /* unreachable: the descent only enters positive totals */
        int negative = 0;
        int w2 = rdme_apply(md, L, v, c, x, status, &negative);
        t = t_new;
        n += 1;
        if (negative) break;
        node[T + v] = voxel_f64(md, L, x + v * N, v, cp, h0, h1, 0.0, NULL);
        if (w2 >= 0) node[T + w2] = voxel_f64(md, L, x + w2 * N, w2, cp, h0, h1, 0.0, NULL);
        /* ancestors, level by level; qb = 0 once the two paths have merged */
        int qa = (T + v) >> 1, qb = w2 >= 0 ? (T + w2) >> 1 : 0;
        while (qa >= 1) {
            if (qb == qa) qb = 0;
            node[qa] = node[2 * qa] + node[2 * qa + 1];
            if (qb) node[qb] = node[2 * qb] + node[2 * qb + 1];
            qa >>= 1;
            qb >>= 1;
        }
    }
    while (k < rp->K) write_lattice(snk, k++, x, status);
    *n_events = n;
    *t_final = t;
}

/* Node q of the tree at epoch e in binary32 arithmetic (kind as voxel_f32). */
static float tree_node_f32(const float *node, int q, int kind, int fmt, int sr, word_stream *wsn, uint32_t e)
{
    float s = node[2 * q] + node[2 * q + 1];
    if (kind != 2) return s;
    rounder R;
    set_tag(wsn, 0x40000000u | (uint32_t)q);
    R.bf16 = fmt; R.sr = sr; R.ws = wsn; R.sr_base = (uint64_t)e << 34; R.op = 0;
    return rnd16(&R, s);
}

/* Voxel v at epoch e in binary32 arithmetic, with its SR stream. */
static float voxel_at_f32(const omodel *md, const olattice *L, const int32_t *x, int v, uint32_t e, const float *cp,
                          const float *h0, const float *h1, const float *Dp, int kind, int fmt, int sr,
                          word_stream *wsv, float r, int *sel)
{
    rounder R;
    set_tag(wsv, 0x80000000u | (uint32_t)v);
    R.bf16 = fmt; R.sr = sr; R.ws = wsv; R.sr_base = (uint64_t)e << 34; R.op = 0;
    return voxel_f32(md, L, x + v * md->N, v, cp, h0, h1, Dp, kind, &R, r, sel);
}

/* One RDME trajectory in binary32 arithmetic: kind 0 fp32, 1 mixed, 2 uniform. */
static void rdme_traj_f32(const omodel *md, const olattice *L, const runp *rp, word_stream *ws, word_stream *wsr,
                          word_stream *wsv, word_stream *wsn, int32_t *x, float *node, uint32_t *epoch,
                          const lsink *snk, uint32_t *status, int64_t *n_events, double *t_final,
                          int kind, int fmt, int sr)
{
    const int N = md->N, S = L->S, T = L->T;
    float cp[OR_MAX_M], h0[OR_MAX_M], h1[OR_MAX_M], Dp[OR_MAX_N];
    for (int j = 0; j < md->M; ++j) {
        cp[j] = (float)md->cprime[j];
        h0[j] = md->law[j] == LAW_HILL ? (float)md->hill[4 * j] : 0.0f;
        h1[j] = md->law[j] == LAW_HILL ? (float)md->hill[4 * j + 1] : 0.0f;
        if (kind != 0) { cp[j] = rn16(fmt, cp[j]); h0[j] = rn16(fmt, h0[j]); h1[j] = rn16(fmt, h1[j]); }
    }
    for (int i = 0; i < N; ++i) Dp[i] = kind != 0 ? rn16(fmt, (float)L->D[i]) : (float)L->D[i];
    float t_end = kind == 2 ? rn16(fmt, (float)rp->t_end) : (float)rp->t_end;
    float smp[1024];
    for (int kk = 0; kk < rp->K; ++kk) smp[kk] = kind == 2 ? rn16(fmt, (float)rp->samples[kk]) : (float)rp->samples[kk];
    const int nsr_ev = 5 + L->depth;
    const uint64_t Ws_ev = 4u * (uint64_t)((nsr_ev + 7) / 8);
    rounder Re;
    Re.bf16 = fmt; Re.sr = sr; Re.ws = wsr; Re.sr_base = 0; Re.op = 0;

    for (int v = 0; v < T; ++v) {
        node[T + v] = v < S ? voxel_at_f32(md, L, x, v, 0u, cp, h0, h1, Dp, kind, fmt, sr, wsv, 0.0f, NULL) : 0.0f;
        if (v < S) epoch[v] = 0;
    }
    for (int q = T - 1; q >= 1; --q) node[q] = tree_node_f32(node, q, kind, fmt, sr, wsn, 0u);
    float t = 0.0f;
    int64_t n = 0;
    int k = 0;
    for (;;) {
        if (n >= rp->max_events) { *status |= ST_MAX_EVENTS; break; }
        float a0 = node[1];
        if (f32_is_nan(a0)) { *status |= ST_NAN; break; }
        if (f32_is_inf(a0)) { *status |= ST_OVERFLOW; break; }
        if (a0 == 0.0f) break;
        uint64_t w = (uint64_t)n * 2u;
        uint32_t w0 = stream_word(ws, w), w1 = stream_word(ws, w + 1);
        float u1 = (float)((w0 >> 8) + 1u) * 0x1p-24f;
        float u2 = (float)(w1 >> 8) * 0x1p-24f;
        float tau, target, t_new;
        Re.sr_base = (uint64_t)n * Ws_ev;
        if (kind == 2) {
            Re.op = 0;
            float E = rnd16(&Re, -oracle_log_f32(u1));
            float U2 = rnd16(&Re, u2);
            tau = rnd16(&Re, E / a0);
            target = rnd16(&Re, U2 * a0);
            t_new = rnd16(&Re, t + tau);
        } else {
            float E = -oracle_log_f32(u1);
            tau = E / a0;
            target = u2 * a0;
            t_new = t + tau;
        }
        while (k < rp->K && smp[k] < t_new) write_lattice(snk, k++, x, status);
        if (t_new > t_end) break;
        int q = 1, level = 0;
        float r = target;
        while (q < T) {
            float lf = node[2 * q], rt = node[2 * q + 1];
            if (lf > r) {
                q = 2 * q;
            } else if (rt > 0.0f) {
                if (kind == 2) { Re.op = 5 + level; r = rnd16(&Re, r - lf); }
                else r = r - lf;
                q = 2 * q + 1;
            } else {
                q = 2 * q;
            }
            level += 1;
        }
        int v = q - T, c = -1;
        voxel_at_f32(md, L, x, v, epoch[v], cp, h0, h1, Dp, kind, fmt, sr, wsv, r, &c);
        if (c < 0) { *status |= ST_NAN; break; }   /* unreachable: the descent only enters positive totals */
        int negative = 0;
        int w2 = rdme_apply(md, L, v, c, x, status, &negative);
        t = t_new;
        n += 1;
        if (negative) break;
        const uint32_t e = (uint32_t)n;            /* epoch n + 1 of the event just applied */
        node[T + v] = voxel_at_f32(md, L, x, v, e, cp, h0, h1, Dp, kind, fmt, sr, wsv, 0.0f, NULL);
        epoch[v] = e;
        if (w2 >= 0) {
            node[T + w2] = voxel_at_f32(md, L, x, w2, e, cp, h0, h1, Dp, kind, fmt, sr, wsv, 0.0f, NULL);
            epoch[w2] = e;
        }
        int qa = (T + v) >> 1, qb = w2 >= 0 ? (T + w2) >> 1 : 0;
        while (qa >= 1) {
            if (qb == qa) qb = 0;
            node[qa] = tree_node_f32(node, qa, kind, fmt, sr, wsn, e);
            if (qb) node[qb] = tree_node_f32(node, qb, kind, fmt, sr, wsn, e);
            qa >>= 1;
            qb >>= 1;
        }
    }
    while (k < rp->K) write_lattice(snk, k++, x, status);
    *n_events = n;
    *t_final = (double)t;
}

/* Public entry: RDME trajectories g0 .. g0+n_traj-1 on an nx x ny x nz      */
/* lattice; D [N] hop rates per direction; x0 [S][N]; snapshots               */
/* out[((k*S + v)*N + i)*n_traj + r].  Returns 0, or -1 on invalid arguments. */
int oracle_rdme_run(int N, int M, const int32_t *order, const int32_t *stoich, const double *rate,
                    const int32_t *law, const double *hill, const uint8_t *constant, int nx, int ny, int nz,
                    const double *D, const int32_t *x0, int64_t n_traj, uint64_t g0, double t_end, int K,
                    const double *samples, int precision, int rounding, int normalise, uint64_t seed,
                    int64_t max_events, int state_bytes, void *out, uint32_t *status, int64_t *n_events,
                    double *t_final)
{
    if (N < 1 || N > OR_MAX_N || M < 1 || M > OR_MAX_M || K < 0 || K > 1024) return -1;
    if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz > OR_MAX_S) return -1;
    if (precision < 0 || precision > 5 || rounding < 0 || rounding > 1) return -1;
    if (rounding == 1 && precision < 2) return -1;
    if (state_bytes != 2 && state_bytes != 4) return -1;
    if (n_traj < 0 || g0 + (uint64_t)n_traj > 0x100000000ull) return -1;
    if (max_events < 0 || max_events > 4294967294ll) return -1;
    olattice L;
    memset(&L, 0, sizeof(L));
    L.nx = nx; L.ny = ny; L.nz = nz; L.S = nx * ny * nz;
    L.T = 1; L.depth = 0;
    while (L.T < L.S) { L.T *= 2; L.depth += 1; }
    for (int i = 0; i < N; ++i) {
        if (!(D[i] >= 0.0) || f64_is_inf(D[i])) return -1;
        if (constant && constant[i] && D[i] != 0.0) return -1;
        L.D[i] = D[i];
        if (constant && constant[i])
            for (int v = 1; v < L.S; ++v) if (x0[v * N + i] != x0[i]) return -1;
    }
    omodel md;
    memset(&md, 0, sizeof(md));
    md.N = N; md.M = M; md.order = order; md.stoich = stoich; md.law = law;
    md.hill = hill; md.constant = constant; md.normalise = normalise;
    for (int j = 0; j < M; ++j) {
        if (law[j] == LAW_HILL) { md.cprime[j] = 0.0; continue; }
        double denom = 1.0;
        for (int i = 0; i < N; ++i) denom = denom * factorial(order[j * N + i]);
        double c = rate[j] / denom;
        if (normalise && constant) {
            for (int i = 0; i < N; ++i) {
                if (!constant[i] || order[j * N + i] == 0) continue;
                for (int m = 0; m < order[j * N + i]; ++m) c = c * (double)(x0[i] - m);
                md.folded[j][i] = 1;
            }
        }
        md.cprime[j] = c;
    }
    runp rp;
    rp.t_end = t_end; rp.K = K; rp.samples = samples; rp.max_events = max_events;
    int32_t *x = (int32_t *)malloc(sizeof(int32_t) * (size_t)L.S * (size_t)N);
    double *node64 = (double *)malloc(sizeof(double) * 2 * (size_t)L.T);
    float *node32 = (float *)malloc(sizeof(float) * 2 * (size_t)L.T);
    uint32_t *epoch = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)L.S);
    if (!x || !node64 || !node32 || !epoch) { free(x); free(node64); free(node32); free(epoch); return -1; }
    for (int64_t r = 0; r < n_traj; ++r) {
        word_stream ws, wsr, wsv, wsn;
        memset(&ws, 0, sizeof(ws));
        ws.key[0] = (uint32_t)seed;
        ws.key[1] = (uint32_t)(seed >> 32);
        ws.traj = (uint32_t)(g0 + (uint64_t)r);
        ws.stream = 0;
        wsr = ws; wsr.stream = 1;
        wsv = ws; wsn = ws;
        memcpy(x, x0, sizeof(int32_t) * (size_t)L.S * (size_t)N);
        lsink snk;
        snk.out = out; snk.state_bytes = state_bytes; snk.n_traj = n_traj; snk.col = r; snk.S = L.S; snk.N = N;
        uint32_t st = 0;
        int64_t ne = 0;
        double tf = 0.0;
        const int fmt = (precision == P_MIXED_BF16 || precision == P_UNIFORM_BF16) ? 1 : 0;
        if (precision == P_FP64)
            rdme_traj_f64(&md, &L, &rp, &ws, x, node64, &snk, &st, &ne, &tf);
        else
            rdme_traj_f32(&md, &L, &rp, &ws, &wsr, &wsv, &wsn, x, node32, epoch, &snk, &st, &ne, &tf,
                          precision == P_FP32 ? 0 : (precision >= P_UNIFORM_F16 ? 2 : 1), fmt, rounding);
        if (status) status[r] = st;
        if (n_events) n_events[r] = ne;
        if (t_final) t_final[r] = tf;
    }
    free(x); free(node64); free(node32); free(epoch);
    return 0;
}
