// ssa_capi.cu -- host side of the C ABI declared in include/ssa.h.
//
// Validates arguments, matches the model against the compiled structure
// families, prepares the rate constants (Gillespie c-convention, binary64)
// and launches the persistent kernel.  Everything that touches trajectory
// data runs in the CUDA kernels; this file only marshals.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/ssa.h"
#include "rdme_device.cuh"
#include "ssa_launch.h"
#include "tau_launch.h"
#include "ssa_models.h"

struct ssa_model {
    int N, M;
    int32_t order[ssa::kMaxM][ssa::kMaxN];
    int32_t stoich[ssa::kMaxM][ssa::kMaxN];
    double rate[ssa::kMaxM];
    int32_t law[ssa::kMaxM];
    double hill[ssa::kMaxM][4];
    uint8_t constant[ssa::kMaxN];
    int family;
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(SSA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Launch shapes.  Until ssa_set_launch_config is called, single-queue
// direct-method runs use kDirectDefault and tau-leaping, RDME and batches use
// kOtherDefault (each the fastest measured for its kernels); afterwards all
// use the shape that was set.
constexpr ssa::LaunchConfig kDirectDefault = {0, 0, 32};   // block size chosen per kernel
constexpr ssa::LaunchConfig kOtherDefault = {128, 0, 16};
ssa::LaunchConfig g_cfg = kDirectDefault;
bool g_cfg_set = false;

ssa::LaunchConfig other_cfg() { return g_cfg_set ? g_cfg : kOtherDefault; }
bool g_tail_compaction = true;
int g_tail_lock_spins = 0;   // 0: the kernels' default bound

// Longest-first scheduling of single-queue direct-method runs: 0 off,
// 1 automatic (runs long and large enough for the launch tail to matter),
// 2 always.  g_park_events: the parking point (0: a0(x0) t_end / 5).
int g_longest_first = 1;
int64_t g_park_events = 0;
constexpr double kLongestFirstMinEvents = 4096.0;   // estimated events per trajectory
constexpr int64_t kLongestFirstMinPerLane = 2;      // trajectories per resident lane
constexpr double kLongestFirstMinSpread = 4.0;      // batches: largest / smallest estimate over the sets
std::atomic<long long> g_direct_launches{0};        // kernels launched by launch_run

}  // namespace

// Counters of the direct-method kernels' tail compaction on each device:
// [0] trajectories moved between warps, [1] lock waits that gave up,
// [2] trajectories resumed from the pool at the end of a block.
__device__ unsigned long long g_tail_counters[3];

namespace {

// Device address of this device's counters, or null when compaction is off.
unsigned long long *tail_counters()
{
    if (!g_tail_compaction) return nullptr;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tail_counters) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<unsigned long long *>(p);
}

template <class S>
bool matches(const ssa_model &m)
{
    if (m.N != S::N || m.M != S::M) return false;
    for (int i = 0; i < S::N; ++i)
        if ((m.constant[i] != 0) != (S::cs[i] != 0)) return false;
    for (int j = 0; j < S::M; ++j) {
        if (m.law[j] != S::lw[j]) return false;
        if (S::lw[j] == SSA_LAW_HILL_REPRESSION) {
            if ((int)m.hill[j][2] != S::hh[j] || (int)m.hill[j][3] != S::hreg[j]) return false;
            continue;
        }
        for (int i = 0; i < S::N; ++i) {
            if (m.order[j][i] != S::ord[j][i]) return false;
            if (!S::cs[i] && m.stoich[j][i] != S::nu[j][i]) return false;
        }
    }
    return true;
}

int detect_family(const ssa_model &m)
{
    if (matches<ssa::models::BirthDeath>(m)) return ssa::models::BirthDeath::family;
    if (matches<ssa::models::Schlogl>(m)) return ssa::models::Schlogl::family;
    if (matches<ssa::models::Telegraph>(m)) return ssa::models::Telegraph::family;
    if (matches<ssa::models::Dimer>(m)) return ssa::models::Dimer::family;
    if (matches<ssa::models::Repressilator>(m)) return ssa::models::Repressilator::family;
    return 0;
}

ssa::Launcher launcher_for(int family)
{
    switch (family) {
    case 1: return ssa::launch_birth_death;
    case 2: return ssa::launch_schlogl;
    case 3: return ssa::launch_telegraph;
    case 4: return ssa::launch_dimer;
    case 5: return ssa::launch_repressilator;
    default: return ssa::launch_general;
    }
}

bool finite_double(double v) { return std::isfinite(v); }

// c'_j = c_j / prod_i r_ij!, then (normalise) times the falling factorials of
// the constant species' counts, species ascending, factor m ascending; all in
// binary64 (reading of Sec. 4.2: k1 A and k3 B formed before rounding).
void rate_constants(const ssa_model &m, const int32_t *x0, int normalise, double *cprime, int8_t folded[][ssa::kMaxN])
{
    for (int j = 0; j < m.M; ++j) {
        for (int i = 0; i < ssa::kMaxN; ++i) folded[j][i] = 0;
        if (m.law[j] == SSA_LAW_HILL_REPRESSION) {
            cprime[j] = 0.0;
            continue;
        }
        double denom = 1.0;
        for (int i = 0; i < m.N; ++i) {
            double f = 1.0;
            for (int q = 2; q <= m.order[j][i]; ++q) f = f * (double)q;
            denom = denom * f;
        }
        double c = m.rate[j] / denom;
        if (normalise) {
            for (int i = 0; i < m.N; ++i) {
                if (!m.constant[i] || m.order[j][i] == 0) continue;
                for (int q = 0; q < m.order[j][i]; ++q) c = c * (double)(x0[i] - q);
                folded[j][i] = 1;
            }
        }
        cprime[j] = c;
    }
}

// Rough events per trajectory, a0(x0) * t_end in binary64: the scale of the
// work a run does per trajectory (used only to pick how host outputs are
// delivered; the order of magnitude is what matters).
double estimated_events(const ssa_model &m, const int32_t *x0, int normalise, double t_end)
{
    double c[ssa::kMaxM];
    int8_t folded[ssa::kMaxM][ssa::kMaxN];
    rate_constants(m, x0, normalise, c, folded);
    double a0 = 0.0;
    for (int j = 0; j < m.M; ++j) {
        if (m.law[j] == SSA_LAW_HILL_REPRESSION) {
            const double P = (double)x0[(int)m.hill[j][3]];
            a0 += m.hill[j][0] + m.hill[j][1] / (1.0 + std::pow(P, m.hill[j][2]));
            continue;
        }
        double a = c[j];
        for (int i = 0; i < m.N; ++i) {
            if (folded[j][i]) continue;
            for (int q = 0; q < m.order[j][i]; ++q) a *= (double)(x0[i] - q > 0 ? x0[i] - q : 0);
        }
        a0 += a;
    }
    return a0 * t_end;
}

int chain_ops(const ssa_model &m, int j, int8_t folded[][ssa::kMaxN])
{
    if (m.law[j] == SSA_LAW_HILL_REPRESSION) return (int)m.hill[j][2] + 3;
    int ops = 0;
    for (int i = 0; i < m.N; ++i)
        if (!folded[j][i]) ops += 2 * m.order[j][i];
    return ops;
}

int validate_run(const ssa_model *model, int64_t n_traj, uint64_t traj_offset, const int32_t *x0, double t_end,
                 int n_samples, const double *sample_times, int precision, int rounding, int64_t max_events,
                 int state_bytes, uint32_t out_species = 0)
{
    if (!model) return fail(SSA_EINVAL, "model is NULL");
    if (n_traj < 0) return fail(SSA_EINVAL, "n_traj must be >= 0");
    if (traj_offset + (uint64_t)n_traj > 0x100000000ull) return fail(SSA_EINVAL, "trajectory ids must fit in 32 bits");
    if (!x0) return fail(SSA_EINVAL, "x0 is NULL");
    for (int i = 0; i < model->N; ++i)
        if (x0[i] < 0) return fail(SSA_EINVAL, "x0[%d] is negative", i);
    if (!finite_double(t_end) || !(t_end > 0.0)) return fail(SSA_EINVAL, "t_end must be finite and > 0");
    if (n_samples < 1 || n_samples > SSA_MAX_SAMPLES) return fail(SSA_EINVAL, "n_samples must be in 1..%d", SSA_MAX_SAMPLES);
    if (!sample_times) return fail(SSA_EINVAL, "sample_times is NULL");
    for (int k = 0; k < n_samples; ++k) {
        const double s = sample_times[k];
        if (!finite_double(s) || s < 0.0 || s > t_end) return fail(SSA_EINVAL, "sample_times[%d] outside [0, t_end]", k);
        if (k > 0 && s < sample_times[k - 1]) return fail(SSA_EINVAL, "sample_times must be ascending");
    }
    if (precision < SSA_FP64 || precision > SSA_UNIFORM_BF16) return fail(SSA_EINVAL, "unknown precision %d", precision);
    if (rounding != SSA_RN && rounding != SSA_SR && rounding != SSA_SR_ACCUM)
        return fail(SSA_EINVAL, "unknown rounding %d", rounding);
    if (rounding == SSA_SR && precision < SSA_MIXED_F16) return fail(SSA_EINVAL, "stochastic rounding needs a 16-bit mode");
    if (rounding == SSA_SR_ACCUM && precision < SSA_UNIFORM_F16)
        return fail(SSA_EINVAL, "selective stochastic rounding needs a uniform 16-bit mode");
    if (max_events < 0) return fail(SSA_EINVAL, "max_events must be >= 0");
    if (state_bytes != 2 && state_bytes != 4) return fail(SSA_EINVAL, "state_bytes must be 2 or 4");
    if (model->N < 32 && (out_species >> model->N) != 0u)
        return fail(SSA_EINVAL, "out_species names species beyond n_species = %d", model->N);
    return SSA_OK;
}

// Stored species of a run: the caller's mask, 0 meaning all.
uint32_t out_mask_of(const ssa_model &m, uint32_t out_species)
{
    return out_species ? out_species : ((1u << m.N) - 1u);
}

// Fill the kernel arguments common to single and batched runs.
void fill_structure(const ssa_model &m, int normalise, const int32_t *x0, ssa::RunArgs &a)
{
    a.N = m.N;
    a.M = m.M;
    a.out_mask = (m.N >= 32) ? 0xFFFFFFFFu : ((1u << m.N) - 1u);   // every species stored
    a.out_N = m.N;
    rate_constants(m, x0, normalise, a.cprime, a.folded);
    int start = 0;
    for (int j = 0; j < m.M; ++j) {
        a.chain_start[j] = (int16_t)start;
        start += chain_ops(m, j, a.folded);
        a.law[j] = (int8_t)m.law[j];
        a.hill_h[j] = (int8_t)(m.law[j] == SSA_LAW_HILL_REPRESSION ? (int)m.hill[j][2] : 0);
        a.hill_reg[j] = (int8_t)(m.law[j] == SSA_LAW_HILL_REPRESSION ? (int)m.hill[j][3] : 0);
        a.hill_a0[j] = m.law[j] == SSA_LAW_HILL_REPRESSION ? m.hill[j][0] : 0.0;
        a.hill_a[j] = m.law[j] == SSA_LAW_HILL_REPRESSION ? m.hill[j][1] : 0.0;
        for (int i = 0; i < m.N; ++i) {
            a.order[j][i] = (int8_t)m.order[j][i];
            a.stoich[j][i] = m.constant[i] ? 0 : m.stoich[j][i];
        }
    }
    a.sr_ops = start;   // rounding operations in the propensity chains of one step
    for (int i = 0; i < m.N; ++i) a.x0[i] = x0[i];
}

// Longest-first scheduling scratch: parked records, keys, the order and the
// counters of the second launch, in one stream-ordered allocation.
size_t longest_first_bytes(int64_t n, int N)
{
    const size_t n8 = (size_t)n * 8, n4 = (size_t)n * 4;
    return 256 + 2 * n8 + (2 + (size_t)N) * n4 + (size_t)n + sizeof(unsigned) * ssa::kOrderBuckets +
           sizeof(unsigned long long) * ssa::kOrderBuckets + 64;
}

ssa::LongestFirstScratch carve_longest_first(char *p, int64_t n, int N)
{
    ssa::LongestFirstScratch L;
    L.head2 = reinterpret_cast<unsigned long long *>(p);
    L.count = L.head2 + 1;
    p += 256;
    L.offs = reinterpret_cast<unsigned long long *>(p); p += sizeof(unsigned long long) * ssa::kOrderBuckets;
    L.t = reinterpret_cast<double *>(p); p += (size_t)n * 8;
    L.order = reinterpret_cast<int64_t *>(p); p += (size_t)n * 8;
    L.hist = reinterpret_cast<unsigned *>(p); p += sizeof(unsigned) * ssa::kOrderBuckets;
    L.k = reinterpret_cast<int32_t *>(p); p += (size_t)n * 4;
    L.status = reinterpret_cast<uint32_t *>(p); p += (size_t)n * 4;
    L.x = reinterpret_cast<int32_t *>(p); p += (size_t)n * 4 * (size_t)N;
    L.parked = reinterpret_cast<uint8_t *>(p);
    return L;
}

// The model as the ordering kernels see it: rate constants of the run (one
// parameter set) in binary32, the structure, and the parked records.
ssa::OrderModel order_model(const ssa::RunArgs &a, const ssa::LongestFirstScratch &L)
{
    ssa::OrderModel m;
    std::memset(&m, 0, sizeof(m));
    m.N = a.N;
    m.M = a.M;
    for (int j = 0; j < a.M; ++j) {
        for (int i = 0; i < a.N; ++i) {
            m.order[j][i] = a.order[j][i];
            m.folded[j][i] = a.folded[j][i];
        }
        m.law[j] = a.law[j];
        m.hill_h[j] = a.hill_h[j];
        m.hill_reg[j] = a.hill_reg[j];
        m.c[j] = (float)a.cprime[j];
        m.h0[j] = (float)a.hill_a0[j];
        m.h1[j] = (float)a.hill_a[j];
    }
    m.n_sets = a.n_sets;
    m.traj_per_set = a.traj_per_set;
    m.cprime_tab = a.cprime_tab;
    m.hill_tab = a.hill_tab;
    m.t_end = a.t_end;
    m.x = L.x;
    m.t = L.t;
    m.parked = L.parked;
    return m;
}

// Whether a single-queue run is split into park / order / resume, and with
// which parking point; returns the scratch (null: one plain launch).  The
// split pays when trajectories are long (the end of a persistent launch waits
// for the trajectories that started last) and every lane runs several.  A
// failed allocation falls back to the plain launch.
char *plan_longest_first(const ssa_model &m, const int32_t *x0, int normalise, double t_end, int64_t n_work,
                         int64_t max_events, cudaStream_t s, int64_t *park)
{
    if (g_longest_first == 0 || n_work < 1) return nullptr;
    const double est = estimated_events(m, x0, normalise, t_end);
    int64_t pe = g_park_events;
    if (pe <= 0) {
        const double p = est / 5.0;
        pe = p < 256.0 ? 256 : (p > 1073741824.0 ? 1073741824 : (int64_t)p);
    }
    pe &= ~(int64_t)1;   // even: parked between step pairs
    if (pe < 2 || pe >= max_events) return nullptr;
    if (g_longest_first == 1) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return nullptr;
        if (!(est >= kLongestFirstMinEvents) || n_work < kLongestFirstMinPerLane * (int64_t)sms * 1024) return nullptr;
    }
    char *p = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&p), longest_first_bytes(n_work, m.N), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    *park = pe;
    return p;
}

// Simulate trajectories traj_offset .. traj_offset + n_work - 1 whose outputs
// sit in columns 0 .. n_work - 1 of arrays with `stride` columns (out,
// status, n_events and t_final already point at the first column): one
// persistent launch, or park / order / resume (longest-first scheduling,
// above) with the same results.  Arguments are validated by the caller.
int launch_run(const ssa_model *model, int64_t n_work, int64_t stride, uint64_t traj_offset, const int32_t *x0,
               double t_end, int n_samples, const double *sample_times, int precision, int rounding, int normalise,
               uint64_t seed, int64_t max_events, int state_bytes, uint32_t out_species, void *out,
               uint32_t *traj_status, int64_t *n_events, double *t_final, cudaStream_t s)
{
    ssa::RunArgs *a = new (std::nothrow) ssa::RunArgs;
    if (!a) return fail(SSA_ENOMEM, "out of host memory");
    std::memset(a, 0, sizeof(*a));
    fill_structure(*model, normalise, x0, *a);
    a->K = n_samples;
    a->n_traj = stride;
    a->n_work = n_work;
    a->slice_pairs = g_cfg.slice_pairs;
    a->traj_offset = (uint32_t)traj_offset;
    a->n_sets = 1;
    a->traj_per_set = n_work;
    a->t_end = t_end;
    for (int k = 0; k < n_samples; ++k) a->samples[k] = sample_times[k];
    a->key0 = (uint32_t)seed;
    a->key1 = (uint32_t)(seed >> 32);
    a->max_events = max_events;
    a->out = out;
    a->state_bytes = state_bytes;
    a->out_mask = out_mask_of(*model, out_species);
    a->out_N = __builtin_popcount(a->out_mask);
    a->status = traj_status;
    a->n_events = n_events;
    a->t_final = t_final;

    unsigned long long *head = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&head), sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        delete a;
        return e == cudaErrorMemoryAllocation ? fail(SSA_ENOMEM, "work-queue counter: out of device memory")
                                              : cuda_fail(e, "cudaMallocAsync");
    }
    e = cudaMemsetAsync(head, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        cudaFreeAsync(head, s);
        delete a;
        return cuda_fail(e, "cudaMemsetAsync");
    }
    a->queue_head = head;
    a->tail_stats = tail_counters();
    a->lock_spins = g_tail_lock_spins;
    int grid = 0;
    const int norm = normalise ? 1 : 0;
    const ssa::Launcher launch = launcher_for(model->family);
    int64_t park = 0;
    char *scratch = plan_longest_first(*model, x0, normalise, t_end, n_work, max_events, s, &park);
    if (scratch) {
        // launch 1: every trajectory up to `park` events; the unfinished are parked
        ssa::LongestFirstScratch L = carve_longest_first(scratch, n_work, model->N);
        a->max_events = park;
        a->cap_events = max_events;
        a->park_t = L.t;
        a->park_k = L.k;
        a->park_status = L.status;
        a->park_x = L.x;
        a->parked = L.parked;
        e = cudaMemsetAsync(L.parked, 0, (size_t)n_work, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(L.head2, 0, sizeof(unsigned long long), s);
        if (e == cudaSuccess) e = launch(*a, precision, rounding, norm, g_cfg, s, &grid);
        int launched = 1;
        if (e == cudaSuccess) {
            ssa::OrderModel om = order_model(*a, L);
            e = ssa::launch_order(om, n_work, L.hist, L.offs, L.count, L.order, s, &launched);
        }
        if (e == cudaSuccess) {
            // launch 2: the parked trajectories, largest predicted remaining work first
            a->max_events = max_events;
            a->cap_events = 0;
            a->parked = nullptr;
            a->resume_order = L.order;
            a->resume_count = L.count;
            a->resume_events = park;
            a->queue_head = L.head2;
            e = launch(*a, precision, rounding, norm, g_cfg, s, &grid);
            launched += 1;
        }
        g_direct_launches += launched;
        cudaFreeAsync(scratch, s);
    } else {
        e = launch(*a, precision, rounding, norm, g_cfg, s, &grid);
        g_direct_launches += 1;
    }
    cudaError_t e2 = cudaFreeAsync(head, s);
    delete a;
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return SSA_OK;
}

}  // namespace

extern "C" {

const char *ssa_last_error(void) { return g_last_error.c_str(); }

int ssa_set_launch_config(int threads_per_block, int blocks_per_sm, int slice_pairs)
{
    if (threads_per_block == 0) {   // back to the library's defaults
        g_cfg = kDirectDefault;
        g_cfg_set = false;
        return SSA_OK;
    }
    if (threads_per_block < 32 || threads_per_block > 256 || threads_per_block % 32 != 0)
        return fail(SSA_EINVAL, "threads_per_block must be a multiple of 32 in 32..256");
    if (blocks_per_sm < 0 || blocks_per_sm > 64) return fail(SSA_EINVAL, "blocks_per_sm must be in 0..64");
    if (slice_pairs < 1 || slice_pairs > 64) return fail(SSA_EINVAL, "slice_pairs must be in 1..64");
    g_cfg_set = true;
    g_cfg.block = threads_per_block;
    g_cfg.blocks_per_sm = blocks_per_sm;
    g_cfg.slice_pairs = slice_pairs;
    return SSA_OK;
}

int ssa_set_tail_compaction(int enabled)
{
    if (enabled != 0 && enabled != 1) return fail(SSA_EINVAL, "enabled must be 0 or 1");
    g_tail_compaction = enabled != 0;
    return SSA_OK;
}

int ssa_set_tail_lock_limit(int spins)
{
    if (spins < 0) return fail(SSA_EINVAL, "spins must be >= 0");
    g_tail_lock_spins = spins;
    return SSA_OK;
}

int ssa_set_longest_first(int mode, int64_t park_events)
{
    if (mode < 0 || mode > 2) return fail(SSA_EINVAL, "mode must be 0 (off), 1 (automatic) or 2 (always)");
    if (park_events < 0 || (park_events > 0 && (park_events < 2 || (park_events & 1))))
        return fail(SSA_EINVAL, "park_events must be 0 (automatic) or an even number >= 2");
    g_longest_first = mode;
    g_park_events = park_events;
    return SSA_OK;
}

int ssa_direct_kernel_launches(int64_t *count)
{
    if (!count) return fail(SSA_EINVAL, "count is NULL");
    *count = (int64_t)g_direct_launches.load();
    return SSA_OK;
}

int ssa_tail_stats(int64_t *moved, int64_t *lock_timeouts, int64_t *resumed)
{
    unsigned long long c[3] = {0, 0, 0};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(c, g_tail_counters, sizeof(c));
    if (e != cudaSuccess) return cuda_fail(e, "tail counters");
    if (moved) *moved = (int64_t)c[0];
    if (lock_timeouts) *lock_timeouts = (int64_t)c[1];
    if (resumed) *resumed = (int64_t)c[2];
    return SSA_OK;
}

int ssa_model_create(int n_species, int n_reactions, const int32_t *reactant_order, const int32_t *stoich,
                     const double *rate, const int32_t *law, const double *hill, const uint8_t *constant_species,
                     ssa_model **out)
{
    if (!out) return fail(SSA_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_species < 1 || n_species > SSA_MAX_SPECIES) return fail(SSA_EINVAL, "n_species must be in 1..%d", SSA_MAX_SPECIES);
    if (n_reactions < 1 || n_reactions > SSA_MAX_REACTIONS)
        return fail(SSA_EINVAL, "n_reactions must be in 1..%d", SSA_MAX_REACTIONS);
    if (!reactant_order || !stoich || !rate) return fail(SSA_EINVAL, "reactant_order, stoich and rate are required");
    ssa_model *m = new (std::nothrow) ssa_model;
    if (!m) return fail(SSA_ENOMEM, "out of host memory");
    std::memset(m, 0, sizeof(*m));
    m->N = n_species;
    m->M = n_reactions;
    for (int i = 0; i < n_species; ++i) m->constant[i] = constant_species ? (constant_species[i] ? 1 : 0) : 0;
    for (int j = 0; j < n_reactions; ++j) {
        m->law[j] = law ? law[j] : SSA_LAW_MASS_ACTION;
        if (m->law[j] != SSA_LAW_MASS_ACTION && m->law[j] != SSA_LAW_HILL_REPRESSION) {
            delete m;
            return fail(SSA_EINVAL, "law[%d] unknown", j);
        }
        m->rate[j] = rate[j];
        if (m->law[j] == SSA_LAW_MASS_ACTION && (!finite_double(rate[j]) || rate[j] < 0.0)) {
            delete m;
            return fail(SSA_EINVAL, "rate[%d] must be finite and >= 0", j);
        }
        for (int i = 0; i < n_species; ++i) {
            const int r = reactant_order[j * n_species + i];
            if (r < 0 || r > SSA_MAX_ORDER) {
                delete m;
                return fail(SSA_EINVAL, "reactant_order[%d][%d] must be in 0..%d", j, i, SSA_MAX_ORDER);
            }
            m->order[j][i] = r;
            m->stoich[j][i] = stoich[j * n_species + i];
        }
        if (m->law[j] == SSA_LAW_HILL_REPRESSION) {
            if (!hill) {
                delete m;
                return fail(SSA_EINVAL, "hill table required for Hill reactions");
            }
            for (int q = 0; q < 4; ++q) m->hill[j][q] = hill[j * 4 + q];
            const double h = m->hill[j][2], reg = m->hill[j][3];
            if (!finite_double(m->hill[j][0]) || !finite_double(m->hill[j][1]) || m->hill[j][0] < 0 || m->hill[j][1] < 0 ||
                h != std::floor(h) || h < 1 || h > SSA_MAX_HILL || reg != std::floor(reg) || reg < 0 || reg >= n_species) {
                delete m;
                return fail(SSA_EINVAL, "hill[%d] must be {alpha0>=0, alpha>=0, h in 1..%d, regulator species}", j, SSA_MAX_HILL);
            }
            for (int i = 0; i < n_species; ++i) m->order[j][i] = 0;
        }
    }
    m->family = detect_family(*m);
    *out = m;
    return SSA_OK;
}

void ssa_model_destroy(ssa_model *model) { delete model; }

int ssa_model_kernel_family(const ssa_model *model) { return model ? model->family : -1; }

int ssa_ensemble_run(const ssa_model *model, int64_t n_traj, uint64_t traj_offset, const int32_t *x0, double t_end,
                     int n_samples, const double *sample_times, int precision, int rounding, int normalise,
                     uint64_t seed, int64_t max_events, int state_bytes, uint32_t out_species, void *out,
                     uint32_t *traj_status, int64_t *n_events, double *t_final, void *stream)
{
    int rc = validate_run(model, n_traj, traj_offset, x0, t_end, n_samples, sample_times, precision, rounding,
                          max_events, state_bytes, out_species);
    if (rc != SSA_OK) return rc;
    if (n_traj > 0 && (!out || !traj_status)) return fail(SSA_EINVAL, "out and traj_status are required");
    if (n_traj == 0) return SSA_OK;
    return launch_run(model, n_traj, n_traj, traj_offset, x0, t_end, n_samples, sample_times, precision, rounding,
                      normalise, seed, max_events, state_bytes, out_species, out, traj_status, n_events, t_final,
                      static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace {

// Staging memory of the host-buffer entry point comes from a stream-ordered
// pool private to this library whose reservation survives between calls
// (release threshold at the maximum): repeated calls reuse the same device
// pages instead of mapping and unmapping hundreds of megabytes each time.
// The reservation is returned when the process exits.
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_staging_pool[kMaxPoolDevices];
bool g_staging_ready[kMaxPoolDevices];

cudaError_t staging_pool(cudaMemPool_t *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_staging_ready[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_staging_pool[dev] = pool;
        g_staging_ready[dev] = true;
    }
    *out = g_staging_pool[dev];
    return cudaSuccess;
}

// Address under which this device reaches page-locked host memory `p`, or
// null when `p` is not page-locked, not mapped for this device, or not
// reachable under its own (unified) address.
void *pinned_for_device(void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || at.devicePointer != p) return nullptr;
    return p;
}

}  // namespace

extern "C" {

int ssa_ensemble_run_host(const ssa_model *model, int64_t n_traj, uint64_t traj_offset, const int32_t *x0,
                          double t_end, int n_samples, const double *sample_times, int precision, int rounding,
                          int normalise, uint64_t seed, int64_t max_events, int state_bytes, uint32_t out_species,
                          void *out, uint32_t *traj_status, int64_t *n_events, double *t_final, void *stream)
{
    int rc = validate_run(model, n_traj, traj_offset, x0, t_end, n_samples, sample_times, precision, rounding,
                          max_events, state_bytes, out_species);
    if (rc != SSA_OK) return rc;
    if (n_traj > 0 && (!out || !traj_status)) return fail(SSA_EINVAL, "out and traj_status are required");
    if (n_traj == 0) return SSA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t out_N = (size_t)__builtin_popcount(out_mask_of(*model, out_species));
    const size_t out_bytes = (size_t)n_samples * out_N * (size_t)n_traj * (size_t)state_bytes;
    // Page-locked outputs: the kernel writes the results straight into them
    // while it runs (over NVLink-C2C on Grace-Blackwell), with no staging
    // buffers and no copy after the kernel -- when the snapshot stream is
    // sparse.  Each snapshot store crosses the link on its own, so a dense
    // stream (more than kDirectBytesPerEvent snapshot bytes per estimated
    // event) goes through device staging and one bulk copy instead.
    constexpr double kDirectBytesPerEvent = 0.05;
    const double bytes_per_event = (double)(out_bytes / (size_t)n_traj) /
                                   std::max(1.0, estimated_events(*model, x0, normalise, t_end));
    if (bytes_per_event <= kDirectBytesPerEvent && pinned_for_device(out) && pinned_for_device(traj_status) &&
        (!n_events || pinned_for_device(n_events)) && (!t_final || pinned_for_device(t_final))) {
        rc = launch_run(model, n_traj, n_traj, traj_offset, x0, t_end, n_samples, sample_times, precision, rounding,
                        normalise, seed, max_events, state_bytes, out_species, out, traj_status, n_events, t_final,
                        s);
        const cudaError_t es = cudaStreamSynchronize(s);
        if (rc == SSA_OK && es != cudaSuccess) rc = cuda_fail(es, "cudaStreamSynchronize");
        return rc;
    }
    const size_t st_bytes = (size_t)n_traj * sizeof(uint32_t);
    const size_t ev_bytes = n_events ? (size_t)n_traj * sizeof(int64_t) : 0;
    const size_t tf_bytes = t_final ? (size_t)n_traj * sizeof(double) : 0;
    char *d = nullptr;
    const size_t total = out_bytes + st_bytes + ev_bytes + tf_bytes + 64;
    cudaMemPool_t pool;
    cudaError_t e = staging_pool(&pool);
    if (e != cudaSuccess) return cuda_fail(e, "staging memory pool");
    e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&d), total, pool, s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? fail(SSA_ENOMEM, "device buffers") : cuda_fail(e, "cudaMallocFromPoolAsync");
    // 8-byte aligned sub-buffers: int64/double arrays first
    char *p = d;
    int64_t *d_ev = ev_bytes ? reinterpret_cast<int64_t *>(p) : nullptr; p += ev_bytes;
    double *d_tf = tf_bytes ? reinterpret_cast<double *>(p) : nullptr; p += tf_bytes;
    uint32_t *d_st = reinterpret_cast<uint32_t *>(p); p += st_bytes;
    void *d_out = p;
    rc = launch_run(model, n_traj, n_traj, traj_offset, x0, t_end, n_samples, sample_times, precision, rounding,
                    normalise, seed, max_events, state_bytes, out_species, d_out, d_st, d_ev, d_tf, s);
    if (rc == SSA_OK) {
        e = cudaMemcpyAsync(out, d_out, out_bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(traj_status, d_st, st_bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && ev_bytes) e = cudaMemcpyAsync(n_events, d_ev, ev_bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && tf_bytes) e = cudaMemcpyAsync(t_final, d_tf, tf_bytes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync");
    }
    cudaFreeAsync(d, s);
    e = cudaStreamSynchronize(s);
    if (rc == SSA_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    return rc;
}


int ssa_rdme_run(const ssa_model *model, int nx, int ny, int nz, const double *diffusion, int64_t n_traj,
                 uint64_t traj_offset, const int32_t *x0, double t_end, int n_samples, const double *sample_times,
                 int precision, int rounding, int normalise, uint64_t seed, int64_t max_events, int state_bytes,
                 void *out, uint32_t *traj_status, int64_t *n_events, double *t_final, void *stream)
{
    if (!model) return fail(SSA_EINVAL, "model is NULL");
    if (nx < 1 || ny < 1 || nz < 1) return fail(SSA_EINVAL, "lattice extents must be >= 1");
    const long long S = (long long)nx * ny * nz;
    if (S > ssa::kMaxVoxels) return fail(SSA_EINVAL, "lattice has %lld voxels (limit %d)", S, ssa::kMaxVoxels);
    if (!x0) return fail(SSA_EINVAL, "x0 is NULL");
    if (!diffusion) return fail(SSA_EINVAL, "diffusion is NULL");
    const int N = model->N;
    for (long long v = 0; v < S; ++v)
        for (int i = 0; i < N; ++i)
            if (x0[v * N + i] < 0) return fail(SSA_EINVAL, "x0[%lld][%d] is negative", v, i);
    int rc = validate_run(model, n_traj, traj_offset, x0, t_end, n_samples, sample_times, precision, rounding,
                          max_events, state_bytes);
    if (rc != SSA_OK) return rc;
    if (rounding == SSA_SR_ACCUM) return fail(SSA_EINVAL, "the RDME supports SSA_RN and SSA_SR only");
    if (max_events > 4294967294ll) return fail(SSA_EINVAL, "max_events must be <= 2^32 - 2 for the RDME");
    for (int i = 0; i < N; ++i) {
        if (!finite_double(diffusion[i]) || diffusion[i] < 0.0)
            return fail(SSA_EINVAL, "diffusion[%d] must be finite and >= 0", i);
        if (model->constant[i]) {
            if (diffusion[i] != 0.0) return fail(SSA_EINVAL, "constant species %d cannot diffuse", i);
            for (long long v = 1; v < S; ++v)
                if (x0[v * N + i] != x0[i])
                    return fail(SSA_EINVAL, "constant species %d must have the same count in every voxel", i);
        }
    }
    if (n_traj > 0 && (!out || !traj_status)) return fail(SSA_EINVAL, "out and traj_status are required");

    ssa::RdmeArgs *A = new (std::nothrow) ssa::RdmeArgs;
    if (!A) return fail(SSA_ENOMEM, "out of host memory");
    std::memset(A, 0, sizeof(*A));
    fill_structure(*model, normalise, x0, A->a);
    A->nx = nx;
    A->ny = ny;
    A->nz = nz;
    A->S = (int)S;
    A->T = 1;
    A->depth = 0;
    while (A->T < A->S) {
        A->T *= 2;
        A->depth += 1;
    }
    for (int i = 0; i < N; ++i) A->D[i] = diffusion[i];
    A->n_stored = N;                      // general model: every species
    if (model->family != 0) {             // compiled structures keep reservoirs out of the lattice
        A->n_stored = 0;
        for (int i = 0; i < N; ++i) A->n_stored += model->constant[i] ? 0 : 1;
    }
    A->a.K = n_samples;
    A->a.n_traj = n_traj;
    A->a.n_work = n_traj;
    A->a.slice_pairs = 1;
    A->a.traj_offset = (uint32_t)traj_offset;
    A->a.n_sets = 1;
    A->a.traj_per_set = n_traj;
    A->a.t_end = t_end;
    for (int k = 0; k < n_samples; ++k) A->a.samples[k] = sample_times[k];
    A->a.key0 = (uint32_t)seed;
    A->a.key1 = (uint32_t)(seed >> 32);
    A->a.max_events = max_events;
    A->a.out = out;
    A->a.state_bytes = state_bytes;
    A->a.status = traj_status;
    A->a.n_events = n_events;
    A->a.t_final = t_final;
    const int elem = precision == SSA_FP64 ? 8 : 4;
    const bool epochs = precision >= SSA_MIXED_F16 && rounding == SSA_SR;
    if (ssa::rdme_block_size(*A, elem, epochs, other_cfg().block) < 32) {
        delete A;
        return fail(SSA_EINVAL, "lattice state of %lld voxels x %d species does not fit in shared memory", S, N);
    }
    if (n_traj == 0) {
        delete A;
        return SSA_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t lat_bytes = sizeof(int32_t) * (size_t)S * (size_t)N;
    char *d = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d), 256 + lat_bytes, s);
    if (e != cudaSuccess) {
        delete A;
        return e == cudaErrorMemoryAllocation ? fail(SSA_ENOMEM, "RDME tables: out of device memory")
                                              : cuda_fail(e, "cudaMallocAsync");
    }
    A->a.queue_head = reinterpret_cast<unsigned long long *>(d);
    A->x0_lat = reinterpret_cast<const int32_t *>(d + 256);
    e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + 256, x0, lat_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(d, s);
        delete A;
        return cuda_fail(e, "RDME table upload");
    }
    int grid = 0, block = 0;
    e = ssa::launch_rdme(*A, model->family, normalise ? 1 : 0, precision, rounding, other_cfg(), s, &grid, &block);
    cudaError_t e2 = cudaFreeAsync(d, s);
    delete A;
    if (e != cudaSuccess) return cuda_fail(e, "RDME kernel launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return SSA_OK;
}

int ssa_tau_run(const ssa_model *model, int64_t n_traj, uint64_t traj_offset, const int32_t *x0, double t_end,
                double tau, int n_samples, const double *sample_times, int precision, int rounding, int normalise,
                uint64_t seed, int state_bytes, void *out, uint32_t *traj_status, int64_t *n_events,
                double *t_final, void *stream)
{
    int rc = validate_run(model, n_traj, traj_offset, x0, t_end, n_samples, sample_times, precision, rounding, 0,
                          state_bytes);
    if (rc != SSA_OK) return rc;
    if (rounding == SSA_SR_ACCUM) return fail(SSA_EINVAL, "tau-leaping supports SSA_RN and SSA_SR only");
    if (!finite_double(tau) || !(tau > 0.0)) return fail(SSA_EINVAL, "tau must be finite and > 0");
    if (!(t_end / tau <= 2147483647.0)) return fail(SSA_EINVAL, "t_end / tau must be <= 2^31 - 1");
    if (n_traj > 0 && (!out || !traj_status)) return fail(SSA_EINVAL, "out and traj_status are required");
    if (n_traj == 0) return SSA_OK;

    ssa::RunArgs *a = new (std::nothrow) ssa::RunArgs;
    if (!a) return fail(SSA_ENOMEM, "out of host memory");
    std::memset(a, 0, sizeof(*a));
    fill_structure(*model, normalise, x0, *a);
    a->K = n_samples;
    a->n_traj = n_traj;
    a->n_work = n_traj;
    a->slice_pairs = 1;
    a->traj_offset = (uint32_t)traj_offset;
    a->n_sets = 1;
    a->traj_per_set = n_traj;
    a->t_end = t_end;
    a->tau = tau;
    a->n_leaps = (int64_t)std::ceil(t_end / tau);
    for (int k = 0; k < n_samples; ++k) a->samples[k] = sample_times[k];
    a->key0 = (uint32_t)seed;
    a->key1 = (uint32_t)(seed >> 32);
    a->out = out;
    a->state_bytes = state_bytes;
    a->status = traj_status;
    a->n_events = n_events;
    a->t_final = t_final;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long *head = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&head), sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        delete a;
        return e == cudaErrorMemoryAllocation ? fail(SSA_ENOMEM, "work-queue counter: out of device memory")
                                              : cuda_fail(e, "cudaMallocAsync");
    }
    e = cudaMemsetAsync(head, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        cudaFreeAsync(head, s);
        delete a;
        return cuda_fail(e, "cudaMemsetAsync");
    }
    a->queue_head = head;
    int grid = 0;
    e = ssa::launch_tau_family(*a, model->family, normalise ? 1 : 0, precision, rounding, other_cfg(), s, &grid);
    cudaError_t e2 = cudaFreeAsync(head, s);
    delete a;
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return SSA_OK;
}

}  // extern "C"

// ======================================================================
// Batched heterogeneous runs
// ======================================================================
struct ssa_batch {
    int n_groups;
    int precision, rounding, normalise;
    bool compact;
    int64_t work;
    ssa::LaunchConfig cfg;
    char *dmem;
    size_t dmem_bytes;
    ssa::RunArgs *d_groups;
    ssa::RunArgs *d_tune_groups;
    unsigned long long *d_heads;
    ssa::RunArgs *h_groups;   // host copies [n_groups] (one launch, no parking)
    ssa::BatchArgs *args;
    cudaGraphExec_t exec;
    bool graph_valid;
    int graph_kernels;                    // kernels in the captured graph
    // longest-first scheduling: launch 1 from d_groups (parking groups get
    // their parking point as the cap), ordering kernels per parking group,
    // launch 2 from d_groups2
    bool split;
    ssa::RunArgs *d_groups2;
    unsigned long long *d_zero;           // resume count of the groups that do not park
    int64_t *park;                        // host [n_groups]: parking point, 0 = not parked
    ssa::LongestFirstScratch *lf;         // host [n_groups]
    ssa::OrderModel *om;                  // host [n_groups]
};

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device bytes of one group's per-set tables: c' [S][M] f64, Hill amplitudes
// [S][M][2] f64, x0 [S][N] i32, each 256-byte aligned.  Used both to size
// the arena and to place the tables in it.
struct GroupTables {
    size_t cprime, hill, x0;
    size_t total() const { return cprime + hill + x0; }
};

GroupTables group_tables(int64_t n_sets, int M, int N)
{
    GroupTables t;
    t.cprime = align_up(sizeof(double) * (size_t)n_sets * (size_t)M, 256);
    t.hill = align_up(sizeof(double) * 2 * (size_t)n_sets * (size_t)M, 256);
    t.x0 = align_up(sizeof(int32_t) * (size_t)n_sets * (size_t)N, 256);
    return t;
}

void batch_free(ssa_batch *b)
{
    if (!b) return;
    if (b->graph_valid) cudaGraphExecDestroy(b->exec);
    if (b->dmem) cudaFree(b->dmem);
    delete[] b->h_groups;
    delete[] b->park;
    delete[] b->lf;
    delete[] b->om;
    delete b->args;
    delete b;
}

// Launch-1 and launch-2 arguments from the plain ones (h_groups), uploaded to
// d_groups and d_groups2; without the split, d_groups gets the plain ones.
cudaError_t batch_upload(ssa_batch *b)
{
    const size_t bytes = sizeof(ssa::RunArgs) * (size_t)b->n_groups;
    if (!b->split) return cudaMemcpy(b->d_groups, b->h_groups, bytes, cudaMemcpyHostToDevice);
    std::vector<ssa::RunArgs> p1(b->h_groups, b->h_groups + b->n_groups), p2 = p1;
    for (int g = 0; g < b->n_groups; ++g) {
        const ssa::LongestFirstScratch &L = b->lf[g];
        if (b->park[g] > 0) {
            p1[g].max_events = b->park[g];
            p1[g].cap_events = b->h_groups[g].max_events;
            p1[g].park_t = L.t;
            p1[g].park_k = L.k;
            p1[g].park_status = L.status;
            p1[g].park_x = L.x;
            p1[g].parked = L.parked;
            p2[g].park_t = L.t;   // launch 2 reads the parked records
            p2[g].park_k = L.k;
            p2[g].park_status = L.status;
            p2[g].park_x = L.x;
            p2[g].resume_order = L.order;
            p2[g].resume_count = L.count;
            p2[g].resume_events = b->park[g];
            p2[g].queue_head = L.head2;
        } else {   // finished in launch 1: nothing to resume
            p2[g].resume_order = reinterpret_cast<const int64_t *>(b->d_zero);
            p2[g].resume_count = b->d_zero;
        }
    }
    cudaError_t e = cudaMemcpy(b->d_groups, p1.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_groups2, p2.data(), bytes, cudaMemcpyHostToDevice);
    return e;
}

// One batched run on stream s: one launch, or (split) launch 1, the ordering
// kernels of every parking group and launch 2.  Stream-ordered throughout,
// so it can be captured in a graph.  Adds the kernels it launched to
// *launches.
cudaError_t batch_enqueue(ssa_batch *b, const ssa::BatchArgs &args, ssa::LaunchConfig cfg, cudaStream_t s,
                          bool split, int *launches)
{
    cudaError_t e = cudaMemsetAsync(b->d_heads, 0, sizeof(unsigned long long) * (size_t)b->n_groups, s);
    if (e != cudaSuccess) return e;
    int grid = 0;
    if (!split) {
        if (launches) *launches += 1;
        return ssa::launch_batch(args, b->work, b->precision, b->rounding, b->compact, cfg, s, &grid);
    }
    for (int g = 0; g < b->n_groups && e == cudaSuccess; ++g) {
        if (b->park[g] <= 0) continue;
        e = cudaMemsetAsync(b->lf[g].parked, 0, (size_t)b->h_groups[g].n_work, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->lf[g].head2, 0, sizeof(unsigned long long), s);
    }
    if (e == cudaSuccess) e = ssa::launch_batch(args, b->work, b->precision, b->rounding, b->compact, cfg, s, &grid);
    int n = 1;
    for (int g = 0; g < b->n_groups && e == cudaSuccess; ++g)
        if (b->park[g] > 0) e = ssa::launch_order(b->om[g], b->h_groups[g].n_work, b->lf[g].hist, b->lf[g].offs,
                                                  b->lf[g].count, b->lf[g].order, s, &n);
    if (e == cudaSuccess) {
        ssa::BatchArgs a2 = args;
        a2.groups = b->d_groups2;
        e = ssa::launch_batch(a2, b->work, b->precision, b->rounding, b->compact, cfg, s, &grid);
        n += 1;
    }
    if (launches) *launches += n;
    return e;
}

}  // namespace

extern "C" {

int ssa_batch_create(int n_groups, const ssa_batch_group *groups, double t_end, int n_samples,
                     const double *sample_times, int precision, int rounding, int normalise, uint64_t seed,
                     int64_t max_events, int state_bytes, ssa_batch **out)
{
    if (!out) return fail(SSA_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_groups < 1 || n_groups > ssa::kMaxGroups) return fail(SSA_EINVAL, "n_groups must be in 1..%d", ssa::kMaxGroups);
    if (!groups) return fail(SSA_EINVAL, "groups is NULL");
    // table sizes, validation
    size_t bytes = align_up(sizeof(ssa::RunArgs) * (size_t)n_groups, 256) * 2 + 256;
    int64_t work = 0;
    bool compact = true;
    double est_events[ssa::kMaxGroups] = {0.0};
    double est_spread[ssa::kMaxGroups] = {0.0};
    for (int g = 0; g < n_groups; ++g) {
        const ssa_batch_group &G = groups[g];
        if (!G.model) return fail(SSA_EINVAL, "group %d: model is NULL", g);
        if (G.n_sets < 1 || G.traj_per_set < 0) return fail(SSA_EINVAL, "group %d: n_sets >= 1 and traj_per_set >= 0", g);
        if (!G.x0) return fail(SSA_EINVAL, "group %d: x0 is NULL", g);
        const int64_t items = G.n_sets * G.traj_per_set;
        for (int64_t q = 0; q < G.n_sets; ++q) {
            const int rc = validate_run(G.model, items, G.traj_offset, G.x0 + q * G.model->N, t_end, n_samples,
                                        sample_times, precision, rounding, max_events, state_bytes);
            if (rc != SSA_OK) return fail(rc, "group %d, set %lld: %s", g, (long long)q, g_last_error.c_str());
            if (G.rates)
                for (int j = 0; j < G.model->M; ++j) {
                    const double c = G.rates[q * G.model->M + j];
                    if (G.model->law[j] == SSA_LAW_MASS_ACTION && (!finite_double(c) || c < 0.0))
                        return fail(SSA_EINVAL, "group %d, set %lld: rate %d must be finite and >= 0", g, (long long)q, j);
                }
            if (G.hill)
                for (int j = 0; j < G.model->M; ++j)
                    for (int c = 0; c < 2; ++c) {
                        const double v = G.hill[(q * G.model->M + j) * 2 + c];
                        if (G.model->law[j] == SSA_LAW_HILL_REPRESSION && (!finite_double(v) || v < 0.0))
                            return fail(SSA_EINVAL, "group %d, set %lld: Hill amplitudes must be finite and >= 0", g, (long long)q);
                    }
        }
        if (items > 0 && (!G.out || !G.traj_status)) return fail(SSA_EINVAL, "group %d: out and traj_status are required", g);
        const int fam = G.model->family;
        if (fam < 3) compact = false;
        work += items;
        bytes += group_tables(G.n_sets, G.model->M, G.model->N).total();
        // mean and spread of the estimated events per trajectory over the
        // group's sets
        double est = 0.0, est_lo = 1e300, est_hi = 0.0;
        for (int64_t q = 0; q < G.n_sets; ++q) {
            ssa_model mq = *G.model;
            for (int j = 0; j < mq.M; ++j) {
                if (G.rates) mq.rate[j] = G.rates[q * mq.M + j];
                if (G.hill && mq.law[j] == SSA_LAW_HILL_REPRESSION)
                    for (int c = 0; c < 2; ++c) mq.hill[j][c] = G.hill[(q * mq.M + j) * 2 + c];
            }
            const double e = estimated_events(mq, G.x0 + q * mq.N, normalise, t_end);
            est += e;
            est_lo = std::min(est_lo, e);
            est_hi = std::max(est_hi, e);
        }
        est_events[g] = est / (double)G.n_sets;
        est_spread[g] = est_hi > 0.0 ? est_hi / std::max(est_lo, 1e-300) : 1.0;
    }
    // longest-first scheduling per group (as for single runs)
    int64_t park[ssa::kMaxGroups] = {0};
    bool split = false;
    if (g_longest_first != 0 && work > 0) {
        int dev = 0, sms = 0;
        const bool ok = cudaGetDevice(&dev) == cudaSuccess &&
                        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
        const bool enough = g_longest_first == 2 || (ok && work >= kLongestFirstMinPerLane * (int64_t)sms * 1024);
        for (int g = 0; g < n_groups && enough; ++g) {
            const int64_t items = groups[g].n_sets * groups[g].traj_per_set;
            if (items < 1) continue;
            // automatic: long trajectories, or sets whose estimated work spreads widely
            if (g_longest_first == 1 && !(est_events[g] >= kLongestFirstMinEvents) &&
                !(est_spread[g] >= kLongestFirstMinSpread))
                continue;
            int64_t pe = g_park_events;
            if (pe <= 0) {
                const double p = est_events[g] / 5.0;
                pe = p < 256.0 ? 256 : (p > 1073741824.0 ? 1073741824 : (int64_t)p);
            }
            pe &= ~(int64_t)1;
            if (pe < 2 || pe >= max_events) continue;
            park[g] = pe;
            split = true;
            bytes += align_up(longest_first_bytes(items, groups[g].model->N), 256);
        }
    }
    if (split) bytes += align_up(sizeof(ssa::RunArgs) * (size_t)n_groups, 256) + 256;
    ssa_batch *b = new (std::nothrow) ssa_batch;
    if (!b) return fail(SSA_ENOMEM, "out of host memory");
    std::memset(b, 0, sizeof(*b));
    b->n_groups = n_groups;
    b->precision = precision;
    b->rounding = rounding;
    b->normalise = normalise ? 1 : 0;
    b->compact = compact;
    b->work = work;
    b->cfg = other_cfg();
    b->h_groups = new (std::nothrow) ssa::RunArgs[n_groups];
    b->args = new (std::nothrow) ssa::BatchArgs;
    b->split = split;
    b->park = new (std::nothrow) int64_t[n_groups];
    b->lf = new (std::nothrow) ssa::LongestFirstScratch[n_groups];
    b->om = new (std::nothrow) ssa::OrderModel[n_groups];
    if (!b->h_groups || !b->args || !b->park || !b->lf || !b->om) {
        batch_free(b);
        return fail(SSA_ENOMEM, "out of host memory");
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&b->dmem), bytes);
    if (e != cudaSuccess) {
        batch_free(b);
        return e == cudaErrorMemoryAllocation ? fail(SSA_ENOMEM, "batch tables: out of device memory")
                                              : cuda_fail(e, "cudaMalloc");
    }
    b->dmem_bytes = bytes;
    char *p = b->dmem;
    b->d_groups = reinterpret_cast<ssa::RunArgs *>(p);
    p += align_up(sizeof(ssa::RunArgs) * (size_t)n_groups, 256);
    b->d_tune_groups = reinterpret_cast<ssa::RunArgs *>(p);
    p += align_up(sizeof(ssa::RunArgs) * (size_t)n_groups, 256);
    b->d_heads = reinterpret_cast<unsigned long long *>(p);
    p += 256;
    if (split) {
        b->d_groups2 = reinterpret_cast<ssa::RunArgs *>(p);
        p += align_up(sizeof(ssa::RunArgs) * (size_t)n_groups, 256);
        b->d_zero = reinterpret_cast<unsigned long long *>(p);
        p += 256;
        e = cudaMemset(b->d_zero, 0, sizeof(unsigned long long));
    }
    for (int g = 0; g < n_groups; ++g) {
        b->park[g] = park[g];
        std::memset(&b->lf[g], 0, sizeof(b->lf[g]));
        std::memset(&b->om[g], 0, sizeof(b->om[g]));
    }

    std::memset(b->args, 0, sizeof(*b->args));
    b->args->n_groups = n_groups;
    b->args->normalise = b->normalise;
    b->args->K = n_samples;
    b->args->t_end = t_end;
    b->args->groups = b->d_groups;
    for (int k = 0; k < n_samples; ++k) b->args->samples[k] = sample_times[k];

    for (int g = 0; g < n_groups && e == cudaSuccess; ++g) {
        const ssa_batch_group &G = groups[g];
        const ssa_model &m = *G.model;
        ssa::RunArgs &a = b->h_groups[g];
        std::memset(&a, 0, sizeof(a));
        fill_structure(m, normalise, G.x0, a);
        const int64_t S = G.n_sets;
        std::vector<double> cp((size_t)S * m.M), hl((size_t)S * m.M * 2);
        for (int64_t q = 0; q < S; ++q) {
            ssa_model mq = m;
            if (G.rates)
                for (int j = 0; j < m.M; ++j) mq.rate[j] = G.rates[q * m.M + j];
            int8_t folded[ssa::kMaxM][ssa::kMaxN];
            rate_constants(mq, G.x0 + q * m.N, normalise, &cp[(size_t)q * m.M], folded);
            for (int j = 0; j < m.M; ++j) {
                const bool hill = m.law[j] == SSA_LAW_HILL_REPRESSION;
                hl[((size_t)q * m.M + j) * 2 + 0] = hill ? (G.hill ? G.hill[(q * m.M + j) * 2 + 0] : m.hill[j][0]) : 0.0;
                hl[((size_t)q * m.M + j) * 2 + 1] = hill ? (G.hill ? G.hill[(q * m.M + j) * 2 + 1] : m.hill[j][1]) : 0.0;
            }
        }
        const GroupTables T = group_tables(S, m.M, m.N);
        if ((size_t)(p - b->dmem) + T.total() > b->dmem_bytes) {   // placement must stay inside the arena
            batch_free(b);
            return fail(SSA_EINVAL, "internal: batch table layout exceeds its arena");
        }
        double *d_cp = reinterpret_cast<double *>(p);
        p += T.cprime;
        double *d_hl = reinterpret_cast<double *>(p);
        p += T.hill;
        int32_t *d_x0 = reinterpret_cast<int32_t *>(p);
        p += T.x0;
        e = cudaMemcpy(d_cp, cp.data(), sizeof(double) * cp.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_hl, hl.data(), sizeof(double) * hl.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_x0, G.x0, sizeof(int32_t) * (size_t)S * m.N, cudaMemcpyHostToDevice);
        a.K = n_samples;
        a.n_traj = S * G.traj_per_set;
        a.n_work = a.n_traj;
        a.slice_pairs = b->cfg.slice_pairs;
        a.traj_offset = (uint32_t)G.traj_offset;
        a.n_sets = (int)S;
        a.traj_per_set = G.traj_per_set > 0 ? G.traj_per_set : 1;
        a.cprime_tab = d_cp;
        a.hill_tab = d_hl;
        a.x0_tab = d_x0;
        a.t_end = t_end;
        for (int k = 0; k < n_samples; ++k) a.samples[k] = sample_times[k];
        a.key0 = (uint32_t)seed;
        a.key1 = (uint32_t)(seed >> 32);
        a.max_events = max_events;
        a.out = G.out;
        a.state_bytes = state_bytes;
        a.status = G.traj_status;
        a.n_events = G.n_events;
        a.t_final = G.t_final;
        a.queue_head = b->d_heads + g;
        b->args->family[g] = (int8_t)m.family;
        if (park[g] > 0) {
            const size_t lb = align_up(longest_first_bytes(a.n_work, m.N), 256);
            if ((size_t)(p - b->dmem) + lb > b->dmem_bytes) {
                batch_free(b);
                return fail(SSA_EINVAL, "internal: batch scratch layout exceeds its arena");
            }
            b->lf[g] = carve_longest_first(p, a.n_work, m.N);
            b->om[g] = order_model(a, b->lf[g]);
            p += lb;
        }
    }
    if (e == cudaSuccess) e = batch_upload(b);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch upload");
    }
    *out = b;
    return SSA_OK;
}

int ssa_batch_launch(ssa_batch *b, void *stream)
{
    if (!b) return fail(SSA_EINVAL, "batch is NULL");
    if (b->work == 0) return SSA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (s == nullptr) {
        int n = 0;
        e = batch_enqueue(b, *b->args, b->cfg, s, b->split, &n);
        g_direct_launches += n;
        return e == cudaSuccess ? SSA_OK : cuda_fail(e, "batch launch");
    }
    if (!b->graph_valid) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        b->graph_kernels = 0;
        const cudaError_t e1 = batch_enqueue(b, *b->args, b->cfg, s, b->split, &b->graph_kernels);
        e = cudaStreamEndCapture(s, &graph);
        if (e1 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e1, "batch capture");
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        b->graph_valid = true;
    }
    e = cudaGraphLaunch(b->exec, s);
    if (e == cudaSuccess) g_direct_launches += b->graph_kernels;
    return e == cudaSuccess ? SSA_OK : cuda_fail(e, "cudaGraphLaunch");
}

int ssa_batch_autotune(ssa_batch *b, void *stream, int *threads_per_block, int *blocks_per_sm, int *slice_pairs,
                       double *best_ms)
{
    if (!b) return fail(SSA_EINVAL, "batch is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    // the same capped proxy workload for every candidate
    const int64_t lanes = (int64_t)sms * 2048;
    std::vector<ssa::RunArgs> tune(b->h_groups, b->h_groups + b->n_groups);
    int64_t tune_work = 0;
    for (auto &a : tune) {
        a.n_work = a.n_traj < 2 * lanes / b->n_groups ? a.n_traj : 2 * lanes / b->n_groups;
        if (a.max_events > 4096) a.max_events = 4096;
        tune_work += a.n_work;
    }
    if (tune_work == 0) return SSA_OK;
    const int blocks[] = {64, 128, 256};
    const int per_sm[] = {0, 4, 2};
    const int slices[] = {1, 4, 16};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    ssa::BatchArgs targs = *b->args;
    targs.groups = b->d_tune_groups;
    double best = 1e300;
    ssa::LaunchConfig best_cfg = b->cfg;
    for (int blk : blocks)
        for (int ps : per_sm)
            for (int sl : slices) {
                for (auto &a : tune) a.slice_pairs = sl;
                e = cudaMemcpyAsync(b->d_tune_groups, tune.data(), sizeof(ssa::RunArgs) * tune.size(),
                                    cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                ssa::LaunchConfig cfg = {blk, ps, sl};
                if (e == cudaSuccess) e = batch_enqueue(b, targs, cfg, s, false, nullptr);   // warm
                if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                if (e == cudaSuccess) e = batch_enqueue(b, targs, cfg, s, false, nullptr);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return cuda_fail(e, "autotune run");
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    best_cfg = cfg;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cfg = best_cfg;
    for (int g = 0; g < b->n_groups; ++g) b->h_groups[g].slice_pairs = best_cfg.slice_pairs;
    e = batch_upload(b);
    if (e != cudaSuccess) return cuda_fail(e, "autotune upload");
    if (b->graph_valid) {
        cudaGraphExecDestroy(b->exec);
        b->graph_valid = false;
    }
    if (threads_per_block) *threads_per_block = best_cfg.block;
    if (blocks_per_sm) *blocks_per_sm = best_cfg.blocks_per_sm;
    if (slice_pairs) *slice_pairs = best_cfg.slice_pairs;
    if (best_ms) *best_ms = best;
    return SSA_OK;
}

void ssa_batch_destroy(ssa_batch *b) { batch_free(b); }

}  // extern "C"

// ======================================================================
// Parameter sweep without allocation
// ======================================================================
// Some callers cannot allocate device memory when they run a simulation:
// programs whose device memory is owned by another allocator or held to a
// fixed budget after start-up, and real-time or embedded loops that forbid
// allocation on their hot path.  For them the sweep's scratch memory (the
// work-queue counter and the per-set rate and initial-state tables) lives in
// one static device array that every GPU loading this library keeps until
// the process exits.  In host code `g_noalloc_scratch` names a host-side
// stand-in, never a device address: the device address is looked up once
// per device with cudaGetSymbolAddress and then passed to the kernel.
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SSA_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices];   // device address of the scratch per device ordinal

int noalloc_scratch(void **ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(SSA_EINVAL, "device ordinal %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
    return SSA_OK;
}

// Copy host values to the device through a fixed stack buffer (no heap).
template <class T, class F>
cudaError_t upload_chunked(T *dst, size_t count, F value, cudaStream_t s)
{
    T buf[512];
    for (size_t at = 0; at < count;) {
        const size_t n = count - at < 512 ? count - at : 512;
        for (size_t q = 0; q < n; ++q) buf[q] = value(at + q);
        // pageable source: the call returns once `buf` has been staged
        const cudaError_t e = cudaMemcpyAsync(dst + at, buf, sizeof(T) * n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        at += n;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

size_t ssa_sweep_noalloc_scratch_bytes(int n_species, int n_reactions, int64_t n_sets)
{
    if (n_sets < 0) return 0;
    // every set needs at least 8 bytes, so larger counts can never fit (and
    // the table sizes below could wrap around)
    if (n_sets > (int64_t)SSA_NOALLOC_SCRATCH_BYTES / 8) return SIZE_MAX;
    const GroupTables T = group_tables(n_sets, n_reactions, n_species);
    return 256 + T.total();
}

int ssa_sweep_run_noalloc(const ssa_model *model, int64_t n_sets, int64_t traj_per_set, const double *rates,
                          const double *hill, const int32_t *x0, uint64_t traj_offset, double t_end, int n_samples,
                          const double *sample_times, int precision, int rounding, int normalise, uint64_t seed,
                          int64_t max_events, int state_bytes, void *out, uint32_t *traj_status, int64_t *n_events,
                          double *t_final, void *stream)
{
    if (!model) return fail(SSA_EINVAL, "model is NULL");
    if (n_sets < 1 || traj_per_set < 0) return fail(SSA_EINVAL, "n_sets >= 1 and traj_per_set >= 0");
    if (n_sets > (int64_t)SSA_NOALLOC_SCRATCH_BYTES / 8)
        return fail(SSA_EINVAL, "n_sets = %lld cannot fit the static scratch of %d bytes", (long long)n_sets,
                    SSA_NOALLOC_SCRATCH_BYTES);
    if (traj_per_set > INT64_MAX / n_sets) return fail(SSA_EINVAL, "n_sets * traj_per_set overflows");
    if (!x0) return fail(SSA_EINVAL, "x0 is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        // The per-set tables are staged from a stack buffer that is gone when
        // the call returns, so a captured copy would replay garbage: refuse.
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const cudaError_t ce = cudaStreamIsCapturing(s, &cs);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamIsCapturing");
        if (cs != cudaStreamCaptureStatusNone)
            return fail(SSA_EINVAL, "stream is capturing: ssa_sweep_run_noalloc stages its tables from host memory "
                                    "that does not outlive the call and cannot be captured");
    }
    const ssa_model &m = *model;
    const size_t need = ssa_sweep_noalloc_scratch_bytes(m.N, m.M, n_sets);
    if (need > (size_t)SSA_NOALLOC_SCRATCH_BYTES)
        return fail(SSA_EINVAL, "sweep needs %zu bytes of scratch, the static scratch holds %d: split it into sweeps "
                                "of fewer parameter sets", need, SSA_NOALLOC_SCRATCH_BYTES);
    const int64_t items = n_sets * traj_per_set;
    for (int64_t q = 0; q < n_sets; ++q) {
        const int rc = validate_run(model, items, traj_offset, x0 + q * m.N, t_end, n_samples, sample_times, precision,
                                    rounding, max_events, state_bytes);
        if (rc != SSA_OK) return rc;
        for (int j = 0; j < m.M; ++j) {
            if (rates && m.law[j] == SSA_LAW_MASS_ACTION && (!finite_double(rates[q * m.M + j]) || rates[q * m.M + j] < 0.0))
                return fail(SSA_EINVAL, "set %lld: rate %d must be finite and >= 0", (long long)q, j);
            if (hill && m.law[j] == SSA_LAW_HILL_REPRESSION)
                for (int c = 0; c < 2; ++c) {
                    const double v = hill[(q * m.M + j) * 2 + c];
                    if (!finite_double(v) || v < 0.0)
                        return fail(SSA_EINVAL, "set %lld: Hill amplitudes must be finite and >= 0", (long long)q);
                }
        }
    }
    if (items > 0 && (!out || !traj_status)) return fail(SSA_EINVAL, "out and traj_status are required");
    if (items == 0) return SSA_OK;

    void *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != SSA_OK) return rc;
    unsigned long long *head = static_cast<unsigned long long *>(scratch);
    const GroupTables T = group_tables(n_sets, m.M, m.N);
    double *d_cp = reinterpret_cast<double *>(static_cast<char *>(scratch) + 256);
    double *d_hl = reinterpret_cast<double *>(reinterpret_cast<char *>(d_cp) + T.cprime);
    int32_t *d_x0 = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(d_hl) + T.hill);

    // per-set c' in binary64 (same folding as every other entry point)
    auto cprime_of = [&](size_t idx) {
        const int64_t q = (int64_t)(idx / (size_t)m.M);
        ssa_model mq = m;
        if (rates)
            for (int j = 0; j < m.M; ++j) mq.rate[j] = rates[q * m.M + j];
        double c[ssa::kMaxM];
        int8_t folded[ssa::kMaxM][ssa::kMaxN];
        rate_constants(mq, x0 + q * m.N, normalise, c, folded);
        return c[idx % (size_t)m.M];
    };
    auto hill_of = [&](size_t idx) {
        const size_t jq = idx / 2;
        const int64_t q = (int64_t)(jq / (size_t)m.M);
        const int j = (int)(jq % (size_t)m.M);
        if (m.law[j] != SSA_LAW_HILL_REPRESSION) return 0.0;
        return hill ? hill[(q * m.M + j) * 2 + (idx & 1)] : m.hill[j][idx & 1];
    };
    ssa::RunArgs a;   // on the stack: no heap allocation either
    std::memset(&a, 0, sizeof(a));
    fill_structure(m, normalise, x0, a);
    for (int j = 0; j < m.M; ++j) {
        a.cprime[j] = cprime_of((size_t)j);
        a.hill_a0[j] = hill_of((size_t)j * 2);
        a.hill_a[j] = hill_of((size_t)j * 2 + 1);
    }
    a.K = n_samples;
    a.n_traj = items;
    a.n_work = items;
    a.slice_pairs = g_cfg.slice_pairs;
    a.traj_offset = (uint32_t)traj_offset;
    a.n_sets = (int)n_sets;
    a.traj_per_set = traj_per_set > 0 ? traj_per_set : 1;
    a.cprime_tab = d_cp;
    a.hill_tab = d_hl;
    a.x0_tab = d_x0;
    a.t_end = t_end;
    for (int k = 0; k < n_samples; ++k) a.samples[k] = sample_times[k];
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.max_events = max_events;
    a.out = out;
    a.state_bytes = state_bytes;
    a.status = traj_status;
    a.n_events = n_events;
    a.t_final = t_final;
    a.queue_head = head;
    a.tail_stats = tail_counters();
    a.lock_spins = g_tail_lock_spins;

    // the scratch keeps the previous call's contents: reset the queue counter
    cudaError_t e = cudaMemsetAsync(head, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = upload_chunked(d_cp, (size_t)n_sets * m.M, cprime_of, s);
    if (e == cudaSuccess) e = upload_chunked(d_hl, (size_t)n_sets * m.M * 2, hill_of, s);
    if (e == cudaSuccess) e = upload_chunked(d_x0, (size_t)n_sets * m.N, [&](size_t i) { return x0[i]; }, s);
    if (e != cudaSuccess) return cuda_fail(e, "scratch upload");
    int grid = 0;
    e = launcher_for(m.family)(a, precision, rounding, normalise ? 1 : 0, g_cfg, s, &grid);
    return e == cudaSuccess ? SSA_OK : cuda_fail(e, "kernel launch");
}

}  // extern "C"
