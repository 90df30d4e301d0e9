/*
 * ssa.h -- C ABI of the GB300 ensemble engine for the reduced-precision
 * Gillespie direct method (Kimpson, Flegg & Flegg, "Reduced-Precision
 * Stochastic Simulation for Mathematical Biology").
 *
 * Problem statement (Sec. 2 of the paper): N species X_1..X_N, M reaction
 * channels R_1..R_M, each with a propensity a_j(x) and a change vector nu_j.
 * The direct method repeats: compute every a_j and a0 = sum_j a_j; draw
 * tau = -ln(u1)/a0; fire the smallest mu with sum_{j<=mu} a_j > u2*a0;
 * x += nu_mu, t += tau.
 *
 * Conventions for every entry point:
 *  - Plain pointers and sizes only.  "host" pointers are read during the call
 *    and may be freed when it returns; "device" pointers are CUDA global
 *    memory owned by the caller and must stay valid until the work queued on
 *    the stream has finished.  A device output may also be page-locked host
 *    memory that the device addresses under the same pointer (cudaHostAlloc,
 *    unified addressing): the kernel then writes its results straight into
 *    host memory (over NVLink-C2C on Grace-Blackwell).
 *  - Functions return SSA_OK (0) or a negative ssa_status.  Invalid arguments
 *    are rejected on the host before anything is launched (SSA_EINVAL); the
 *    message is available from ssa_last_error() on the calling thread.
 *  - Launches are asynchronous on the given CUDA stream (NULL = legacy default
 *    stream) unless the entry point says otherwise.
 *  - Per-trajectory problems (overflow, event cap, ...) never abort a launch:
 *    they are reported as status bits in traj_status[].
 *  - Results of a trajectory depend only on (model, x0, rates, t_end, sample
 *    times, precision, rounding, normalise, seed, max_events, global
 *    trajectory id); never on the launch configuration or on other
 *    trajectories.
 */
#ifndef SSA_H
#define SSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ssa_model ssa_model;   /* opaque, owned by the library */

/* Propensity laws.
 * SSA_LAW_MASS_ACTION: a_j = c'_j * prod_i prod_{m<r_ij} (x_i - m), with
 *   c'_j = c_j / prod_i r_ij!  (Gillespie's c-convention: c_j times the number
 *   of distinct reactant combinations; Sec. 4.2 Schloegl k2 n(n-1)(n-2),
 *   Sec. 4.4 dimer kf nA(nA-1)/2).  a_j = 0 when any x_i < r_ij.
 * SSA_LAW_HILL_REPRESSION: a_j = alpha0 + alpha / (1 + P^h) with P the count
 *   of the regulator species (Sec. 4.5, repressilator transcription); the
 *   rate c_j is not used. */
typedef enum { SSA_LAW_MASS_ACTION = 0, SSA_LAW_HILL_REPRESSION = 1 } ssa_law;

/* Precision modes (Sec. 3.2 and Sec. 4 mode list).  Tp = propensity type,
 * Ta = type of the propensity sum, Tt = time type; state is int32 in all.
 *   SSA_FP64          Tp = Ta = Tt = binary64
 *   SSA_FP32          Tp = Ta = Tt = binary32
 *   SSA_MIXED_F16     Tp = binary16, Ta = Tt = binary32
 *   SSA_MIXED_BF16    Tp = bfloat16, Ta = Tt = binary32
 *   SSA_UNIFORM_F16   every operation rounded to binary16
 *   SSA_UNIFORM_BF16  every operation rounded to bfloat16 */
typedef enum {
    SSA_FP64 = 0, SSA_FP32 = 1, SSA_MIXED_F16 = 2, SSA_MIXED_BF16 = 3,
    SSA_UNIFORM_F16 = 4, SSA_UNIFORM_BF16 = 5
} ssa_precision;

/* Rounding of 16-bit operations (Sec. 3.3): round-to-nearest-even, or
 * stochastic rounding applied after every operation whose result has the
 * 16-bit type (valid with the four 16-bit modes), or selective stochastic
 * rounding: SR only at the accumulation points -- the partial sums of the
 * propensities and the clock update -- and round-to-nearest elsewhere (the
 * strategy Sec. 3.3 names without testing; valid with the uniform modes,
 * since mixed modes accumulate in binary32). */
typedef enum { SSA_RN = 0, SSA_SR = 1, SSA_SR_ACCUM = 2 } ssa_rounding;

typedef enum {
    SSA_OK = 0, SSA_EINVAL = -1, SSA_ENOMEM = -2, SSA_ECUDA = -3, SSA_ETIMEDOUT = -4
} ssa_status;

/* Per-trajectory status bits written to traj_status[]. */
enum {
    SSA_TRAJ_OVERFLOW = 1,     /* a0 = +inf: the trajectory stops at its current state */
    SSA_TRAJ_MAX_EVENTS = 2,   /* the event cap was reached before t_end */
    SSA_TRAJ_STATE_RANGE = 4,  /* a count went negative, or did not fit int16 storage */
    SSA_TRAJ_NAN = 8,          /* a0 = NaN */
    SSA_TRAJ_TAU_CLAMPED = 16  /* tau-leaping: a leap drove a count below 0; it was set to 0 */
};

/* Limits of this build. */
enum { SSA_MAX_SPECIES = 8, SSA_MAX_REACTIONS = 16, SSA_MAX_ORDER = 3, SSA_MAX_HILL = 4,
       SSA_MAX_SAMPLES = 1024 };

/*
 * ssa_model_create -- describe a reaction network (Sec. 2 problem statement).
 *   n_species         N, 1..SSA_MAX_SPECIES
 *   n_reactions       M, 1..SSA_MAX_REACTIONS
 *   reactant_order    host [M][N] row-major, r_ij in 0..SSA_MAX_ORDER
 *   stoich            host [M][N] row-major, net change nu_ij
 *   rate              host [M] c-convention constants c_j >= 0 (finite)
 *   law               host [M] ssa_law, or NULL for all mass action
 *   hill              host [M][4] {alpha0, alpha, h, regulator} for Hill rows
 *                     (h integer 1..SSA_MAX_HILL, regulator a species index),
 *                     or NULL when no row uses SSA_LAW_HILL_REPRESSION
 *   constant_species  host [N], 1 = reservoir held at its initial count
 *                     (its nu entries are ignored), or NULL for none
 *   out               receives the model handle
 * Errors: SSA_EINVAL on any out-of-range entry; SSA_ENOMEM.
 */
int ssa_model_create(int n_species, int n_reactions, const int32_t *reactant_order,
                     const int32_t *stoich, const double *rate, const int32_t *law,
                     const double *hill, const uint8_t *constant_species, ssa_model **out);

/* Release a model (NULL is allowed).  No launch may still be using it. */
void ssa_model_destroy(ssa_model *model);

/* Which compiled kernel family serves this model: 0 = general table-driven
 * kernel, >0 = a structure-specialised kernel (1 birth-death, 2 Schloegl,
 * 3 telegraph, 4 dimer, 5 repressilator).  Negative on a NULL model. */
int ssa_model_kernel_family(const ssa_model *model);

/*
 * ssa_ensemble_run -- simulate n_traj independent trajectories of one model
 * from one initial state, one trajectory per GPU lane.
 *   n_traj        number of trajectories, >= 0
 *   traj_offset   global id of the first trajectory; ids offset..offset+n_traj-1
 *                 must fit in 32 bits.  Trajectory r draws its random numbers
 *                 from Philox4x32-10 streams keyed by (seed, offset + r).
 *   x0            host [N] initial counts (>= 0)
 *   t_end         final time, finite, > 0
 *   n_samples     K, 1..SSA_MAX_SAMPLES
 *   sample_times  host [K] ascending, 0 <= s_k <= t_end.  Snapshot k holds
 *                 the state after every event at time <= s_k.
 *   precision, rounding   see above
 *   normalise     1: fold constant species into the rate constants in
 *                 binary64 before rounding to Tp (Sec. 4.2 rescaling)
 *   seed          64-bit Philox key
 *   max_events    event cap per trajectory, >= 0
 *   state_bytes   4 (int32 snapshots) or 2 (int16; values are clamped and
 *                 flagged SSA_TRAJ_STATE_RANGE when out of range)
 *   out_species   bit i set: species i is stored in the snapshots; 0 means
 *                 every species.  A run stores only what the caller needs --
 *                 e.g. not the reservoir species that normalisation holds
 *                 fixed -- and its snapshot stream shrinks accordingly.  The
 *                 simulation itself never depends on it; int16 clamping (and
 *                 its status bit) applies to stored species only.  Bits
 *                 beyond n_species are rejected (SSA_EINVAL).
 *   out           device [K][Ns][n_traj], Ns = number of stored species (in
 *                 ascending species order), trajectory index fastest
 *   traj_status   device [n_traj] status bits
 *   n_events      device [n_traj] events fired per trajectory, or NULL
 *   t_final       device [n_traj] time of the last event (widened), or NULL
 *   stream        cudaStream_t, or NULL
 * The call allocates an 8-byte work-queue counter with stream-ordered
 * allocation and frees it after the launch.
 * Errors: SSA_EINVAL (arguments), SSA_ENOMEM, SSA_ECUDA (launch failure).
 */
int ssa_ensemble_run(const ssa_model *model, int64_t n_traj, uint64_t traj_offset,
                     const int32_t *x0, double t_end, int n_samples, const double *sample_times,
                     int precision, int rounding, int normalise, uint64_t seed,
                     int64_t max_events, int state_bytes, uint32_t out_species, void *out,
                     uint32_t *traj_status, int64_t *n_events, double *t_final, void *stream);

/*
 * ssa_ensemble_run_host -- ssa_ensemble_run with HOST output buffers;
 * synchronises the stream before returning.  out, traj_status, n_events and
 * t_final are host pointers with the layouts above (n_events, t_final may be
 * NULL).
 *  - If every given output is page-locked host memory that the current
 *    device addresses under the same pointer (cudaHostAlloc, or
 *    cudaHostRegister with mapping; unified addressing) and the snapshot
 *    stream is sparse (at most 0.05 snapshot bytes per event, events
 *    estimated as a0(x0) * t_end), the kernel writes the results straight
 *    into it as the ensemble runs -- on Grace-Blackwell over NVLink-C2C --
 *    with no device buffers and no copy afterwards.  A denser stream would
 *    cross the link one small store at a time, so it is staged instead.
 *  - Otherwise the call stages the results in device buffers and copies them
 *    back after the kernel.  The device buffers come from a memory pool
 *    private to the library that keeps its reservation between calls (the
 *    largest call's size, per device, until the process exits), so repeated
 *    calls do not remap device memory.
 * Results are the same either way.
 */
int ssa_ensemble_run_host(const ssa_model *model, int64_t n_traj, uint64_t traj_offset,
                          const int32_t *x0, double t_end, int n_samples, const double *sample_times,
                          int precision, int rounding, int normalise, uint64_t seed,
                          int64_t max_events, int state_bytes, uint32_t out_species, void *out,
                          uint32_t *traj_status, int64_t *n_events, double *t_final, void *stream);

/*
 * ssa_tau_run -- explicit tau-leaping with a fixed leap (the approximate
 * family of Table 1 and Sec. 2, run in the reduced-precision modes; Sec. 5
 * lists this interaction as untested and Sec. 6 as future work).  Leap n covers
 * [n tau, (n+1) tau), n = 0 .. ceil(t_end / tau) - 1; in each leap every
 * reaction j fires k_j ~ Poisson(a_j(x) tau) times at once and
 * x += sum_j nu_j k_j.
 *   a_j           the direct method's propensity arithmetic (same rounding
 *                 chain, same SR operation indices 0 .. S-1 per leap)
 *   lambda_j      a_j * tau in binary64 (SSA_FP64), binary32 (SSA_FP32 and
 *                 mixed modes), or in uniform modes rnd16(a_j * rnd16(tau))
 *                 with SR operation index S + j
 *   k_j           Poisson sampler in binary64 (SSA_FP64) or binary32:
 *                 multiplication method below lambda = 10, Hoermann's
 *                 transformed rejection (PTRS) from 10; its uniforms come from
 *                 Philox4x32-10 with counter (word / 4, n, trajectory id, 2 + j)
 *   counts        updated in 64-bit integers; a count that would go negative
 *                 is set to 0 and flagged SSA_TRAJ_TAU_CLAMPED; counts are
 *                 capped at 2^31 - 1
 * Arguments as ssa_ensemble_run, except:
 *   tau           leap length, finite, > 0, t_end / tau <= 2^31 - 1
 *   rounding      SSA_RN or SSA_SR (SSA_SR_ACCUM is rejected)
 *   sample_times  snapshot k holds the state after every leap that ends at
 *                 or before s_k (leaps end at (n+1) tau)
 *   n_events      device [n_traj] total reactions fired (sum of the k_j), or NULL
 *   t_final       device [n_traj] end time of the last completed leap, or NULL
 * A propensity that evaluates to +inf or NaN stops the trajectory at the
 * start of that leap with SSA_TRAJ_OVERFLOW or SSA_TRAJ_NAN.  The model may
 * use any structure (the general table-driven kernel serves every model).
 * Allocates an 8-byte work-queue counter as ssa_ensemble_run does.
 * Errors: SSA_EINVAL, SSA_ENOMEM, SSA_ECUDA.
 */
int ssa_tau_run(const ssa_model *model, int64_t n_traj, uint64_t traj_offset, const int32_t *x0,
                double t_end, double tau, int n_samples, const double *sample_times, int precision,
                int rounding, int normalise, uint64_t seed, int state_bytes, void *out,
                uint32_t *traj_status, int64_t *n_events, double *t_final, void *stream);

/*
 * ssa_rdme_run -- reaction-diffusion master equation on an nx x ny x nz
 * lattice of well-mixed voxels (the spatial setting of Sec. 1 and Sec. 5,
 * future work in Sec. 6; the paper gives no algorithm).  Every voxel runs the
 * model's reactions; species i hops to each existing neighbour (reflecting
 * boundaries) at rate diffusion[i] * x_vi.  One trajectory = one lattice,
 * simulated exactly by the direct method over all channels of all voxels:
 *   channels of voxel v  reactions 0..M-1 (the propensity chain of
 *                        ssa_ensemble_run on the voxel's counts), then for
 *                        each species with diffusion > 0 and each existing
 *                        neighbour direction (-x, +x, -y, +y, -z, +z) a hop
 *                        of value rnd(D_i * rnd(x_vi))
 *   selection            voxel totals (last partial sum, accumulator type) in
 *                        a binary sum tree; descent from the root with
 *                        r = u2 a0 (go right with r = r - left when left <= r
 *                        and right > 0), then the first channel of the voxel
 *                        whose partial sum exceeds r
 *   rounding             as ssa_ensemble_run; stochastic-rounding bits are
 *                        keyed by (voxel or tree node, epoch of its last
 *                        recomputation); SSA_SR_ACCUM is rejected
 * With one voxel the result equals ssa_ensemble_run's in the RN modes.
 *   nx, ny, nz    lattice extent, each >= 1; S = nx*ny*nz voxels (<= 1024,
 *                 and the per-lane state -- S*N counts, 2*T tree nodes with T
 *                 the smallest power of two >= S, S epochs in SR modes --
 *                 must fit in shared memory for 32 lanes)
 *   diffusion     host [N] hop rate per direction, finite, >= 0; constant
 *                 species must have 0 and the same count in every voxel
 *   x0            host [S][N] initial counts (>= 0), voxel-major
 *   max_events    events (reactions + hops) per trajectory, 0..2^32-2
 *   out           device [K][S][N][n_traj], trajectory index fastest
 *   other arguments as ssa_ensemble_run (n_events counts reactions and hops)
 * Allocates a work-queue counter and the [S][N] initial-state table with
 * stream-ordered allocation and frees them after the launch.
 * Errors: SSA_EINVAL (arguments; lattice too large), SSA_ENOMEM, SSA_ECUDA.
 */
int ssa_rdme_run(const ssa_model *model, int nx, int ny, int nz, const double *diffusion, int64_t n_traj,
                 uint64_t traj_offset, const int32_t *x0, double t_end, int n_samples,
                 const double *sample_times, int precision, int rounding, int normalise, uint64_t seed,
                 int64_t max_events, int state_bytes, void *out, uint32_t *traj_status, int64_t *n_events,
                 double *t_final, void *stream);

/*
 * ssa_set_launch_config -- launch shape for subsequent runs in this process.
 *   threads_per_block  multiple of 32 in 32..256
 *   blocks_per_sm      resident blocks per SM to launch (0 = as many as the
 *                      occupancy calculator allows)
 *   slice_pairs        pairs of steps each lane runs between two checks for
 *                      finished lanes to refill, 1..64
 * threads_per_block = 0 restores the library's defaults (the other arguments
 * are then ignored): for single-queue direct-method runs 32 step pairs per
 * check and, per kernel, 256 threads per block unless that keeps fewer than
 * 85% of the resident warps 128-thread blocks would (then 128); (128, 0, 16)
 * for tau-leaping, RDME and batches.  These were the fastest measured.  Once a shape is set, every kind of run uses it.  Tau-leaping and
 * RDME kernels take only the block size and check for refills after every
 * step.
 * Results never depend on the launch shape; only speed does.  Not
 * synchronised with concurrent launches from other threads.
 * Errors: SSA_EINVAL.
 */
int ssa_set_launch_config(int threads_per_block, int blocks_per_sm, int slice_pairs);

/*
 * ssa_set_tail_compaction -- tail compaction for subsequent direct-method
 * runs (ssa_ensemble_run, ssa_ensemble_run_host, ssa_sweep_run_noalloc):
 * 1 (the default) or 0.  Once the work queue has drained, a warp whose
 * unfinished trajectories fit into the idle lanes of the other warps of its
 * block hands them over (through shared memory) and stops, so the last
 * trajectories of a launch run on fewer, fuller warps.  A trajectory's state
 * moves whole, so results never depend on this; only speed does.  No paper
 * counterpart (the paper runs trajectories one after another on a CPU).
 * Errors: SSA_EINVAL.
 */
int ssa_set_tail_compaction(int enabled);

/*
 * ssa_set_tail_lock_limit -- bound on one wait for a block's hand-off lock in
 * subsequent direct-method launches: at most `spins` attempts (0, the
 * default, means 2^22 attempts, under a second).  A wait that runs out is
 * counted and decides nothing; small limits exist to exercise that path.
 * Results never depend on it: stranded trajectories are resumed at the end
 * of the block (below).  Errors: SSA_EINVAL (spins < 0).
 */
int ssa_set_tail_lock_limit(int spins);

/*
 * ssa_tail_stats -- synchronises the current device, then reports, for all
 * direct-method launches of this process on it so far, the trajectories moved
 * between warps by tail compaction (*moved), the hand-off lock waits that
 * gave up (*lock_timeouts; each wait is bounded) and the trajectories a
 * block resumed from its pool after all its warps had left (*resumed: a warp
 * whose lock wait gave up can leave while records wait for it; once every
 * warp is out, warp 0 runs whatever the pool still holds, so outputs stay
 * complete and identical).  Any pointer may be NULL.
 * Errors: SSA_ECUDA.
 */
int ssa_tail_stats(int64_t *moved, int64_t *lock_timeouts, int64_t *resumed);

/*
 * ssa_set_longest_first -- scheduling of subsequent ssa_ensemble_run and
 * ssa_ensemble_run_host calls.  A persistent launch ends when the trajectories
 * that started last are done, and a long one among them keeps the GPU
 * waiting on a few lanes.  Longest-first scheduling splits the run in two
 * launches of the same kernel: the first runs every trajectory up to
 * `park_events` events and parks those still unfinished (state, clock, next
 * snapshot, and a predicted remaining work a0(x) * (t_end - t)); three small
 * kernels sort the parked trajectories by that prediction; the second launch
 * resumes them, largest first, so the launch ends on short ones.
 *   mode         0 off; 1 automatic (the default: when a0(x0) * t_end >= 4096
 *                events and there are at least 2 trajectories per resident
 *                lane, 2 * SMs * 1024); 2 always
 *   park_events  the parking point: 0 (the default) for a0(x0) * t_end / 5
 *                (at least 256), else an even number >= 2; no split when it
 *                is >= the run's max_events
 * Random numbers are keyed by (trajectory id, event count) and a parked
 * trajectory resumes whole, so results never depend on this; only speed
 * does.  The split allocates its scratch (about 29 + 4 N bytes per
 * trajectory) with stream-ordered allocation and runs one plain launch if
 * that fails.  ssa_batch_create applies the setting in force when it is
 * called, per group, to that batch's launches: a group parks by the same
 * rule with its mean a0(x0) * t_end over its sets, and in automatic mode
 * also when that estimate differs by 4x or more between its sets (the
 * ordering uses each set's own rate constants), the batch's scratch is part of its device
 * tables, and ssa_batch_launch then runs launch 1, the ordering kernels of
 * every parking group and launch 2 (all captured in its graph); the
 * autotuner times plain launches.  ssa_sweep_run_noalloc never splits.  Not
 * synchronised with concurrent calls from other threads.  No paper
 * counterpart.
 * Errors: SSA_EINVAL (mode outside 0..2; park_events odd, or 1).
 */
int ssa_set_longest_first(int mode, int64_t park_events);

/*
 * ssa_direct_kernel_launches -- *count = kernels launched by
 * ssa_ensemble_run, ssa_ensemble_run_host and ssa_batch_launch in this
 * process so far: one per call, or with longest-first scheduling two
 * direct-method launches plus three ordering kernels (per parking group for
 * a batch).  Errors: SSA_EINVAL (count is NULL).
 */
int ssa_direct_kernel_launches(int64_t *count);

/*
 * Batched heterogeneous runs: several groups, each a model with a sweep of
 * parameter sets, simulated by ONE persistent kernel with one device work
 * queue per group.  Lanes that finish a trajectory take the next one from
 * their warp's current group; a warp moves to the next group once it has
 * drained the current one.  All groups share t_end, the sample times, the
 * precision, rounding, normalisation, seed, event cap and state storage.
 *
 * ssa_batch_group:
 *   model         the network (its structure; its rates are defaults)
 *   n_sets        parameter sets, >= 1
 *   traj_per_set  trajectories per set, >= 0; item r of the group belongs to
 *                 set r / traj_per_set and has global trajectory id
 *                 traj_offset + r (ids must fit in 32 bits)
 *   rates         host [n_sets][M] c-convention rates, or NULL (model's)
 *   hill          host [n_sets][M][2] {alpha0, alpha} for Hill rows, or NULL
 *   x0            host [n_sets][N] initial counts
 *   out           device [K][N][n_sets * traj_per_set]
 *   traj_status   device [n_sets * traj_per_set]
 *   n_events      device [n_sets * traj_per_set] or NULL
 *   t_final       device [n_sets * traj_per_set] or NULL
 * Results of every trajectory equal those of ssa_ensemble_run with the same
 * rates, x0 and global trajectory id.
 */
typedef struct {
    const ssa_model *model;
    int64_t n_sets;
    int64_t traj_per_set;
    const double *rates;
    const double *hill;
    const int32_t *x0;
    uint64_t traj_offset;
    void *out;
    uint32_t *traj_status;
    int64_t *n_events;
    double *t_final;
} ssa_batch_group;

typedef struct ssa_batch ssa_batch;   /* opaque, owned by the library */

/* Validate the groups, compute every set's c' in binary64, upload the
 * per-set tables to device memory owned by the batch (synchronous), and
 * decide per group whether its launches park and resume longest-first
 * (ssa_set_longest_first; the scratch, about 29 + 4 N bytes per trajectory
 * of a parking group, is part of the batch's device memory).
 * n_groups in 1..16.  Errors: SSA_EINVAL, SSA_ENOMEM, SSA_ECUDA. */
int ssa_batch_create(int n_groups, const ssa_batch_group *groups, double t_end, int n_samples,
                     const double *sample_times, int precision, int rounding, int normalise,
                     uint64_t seed, int64_t max_events, int state_bytes, ssa_batch **out);

/* Run the whole batch on `stream`.  On a non-NULL stream the queue reset and
 * the kernels (one launch, or launch 1, the ordering kernels and launch 2
 * when groups park) are captured once into a CUDA graph and replayed on
 * later calls; on the NULL stream they are launched directly.  Asynchronous. */
int ssa_batch_launch(ssa_batch *batch, void *stream);

/* Pick threads per block, resident blocks per SM and step pairs per refill
 * check by timing short runs of this batch (at most 2 lanes' worth of
 * trajectories per lane, events capped at 4096 per trajectory).  Writes
 * provisional results into the output buffers; launch again afterwards.
 * Synchronous.  Any of the out pointers may be NULL. */
int ssa_batch_autotune(ssa_batch *batch, void *stream, int *threads_per_block, int *blocks_per_sm,
                       int *slice_pairs, double *best_ms);

/* Release the batch and its device memory (NULL is allowed).  No launch of
 * it may still be running. */
void ssa_batch_destroy(ssa_batch *batch);

/*
 * ssa_sweep_run_noalloc -- a parameter sweep of one model that allocates no
 * memory (the paper has no counterpart; this is a deployment entry point).
 *
 * For callers that cannot allocate device memory while they simulate:
 * programs whose device memory belongs to another allocator or is held to a
 * fixed budget after start-up, and real-time or embedded loops that forbid
 * allocation on their hot path.  A successful call makes no cudaMalloc,
 * cudaFree or other allocating call, on the device or the host; the caller
 * passes the inputs and owns the outputs.  Two exceptions: the first call on
 * a device and the first call in each precision / rounding mode may load
 * code (lazy module loading, the symbol lookup below), which can allocate
 * device memory, so allocation-sensitive callers make one warm-up call in
 * every mode they use; and the error path formats its message into
 * heap-allocated host memory.  Its scratch (the work-queue counter and the
 * per-set tables) lives in one static device array of
 * SSA_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until
 * the process exits.
 *
 * Semantics equal n_sets calls of ssa_ensemble_run: trajectory r belongs to
 * set r / traj_per_set, uses rates[set] (host [n_sets][M] c-convention, or
 * NULL for the model's), hill[set] (host [n_sets][M][2] {alpha0, alpha}, or
 * NULL) and x0[set] (host [n_sets][N]), and has global id traj_offset + r.
 * Outputs: device [K][N][n_sets*traj_per_set], [n_sets*traj_per_set] ...
 * as in ssa_ensemble_run.
 *
 *  - Sweeps needing more than SSA_NOALLOC_SCRATCH_BYTES of scratch
 *    (ssa_sweep_noalloc_scratch_bytes) are rejected with SSA_EINVAL and a
 *    message; split them into smaller sweeps.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) for that device; make that first call before any
 *    stream capture.
 *  - The per-set tables are staged from a host buffer that lives only during
 *    the call, so a call on a stream that is capturing is refused with
 *    SSA_EINVAL.
 *  - n_sets above SSA_NOALLOC_SCRATCH_BYTES / 8, or n_sets * traj_per_set
 *    beyond int64, is rejected with SSA_EINVAL before any table is sized.
 *  - Every call shares the one array, which keeps the previous call's
 *    contents (the call resets what must start at zero).  Calls whose work
 *    overlaps on the GPU (other streams, other threads) race on it:
 *    serialise them.
 *  - Asynchronous on `stream`, except that the per-set tables are staged from
 *    pageable host memory before the call returns.
 */
enum { SSA_NOALLOC_SCRATCH_BYTES = 1 << 20 };

size_t ssa_sweep_noalloc_scratch_bytes(int n_species, int n_reactions, int64_t n_sets);

int ssa_sweep_run_noalloc(const ssa_model *model, int64_t n_sets, int64_t traj_per_set,
                          const double *rates, const double *hill, const int32_t *x0,
                          uint64_t traj_offset, double t_end, int n_samples, const double *sample_times,
                          int precision, int rounding, int normalise, uint64_t seed,
                          int64_t max_events, int state_bytes, void *out, uint32_t *traj_status,
                          int64_t *n_events, double *t_final, void *stream);

/*
 * Learned surrogate for the telegraph model (an extension beyond the paper; it
 * trains no network).  A multilayer perceptron maps 4 standardised
 * log-parameters (log kon, log koff, log km, log gamma) through three hidden
 * layers of 256 GELU units to a 128-bin softmax over the mRNA count (bins
 * 0..127, the last holding >= 127).  bf16 weights and activations, fp32
 * accumulation in tensor memory (tcgen05), fp32 master weights with AdamW,
 * cross-entropy against SSA histograms.  Parameter vector (fp32, host or
 * device as stated): W1 [256][16] (input columns 4..15 are padding, kept 0),
 * b1 [256], W2 [256][256], b2 [256], W3 [256][256], b3 [256], W4 [128][256],
 * b4 [128]; ssa_surrogate_param_count() values.
 */
typedef struct ssa_surrogate ssa_surrogate;

int64_t ssa_surrogate_param_count(void);

/* Allocate weights, optimiser state and activations for batches of up to
 * max_batch rows (1..2^20); He-normal initialisation from `seed`.
 * Synchronous.  Errors: SSA_EINVAL, SSA_ENOMEM, SSA_ECUDA. */
int ssa_surrogate_create(int max_batch, uint64_t seed, ssa_surrogate **out);
void ssa_surrogate_destroy(ssa_surrogate *s);

/* Replace / read the fp32 parameter vector (host [param_count]); setting
 * resets the optimiser state.  Synchronous. */
int ssa_surrogate_set_params(ssa_surrogate *s, const float *params);
int ssa_surrogate_get_params(ssa_surrogate *s, float *params);

/* probs (device [B][128]) = softmax(network(features)), features device
 * [B][4].  Asynchronous on stream. */
int ssa_surrogate_predict(ssa_surrogate *s, int B, const float *features, float *probs, void *stream);

/*
 * ssa_surrogate_train -- n_steps AdamW steps (as ssa_surrogate_train_step)
 * driven from the device: step 0 runs directly, the rest replay one captured
 * CUDA graph, with the step counters, learning rate and bias corrections kept
 * in device memory.  No paper counterpart (the surrogate is this project's).
 *   features, targets  device [n_rows][4] and [n_rows][128] (rows sum to 1)
 *   batch              rows per step, 1..max_batch; step k trains on rows
 *                      (k * batch + j) mod n_rows, j < batch -- shuffle the
 *                      rows beforehand for random minibatches
 *   lr_max, lr_min     cosine schedule: lr_k = lr_min + (lr_max - lr_min)
 *                      (1 + cos(pi k / (n_steps - 1))) / 2, in binary64,
 *                      rounded to binary32
 *   loss_every, loss_trace  device [ceil(n_steps / loss_every)]: the loss of
 *                      steps 0, loss_every, 2 loss_every, ...; or NULL
 *   stream             the caller's stream, or NULL (then a private stream
 *                      ordered after the legacy default stream)
 * Each step equals ssa_surrogate_train_step on that minibatch with that
 * learning rate.  Synchronous: returns once the run has finished.
 * Errors: SSA_EINVAL, SSA_ECUDA.
 */
int ssa_surrogate_train(ssa_surrogate *s, int64_t n_steps, int64_t n_rows, const float *features,
                        const float *targets, int batch, float lr_max, float lr_min, float weight_decay,
                        int64_t loss_every, float *loss_trace, void *stream);

/* One AdamW step (beta = 0.9, 0.999; eps = 1e-8; decoupled weight decay on
 * the weights) on the mean cross-entropy of the batch against targets
 * (device [B][128], rows summing to 1).  loss_out: device float or NULL.
 * Asynchronous on stream. */
int ssa_surrogate_train_step(ssa_surrogate *s, int B, const float *features, const float *targets, float lr,
                             float weight_decay, float *loss_out, void *stream);

/* Gradient of the mean cross-entropy (host [param_count]) and the loss
 * (host float or NULL) without updating anything.  Synchronous. */
int ssa_surrogate_gradients(ssa_surrogate *s, int B, const float *features, const float *targets,
                            float *grads, float *loss);

/* Optimiser state after synchronising: fp32 master parameters, AdamW first
 * and second moments and the gradient of the last step (host [param_count]
 * each, any may be NULL) and the number of AdamW steps taken (t of the bias
 * corrections 1 - beta^t; NULL allowed).  AdamW (Loshchilov & Hutter,
 * decoupled weight decay) is not in the paper; hyperparameters beta1 = 0.9f,
 * beta2 = 0.999f, eps = 1e-8f, decay on weights only.  Synchronous. */
int ssa_surrogate_get_state(ssa_surrogate *s, float *theta, float *m, float *v, float *grad,
                            int64_t *adam_steps);

/* Synchronise and report a tensor-core pipeline timeout (SSA_ETIMEDOUT) if a
 * GEMM's bounded wait gave up since creation. */
int ssa_surrogate_status(ssa_surrogate *s);

/* hist (device [n_sets][bins]) = normalised histogram of counts (device
 * [n_sets * traj_per_set], set-major), counts clamped to [0, bins-1]. */
int ssa_histogram(const int32_t *counts, int64_t n_sets, int64_t traj_per_set, int bins, float *hist,
                  void *stream);

/* w1 (device [rows]) = sum_b |CDF_p(b) - CDF_q(b)| for histograms p, q
 * (device [rows][bins]): the Wasserstein-1 distance on the integers. */
int ssa_hist_w1(const float *p, const float *q, int64_t rows, int bins, float *w1, void *stream);

/* Expected Wasserstein-1 distance between a law and the empirical histogram
 * of n_draws independent draws from it, per row of p (device [rows][bins],
 * rows summing to 1): sum over b < bins-1 of sqrt(2 F(b)(1 - F(b)) / (pi n)),
 * the normal approximation of E|F_n(b) - F(b)| (F the cumulative law).  The
 * surrogate's check uses it as the sampling noise of a small SSA ensemble.
 * No paper counterpart.  Asynchronous.  Errors: SSA_EINVAL, SSA_ECUDA. */
int ssa_hist_w1_noise(const float *p, int64_t rows, int bins, double n_draws, float *out, void *stream);

/*
 * On-device ensemble statistics (the comparisons of Sec. 4: two-sample
 * Kolmogorov-Smirnov statistic and Wasserstein-1 distance between the
 * ensembles of two precision modes; dwell times of the telegraph gene,
 * Sec. 4.3).  Integer-exact definitions:
 *
 * ssa_count_histogram -- hist[k] += #{values == k}, k = 0..bins-1 (device
 *   uint64 [bins], ACCUMULATED: zero it first); values below 0 or above
 *   bins-1 are counted in the end bins and added to *n_clamped (device).
 *   values: device int32 (elem_bytes 4) or int16 (2), n of them; 1 <= bins
 *   <= 2^24.  Asynchronous on stream.
 *
 * ssa_hist_ks_w1 -- out (device double [2]) = {D, W1} of the two samples
 *   whose histograms are ha, hb (device uint64 [bins]): with cumulative
 *   counts C_a, C_b and totals n_a, n_b, diff(k) = |C_a(k) n_b - C_b(k) n_a|
 *   (64-bit integers), D = max diff / (n_a n_b), W1 = sum diff / (n_a n_b),
 *   each the binary64 quotient of the two integers rounded to binary64.
 *   NaN when a sample is empty or bins * n_a * n_b >= 2^63.  Asynchronous.
 *
 * ssa_dwell_histogram -- hist[d] += the number of completed OFF intervals of
 *   d samples (device uint64 [K], ACCUMULATED) in the series
 *   s[k * k_stride + j] (k = 0..K-1, trajectory j = 0..n-1, k_stride >= n;
 *   device int32 or int16; nonzero = OFF): an interval starts at the first
 *   OFF sample after an ON sample and ends at the first ON sample after it.
 *   For snapshots [K][N][n] of species i: pass the address of element
 *   (0, i, 0) and k_stride = N * n.  Asynchronous.
 * Errors: SSA_EINVAL (arguments), SSA_ECUDA (launch).
 */
int ssa_count_histogram(const void *values, int elem_bytes, int64_t n, int bins, uint64_t *hist,
                        uint64_t *n_clamped, void *stream);
int ssa_hist_ks_w1(const uint64_t *ha, const uint64_t *hb, int bins, double *out, void *stream);
int ssa_dwell_histogram(const void *series, int elem_bytes, int K, int64_t n, int64_t k_stride, uint64_t *hist,
                        void *stream);

/*
 * ssa_round16 -- one 16-bit rounding of the engine applied to an array: the
 * rounding that ends every reduced-precision operation (paper Sec. 3.1
 * formats, Sec. 3.3 stochastic rounding: round up with probability
 * (x - x-)/(x+ - x-)).  The kernels' own device functions are used, so this
 * is the engine's rounding contract, checkable value by value.
 *
 * x: device [n] binary32 inputs.  format: 0 binary16, 1 bfloat16.
 * rounding: 0 round to nearest even (rbits unused, may be NULL), 1 SR.
 * rbits: device [n] random words; SR uses the low 16 bits (half = 0) or the
 * high 16 bits (half = 1) of each word, as operation slots 2i and 2i+1 of a
 * step do.  binary16 uses the low 13 of those 16 bits aligned with the most
 * significant discarded bit (13-bit resolution, also for subnormal results),
 * bfloat16 all 16; a magnitude rounded past the largest finite value becomes
 * infinity.  out: device [n] results widened to binary32 (exact).
 * Asynchronous on `stream`.  Errors: SSA_EINVAL, SSA_ECUDA.
 */
int ssa_round16(const float *x, const uint32_t *rbits, int64_t n, int format, int rounding, int half,
                float *out, void *stream);

/* Tensor-core GEMM check: D (device [M][N] fp32) = A (device [M][K] bf16,
 * row-major) times B (device [N][K] bf16, row-major) transposed.
 * N in 16..256 and a multiple of 16; K a multiple of 16 (of 256 above 256).
 * Synchronous; SSA_ETIMEDOUT if a bounded wait gave up. */
int ssa_mlp_gemm_bf16(int M, int N, int K, const uint16_t *A, const uint16_t *B, float *D, void *stream);

/*
 * Stage checks of the surrogate's training step (no paper counterpart): the
 * fused kernels of ssa_surrogate_train_step on caller inputs, so each can be
 * compared element by element with a CPU reference.  Synchronous; device
 * pointers; row-major.
 *
 * ssa_mlp_gemm_epi: acc = A (bf16 [M][K]) times B (bf16 [N][K]) transposed,
 * fp32 accumulation in tensor memory, then epilogue
 *   0  fout = acc                                   (weight gradients)
 *   1  fout = z = acc + bias;  hout = bf16(gelu(z)) (hidden layer forward)
 *   2  fout = acc + bias                            (logits)
 *   3  d = acc * gelu'(zin) (zin fp32 [M][N]); hout = bf16(d);
 *      bias_grad[n] += sum over rows of d (fp32 atomics)  (hidden backward)
 * gelu(z) = z Phi(z) (exact form, Phi the normal CDF).  Sizes as
 * ssa_mlp_gemm_bf16.  Errors: SSA_EINVAL, SSA_ENOMEM, SSA_ECUDA,
 * SSA_ETIMEDOUT (a bounded wait gave up).
 *
 * ssa_mlp_softmax_xent: per row of logits (fp32 [B][128]): without targets,
 * probs = softmax; with targets (fp32 [B][128], rows summing to 1),
 * dz = bf16((softmax - targets) / B) (bf16 [B][128]), bias_grad[k] += sum of
 * the unrounded (softmax - targets) / B over rows, *loss += mean
 * cross-entropy (caller zeroes the accumulators).  Errors: SSA_EINVAL,
 * SSA_ENOMEM, SSA_ECUDA.
 */
int ssa_mlp_gemm_epi(int epi, int M, int N, int K, const uint16_t *A, const uint16_t *B, const float *bias,
                     const float *zin, float *fout, uint16_t *hout, float *bias_grad, void *stream);
int ssa_mlp_softmax_xent(int B, const float *logits, const float *targets, float *probs, uint16_t *dz,
                         float *bias_grad, float *loss, void *stream);

/*
 * ssa_mlp_set_wait_test -- failure detection of the tensor-core GEMM (no
 * paper counterpart).  Every wait of the GEMM (operands landed, MMAs done) is
 * bounded; when one runs out, the kernel records an error word, lets its own
 * copies and MMAs in flight land (bounded), frees its tensor memory and
 * returns, and the caller sees SSA_ETIMEDOUT (ssa_mlp_gemm_bf16,
 * ssa_surrogate_status).  This setting makes that happen on purpose for all
 * later GEMMs of the process: withhold 1 issues no operand loads, withhold 2
 * no MMAs, so that wait never completes; spin_limit is the number of polls
 * per wait (0: 2^22).  (0, 0) restores normal operation.  Not synchronised
 * with launches from other threads.  Errors: SSA_EINVAL.
 */
int ssa_mlp_set_wait_test(int withhold, int spin_limit);

/* Thread-local description of the last error on the calling thread. */
const char *ssa_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SSA_H */
