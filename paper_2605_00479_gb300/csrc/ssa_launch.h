// ssa_launch.h -- per-family kernel launchers (one translation unit each, so
// the kernel instantiations compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include "ssa_device.cuh"

namespace ssa {

struct LaunchConfig {
    int block;          // threads per block (multiple of 32, <= 256); 0: chosen per kernel
    int blocks_per_sm;  // 0: as many as occupancy allows
    int slice_pairs;    // step pairs between refill checks
};

// Launch the persistent kernel of one family for precision `prec`, rounding
// `sr` (0 RN, 1 SR) and `norm` (fold constant species).  Writes the grid size
// used to *grid_out.  Returns the CUDA error of the launch.
using Launcher = cudaError_t (*)(const RunArgs &a, int prec, int sr, int norm, LaunchConfig cfg,
                                 cudaStream_t stream, int *grid_out);

cudaError_t launch_general(const RunArgs &, int, int, int, LaunchConfig, cudaStream_t, int *);
cudaError_t launch_birth_death(const RunArgs &, int, int, int, LaunchConfig, cudaStream_t, int *);
cudaError_t launch_schlogl(const RunArgs &, int, int, int, LaunchConfig, cudaStream_t, int *);
cudaError_t launch_telegraph(const RunArgs &, int, int, int, LaunchConfig, cudaStream_t, int *);
cudaError_t launch_dimer(const RunArgs &, int, int, int, LaunchConfig, cudaStream_t, int *);
cudaError_t launch_repressilator(const RunArgs &, int, int, int, LaunchConfig, cudaStream_t, int *);

// Longest-first scheduling (ssa_order.cu): order the parked items by
// descending predicted remaining work into order[0 .. *count-1].  hist
// [kOrderBuckets] and offs [kOrderBuckets] are scratch.  Adds the kernels it
// launched to *launches.
constexpr int kOrderBuckets = 1024;
struct OrderModel {
    int N, M;
    int8_t order[kMaxM][kMaxN];
    int8_t folded[kMaxM][kMaxN];
    int8_t law[kMaxM];
    int8_t hill_h[kMaxM];
    int8_t hill_reg[kMaxM];
    float c[kMaxM];              // c'_j (mass action), binary32 (one parameter set)
    float h0[kMaxM], h1[kMaxM];  // Hill alpha0, alpha (one parameter set)
    int n_sets;                  // > 1: item i uses set i / traj_per_set from the tables below
    int64_t traj_per_set;
    const double *cprime_tab;    // [n_sets][M]
    const double *hill_tab;      // [n_sets][M][2] or null
    double t_end;
    const int32_t *x;            // parked state [N][n]
    const double *t;             // parked clock [n]
    const uint8_t *parked;       // [n] nonzero: parked
};
struct LongestFirstScratch {
    unsigned long long *head2;   // work-queue counter of launch 2
    unsigned long long *count;   // parked trajectories
    unsigned long long *offs;    // [kOrderBuckets]
    unsigned *hist;              // [kOrderBuckets]
    double *t;                   // [n] parked records (RunArgs::park_*)
    int32_t *k;
    uint32_t *status;
    int32_t *x;                  // [N][n]
    uint8_t *parked;             // [n]
    int64_t *order;              // [n]
};
cudaError_t launch_order(const OrderModel &m, int64_t n, unsigned *hist, unsigned long long *offs,
                         unsigned long long *count, int64_t *order, cudaStream_t stream, int *launches);

// Tau-leaping kernel (ssa_k_tau.cu): precision `prec`, rounding `sr` (0 RN,
// 1 SR), leap a.tau, a.n_leaps leaps.
cudaError_t launch_tau(const RunArgs &a, int prec, int sr, LaunchConfig cfg, cudaStream_t stream, int *grid_out);

// RDME kernels (ssa_k_rdme*.cu).  rdme_block_size: threads per block, the
// largest multiple of 32 (at most max_block) whose lattice columns fit in
// shared memory, 0 if not even one warp fits.  launch_rdme picks the compiled
// structure `family` (0 = general; norm selects the folded Schloegl variant)
// and writes the grid and block it used.
struct RdmeArgs;
int rdme_block_size(const RdmeArgs &A, int elem_bytes, bool epochs, int max_block);
cudaError_t launch_rdme(const RdmeArgs &A, int family, int norm, int prec, int sr, LaunchConfig cfg,
                        cudaStream_t stream, int *grid_out, int *block_out);

// Shared launch logic: choose the kernel for (prec, sr), size the grid from
// occupancy (persistent: enough lanes to fill the GPU, no more than the work).
template <class ModelF>
cudaError_t launch_family(const RunArgs &a, int prec, int sr, LaunchConfig cfg, cudaStream_t stream, int *grid_out)
{
    using K = void (*)(const RunArgs);
    K k = nullptr;
    switch (prec) {
    case FP64: k = ssa_kernel<ModelF, FP64, 0>; break;
    case FP32: k = ssa_kernel<ModelF, FP32, 0>; break;
    case MIXED_F16: k = sr ? ssa_kernel<ModelF, MIXED_F16, 1> : ssa_kernel<ModelF, MIXED_F16, 0>; break;
    case MIXED_BF16: k = sr ? ssa_kernel<ModelF, MIXED_BF16, 1> : ssa_kernel<ModelF, MIXED_BF16, 0>; break;
    case UNIFORM_F16:
        k = sr == 2 ? ssa_kernel<ModelF, UNIFORM_F16, 2>
                    : (sr ? ssa_kernel<ModelF, UNIFORM_F16, 1> : ssa_kernel<ModelF, UNIFORM_F16, 0>);
        break;
    case UNIFORM_BF16:
        k = sr == 2 ? ssa_kernel<ModelF, UNIFORM_BF16, 2>
                    : (sr ? ssa_kernel<ModelF, UNIFORM_BF16, 1> : ssa_kernel<ModelF, UNIFORM_BF16, 0>);
        break;
    default: return cudaErrorInvalidValue;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int block = cfg.block;
    if (block == 0) {
        // 256 threads (eight warps per block pack better under tail compaction)
        // unless they keep fewer than 85% of the warps 128-thread blocks would
        int p256 = 0, p128 = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p256, k, 256, 0);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p128, k, 128, 0);
        if (e != cudaSuccess) return e;
        block = (p256 * 8 * 100 >= p128 * 4 * 85) ? 256 : 128;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (cfg.blocks_per_sm > 0 && cfg.blocks_per_sm < per_sm) per_sm = cfg.blocks_per_sm;
    long long grid = (long long)sms * per_sm;
    const long long need = (a.n_work + block - 1) / block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    *grid_out = (int)grid;
    k<<<(unsigned)grid, (unsigned)block, 0, stream>>>(a);
    return cudaGetLastError();
}

// Batched launch over heterogeneous groups (ssa_k_batch_*.cu).  `work` is the
// total number of items over all groups (caps the grid).  `compact` selects
// the instantiation holding only the telegraph, dimer and repressilator
// structures (fewer registers, higher occupancy) instead of every family.
cudaError_t launch_batch(const BatchArgs &b, int64_t work, int prec, int sr, bool compact, LaunchConfig cfg,
                         cudaStream_t stream, int *grid_out);

template <int PREC, int SR>
cudaError_t launch_batch_mode(const BatchArgs &b, int64_t work, bool compact, LaunchConfig cfg, cudaStream_t stream,
                              int *grid_out)
{
    auto k = compact ? ssa_batch_kernel<PREC, SR, 3, 4, 5> : ssa_batch_kernel<PREC, SR, 1, 2, 3, 4, 5, 0>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, cfg.block, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (cfg.blocks_per_sm > 0 && cfg.blocks_per_sm < per_sm) per_sm = cfg.blocks_per_sm;
    long long grid = (long long)sms * per_sm;
    const long long need = (work + cfg.block - 1) / cfg.block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    *grid_out = (int)grid;
    k<<<(unsigned)grid, (unsigned)cfg.block, 0, stream>>>(b);
    return cudaGetLastError();
}

}  // namespace ssa
