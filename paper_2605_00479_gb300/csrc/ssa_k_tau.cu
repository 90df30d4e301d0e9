// Kernel instantiations of the tau-leaping engine (general model tables).
#include "ssa_launch.h"
#include "tau_device.cuh"

namespace ssa {

cudaError_t launch_tau(const RunArgs &a, int prec, int sr, LaunchConfig cfg, cudaStream_t stream, int *grid_out)
{
    using K = void (*)(const RunArgs);
    K k = nullptr;
    switch (prec) {
    case FP64: k = tau_kernel<FP64, 0>; break;
    case FP32: k = tau_kernel<FP32, 0>; break;
    case MIXED_F16: k = sr ? tau_kernel<MIXED_F16, 1> : tau_kernel<MIXED_F16, 0>; break;
    case MIXED_BF16: k = sr ? tau_kernel<MIXED_BF16, 1> : tau_kernel<MIXED_BF16, 0>; break;
    case UNIFORM_F16: k = sr ? tau_kernel<UNIFORM_F16, 1> : tau_kernel<UNIFORM_F16, 0>; break;
    case UNIFORM_BF16: k = sr ? tau_kernel<UNIFORM_BF16, 1> : tau_kernel<UNIFORM_BF16, 0>; break;
    default: return cudaErrorInvalidValue;
    }
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
    const long long need = (a.n_work + cfg.block - 1) / cfg.block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    *grid_out = (int)grid;
    k<<<(unsigned)grid, (unsigned)cfg.block, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace ssa
