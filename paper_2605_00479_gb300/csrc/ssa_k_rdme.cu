// Kernel instantiations of the RDME engine and its launch-shape choice.
#include "ssa_launch.h"
#include "rdme_device.cuh"

namespace ssa {

namespace {

constexpr size_t kSmemPerBlock = 227 * 1024;   // opt-in dynamic shared memory per block on sm_103a

template <int PREC, int SR>
cudaError_t launch_mode(const RdmeArgs &A, LaunchConfig cfg, cudaStream_t stream, int *grid_out, int *block_out)
{
    using P = typename ModeTraits<PREC>::P;
    constexpr bool kEpochs = ModeTraits<PREC>::k16 && SR != 0;
    auto k = rdme_kernel<PREC, SR>;
    int block = rdme_block_size(A, (int)sizeof(P), kEpochs, cfg.block);
    if (block < 32) return cudaErrorInvalidConfiguration;
    const size_t bytes = rdme_layout(A.a.K, A.S, A.T, A.a.N, block, (int)sizeof(P), kEpochs).total;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (cfg.blocks_per_sm > 0 && cfg.blocks_per_sm < per_sm) per_sm = cfg.blocks_per_sm;
    long long grid = (long long)sms * per_sm;
    const long long need = (A.a.n_work + block - 1) / block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    *grid_out = (int)grid;
    *block_out = block;
    k<<<(unsigned)grid, (unsigned)block, bytes, stream>>>(A);
    return cudaGetLastError();
}

}  // namespace

int rdme_block_size(const RdmeArgs &A, int elem_bytes, bool epochs, int max_block)
{
    const size_t fixed = rdme_layout(A.a.K, A.S, A.T, A.a.N, 0, elem_bytes, epochs).total + 64;
    const size_t per_lane = (size_t)A.S * A.a.N * 4 + (size_t)2 * A.T * elem_bytes + (epochs ? (size_t)A.S * 4 : 0);
    if (fixed >= kSmemPerBlock) return 0;
    long long lanes = (long long)((kSmemPerBlock - fixed) / per_lane);
    long long block = (lanes / 32) * 32;
    if (block > max_block) block = max_block;
    // the interleaved columns need 16-byte alignment slack per region
    while (block >= 32 && rdme_layout(A.a.K, A.S, A.T, A.a.N, (int)block, elem_bytes, epochs).total > kSmemPerBlock)
        block -= 32;
    return (int)block;
}

cudaError_t launch_rdme(const RdmeArgs &A, int prec, int sr, LaunchConfig cfg, cudaStream_t stream, int *grid_out,
                        int *block_out)
{
    switch (prec) {
    case FP64: return launch_mode<FP64, 0>(A, cfg, stream, grid_out, block_out);
    case FP32: return launch_mode<FP32, 0>(A, cfg, stream, grid_out, block_out);
    case MIXED_F16:
        return sr ? launch_mode<MIXED_F16, 1>(A, cfg, stream, grid_out, block_out)
                  : launch_mode<MIXED_F16, 0>(A, cfg, stream, grid_out, block_out);
    case MIXED_BF16:
        return sr ? launch_mode<MIXED_BF16, 1>(A, cfg, stream, grid_out, block_out)
                  : launch_mode<MIXED_BF16, 0>(A, cfg, stream, grid_out, block_out);
    case UNIFORM_F16:
        return sr ? launch_mode<UNIFORM_F16, 1>(A, cfg, stream, grid_out, block_out)
                  : launch_mode<UNIFORM_F16, 0>(A, cfg, stream, grid_out, block_out);
    case UNIFORM_BF16:
        return sr ? launch_mode<UNIFORM_BF16, 1>(A, cfg, stream, grid_out, block_out)
                  : launch_mode<UNIFORM_BF16, 0>(A, cfg, stream, grid_out, block_out);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ssa
