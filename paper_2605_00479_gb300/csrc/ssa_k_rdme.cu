// RDME launch dispatch and the general-model instantiations.
#include "ssa_launch.h"
#include "rdme_device.cuh"

namespace ssa {

constexpr size_t kRdmeSmemPerBlock = 227 * 1024;   // opt-in dynamic shared memory per block on sm_103a

cudaError_t launch_rdme_schlogl(const RdmeArgs &, int, int, int, int, int, size_t, cudaStream_t, int *, int *);
cudaError_t launch_rdme_small(const RdmeArgs &, int, int, int, int, int, size_t, cudaStream_t, int *, int *);
cudaError_t launch_rdme_repressilator(const RdmeArgs &, int, int, int, int, size_t, cudaStream_t, int *, int *);

int rdme_block_size(const RdmeArgs &A, int elem_bytes, bool epochs, int max_block)
{
    return rdme_block_size_for(A, elem_bytes, epochs, max_block, kRdmeSmemPerBlock);
}

cudaError_t launch_rdme(const RdmeArgs &A, int family, int norm, int prec, int sr, LaunchConfig cfg,
                        cudaStream_t stream, int *grid_out, int *block_out)
{
    const int mb = cfg.block, bps = cfg.blocks_per_sm;
    const size_t lim = kRdmeSmemPerBlock;
    switch (family) {
    case 2: return launch_rdme_schlogl(A, norm, prec, sr, mb, bps, lim, stream, grid_out, block_out);
    case 1:
    case 3:
    case 4: return launch_rdme_small(A, family, prec, sr, mb, bps, lim, stream, grid_out, block_out);
    case 5: return launch_rdme_repressilator(A, prec, sr, mb, bps, lim, stream, grid_out, block_out);
    default: return rdme_launch_model<GeneralModel>(A, prec, sr, mb, bps, lim, stream, grid_out, block_out);
    }
}

}  // namespace ssa
