// RDME instantiations for the Schloegl structure (reservoirs folded or not).
#include "rdme_device.cuh"
#include "ssa_models.h"

namespace ssa {

cudaError_t launch_rdme_schlogl(const RdmeArgs &A, int norm, int prec, int sr, int max_block, int bps,
                                size_t smem_limit, cudaStream_t s, int *grid, int *block)
{
    if (norm)
        return rdme_launch_model<StaticModel<models::Schlogl, true>>(A, prec, sr, max_block, bps, smem_limit, s,
                                                                      grid, block);
    return rdme_launch_model<StaticModel<models::Schlogl, false>>(A, prec, sr, max_block, bps, smem_limit, s, grid,
                                                                   block);
}

}  // namespace ssa
