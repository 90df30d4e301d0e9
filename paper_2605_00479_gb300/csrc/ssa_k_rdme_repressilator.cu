// RDME instantiations for the repressilator structure.
#include "rdme_device.cuh"
#include "ssa_models.h"

namespace ssa {

cudaError_t launch_rdme_repressilator(const RdmeArgs &A, int prec, int sr, int max_block, int bps, size_t smem_limit,
                                      cudaStream_t s, int *grid, int *block)
{
    return rdme_launch_model<StaticModel<models::Repressilator, false>>(A, prec, sr, max_block, bps, smem_limit, s,
                                                                         grid, block);
}

}  // namespace ssa
