// RDME instantiations for the birth-death, telegraph and dimerisation structures.
#include "rdme_device.cuh"
#include "ssa_models.h"

namespace ssa {

cudaError_t launch_rdme_small(const RdmeArgs &A, int family, int prec, int sr, int max_block, int bps,
                              size_t smem_limit, cudaStream_t s, int *grid, int *block)
{
    switch (family) {
    case 1:
        return rdme_launch_model<StaticModel<models::BirthDeath, false>>(A, prec, sr, max_block, bps, smem_limit,
                                                                          s, grid, block);
    case 3:
        return rdme_launch_model<StaticModel<models::Telegraph, false>>(A, prec, sr, max_block, bps, smem_limit, s,
                                                                         grid, block);
    default:
        return rdme_launch_model<StaticModel<models::Dimer, false>>(A, prec, sr, max_block, bps, smem_limit, s,
                                                                     grid, block);
    }
}

}  // namespace ssa
