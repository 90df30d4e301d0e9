// Tau-leaping instantiations for the birth-death, telegraph and dimerisation structures.
#include "ssa_models.h"
#include "tau_device.cuh"
#include "tau_launch.h"

namespace ssa {

cudaError_t launch_tau_small(const RunArgs &a, int family, int prec, int sr, LaunchConfig cfg, cudaStream_t stream,
                             int *grid_out)
{
    switch (family) {
    case 1:
        return tau_launch_model<StaticModel<models::BirthDeath, false>>(a, prec, sr, cfg.block, cfg.blocks_per_sm,
                                                                         stream, grid_out);
    case 3:
        return tau_launch_model<StaticModel<models::Telegraph, false>>(a, prec, sr, cfg.block, cfg.blocks_per_sm,
                                                                        stream, grid_out);
    default:
        return tau_launch_model<StaticModel<models::Dimer, false>>(a, prec, sr, cfg.block, cfg.blocks_per_sm, stream,
                                                                    grid_out);
    }
}

}  // namespace ssa
