// Tau-leaping instantiations for the Schloegl structure (reservoirs folded or not).
#include "ssa_models.h"
#include "tau_device.cuh"
#include "tau_launch.h"

namespace ssa {

cudaError_t launch_tau_schlogl(const RunArgs &a, int norm, int prec, int sr, LaunchConfig cfg, cudaStream_t stream,
                               int *grid_out)
{
    if (norm)
        return tau_launch_model<StaticModel<models::Schlogl, true>>(a, prec, sr, cfg.block, cfg.blocks_per_sm, stream,
                                                                     grid_out);
    return tau_launch_model<StaticModel<models::Schlogl, false>>(a, prec, sr, cfg.block, cfg.blocks_per_sm, stream,
                                                                  grid_out);
}

}  // namespace ssa
