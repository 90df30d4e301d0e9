// Tau-leaping instantiations for the repressilator structure.
#include "ssa_models.h"
#include "tau_device.cuh"
#include "tau_launch.h"

namespace ssa {

cudaError_t launch_tau_repressilator(const RunArgs &a, int prec, int sr, LaunchConfig cfg, cudaStream_t stream,
                                     int *grid_out)
{
    return tau_launch_model<StaticModel<models::Repressilator, false>>(a, prec, sr, cfg.block, cfg.blocks_per_sm,
                                                                        stream, grid_out);
}

}  // namespace ssa
