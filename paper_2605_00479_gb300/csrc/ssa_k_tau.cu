// Tau-leaping: the general-model instantiations and the family dispatch.
#include "tau_device.cuh"
#include "tau_launch.h"

namespace ssa {

cudaError_t launch_tau(const RunArgs &a, int prec, int sr, LaunchConfig cfg, cudaStream_t stream, int *grid_out)
{
    return tau_launch_model<GeneralModel>(a, prec, sr, cfg.block, cfg.blocks_per_sm, stream, grid_out);
}

cudaError_t launch_tau_family(const RunArgs &a, int family, int norm, int prec, int sr, LaunchConfig cfg,
                              cudaStream_t stream, int *grid_out)
{
    switch (family) {
    case 2: return launch_tau_schlogl(a, norm, prec, sr, cfg, stream, grid_out);
    case 1:
    case 3:
    case 4: return launch_tau_small(a, family, prec, sr, cfg, stream, grid_out);
    case 5: return launch_tau_repressilator(a, prec, sr, cfg, stream, grid_out);
    default: return launch_tau(a, prec, sr, cfg, stream, grid_out);
    }
}

}  // namespace ssa
