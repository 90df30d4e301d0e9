// Kernel instantiations for the Schloegl structure family (with and without
// the reservoir species folded into the rate constants).
#include "ssa_launch.h"
#include "ssa_models.h"

namespace ssa {

cudaError_t launch_schlogl(const RunArgs &a, int prec, int sr, int norm, LaunchConfig cfg, cudaStream_t s, int *grid)
{
    if (norm) return launch_family<StaticModel<models::Schlogl, true>>(a, prec, sr, cfg, s, grid);
    return launch_family<StaticModel<models::Schlogl, false>>(a, prec, sr, cfg, s, grid);
}

}  // namespace ssa
