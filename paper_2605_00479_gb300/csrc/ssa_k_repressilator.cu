// Kernel instantiations for the repressilator structure family.
#include "ssa_launch.h"
#include "ssa_models.h"

namespace ssa {

cudaError_t launch_repressilator(const RunArgs &a, int prec, int sr, int norm, LaunchConfig cfg, cudaStream_t s, int *grid)
{
    (void)norm;  // no constant species: folding never applies
    return launch_family<StaticModel<models::Repressilator, false>>(a, prec, sr, cfg, s, grid);
}

}  // namespace ssa
