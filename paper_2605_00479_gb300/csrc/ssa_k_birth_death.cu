// Kernel instantiations for the birth-death structure family.
#include "ssa_launch.h"
#include "ssa_models.h"

namespace ssa {

cudaError_t launch_birth_death(const RunArgs &a, int prec, int sr, int norm, LaunchConfig cfg, cudaStream_t s, int *grid)
{
    (void)norm;  // no constant species: folding never applies
    return launch_family<StaticModel<models::BirthDeath, false>>(a, prec, sr, cfg, s, grid);
}

}  // namespace ssa
