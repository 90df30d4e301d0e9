// Kernel instantiations for the general structure family.
#include "ssa_launch.h"
#include "ssa_models.h"

namespace ssa {

cudaError_t launch_general(const RunArgs &a, int prec, int sr, int norm, LaunchConfig cfg, cudaStream_t s, int *grid)
{
    (void)norm;  // the folding table travels in the kernel arguments
    return launch_family<GeneralModel>(a, prec, sr, cfg, s, grid);
}

}  // namespace ssa
