// Batched-kernel instantiations: uniform binary16.
#include "ssa_launch.h"

namespace ssa {

cudaError_t launch_batch_uniform_f16(const BatchArgs &b, int64_t work, int prec, int sr, bool compact, LaunchConfig cfg,
                               cudaStream_t s, int *grid)
{
    if (prec == UNIFORM_F16 && sr == 0) return launch_batch_mode<UNIFORM_F16, 0>(b, work, compact, cfg, s, grid);
    if (prec == UNIFORM_F16 && sr == 1) return launch_batch_mode<UNIFORM_F16, 1>(b, work, compact, cfg, s, grid);
    if (prec == UNIFORM_F16 && sr == 2) return launch_batch_mode<UNIFORM_F16, 2>(b, work, compact, cfg, s, grid);
    return cudaErrorInvalidValue;
}

}  // namespace ssa
