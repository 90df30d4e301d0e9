// Batched-kernel instantiations: fp64 and fp32.
#include "ssa_launch.h"

namespace ssa {

cudaError_t launch_batch_f64_f32(const BatchArgs &b, int64_t work, int prec, int sr, bool compact, LaunchConfig cfg,
                               cudaStream_t s, int *grid)
{
    if (prec == FP64 && sr == 0) return launch_batch_mode<FP64, 0>(b, work, compact, cfg, s, grid);
    if (prec == FP32 && sr == 0) return launch_batch_mode<FP32, 0>(b, work, compact, cfg, s, grid);
    return cudaErrorInvalidValue;
}

}  // namespace ssa
