// Batched-kernel instantiations: uniform bfloat16.
#include "ssa_launch.h"

namespace ssa {

cudaError_t launch_batch_uniform_bf16(const BatchArgs &b, int64_t work, int prec, int sr, bool compact, LaunchConfig cfg,
                               cudaStream_t s, int *grid)
{
    if (prec == UNIFORM_BF16 && sr == 0) return launch_batch_mode<UNIFORM_BF16, 0>(b, work, compact, cfg, s, grid);
    if (prec == UNIFORM_BF16 && sr == 1) return launch_batch_mode<UNIFORM_BF16, 1>(b, work, compact, cfg, s, grid);
    if (prec == UNIFORM_BF16 && sr == 2) return launch_batch_mode<UNIFORM_BF16, 2>(b, work, compact, cfg, s, grid);
    return cudaErrorInvalidValue;
}

}  // namespace ssa

namespace ssa {

cudaError_t launch_batch_f64_f32(const BatchArgs &, int64_t, int, int, bool, LaunchConfig, cudaStream_t, int *);
cudaError_t launch_batch_mixed_f16(const BatchArgs &, int64_t, int, int, bool, LaunchConfig, cudaStream_t, int *);
cudaError_t launch_batch_mixed_bf16(const BatchArgs &, int64_t, int, int, bool, LaunchConfig, cudaStream_t, int *);
cudaError_t launch_batch_uniform_f16(const BatchArgs &, int64_t, int, int, bool, LaunchConfig, cudaStream_t, int *);

cudaError_t launch_batch(const BatchArgs &b, int64_t work, int prec, int sr, bool compact, LaunchConfig cfg,
                         cudaStream_t s, int *grid)
{
    switch (prec) {
    case FP64:
    case FP32: return launch_batch_f64_f32(b, work, prec, sr, compact, cfg, s, grid);
    case MIXED_F16: return launch_batch_mixed_f16(b, work, prec, sr, compact, cfg, s, grid);
    case MIXED_BF16: return launch_batch_mixed_bf16(b, work, prec, sr, compact, cfg, s, grid);
    case UNIFORM_F16: return launch_batch_uniform_f16(b, work, prec, sr, compact, cfg, s, grid);
    default: return launch_batch_uniform_bf16(b, work, prec, sr, compact, cfg, s, grid);
    }
}

}  // namespace ssa
