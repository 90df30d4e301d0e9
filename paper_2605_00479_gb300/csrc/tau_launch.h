// tau_launch.h -- launchers of the tau-leaping kernels, one per compiled
// structure family (ssa_k_tau*.cu) plus the runtime-table general model.
#pragma once

#include "ssa_launch.h"

namespace ssa {

// Picks the kernel of the model's structure family (0 = general; norm selects
// the folded Schloegl variant) and launches it; writes the grid it used.
cudaError_t launch_tau_family(const RunArgs &a, int family, int norm, int prec, int sr, LaunchConfig cfg,
                              cudaStream_t stream, int *grid_out);

cudaError_t launch_tau_schlogl(const RunArgs &a, int norm, int prec, int sr, LaunchConfig cfg, cudaStream_t stream,
                               int *grid_out);
cudaError_t launch_tau_small(const RunArgs &a, int family, int prec, int sr, LaunchConfig cfg, cudaStream_t stream,
                             int *grid_out);
cudaError_t launch_tau_repressilator(const RunArgs &a, int prec, int sr, LaunchConfig cfg, cudaStream_t stream,
                                     int *grid_out);

}  // namespace ssa
