// Instantiations of the grid step for kernel label count 12 (see grid_step.cuh).
#include "grid_step.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l12(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<12>(a, st);
}

}  // namespace proxmf
