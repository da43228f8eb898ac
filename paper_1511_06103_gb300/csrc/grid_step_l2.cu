// Instantiations of the grid step for kernel label count 2 (see grid_step.cuh).
#include "grid_step.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l2(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<2>(a, st);
}

}  // namespace proxmf
