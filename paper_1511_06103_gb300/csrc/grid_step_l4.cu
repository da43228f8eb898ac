// Instantiations of the grid step for kernel label count 4 (see grid_step.cuh).
#include "grid_step.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l4(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<4>(a, st);
}

}  // namespace proxmf
