// Instantiations of the grid step for kernel label count 8 (see grid_step.cuh).
#include "grid_step.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l8(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<8>(a, st);
}

}  // namespace proxmf
