// Instantiations of the grid step for kernel label count 21 (see grid_step.cuh).
#include "grid_step.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l21(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<21>(a, st);
}

}  // namespace proxmf
