// Instantiations of the grid step for kernel label count 28 (see grid_step.cuh).
#include "grid_step.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l28(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<28>(a, st);
}

}  // namespace proxmf
