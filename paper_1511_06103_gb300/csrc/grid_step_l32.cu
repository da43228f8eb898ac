// Instantiations of the grid step for kernel label count 32 (see grid_step.cuh).
#include "grid_step.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l32(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<32>(a, st);
}

}  // namespace proxmf
