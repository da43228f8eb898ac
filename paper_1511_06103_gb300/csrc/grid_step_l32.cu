// Instantiations of the grid step and the serving step for kernel label count 32 (see grid_step.cuh).
#include "grid_step.cuh"
#include "serve.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l32(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<32>(a, st);
}

cudaError_t launch_serve_l32(int conn, bool sym, ServeSlot *slots, const ServeBucket *bucket, ServeResult *res,
                            int grid, cudaStream_t st) {
    return launch_serve_lt<32>(conn, sym, slots, bucket, res, grid, st);
}

}  // namespace proxmf
