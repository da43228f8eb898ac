// Instantiations of the grid step and the serving step for kernel label count 28 (see grid_step.cuh).
#include "grid_step.cuh"
#include "serve.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l28(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<28>(a, st);
}

cudaError_t launch_serve_l28(int conn, bool sym, ServeSlot *slots, const ServeBucket *bucket, ServeResult *res,
                            int grid, cudaStream_t st) {
    return launch_serve_lt<28>(conn, sym, slots, bucket, res, grid, st);
}

}  // namespace proxmf
