// Instantiations of the grid step and the serving step for kernel label count 2 (see grid_step.cuh).
#include "grid_step.cuh"
#include "serve.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l2(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<2>(a, st);
}

cudaError_t launch_serve_l2(int conn, bool sym, ServeSlot *slots, const ServeBucket *bucket, ServeResult *res,
                            int grid, cudaStream_t st) {
    return launch_serve_lt<2>(conn, sym, slots, bucket, res, grid, st);
}

}  // namespace proxmf
