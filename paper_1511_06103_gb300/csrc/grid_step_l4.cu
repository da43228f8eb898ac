// Instantiations of the grid step and the serving step for kernel label count 4 (see grid_step.cuh).
#include "grid_step.cuh"
#include "serve.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l4(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<4>(a, st);
}

cudaError_t launch_serve_l4(int conn, bool sym, ServeSlot *slots, const ServeBucket *bucket, ServeResult *res,
                            int grid, cudaStream_t st) {
    return launch_serve_lt<4>(conn, sym, slots, bucket, res, grid, st);
}

}  // namespace proxmf
