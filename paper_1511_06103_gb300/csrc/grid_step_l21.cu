// Instantiations of the grid step and the serving step for kernel label count 21 (see grid_step.cuh).
#include "grid_step.cuh"
#include "serve.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l21(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<21>(a, st);
}

cudaError_t launch_serve_l21(int conn, bool sym, ServeSlot *slots, const ServeBucket *bucket, ServeResult *res,
                            int grid, cudaStream_t st) {
    return launch_serve_lt<21>(conn, sym, slots, bucket, res, grid, st);
}

}  // namespace proxmf
