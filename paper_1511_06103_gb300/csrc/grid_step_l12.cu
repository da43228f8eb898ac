// Instantiations of the grid step and the serving step for kernel label count 12 (see grid_step.cuh).
#include "grid_step.cuh"
#include "serve.cuh"

namespace proxmf {

cudaError_t launch_grid_step_l12(const GridStepLaunch &a, cudaStream_t st) {
    return launch_grid_step_lt<12>(a, st);
}

cudaError_t launch_serve_l12(int conn, bool sym, ServeSlot *slots, const ServeBucket *bucket, ServeResult *res,
                            int grid, cudaStream_t st) {
    return launch_serve_lt<12>(conn, sym, slots, bucket, res, grid, st);
}

}  // namespace proxmf
