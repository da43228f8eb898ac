// grid_f_deferred.cu -- the free energy of the last deferring grid step.
//
// In a step loop the TMA-staged grid kernels store one F partial per tile and
// leave the sum to the next step (grid_step_prologue), which takes it while
// its own tile loads are in flight.  After the last such step this kernel
// takes it: the fixed-order sum of the tile partials, the trace entry, F_cur
// and the stopping rule, exactly as the next step would have.
#include "grid_step.cuh"

namespace proxmf {

__global__ void __launch_bounds__(128) grid_f_flush_kernel(const __grid_constant__ GridStepArgs a) {
    __shared__ double red[4];
    const int b = blockIdx.x;
    if (a.done != nullptr && a.done[b] != 0) return;   // the step copied a stopped instance: no partials
    deferred_f<128>(a, b, a.t, a.prev_pending, true, red);
}

cudaError_t launch_grid_f_flush(const GridStepLaunch &l, int t, int parts, cudaStream_t st) {
    if (parts < 1 || parts > kMaxFParts) return cudaErrorInvalidValue;
    GridStepArgs a{};
    int nbx, nby;
    grid_tiles(l.H, l.W, &nbx, &nby);
    a.nbx = nbx;
    a.nblk = nbx * nby;
    a.pslot = (size_t)l.B * a.nblk * kMaxFParts;
    a.prev_pending = parts;
    a.partial = l.partial;
    a.f_trace = l.f_trace;
    a.f_cur = l.f_cur;
    a.done = l.done;
    a.status = l.status;
    a.t = t;
    a.trace_cap = l.trace_cap;
    a.update = 1;
    a.rel_tol = l.rel_tol;
    grid_f_flush_kernel<<<l.B, 128, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace proxmf
