// serve.cuh -- device side of the serving loop: one persistent launch per
// label class per iteration advances every in-flight grid CRF of that class.
//
// The host keeps a table of slots in device memory (one admitted request
// each) and, per class ("bucket": kernel label count, connectivity, symmetry
// of mu), the list of its slots with the prefix sums of their tile counts.
// A launch walks all tiles of the bucket with a grid-stride loop, runs the
// same tile step as a single-instance solve (grid_tile), and the last tile of
// a slot finishes that slot's free energy in a fixed order, advances its
// iteration count and retires it when the stopping rule holds -- so a
// request's result does not depend on which other requests share the GPU.
// Results are published to host-mapped memory.
#pragma once

#include "grid_step.cuh"

namespace proxmf {

struct ServeSlot {
    const float *U;          // [N][LP]
    float *s[2];             // [N][LP] ping-pong log q
    const float *w;          // [N][nd]
    const float2 *mu_out, *mu_in;
    double *partial;         // [nblk]
    unsigned *counter;       // [1]
    const float *eta;        // [1] device
    int L, H, W, nbx, nblk;
    int max_iters;
    double rel_tol;
    // device-maintained
    int it;                  // steps taken (state parity)
    int active;              // 1 while running
    double F_prev;
};

struct ServeResult {         // host-mapped
    int done;                // 1 once retired
    int iters;
    double F;                // F of the state before the last step
};

struct ServeBucket {
    int count;               // slots in this bucket
    int slots[kMaxServeSlots];
    int prefix[kMaxServeSlots + 1];   // tile offsets
};

template <int LT, int CONN, bool SYM>
__global__ void __launch_bounds__(GT, (LT >= 24) ? 1 : 2)
serve_step_kernel(ServeSlot *slots, const ServeBucket *bucket, ServeResult *results) {
    __shared__ int sh_slot, sh_local, sh_last;
    __shared__ double red[GT / 32];
    const int tid = threadIdx.y * GX + threadIdx.x;
    const int count = bucket->count;
    const int total = bucket->prefix[count];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        if (tid == 0) {
            int k = 0;
            while (k + 1 < count && bucket->prefix[k + 1] <= t) ++k;
            sh_slot = bucket->slots[k];
            sh_local = t - bucket->prefix[k];
        }
        __syncthreads();
        const int si = sh_slot, local = sh_local;
        ServeSlot &sl = slots[si];
        const int active = *(volatile int *)&sl.active;
        const int it = *(volatile int *)&sl.it;
        if (!active) {
            __syncthreads();
            continue;
        }
        TileJob j;
        j.s_in = sl.s[it & 1];
        j.s_out = sl.s[(it + 1) & 1];
        j.U = sl.U;
        j.w = sl.w;
        j.mu_out = sl.mu_out;
        j.mu_in = sl.mu_in;
        j.mu_p = sl.mu_out;   // the serving step reads the column pairs from global memory
        j.eta = *sl.eta;
        j.adaptive = false;
        j.adapt_d = 0.f;
        j.L = sl.L;
        j.H = sl.H;
        j.W = sl.W;
        j.update = 1;
        const double bs = grid_tile<LT, CONN, SYM>(j, local % sl.nbx, local / sl.nbx);
        if (tid == 0) {
            sl.partial[local] = bs;
            __threadfence();
            sh_last = atomicAdd(sl.counter, 1u) == (unsigned)(sl.nblk - 1);
        }
        __syncthreads();
        if (sh_last) {
            __threadfence();
            double acc = 0.0;
            for (int k = tid; k < sl.nblk; k += GT) acc += __ldcg(sl.partial + k);
            acc = warp_sum_f64(acc);
            if ((tid & 31) == 0) red[tid >> 5] = acc;
            __syncthreads();
            if (tid == 0) {
                double F = 0.0;
#pragma unroll
                for (int k = 0; k < GT / 32; ++k) F += red[k];
                *sl.counter = 0u;
                const int nit = it + 1;
                bool stop = nit >= sl.max_iters || !isfinite(F);
                if (sl.rel_tol > 0.0 && it > 0 && fabs(F - sl.F_prev) <= sl.rel_tol * fabs(F)) stop = true;
                sl.F_prev = F;
                sl.it = nit;
                if (stop) {
                    sl.active = 0;
                    ServeResult *r = results + si;
                    r->F = F;
                    r->iters = nit;
                    __threadfence_system();
                    *(volatile int *)&r->done = 1;
                    __threadfence_system();
                }
                __threadfence();
            }
        }
        __syncthreads();
    }
}

template <int LT>
cudaError_t launch_serve_lt(int conn, bool sym, ServeSlot *slots, const ServeBucket *bucket, ServeResult *res,
                            int grid, cudaStream_t st) {
    dim3 block(GX, GY, 1);
    if (conn == 8) {
        if (sym)
            serve_step_kernel<LT, 8, true><<<grid, block, 0, st>>>(slots, bucket, res);
        else
            serve_step_kernel<LT, 8, false><<<grid, block, 0, st>>>(slots, bucket, res);
    } else {
        if (sym)
            serve_step_kernel<LT, 4, true><<<grid, block, 0, st>>>(slots, bucket, res);
        else
            serve_step_kernel<LT, 4, false><<<grid, block, 0, st>>>(slots, bucket, res);
    }
    return cudaGetLastError();
}

}  // namespace proxmf
