// internal.h -- declarations shared by the library's translation units.
// Not part of the public ABI (include/proxmf.h is).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace proxmf {

constexpr int kMaxLabels = 32;

// Grid tile of the step kernel: GX x GY pixels, one thread per pixel.
constexpr int GX = 32;
constexpr int GY = 8;
constexpr int GT = GX * GY;

// Everything one launch of the grid step needs, in a layout-agnostic form.
// State, unaries and weights are label-planar: element (b, l, y, x) lives at
// ((b * L + l) * H + y) * P + x (weights: (b * n_dirs + k) instead of l).
struct GridStepLaunch {
    const float *s_in;       // log q^t
    float *s_out;            // log q^{t+1}
    const float *U;          // unary costs
    const float *w;          // edge weights, zero on edges that leave the image
    const float *eta;        // [B] step per instance
    double *partial;         // [B][nblk] per-tile free-energy partials (scratch)
    unsigned int *counter;   // [B] tiles finished in this launch (scratch, self-resetting)
    double *f_trace;         // [B][trace_cap]
    double *f_cur;           // [B] F of the state read by this launch
    int *done;               // [B] 0 = running, k = stopped after k steps (may be null)
    int *status;             // device error word
    int B, L, H, W, P, conn;
    int t, trace_cap, update;
    double rel_tol;
    bool mu_sym;
    const float *mu_host;    // [L][L] row-major host copy
};

// Number of tiles per instance.
inline void grid_tiles(int H, int W, int *nbx, int *nby) {
    *nbx = (W + GX - 1) / GX;
    *nby = (H + GY - 1) / GY;
}

// Per-label-bucket launchers (one translation unit each).
cudaError_t launch_grid_step_l2(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l4(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l8(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l16(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l21(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l32(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step(const GridStepLaunch &a, cudaStream_t st);

// Layout conversion and initialisation (layout.cu).
// rows [B][N][L] <-> planar [B][L][H][P]; mode selects the element transform.
enum ConvMode { CONV_COPY = 0, CONV_EXP = 1 };
cudaError_t launch_rows_to_planar(const float *src, float *dst, int B, int L, int H, int W, int P,
                                  cudaStream_t st);
cudaError_t launch_planar_to_rows(const float *src, float *dst, int B, int L, int H, int W, int P,
                                  int mode, cudaStream_t st);
// [B][nd][H][W] -> [B][nd][H][P], zeroing entries whose edge leaves the image.
cudaError_t launch_weights_to_planar(const float *src, float *dst, int B, int nd, int H, int W,
                                     int P, cudaStream_t st);
// s = log softmax(-U) per variable (planar).
cudaError_t launch_init_logq(const float *U, float *s, int B, int L, int H, int W, int P,
                             cudaStream_t st);
// eta[b] = value for all b.
cudaError_t launch_fill_eta(float *eta, int B, double value, cudaStream_t st);

// Step-size constant (lanczos.cu).  Fills Lambda[b] (device, FP64) and
// eta[b] = 1/(1+max(Lambda,0)) (device, FP32).  Returns CRF status codes.
struct LipschitzJob {
    const float *w;          // planar weights
    const float *mu_host;    // [L][L]
    bool mu_sym;
    int B, L, H, W, P, conn;
    double *Lambda;          // [B] device
    float *eta;              // [B] device
    int max_steps;
    double tol;
};
int estimate_lipschitz_grid(const LipschitzJob &job, cudaStream_t st, int *steps_out,
                            long long *launches_out);

}  // namespace proxmf
