// internal.h -- declarations shared by the library's translation units.
// Not part of the public ABI (include/proxmf.h is).
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace proxmf {

constexpr int kMaxLabels = 32;
constexpr int kMaxServeSlots = 256;   // requests in flight in one server

// Grid tile of the step kernel: GX x GY pixels, one thread per pixel.
constexpr int GX = 32;
constexpr int GY = 8;
constexpr int GT = GX * GY;

// Labels stored per pixel in HBM: L rounded up to a multiple of 4 (2 when
// L <= 2), so that one pixel is a whole number of 16-byte vectors.
// Padding labels hold log q = kPadLogQ (q = 0) and U = 0.
__host__ __device__ constexpr int storage_labels(int L) { return L <= 2 ? 2 : (L + 3) / 4 * 4; }
constexpr float kPadLogQ = -1e30f;

// Label count a step kernel is compiled for, given the runtime L: the exact
// count for the segmentation workload's 21, else the storage count (the
// kernel then masks labels >= L).
inline int kernel_labels(int L) { return L == 21 ? 21 : storage_labels(L); }

// Pairs of mu used by the step kernel for a kernel label count LT:
// NPP = pair slots per row (ceil(LT/2) rounded up to even);
// out[k*NPP + j] = (mu[2j][k], mu[2j+1][k]), in[k*NPP + j] = (mu[k][2j], mu[k][2j+1]),
// zero outside the L x L matrix.
inline int mu_pair_slots(int LT) { return ((LT + 1) / 2 + 1) / 2 * 2; }

// Tensor-core form of the grid step: the L x L product runs as BF16 MMAs
// with K = N = tc_k(LT) labels.  Operands use the no-swizzle K-major layout:
// 8 x 8 BF16 core matrices of 128 contiguous bytes, K-adjacent core matrices
// 128 bytes apart (leading byte offset), 8-row groups tc_sbo bytes apart
// (stride byte offset).  Element (r, k) of an operand sits at byte
// (r / 8) * tc_sbo + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
__host__ __device__ constexpr int tc_k(int LT) { return LT <= 16 ? 16 : 32; }
__host__ __device__ constexpr int tc_sbo(int KP) { return KP / 8 * 128; }
constexpr int kTcImageBytes = 2 * 32 * 32 * 2;   // mu and mu^T images at the largest tc_k

// Everything one launch of the grid step needs.  State and unaries are
// pixel-major [B][N][storage_labels(L)], N = H*W, pixel p = y*W + x; edge
// weights are [B][N][n_dirs] with zero on edges that leave the image.
// The whole iteration loop of a small grid instance in one launch, one
// thread-block cluster per instance with the iterates in shared memory
// (grid_resident.cu).
constexpr size_t kResidentMaxSmem = 200 * 1024;
constexpr int kResidentCtas = 8;   // CTAs per instance (one cluster), rows split among them
struct GridResidentLaunch {
    const float *s_in;       // [B][N][LP] log q^0 (padding kPadLogQ)
    float *s_out;            // [B][N][LP] log q after the loop (may equal s_in)
    const float *U;          // [B][N][LP]
    const float *w;          // [B][N][n_dirs] pixel-major edge weights
    const float *mu;         // [L][L] device
    const float *eta;        // [B]
    double *f_trace;         // [B][trace_cap]: F(q^t) of each step
    double *f_cur;           // [B]: F of the last iterate read
    int *done;               // [B]: step count at which the stopping rule held
    int *status;
    int B, H, W, L, LP, conn, mu_sym, nsteps, trace_cap;
    double rel_tol;
};
size_t grid_resident_smem(int H, int W, int L, int LP);
bool grid_resident_fits(int H, int W, int L, int LP);
cudaError_t launch_grid_resident(const GridResidentLaunch &a, cudaStream_t st);

struct GridStepLaunch {
    const float *s_in;       // log q^t
    float *s_out;            // log q^{t+1}
    const float *U;          // unary costs
    const float *w;          // edge weights
    const float *eta;        // [B] step per instance
    const float2 *mu_out;    // device [LT][NPP] column pairs (see mu_pair_slots)
    const float2 *mu_in;     // device [LT][NPP] row pairs
    const float2 *mu_host;   // host copy of the column pairs (first LT * mu_pair_slots(LT)); required
                             // for symmetric mu with LT <= 21 (copied into the launch parameters)
    const uint4 *mu_tc;      // tensor-core form: device BF16 operand images of mu, mu^T
    const __nv_bfloat16 *U16;  // tensor-core form: unaries in BF16, [B][N][u16_pitch(LP)] (may be null)
    bool tc;                 // BF16 tensor-core messages (else FP32)
    const float *adapt_d;    // [B] adaptive binary step: eta_i = 1/(1 + d q_i0 q_i1); null = fixed eta;
                             // for rule 2 (Adam): d0 per instance
    int rule;                // 0 fixed / adaptive, 1 momentum (Sec. 3.4), 2 Adam (Sec. 3.5),
                             // 3 ADHOC mean-parameter damping (Sec. 2.2.2); FP32 form only
    float *mom, *vv;         // [B][N][LP] momentum average and second moment (rules 1, 2)
    float gamma1, gamma2, eps;
    int rule_first;          // 1 on the first step of a run (no history)
    double *partial;         // [2][B][nblk][kMaxFParts] free-energy partials (scratch; slot t & 1 when deferred)
    unsigned int *counter;   // [B] tiles finished in this launch (scratch, self-resetting)
    double *f_trace;         // [B][trace_cap]
    double *f_cur;           // [B] F of the state read by this launch
    int *done;               // [B] 0 = running, k = stopped after k steps (may be null)
    int *status;             // device error word
    int B, L, H, W, conn;
    int t, trace_cap, update;
    double rel_tol;
    bool mu_sym;
    // Deferred free energy (step loops of mf_iterate): with defer = n > 0
    // each tile stores n partials of step t (one per warp of the two-pixel
    // kernel, else one) in slot t & 1 of partial and takes no ticket;
    // prev_pending = n > 0 makes this launch first sum the n partials per
    // tile of step t - 1 (trace entry, stopping rule).  0: none.
    int defer, prev_pending;
};

// Opt-in of one kernel to more than 48 KB of dynamic shared memory.  The
// attribute belongs to the device that is current when it is set, so each
// call site keeps one bit per device (devices 0..63; others set it on every
// launch) and sets it the first time it launches on that device.
struct SmemOptIn {
    std::atomic<unsigned long long> devices{0ull};
};
template <typename Kernel>
inline cudaError_t smem_optin(SmemOptIn &o, Kernel k, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;
    if (bit != 0ull && (o.devices.load(std::memory_order_acquire) & bit) != 0ull) return cudaSuccess;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && bit != 0ull) o.devices.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// Number of tiles per instance.
inline void grid_tiles(int H, int W, int *nbx, int *nby) {
    *nbx = (W + GX - 1) / GX;
    *nby = (H + GY - 1) / GY;
}

// Per-label-bucket launchers (one translation unit each).
// Column / row pairs of mu for a kernel label count LT (api.cu).
void build_mu_pairs_host(const float *mu, int L, int LT, float2 *out);

// Step-size bound for serving: eta = 1/(1 + D max|nu|), D the largest weighted
// degree, nu the eigenvalues of C mu C (symmetric mu).
cudaError_t launch_eta_bound(const float *w, int H, int W, int nd, const float *mu, int L, float *eta,
                             double *scratch, cudaStream_t st);

// Per-label-count launchers (grid_step_l*.cu), dispatched by launch_grid_step.
cudaError_t launch_grid_step_l2(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l4(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l8(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l12(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l16(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l20(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l21(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l24(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l28(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step_l32(const GridStepLaunch &a, cudaStream_t st);
cudaError_t launch_grid_step(const GridStepLaunch &a, cudaStream_t st);

// True when launch_grid_step runs one of the TMA-staged grid kernels for l
// (grid_tma.cuh, grid_tma_tc.cuh): those alone take the deferred free energy.
inline bool grid_step_uses_tma(const GridStepLaunch &l) {
    return l.L > 2 && l.rule == 0 && l.adapt_d == nullptr && (!l.tc || (l.mu_sym && l.U16 != nullptr));
}
// Free-energy partials per tile of a deferring launch: one per warp of the
// two-pixel FP32 kernel (symmetric mu), one for the other TMA kernels.
constexpr int kMaxFParts = 4;
inline int grid_step_fparts(const GridStepLaunch &l) {
    return grid_step_uses_tma(l) ? ((!l.tc && l.mu_sym) ? kMaxFParts : 1) : 0;
}

// The deferred free energy of step t (the last step of a loop, or of a run
// of deferring steps): trace entry, F_cur and the stopping rule, one block per
// instance (grid_f_deferred.cu).
cudaError_t launch_grid_f_flush(const GridStepLaunch &l, int t, int parts, cudaStream_t st);

// Layout conversion and initialisation (layout.cu).
// rows [B][N][L] <-> padded [B][N][LP]; pad fills the padding labels.
enum ConvMode { CONV_COPY = 0, CONV_EXP = 1 };
cudaError_t launch_rows_to_padded(const float *src, float *dst, long long rows, int L, int LP, float pad,
                                  cudaStream_t st);
cudaError_t launch_padded_to_rows(const float *src, float *dst, long long rows, int L, int LP, int mode,
                                  cudaStream_t st);
// [B][nd][H][W] -> [B][H*W][nd], zeroing entries whose edge leaves the image.
cudaError_t launch_weights_to_pixel_major(const float *src, float *dst, int B, int nd, int H, int W,
                                          cudaStream_t st);
// s = log softmax(-U) per variable (padded layout; padding labels get kPadLogQ).
cudaError_t launch_init_logq(const float *U, float *s, long long rows, int L, int LP, cudaStream_t st);
// eta[b] = value for all b.
cudaError_t launch_fill_eta(float *eta, int B, double value, cudaStream_t st);
// BF16 unaries of the tensor-core grid step: LP labels padded to a multiple
// of 8 (whole 16-byte rows for the TMA).
__host__ __device__ constexpr int u16_pitch(int LP) { return (LP + 7) / 8 * 8; }
// dst[r][0..pitch) = src[r][0..LP) rounded to BF16 (nearest even), zero past LP.
cudaError_t launch_to_bf16(const float *src, __nv_bfloat16 *dst, long long rows, int LP, int pitch,
                           cudaStream_t st);
// d[b] = max(Lambda[b], 0) (FP32)
cudaError_t launch_lambda_to_d(const double *Lambda, float *d, int B, cudaStream_t st);

// Fully connected Gaussian model (dense.cu, dense_tc.cu).
struct DenseStepLaunch {
    const float *K32;            // [B][N][N] FP32 weights (FP32 form)
    const __nv_bfloat16 *K16;    // [B][N][N] BF16 weights (tensor-core form)
    const float *q_in;           // [B][N][LP] q of the state read
    const __nv_bfloat16 *qt_in;  // [B][32][N] BF16 q, label-major (tensor-core form)
    const float *s_in;           // [B][N][LP]
    const float *U;              // [B][N][LP]
    float *s_out;                // [B][N][LP]
    float *q_out;                // [B][N][LP]
    __nv_bfloat16 *qt_out;       // [B][32][N] or null
    const float *eta;            // [B]
    const float *mu;             // [L][L] device
    const float *featsT;         // tensor-core form computing K in the kernel: [B][nchunk][6][64]
                                 // (launch_dense_fly_features), else null (K16 is read)
    double *partial;             // [B][dense_nblk(N)]; deferred: two slots of [B][dense_tc_tiles(N)]
    unsigned *counter;           // [B]
    double *f_trace, *f_cur;
    int *done, *status;
    int B, N, L;
    int t, trace_cap, update;
    double rel_tol;
    // Deferred free energy of the tensor-core step in a loop (as for the
    // grid step): defer = 1 stores the row tile's partial in slot t & 1 and
    // takes no ticket; prev_pending = 1 sums step t - 1's partials first.
    int defer, prev_pending;
};
// The pending free energy of tensor-core step t (dense_tc.cu).
cudaError_t launch_dense_f_flush(const DenseStepLaunch &l, int t, cudaStream_t st);
// Prescaled features of the on-the-fly tensor-core form, per chunk of 64
// columns: sqrt(2) s f_k (k = 0..4; s = sqrt(log2 e / (2 theta^2)) of the
// position or colour group) and -|s f|^2; columns past N get 0 and -1e30.
cudaError_t launch_dense_fly_features(const float *feats, float *featsT, int B, int N, double theta_pos,
                                      double theta_rgb, cudaStream_t st);
int dense_nblk(int N);
int dense_tc_tiles(int N);
int dense_tc_pitch(int N);   // row pitch (elements) of the BF16 K and q^T copies
// K32 [B][N][N] and/or K16 [B][N][pitch] (padding columns zero)
cudaError_t launch_dense_kernel_build(const float *feats, float *K32, __nv_bfloat16 *K16, int B, int N,
                                      double theta_pos, double theta_rgb, cudaStream_t st);
// q = exp(s): FP32 [B][N][LP] and/or BF16 label-major [B][32][pitch]
cudaError_t launch_dense_export_q(const float *s, float *q32, __nv_bfloat16 *qt16, int B, int N, int L, int LP,
                                  cudaStream_t st);
cudaError_t launch_dense_step_f32(const DenseStepLaunch &a, cudaStream_t st);
struct DenseTcBuffers {
    float *split_part;       // [B][tiles][2][128][32] split-K partial sums
    unsigned *tile_count;    // [B][tiles] (zero, self-resetting)
};
cudaError_t launch_dense_step_tc(const DenseStepLaunch &a, const DenseTcBuffers &tb, cudaStream_t st);

// Extreme eigenvalues of C mu C into nu[0] (min), nu[1] (max) (lanczos.cu).
cudaError_t launch_mu_tilde_extremes(const float *mu_dev, int L, double *nu, cudaStream_t st);

// Step-size constant (lanczos.cu).  Fills Lambda[b] (device, FP64) and
// eta[b] = 1/(1+max(Lambda,0)) (device, FP32).  Returns CRF status codes.
struct LipschitzJob {
    const float *w;          // pixel-major weights [B][N][n_dirs]
    const float *Kdense;     // dense model: FP32 weights [B][N][N] (then H = 1, W = N)
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


// General pairwise graphs (sparse.cu): CSR adjacency, one warp per variable.
struct SparseStepLaunch {
    const float *s_in;       // [B][N][LP] log q^t
    float *s_out;            // [B][N][LP] log q^{t+1}
    const float *q_in;       // [B][N][LP] q^t
    float *q_out;            // [B][N][LP] q^{t+1}
    const float *U;          // [B][N][LP]
    const int *out_ptr, *out_col;   // adjacency: symmetric mu -> both directions of every edge
    const float *out_w;
    const int *in_ptr, *in_col;     // asymmetric mu: edges entering each variable
    const float *in_w;
    const float *mu;         // [L][L] device
    const float *eta;        // [B]
    double *partial;         // [B][nblk]
    unsigned *counter;       // [B]
    double *f_trace, *f_cur;
    int *done, *status;
    int B, N, L, LP, nblk;
    int t, trace_cap, update;
    double rel_tol;
    bool sym;
};
int sparse_blocks(int N);
cudaError_t launch_sparse_step(const SparseStepLaunch &a, cudaStream_t st);
cudaError_t launch_sparse_degree(const int *ptr, const float *w, int N, unsigned *out_bits, cudaStream_t st);

// Reverse mode through unrolled grid steps (adjoint.cu).  All arrays are in
// the padded pixel-major layout of the step kernel; L <= 24.
constexpr int kAdjointMaxLabels = 24;
struct AdjointStep {
    const float *gs_in;      // [B][N][LP] d loss / d s^{t+1} (padding 0)
    float *gs_out;           // [B][N][LP] d loss / d s^t (padding written 0)
    float *dU;               // [B][N][LP] accumulated
    float *dw;               // [B][N][n_dirs] accumulated
    float *dmu_part;         // [adjoint_blocks][L][L] accumulated per-block partials
    const float *s;          // s^t
    const float *s_next;     // s^{t+1}
    const float *w;          // [B][N][n_dirs]
    const float *mu;         // [L][L] device
    const float *eta;        // [B]
    int *status;             // device error word (bounded waits)
    int B, L, H, W, conn;
    bool mu_sym;
};
struct AdjointFinish {
    const float *gs;         // d/ds^0
    const float *s0;         // s^0 = log softmax(-U)
    float *dU;               // accumulated, padded layout
    const float *dw;         // pixel-major accumulated
    float *dw_out;           // [B][n_dirs][H][W]
    const float *dmu_part;
    float *dmu_out;          // [L][L]
    int B, L, H, W, conn;
};
// Blocks of one reverse-step launch (32 x 4 pixel tiles per instance).
int adjoint_blocks(int B, int H, int W);
cudaError_t launch_adjoint_step(const AdjointStep &a, cudaStream_t st);
cudaError_t launch_adjoint_finish(const AdjointFinish &a, cudaStream_t st);

}  // namespace proxmf
