// layout.cu -- conversions between the external [B][N][L] row layout and the
// internal padded pixel-major [B][N][LP] layout, the initial state q^0, and
// small fills.  None of this runs inside the iteration loop.
#include <cmath>

#include "internal.h"

namespace proxmf {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(size_t n) {
    size_t b = (n + kThreads - 1) / kThreads;
    return (int)(b > 0x7fffffff ? 0x7fffffff : (b == 0 ? 1 : b));
}

// rows [R][L] -> padded rows [R][LP]; one thread per output element.
__global__ void rows_to_padded_kernel(const float *__restrict__ src, float *__restrict__ dst, long long rows,
                                      int L, int LP, float pad) {
    const long long n = rows * LP;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / LP;
        const int l = (int)(i - r * LP);
        dst[i] = l < L ? src[r * L + l] : pad;
    }
}

__global__ void padded_to_rows_kernel(const float *__restrict__ src, float *__restrict__ dst, long long rows,
                                      int L, int LP, int mode) {
    const long long n = rows * L;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / L;
        const int l = (int)(i - r * L);
        const float v = src[r * LP + l];
        dst[i] = mode == CONV_EXP ? expf(v) : v;
    }
}

// Direction k of the grid: 0 right, 1 down, 2 down-right, 3 down-left.
__device__ __forceinline__ void dir_offset(int k, int *dy, int *dx) {
    *dy = k == 0 ? 0 : 1;
    *dx = k == 0 ? 1 : (k == 1 ? 0 : (k == 2 ? 1 : -1));
}

// [B][nd][H][W] -> [B][H*W][nd], zero where the edge would leave the image.
__global__ void weights_to_pixel_major_kernel(const float *__restrict__ src, float *__restrict__ dst, int B,
                                              int nd, int H, int W) {
    const long long n = (long long)B * H * W * nd;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % nd);
        const long long bp = i / nd;
        const long long pix = bp % ((long long)H * W);
        const long long b = bp / ((long long)H * W);
        const int y = (int)(pix / W), x = (int)(pix % W);
        int dy, dx;
        dir_offset(k, &dy, &dx);
        const int yy = y + dy, xx = x + dx;
        float v = 0.f;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = src[((b * nd + k) * H + y) * (long long)W + x];
        dst[i] = v;
    }
}

// q^0 = softmax(-U): unary-only marginals, written as log q (padded rows).
__global__ void init_logq_kernel(const float *__restrict__ U, float *__restrict__ s, long long rows, int L,
                                 int LP) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        const float *u = U + r * LP;
        float *o = s + r * LP;
        float mx = -INFINITY;
        for (int l = 0; l < L; ++l) mx = fmaxf(mx, -u[l]);
        float z = 0.f;
        for (int l = 0; l < L; ++l) z += expf(-u[l] - mx);
        const float lse = mx + logf(z);
        for (int l = 0; l < L; ++l) o[l] = -u[l] - lse;
        for (int l = L; l < LP; ++l) o[l] = kPadLogQ;
    }
}

__global__ void lambda_to_d_kernel(const double *Lambda, float *d, int B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B) d[i] = (float)fmax(Lambda[i], 0.0);
}

__global__ void fill_eta_kernel(float *eta, int B, float v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B) eta[i] = v;
}

}  // namespace

cudaError_t launch_rows_to_padded(const float *src, float *dst, long long rows, int L, int LP, float pad,
                                  cudaStream_t st) {
    rows_to_padded_kernel<<<blocks_for((size_t)(rows * LP)), kThreads, 0, st>>>(src, dst, rows, L, LP, pad);
    return cudaGetLastError();
}

cudaError_t launch_padded_to_rows(const float *src, float *dst, long long rows, int L, int LP, int mode,
                                  cudaStream_t st) {
    padded_to_rows_kernel<<<blocks_for((size_t)(rows * L)), kThreads, 0, st>>>(src, dst, rows, L, LP, mode);
    return cudaGetLastError();
}

cudaError_t launch_weights_to_pixel_major(const float *src, float *dst, int B, int nd, int H, int W,
                                          cudaStream_t st) {
    weights_to_pixel_major_kernel<<<blocks_for((size_t)B * nd * H * W), kThreads, 0, st>>>(src, dst, B, nd,
                                                                                          H, W);
    return cudaGetLastError();
}

cudaError_t launch_init_logq(const float *U, float *s, long long rows, int L, int LP, cudaStream_t st) {
    init_logq_kernel<<<blocks_for((size_t)rows), kThreads, 0, st>>>(U, s, rows, L, LP);
    return cudaGetLastError();
}

cudaError_t launch_lambda_to_d(const double *Lambda, float *d, int B, cudaStream_t st) {
    lambda_to_d_kernel<<<(B + 127) / 128, 128, 0, st>>>(Lambda, d, B);
    return cudaGetLastError();
}

__global__ void to_bf16_kernel(const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst, long long rows,
                               int LP, int pitch) {
    const long long n = rows * pitch;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / pitch;
        const int l = (int)(i - r * pitch);
        dst[i] = __float2bfloat16_rn(l < LP ? src[r * LP + l] : 0.f);
    }
}

cudaError_t launch_to_bf16(const float *src, __nv_bfloat16 *dst, long long rows, int LP, int pitch,
                           cudaStream_t st) {
    const long long blocks = (rows * pitch + 255) / 256;
    to_bf16_kernel<<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), 256, 0, st>>>(src, dst, rows, LP, pitch);
    return cudaGetLastError();
}

cudaError_t launch_fill_eta(float *eta, int B, double value, cudaStream_t st) {
    fill_eta_kernel<<<(B + 127) / 128, 128, 0, st>>>(eta, B, (float)value);
    return cudaGetLastError();
}

}  // namespace proxmf
