// layout.cu -- conversions between the external [B][N][L] row layout and the
// internal label-planar [B][L][H][P] layout, the initial state q^0, and small
// fills.  None of this runs inside the iteration loop.
#include <cmath>

#include "internal.h"

namespace proxmf {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(size_t n) {
    size_t b = (n + kThreads - 1) / kThreads;
    return (int)(b > 0x7fffffff ? 0x7fffffff : (b == 0 ? 1 : b));
}

// One thread per (b, y, x): reads L consecutive values, writes one per plane.
__global__ void rows_to_planar_kernel(const float *__restrict__ src, float *__restrict__ dst, int B,
                                      int L, int H, int W, int P) {
    const size_t n = (size_t)B * H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / ((size_t)H * W);
        const size_t p = i - b * H * W;
        const size_t y = p / W, x = p - y * W;
        const float *r = src + i * L;
        float *d = dst + b * L * H * P + y * P + x;
        for (int l = 0; l < L; ++l) d[(size_t)l * H * P] = r[l];
    }
}

__global__ void planar_to_rows_kernel(const float *__restrict__ src, float *__restrict__ dst, int B,
                                      int L, int H, int W, int P, int mode) {
    const size_t n = (size_t)B * H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / ((size_t)H * W);
        const size_t p = i - b * H * W;
        const size_t y = p / W, x = p - y * W;
        const float *s = src + b * L * H * P + y * P + x;
        float *r = dst + i * L;
        for (int l = 0; l < L; ++l) {
            const float v = s[(size_t)l * H * P];
            r[l] = mode == CONV_EXP ? expf(v) : v;
        }
    }
}

// Direction k of the grid: 0 right, 1 down, 2 down-right, 3 down-left.
__device__ __forceinline__ void dir_offset(int k, int *dy, int *dx) {
    *dy = k == 0 ? 0 : 1;
    *dx = k == 0 ? 1 : (k == 1 ? 0 : (k == 2 ? 1 : -1));
}

__global__ void weights_to_planar_kernel(const float *__restrict__ src, float *__restrict__ dst,
                                         int B, int nd, int H, int W, int P) {
    const size_t n = (size_t)B * nd * H * P;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t x = i % P;
        const size_t r = i / P;
        const size_t y = r % H;
        const size_t bk = r / H;
        const int k = (int)(bk % nd);
        int dy, dx;
        dir_offset(k, &dy, &dx);
        const long long yy = (long long)y + dy, xx = (long long)x + dx;
        float v = 0.f;
        if (x < (size_t)W && yy >= 0 && yy < H && xx >= 0 && xx < W) v = src[(bk * H + y) * W + x];
        dst[i] = v;
    }
}

// q^0 = softmax(-U): unary-only marginals, written as log q.
__global__ void init_logq_kernel(const float *__restrict__ U, float *__restrict__ s, int B, int L,
                                 int H, int W, int P) {
    const size_t n = (size_t)B * H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / ((size_t)H * W);
        const size_t p = i - b * H * W;
        const size_t y = p / W, x = p - y * W;
        const size_t base = b * L * H * P + y * P + x;
        const size_t plane = (size_t)H * P;
        float mx = -INFINITY;
        for (int l = 0; l < L; ++l) mx = fmaxf(mx, -U[base + l * plane]);
        float z = 0.f;
        for (int l = 0; l < L; ++l) z += expf(-U[base + l * plane] - mx);
        const float lse = mx + logf(z);
        for (int l = 0; l < L; ++l) s[base + l * plane] = -U[base + l * plane] - lse;
    }
}

__global__ void fill_eta_kernel(float *eta, int B, float v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B) eta[i] = v;
}

}  // namespace

cudaError_t launch_rows_to_planar(const float *src, float *dst, int B, int L, int H, int W, int P,
                                  cudaStream_t st) {
    rows_to_planar_kernel<<<blocks_for((size_t)B * H * W), kThreads, 0, st>>>(src, dst, B, L, H, W, P);
    return cudaGetLastError();
}

cudaError_t launch_planar_to_rows(const float *src, float *dst, int B, int L, int H, int W, int P,
                                  int mode, cudaStream_t st) {
    planar_to_rows_kernel<<<blocks_for((size_t)B * H * W), kThreads, 0, st>>>(src, dst, B, L, H, W, P,
                                                                              mode);
    return cudaGetLastError();
}

cudaError_t launch_weights_to_planar(const float *src, float *dst, int B, int nd, int H, int W,
                                     int P, cudaStream_t st) {
    weights_to_planar_kernel<<<blocks_for((size_t)B * nd * H * P), kThreads, 0, st>>>(src, dst, B, nd,
                                                                                      H, W, P);
    return cudaGetLastError();
}

cudaError_t launch_init_logq(const float *U, float *s, int B, int L, int H, int W, int P,
                             cudaStream_t st) {
    init_logq_kernel<<<blocks_for((size_t)B * H * W), kThreads, 0, st>>>(U, s, B, L, H, W, P);
    return cudaGetLastError();
}

cudaError_t launch_fill_eta(float *eta, int B, double value, cudaStream_t st) {
    fill_eta_kernel<<<(B + 127) / 128, 128, 0, st>>>(eta, B, (float)value);
    return cudaGetLastError();
}

}  // namespace proxmf
