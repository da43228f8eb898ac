// dense.cu -- fully connected CRF with a Gaussian appearance kernel
// (the dense segmentation model of Sec. 4.2), FP32 CUDA-core form.
//
// The pairwise weights are K_ij = exp(-|p_i-p_j|^2/(2 theta_pos^2)
// - |c_i-c_j|^2/(2 theta_rgb^2)) for i != j over (x, y, r, g, b) features, each
// unordered pair counted once, with one symmetric label matrix mu.  One step:
//   a1  S = K Q (N x N times N x L), m_i = mu S_i
//   a2  g_i = U_i + m_i
//   a3  a_i = -eta g_i + (1 - eta) log q_i
//   a4  log q'_i = a_i - logsumexp(a_i)
//   a5  F = sum_i q_i . (U_i + m_i / 2 + log q_i)
//
// K is materialised once per model ([B][N][N], FP32 here; BF16 for the
// tensor-core form in dense_tc.cu), so a step streams it from HBM: the FP32
// form reads 4 N^2 bytes per iteration and is bound by HBM bandwidth.
// A CTA owns 64 rows of K and all label columns; K is read in 64 x 32
// chunks, copied asynchronously (cp.async, 16 bytes per copy, coalesced
// along the rows) into a padded row-major shared-memory tile.  Each thread
// owns 4 rows (16 apart) x 6 labels and the four k of its slice of a chunk:
// one 128-bit shared load per row and three 64-bit loads of q per k feed
// 12 paired FMAs per k; the 512 threads split each chunk eight ways along k.
// A ring of six chunks (K and Q, 74 KB) is in flight per SM while one is
// multiplied.  The epilogue (mu product, update,
// renormalisation, free energy) runs on the CTA's 64 rows.
#include <cmath>

#include "dense_common.cuh"
#include "f32x2.cuh"
#include "internal.h"

namespace proxmf {

namespace {

constexpr int kDR = 64;        // rows of K per CTA
constexpr int kDK = 32;        // k per chunk
constexpr int kDT = 512;       // threads per CTA
constexpr int kSlices = kDT / 64;   // k slices of a chunk (64 threads each)
constexpr int kStages = 6;     // chunks in flight in the shared-memory ring

constexpr int kKsRow = kDK + 4;   // padded K tile row (16-byte aligned, conflict-free 128-bit reads)

template <int LP>
constexpr size_t dense_f32_dyn_smem() {
    return (size_t)kStages * (kDR * kKsRow + kDK * LP) * sizeof(float);
}

// ---------------------------------------------------------------- K build --

template <typename T>
__device__ __forceinline__ T to_out(float v);
template <>
__device__ __forceinline__ float to_out<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// K[b][i][j] from features [b][N][5]; one thread per (i, 4 consecutive j).
template <typename T>
__global__ void dense_kernel_build_kernel(const float *__restrict__ feats, T *__restrict__ K, int N, int pitch,
                                          float inv2p, float inv2c) {
    const int b = blockIdx.z;
    const int i = blockIdx.y;
    const float *f = feats + (size_t)b * N * 5;
    const float xi = f[i * 5 + 0], yi = f[i * 5 + 1], ri = f[i * 5 + 2], gi = f[i * 5 + 3], bi = f[i * 5 + 4];
    T *row = K + ((size_t)b * N + i) * pitch;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < pitch; j += gridDim.x * blockDim.x) {
        if (j >= N) {
            row[j] = to_out<T>(0.f);
            continue;
        }
        const float dx = xi - f[j * 5 + 0], dy = yi - f[j * 5 + 1];
        const float dr = ri - f[j * 5 + 2], dg = gi - f[j * 5 + 3], db = bi - f[j * 5 + 4];
        const float p2 = dx * dx + dy * dy, c2 = dr * dr + dg * dg + db * db;
        const float v = (j == i) ? 0.f : expf(-p2 * inv2p - c2 * inv2c);
        row[j] = to_out<T>(v);
    }
}

// The BF16 copy of K for the tensor-core step, in blocks of 128 rows by 64
// columns: block (tile, chunk) of instance b starts at element
// ((b * nchunk + chunk) * ntiles + tile) * 8192 (chunk-major, so the blocks
// that all row tiles read at the same moment lie side by side in memory and
// spread over every memory channel) and holds row r, column k at
// byte r * 128 + (((k / 8) ^ (r % 8)) * 16) + (k % 8) * 2 -- the 128-byte
// swizzled K-major layout the MMA reads from shared memory, so one block is
// one contiguous 16 KiB bulk copy.  Rows and columns past N are zero.
__global__ void dense_kernel_build_tiled_kernel(const float *__restrict__ feats, __nv_bfloat16 *__restrict__ K,
                                                int N, int ntiles, int nchunk, float inv2p, float inv2c) {
    const int b = blockIdx.z;
    const int i = blockIdx.y;                 // row, < ntiles * 128
    const float *f = feats + (size_t)b * N * 5;
    const bool row_ok = i < N;
    float xi = 0.f, yi = 0.f, ri = 0.f, gi = 0.f, bi = 0.f;
    if (row_ok) {
        xi = f[i * 5 + 0];
        yi = f[i * 5 + 1];
        ri = f[i * 5 + 2];
        gi = f[i * 5 + 3];
        bi = f[i * 5 + 4];
    }
    const int tile = i / 128, r = i % 128;
    uint8_t *tb = reinterpret_cast<uint8_t *>(K) + ((size_t)b * nchunk * ntiles + tile) * 16384 + (size_t)r * 128;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nchunk * 64; j += gridDim.x * blockDim.x) {
        float v = 0.f;
        if (row_ok && j < N && j != i) {
            const float dx = xi - f[j * 5 + 0], dy = yi - f[j * 5 + 1];
            const float dr = ri - f[j * 5 + 2], dg = gi - f[j * 5 + 3], db = bi - f[j * 5 + 4];
            const float p2 = dx * dx + dy * dy, c2 = dr * dr + dg * dg + db * db;
            v = expf(-p2 * inv2p - c2 * inv2c);
        }
        const int chunk = j / 64, k = j % 64;
        *reinterpret_cast<__nv_bfloat16 *>(tb + (size_t)chunk * ntiles * 16384 + (((k >> 3) ^ (r & 7)) << 4) +
                                           (k & 7) * 2) =
            __float2bfloat16_rn(v);
    }
}

// q = exp(log q) as FP32 rows [B][N][LP] (padding 0) and, if qt16 is given,
// BF16 label-major [B][32][pitch] (labels >= L zero) for the tensor-core form.
__global__ void dense_export_q_kernel(const float *__restrict__ s, float *__restrict__ q32,
                                      __nv_bfloat16 *__restrict__ qt16, int B, int N, int L, int LP, int pitch) {
    const long long n = (long long)B * N * LP;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(idx % LP);
        const long long bi = idx / LP;
        const int b = (int)(bi / N), i = (int)(bi % N);
        const float q = l < L ? expf(s[idx]) : 0.f;
        if (q32) q32[idx] = q;
        if (qt16 && l < 32) qt16[((size_t)b * 32 + l) * pitch + i] = __float2bfloat16_rn(q);
    }
}

// ---------------------------------------------------------------- step --

struct DenseStepArgs {
    const float *K;          // [B][N][N]
    const float *q_in;       // [B][N][LP] q of the state read
    const float *s_in;       // [B][N][LP] log q
    const float *U;          // [B][N][LP]
    float *s_out;            // [B][N][LP]
    float *q_out;            // [B][N][LP] q of the new state (for the next step)
    __nv_bfloat16 *qt_out;   // [B][32][pitch] BF16 copy of q_out (tensor-core form) or null
    const float *eta;        // [B]
    const float *mu;         // [L][L] device
    double *partial;         // [B][nblk]
    unsigned *counter;       // [B]
    double *f_trace, *f_cur;
    int *done, *status;
    int N, L, nblk, pitch;
    int t, trace_cap, update;
    double rel_tol;
};

}  // namespace

namespace {

// cp.async helpers: 4-byte copy with zero fill when !valid (no bytes read),
// 16-byte copy, group commit and wait.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(gmem), "r"(valid ? 4 : 0) : "memory");
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}

// 16-byte copy of the first nbytes (0..16) of the source, the rest zero
__device__ __forceinline__ void cp_async16z(void *smem, const void *gmem, int nbytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gmem), "r"(nbytes) : "memory");
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int LP>
__global__ void __launch_bounds__(kDT, 1) dense_step_f32_kernel(const __grid_constant__ DenseStepArgs a) {
    constexpr int NC = (LP + 5) / 6;             // column groups of 6 (last may be partial)
    constexpr int CG = 4;                        // column groups handled by the thread grid
    static_assert(NC <= CG, "LP <= 24");
    extern __shared__ __align__(16) float dsm[];
    float *Ks = dsm;                                     // [kStages][kDR][kKsRow]  (row-major K tile)
    float *Qs = Ks + (size_t)kStages * kDR * kKsRow;     // [kStages][kDK][LP]
    __shared__ __align__(16) float Sred[kDR][LP + 1];
    __shared__ __align__(16) float mus[kMaxLabels * kMaxLabels];   // mu^T, zero-padded
    __shared__ double red[kDT / 32];
    __shared__ int is_last;

    const int b = blockIdx.y;
    const int tid = threadIdx.x;
    const int N = a.N, L = a.L;
    const int row0 = blockIdx.x * kDR;
    const float *Kb = a.K + (size_t)b * N * N;
    const float *qb = a.q_in + (size_t)b * N * LP;

    if (a.done != nullptr && a.done[b] != 0) {
        if (a.update)
            for (int idx = tid; idx < kDR * LP; idx += kDT) {
                const int r = row0 + idx / LP;
                if (r < N) {
                    const size_t o = ((size_t)b * N + r) * LP + idx % LP;
                    a.s_out[o] = a.s_in[o];
                    a.q_out[o] = a.q_in[o];
                }
            }
        return;
    }

    load_mu_transposed(mus, a.mu, L, tid, kDT);

    // micro-tile: rows ig + 16 r (r < 4), label columns 6*cg .. 6*cg+5, the
    // four k of slice ks of each chunk
    const int ig = tid & 15, cg = (tid >> 4) & 3, ks = tid >> 6;
    // loader: row tid >> 3, k = 4 * (tid & 7) .. +3 of the chunk: one 16-byte
    // asynchronous copy (rows of K start on 16-byte boundaries when N % 4 == 0;
    // otherwise four 4-byte copies), zero past N
    const int lrow = tid >> 3, lk = 4 * (tid & 7);
    const bool rvalid = row0 + lrow < N;
    const float *ksrc = Kb + (size_t)(rvalid ? row0 + lrow : 0) * N;
    const bool vec16 = (N & 3) == 0;
    // Q chunk in 16-byte pieces (8-byte for LP = 2: an instance's rows then
    // start on an 8-byte boundary only); rows past N read the zero padding
    constexpr int kQV = LP % 4 == 0 ? 4 : 2;
    constexpr int kQn = kDK * LP / kQV;

    float2 acc[4][3];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[r][c] = splat2(0.f);

    const int nchunk = (N + kDK - 1) / kDK;
    auto issue = [&](int c) {
        const int stg = c % kStages, k0 = c * kDK;
        float *kd = Ks + (size_t)stg * kDR * kKsRow + lrow * kKsRow + lk;
        const int k = k0 + lk;
        if (vec16) {
            const int nb = rvalid ? max(0, min(16, 4 * (N - k))) : 0;
            cp_async16z(kd, nb > 0 ? ksrc + k : Kb, nb);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const bool v = rvalid && k + e < N;
                cp_async4(kd + e, v ? ksrc + k + e : Kb, v);
            }
        }
        if (tid < kQn) {
            float *qd = Qs + (size_t)stg * kDK * LP + kQV * tid;
            const float *qsrc = qb + (size_t)k0 * LP + kQV * tid;
            if constexpr (kQV == 4)
                cp_async16(qd, qsrc);
            else
                cp_async8(qd, qsrc);
        }
    };
    auto compute = [&](int stg) {
        if (cg >= NC) return;
        const float *kb = Ks + (size_t)stg * kDR * kKsRow + ks * (kDK / kSlices);
        const float *qs = Qs + (size_t)stg * kDK * LP + ks * (kDK / kSlices) * LP;
        float kr[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float4 kv = *reinterpret_cast<const float4 *>(kb + (ig + 16 * r) * kKsRow);
            kr[r][0] = kv.x;
            kr[r][1] = kv.y;
            kr[r][2] = kv.z;
            kr[r][3] = kv.w;
        }
#pragma unroll
        for (int kk = 0; kk < kDK / kSlices; ++kk) {
            float2 qv[3];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const int col = 6 * cg + 2 * p;
                qv[p] = col + 1 < LP ? *reinterpret_cast<const float2 *>(qs + kk * LP + col) : splat2(0.f);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float2 kk2 = splat2(kr[r][kk]);
#pragma unroll
                for (int p = 0; p < 3; ++p) acc[r][p] = fma2(kk2, qv[p], acc[r][p]);
            }
        }
    };

    // multistage ring: chunk c lands in stage c % kStages; the copy of chunk
    // c + kStages - 1 goes into the stage computed one iteration earlier
#pragma unroll
    for (int c = 0; c < kStages - 1; ++c) {
        if (c < nchunk) issue(c);
        cp_async_commit();
    }
    for (int c = 0; c < nchunk; ++c) {
        cp_async_wait<kStages - 2>();
        __syncthreads();
        compute(c % kStages);
        if (c + kStages - 1 < nchunk) issue(c + kStages - 1);
        cp_async_commit();
    }
    cp_async_wait<0>();
    __syncthreads();

    // reduce the k slices: slice 0 writes, the others add, in a fixed order
    for (int sl = 0; sl < kSlices; ++sl) {
        if (ks == sl && cg < NC) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    const int col = 6 * cg + 2 * p;
                    if (col + 1 < LP) {
                        float *d = &Sred[ig + 16 * r][col];
                        if (sl == 0) {
                            d[0] = acc[r][p].x;
                            d[1] = acc[r][p].y;
                        } else {
                            d[0] += acc[r][p].x;
                            d[1] += acc[r][p].y;
                        }
                    }
                }
        }
        __syncthreads();
    }

    // epilogue: one thread per row
    float f = 0.f;
    if (tid < kDR && row0 + tid < N) {
        const int i = row0 + tid;
        const size_t o = ((size_t)b * N + i) * LP;
        f = dense_row_update<LP>(Sred[tid], mus, L, a.eta[b], a.s_in + o, a.U + o, a.s_out + o, a.q_out + o,
                                 a.qt_out ? a.qt_out + (size_t)b * 32 * a.pitch + i : nullptr, (size_t)a.pitch,
                                 a.update != 0);
    }
    double fd = (double)f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) fd += __shfl_down_sync(0xffffffffu, fd, off);
    if ((tid & 31) == 0) red[tid >> 5] = fd;
    __syncthreads();
    if (tid == 0) {
        double bs = 0.0;
        for (int k = 0; k < kDT / 32; ++k) bs += red[k];
        a.partial[(size_t)b * a.nblk + blockIdx.x] = bs;
        __threadfence();
        is_last = atomicAdd(a.counter + b, 1u) == (unsigned)(a.nblk - 1);
    }
    __syncthreads();
    if (!is_last) return;
    // last block of the instance: all threads sum fixed strided subsets of
    // the partials, then a fixed-shape tree (deterministic)
    __threadfence();
    double tot = 0.0;
    for (int k = tid; k < a.nblk; k += kDT) tot += __ldcg(a.partial + (size_t)b * a.nblk + k);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, off);
    __syncthreads();   // red is reused
    if ((tid & 31) == 0) red[tid >> 5] = tot;
    __syncthreads();
    if (tid == 0) {
        double F = 0.0;
        for (int k = 0; k < kDT / 32; ++k) F += red[k];
        a.f_cur[b] = F;
        if (!isfinite(F)) atomicExch(a.status, -6);
        if (a.update) {
            if (a.t < a.trace_cap) a.f_trace[(size_t)b * a.trace_cap + a.t] = F;
            if (a.rel_tol > 0.0 && a.t > 0 && a.t - 1 < a.trace_cap && a.done != nullptr) {
                const double Fp = a.f_trace[(size_t)b * a.trace_cap + a.t - 1];
                if (fabs(F - Fp) <= a.rel_tol * fabs(F)) a.done[b] = a.t + 1;
            }
        }
        a.counter[b] = 0u;
    }
}

}  // namespace

cudaError_t launch_dense_kernel_build(const float *feats, float *K32, __nv_bfloat16 *K16, int B, int N,
                                      double theta_pos, double theta_rgb, cudaStream_t st) {
    const float inv2p = (float)(1.0 / (2.0 * theta_pos * theta_pos));
    const float inv2c = (float)(1.0 / (2.0 * theta_rgb * theta_rgb));
    dim3 grid((N + 255) / 256 < 8 ? (N + 255) / 256 : 8, N, B);
    if (K32) dense_kernel_build_kernel<float><<<grid, 256, 0, st>>>(feats, K32, N, N, inv2p, inv2c);
    if (K16) {
        const int ntiles = dense_tc_tiles(N), nchunk = dense_tc_pitch(N) / 64;
        dim3 g2((nchunk * 64 + 255) / 256 < 8 ? (nchunk * 64 + 255) / 256 : 8, ntiles * 128, B);
        dense_kernel_build_tiled_kernel<<<g2, 256, 0, st>>>(feats, K16, N, ntiles, nchunk, inv2p, inv2c);
    }
    return cudaGetLastError();
}

namespace {

// One thread per (instance, chunk, column): the six rows of a chunk's column
// (see launch_dense_fly_features).
__global__ void dense_fly_features_kernel(const float *__restrict__ feats, float *__restrict__ featsT, int B, int N,
                                          int nchunk, float sp, float sc) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)B * nchunk * 64) return;
    const int j = (int)(idx % 64);
    const long long bc = idx / 64;                 // b * nchunk + chunk
    const int chunk = (int)(bc % nchunk), b = (int)(bc / nchunk);
    const int J = chunk * 64 + j;
    float *out = featsT + bc * 6 * 64 + j;
    if (J >= N) {
        for (int k = 0; k < 5; ++k) out[k * 64] = 0.f;
        out[5 * 64] = -1e30f;
        return;
    }
    const float *f = feats + ((size_t)b * N + J) * 5;
    float g[5];
    g[0] = sp * f[0];
    g[1] = sp * f[1];
    g[2] = sc * f[2];
    g[3] = sc * f[3];
    g[4] = sc * f[4];
    float n2 = 0.f;
    for (int k = 0; k < 5; ++k) {
        out[k * 64] = 1.41421356f * g[k];
        n2 = fmaf(g[k], g[k], n2);
    }
    out[5 * 64] = -n2;
}

}  // namespace

cudaError_t launch_dense_fly_features(const float *feats, float *featsT, int B, int N, double theta_pos,
                                      double theta_rgb, cudaStream_t st) {
    // K = exp(-d^2 / (2 theta^2)) = 2^(-(s d)^2) with s = sqrt(log2(e) / (2 theta^2))
    const double log2e = 1.4426950408889634;
    const float sp = (float)std::sqrt(log2e / (2.0 * theta_pos * theta_pos));
    const float sc = (float)std::sqrt(log2e / (2.0 * theta_rgb * theta_rgb));
    const int nchunk = dense_tc_pitch(N) / 64;
    const long long n = (long long)B * nchunk * 64;
    dense_fly_features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(feats, featsT, B, N, nchunk, sp, sc);
    return cudaGetLastError();
}

cudaError_t launch_dense_export_q(const float *s, float *q32, __nv_bfloat16 *qt16, int B, int N, int L, int LP,
                                  cudaStream_t st) {
    const long long n = (long long)B * N * LP;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 1 << 20);
    dense_export_q_kernel<<<blocks, 256, 0, st>>>(s, q32, qt16, B, N, L, LP, dense_tc_pitch(N));
    return cudaGetLastError();
}

int dense_nblk(int N) { return (N + kDR - 1) / kDR; }

namespace {

template <int LP>
cudaError_t launch_f32(dim3 grid, const DenseStepArgs &a, cudaStream_t st) {
    constexpr size_t smem = dense_f32_dyn_smem<LP>();
    static SmemOptIn optin;   // the opt-in above 48 KB, once per device
    const cudaError_t attr = smem_optin(optin, dense_step_f32_kernel<LP>, smem);
    if (attr != cudaSuccess) return attr;
    dense_step_f32_kernel<LP><<<grid, kDT, smem, st>>>(a);
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_dense_step_f32(const DenseStepLaunch &l, cudaStream_t st) {
    DenseStepArgs a;
    a.K = l.K32;
    a.q_in = l.q_in;
    a.s_in = l.s_in;
    a.U = l.U;
    a.s_out = l.s_out;
    a.q_out = l.q_out;
    a.qt_out = l.qt_out;
    a.eta = l.eta;
    a.mu = l.mu;
    a.partial = l.partial;
    a.counter = l.counter;
    a.f_trace = l.f_trace;
    a.f_cur = l.f_cur;
    a.done = l.done;
    a.status = l.status;
    a.N = l.N;
    a.L = l.L;
    a.nblk = dense_nblk(l.N);
    a.pitch = dense_tc_pitch(l.N);
    a.t = l.t;
    a.trace_cap = l.trace_cap;
    a.update = l.update;
    a.rel_tol = l.rel_tol;
    dim3 grid(a.nblk, l.B);
    cudaError_t e = cudaSuccess;
    switch (storage_labels(l.L)) {
    case 2: e = launch_f32<2>(grid, a, st); break;
    case 4: e = launch_f32<4>(grid, a, st); break;
    case 8: e = launch_f32<8>(grid, a, st); break;
    case 12: e = launch_f32<12>(grid, a, st); break;
    case 16: e = launch_f32<16>(grid, a, st); break;
    case 20: e = launch_f32<20>(grid, a, st); break;
    case 24: e = launch_f32<24>(grid, a, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace proxmf
