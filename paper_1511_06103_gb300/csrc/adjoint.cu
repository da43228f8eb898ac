// adjoint.cu -- reverse mode through K unrolled proximal steps on a grid CRF.
//
// Forward (per step, eta fixed):  q = exp(s),  m = H q,
//   a = -eta (U + m) + (1 - eta) s,  s' = a - logsumexp(a),
// from s^0 = logsoftmax(-U), with H the constant potential matrix
// (H v)_i = mu sum_{i->j} w_ij v_j + mu^T sum_{k->i} w_ki v_k.
// Backward, with gs = d loss / d s' given:
//   ga = gs - q' sum_l gs                     (log-softmax)
//   dU += -eta ga,  gm = -eta ga              (affine step)
//   gs_prev = (1 - eta) ga + q (.) (H gm)     (H is symmetric)
//   dw_{i->j} += gm_i^T mu q_j + q_i^T mu gm_j
//   dmu += sum_i gm_i S_i^T + T_i gm_i^T,  S_i = sum_{i->j} w q_j, T_i = sum_{k->i} w q_k
// and finally through s^0: dU += -(gs - q^0 sum_l gs).
// The forward keeps every s^t (checkpoints) so the backward needs no
// recomputation of the trajectory; each backward step is two kernels over the
// pixels.  Every gradient is accumulated by the thread or block that owns it
// (dmu through per-block partials reduced in a fixed order), so results do
// not depend on scheduling.
#include <cmath>

#include "internal.h"

namespace proxmf {

namespace {

constexpr int kAT = 128;   // 3 x kAT x 24 floats of shared memory stay under 48 KB

__device__ __forceinline__ void adj_dir(int k, int *dy, int *dx) {
    *dy = k == 0 ? 0 : 1;
    *dx = k == 0 ? 1 : (k == 1 ? 0 : (k == 2 ? 1 : -1));
}

// Keeps the compiler from carrying shared-memory loads (the L x L matrix)
// in registers from one phase of a kernel to the next.
__device__ __forceinline__ void reload_fence() { asm volatile("" ::: "memory"); }

// ga = gs - q' sum gs; gm = -eta ga; gs <- (1 - eta) ga; dU += -eta ga.
template <int LP>
__global__ void adj_softmax_kernel(float *gs, float *gm, float *dU, const float *s_next, const float *eta, int B,
                                   int N, int L) {
    const long long n = (long long)B * N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
         r += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(r / N);
        const float e = eta[b];
        const size_t o = (size_t)r * LP;
        float g[LP], sum = 0.f;
#pragma unroll
        for (int l = 0; l < LP; ++l) {
            g[l] = l < L ? gs[o + l] : 0.f;
            sum += g[l];
        }
#pragma unroll
        for (int l = 0; l < LP; ++l) {
            if (l >= L) continue;
            const float ga = g[l] - __expf(s_next[o + l]) * sum;
            gm[o + l] = -e * ga;
            gs[o + l] = (1.f - e) * ga;
            dU[o + l] += -e * ga;
        }
    }
}

// gs += q (.) (H gm); dw and the per-block dmu partial.  Per-thread
// registers hold at most four label vectors at a time; S, T and gm of the
// block's pixels go to shared memory ([label][pixel], stride kAT + 1 so that
// both the per-pixel and the per-entry access patterns are conflict free).
template <int LP>
__global__ void __launch_bounds__(kAT) adj_message_kernel(float *gs, const float *gm, const float *s, const float *w,
                                                        const float *mu, float *dw, float *dmu_part, int B, int H,
                                                        int W, int L, int conn) {
    constexpr int SP = kAT + 1;
    __shared__ float mus[LP * LP];   // mu zero padded to LP x LP
    __shared__ float sg[LP * SP], sS[LP * SP], sT[LP * SP];
    const int nd = conn == 8 ? 4 : 2;
    for (int i = threadIdx.x; i < LP * LP; i += blockDim.x) {
        const int r = i / LP, c = i - r * LP;
        mus[i] = (r < L && c < L) ? mu[r * L + c] : 0.f;
    }
    const int N = H * W;
    const int tid = threadIdx.x;
    const long long r = blockIdx.x * (long long)kAT + tid;
    const bool act = r < (long long)B * N;
    const int b = act ? (int)(r / N) : 0;
    const int p = act ? (int)(r - (long long)b * N) : 0;
    const int y = p / W, x = p - y * W;
    const size_t base = (size_t)b * N;
    const size_t o = (base + p) * LP;
    float qi[LP], v1[LP], v2[LP];
#pragma unroll
    for (int l = 0; l < LP; ++l) {
        const float g = (act && l < L) ? gm[o + l] : 0.f;
        sg[l * SP + tid] = g;
        sS[l * SP + tid] = 0.f;
        sT[l * SP + tid] = 0.f;
        qi[l] = (act && l < L) ? __expf(s[o + l]) : 0.f;
    }
    __syncthreads();
    // v1 = mu^T gm_i, v2 = mu^T q_i (edge gradients of out-going edges)
#pragma unroll
    for (int l = 0; l < LP; ++l) {
        float a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int k = 0; k < LP; ++k) {
            a1 = fmaf(mus[k * LP + l], sg[k * SP + tid], a1);
            a2 = fmaf(mus[k * LP + l], qi[k], a2);
        }
        v1[l] = a1;
        v2[l] = a2;
    }
    float hacc[LP];
    reload_fence();
    {
        float G[LP];
#pragma unroll
        for (int l = 0; l < LP; ++l) G[l] = 0.f;
        for (int d = 0; act && d < nd; ++d) {                    // out-going edges p -> j
            int dy, dx;
            adj_dir(d, &dy, &dx);
            const int yo = y + dy, xo = x + dx;
            if (yo >= H || xo < 0 || xo >= W) continue;
            const size_t j = (base + (size_t)yo * W + xo) * LP;
            const float wv = w[(base + p) * nd + d];
            float de = 0.f;
#pragma unroll
            for (int l = 0; l < LP; ++l) {
                if (l >= L) continue;
                const float gj = gm[j + l], qj = __expf(s[j + l]);
                G[l] = fmaf(wv, gj, G[l]);
                sS[l * SP + tid] = fmaf(wv, qj, sS[l * SP + tid]);
                de = fmaf(v1[l], qj, fmaf(v2[l], gj, de));
            }
            dw[(base + p) * nd + d] += de;
        }
        reload_fence();
#pragma unroll
        for (int l = 0; l < LP; ++l) {                          // hacc = mu G
            float h = 0.f;
#pragma unroll
            for (int k = 0; k < LP; ++k) h = fmaf(mus[l * LP + k], G[k], h);
            hacc[l] = h;
        }
    }
    reload_fence();
    {
        float G[LP];
#pragma unroll
        for (int l = 0; l < LP; ++l) G[l] = 0.f;
        for (int d = 0; act && d < nd; ++d) {                    // in-coming edges k -> p
            int dy, dx;
            adj_dir(d, &dy, &dx);
            const int yi = y - dy, xi = x - dx;
            if (yi < 0 || xi < 0 || xi >= W) continue;
            const size_t k = base + (size_t)yi * W + xi;
            const float wv = w[k * nd + d];
#pragma unroll
            for (int l = 0; l < LP; ++l) {
                if (l >= L) continue;
                G[l] = fmaf(wv, gm[k * LP + l], G[l]);
                sT[l * SP + tid] = fmaf(wv, __expf(s[k * LP + l]), sT[l * SP + tid]);
            }
        }
        reload_fence();
#pragma unroll
        for (int l = 0; l < LP; ++l) {                          // hacc += mu^T G
            float h = hacc[l];
#pragma unroll
            for (int k = 0; k < LP; ++k) h = fmaf(mus[k * LP + l], G[k], h);
            hacc[l] = h;
        }
    }
    if (act) {
#pragma unroll
        for (int l = 0; l < LP; ++l)
            if (l < L) gs[o + l] += qi[l] * hacc[l];
    }
    __syncthreads();
    // dmu partial of this block: sum over its pixels of gm_i S_i^T + T_i gm_i^T
    for (int e = tid; e < L * L; e += kAT) {
        const int a = e / L, c = e - a * L;
        float acc = 0.f;
        for (int t = 0; t < kAT; ++t)
            acc = fmaf(sg[a * SP + t], sS[c * SP + t], fmaf(sT[a * SP + t], sg[c * SP + t], acc));
        dmu_part[(size_t)blockIdx.x * L * L + e] += acc;
    }
}

// Through s^0 = logsoftmax(-U): dU += -(gs - q^0 sum gs).
template <int LP>
__global__ void adj_init_kernel(const float *gs, const float *s0, float *dU, long long rows, int L) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        const size_t o = (size_t)r * LP;
        float sum = 0.f;
        for (int l = 0; l < L; ++l) sum += gs[o + l];
        for (int l = 0; l < L; ++l) dU[o + l] += -(gs[o + l] - __expf(s0[o + l]) * sum);
    }
}

// dmu[e] = sum of the per-block partials: one block per entry, each thread a
// fixed strided subset in FP64, then a fixed-shape tree (deterministic).
__global__ void adj_dmu_reduce_kernel(const float *part, int nblk, int LL, float *dmu) {
    __shared__ double red[256];
    const int e = blockIdx.x;
    double acc = 0.0;
    for (int k = threadIdx.x; k < nblk; k += 256) acc += (double)part[(size_t)k * LL + e];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) dmu[e] = (float)red[0];
}

// [B][N][nd] -> [B][nd][H][W]
__global__ void adj_dw_out_kernel(const float *dw, float *out, int B, int nd, int H, int W) {
    const long long n = (long long)B * nd * H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % W);
        const long long r = i / W;
        const int y = (int)(r % H);
        const long long bk = r / H;
        const int k = (int)(bk % nd);
        const long long b = bk / nd;
        out[i] = dw[((size_t)b * H * W + (size_t)y * W + x) * nd + k];
    }
}

inline int nb(long long n, int t) { return (int)std::min<long long>((n + t - 1) / t, 1 << 20); }

}  // namespace

cudaError_t launch_adjoint_step(const AdjointStep &a, cudaStream_t st) {
    const long long rows = (long long)a.B * a.H * a.W;
    const int LP = storage_labels(a.L);
    const int nblk = (int)((rows + kAT - 1) / kAT);
#define PROXMF_ADJ(LPV)                                                                                         \
    case LPV:                                                                                                   \
        adj_softmax_kernel<LPV><<<nb(rows, 256), 256, 0, st>>>(a.gs, a.gm, a.dU, a.s_next, a.eta, a.B,          \
                                                               a.H * a.W, a.L);                                \
        adj_message_kernel<LPV><<<nblk, kAT, 0, st>>>(a.gs, a.gm, a.s, a.w, a.mu, a.dw, a.dmu_part, a.B, a.H,   \
                                                      a.W, a.L, a.conn);                                        \
        break;
    switch (LP) {
        PROXMF_ADJ(2)
        PROXMF_ADJ(4)
        PROXMF_ADJ(8)
        PROXMF_ADJ(12)
        PROXMF_ADJ(16)
        PROXMF_ADJ(20)
        PROXMF_ADJ(24)
    default:
        return cudaErrorInvalidValue;
    }
#undef PROXMF_ADJ
    return cudaGetLastError();
}

int adjoint_blocks(long long rows) { return (int)((rows + kAT - 1) / kAT); }

cudaError_t launch_adjoint_finish(const AdjointFinish &a, cudaStream_t st) {
    const long long rows = (long long)a.B * a.H * a.W;
    const int LP = storage_labels(a.L);
    switch (LP) {
    case 2: adj_init_kernel<2><<<nb(rows, 256), 256, 0, st>>>(a.gs, a.s0, a.dU, rows, a.L); break;
    case 4: adj_init_kernel<4><<<nb(rows, 256), 256, 0, st>>>(a.gs, a.s0, a.dU, rows, a.L); break;
    case 8: adj_init_kernel<8><<<nb(rows, 256), 256, 0, st>>>(a.gs, a.s0, a.dU, rows, a.L); break;
    case 12: adj_init_kernel<12><<<nb(rows, 256), 256, 0, st>>>(a.gs, a.s0, a.dU, rows, a.L); break;
    case 16: adj_init_kernel<16><<<nb(rows, 256), 256, 0, st>>>(a.gs, a.s0, a.dU, rows, a.L); break;
    case 20: adj_init_kernel<20><<<nb(rows, 256), 256, 0, st>>>(a.gs, a.s0, a.dU, rows, a.L); break;
    case 24: adj_init_kernel<24><<<nb(rows, 256), 256, 0, st>>>(a.gs, a.s0, a.dU, rows, a.L); break;
    default: return cudaErrorInvalidValue;
    }
    adj_dmu_reduce_kernel<<<a.L * a.L, 256, 0, st>>>(a.dmu_part, adjoint_blocks(rows), a.L * a.L, a.dmu_out);
    const int nd = a.conn == 8 ? 4 : 2;
    adj_dw_out_kernel<<<nb(rows * nd, 256), 256, 0, st>>>(a.dw, a.dw_out, a.B, nd, a.H, a.W);
    return cudaGetLastError();
}

}  // namespace proxmf
