// sparse.cu -- the parallel proximal step on a general pairwise graph given
// as an edge list (Sec. 2.1, Eq. related:pairwise-mrf with an arbitrary edge
// set; the DBN-shaped layers of the paper's benchmarks are one instance).
//
// One warp per variable, one lane per label (L <= 32): the lanes walk the
// variable's adjacency list in CSR form and accumulate the weighted
// neighbour marginals with one coalesced 4*LP-byte read per neighbour (for
// L <= 8 the lanes split the list instead and reduce in a fixed order), then
//   m = mu S_out + mu^T S_in      (m = mu S for symmetric mu, S over both
//                                  directions of every edge),
// the L x L product with the other lanes' S through warp shuffles, and the
// log-domain step, renormalisation and free-energy term of Eq.
// method:update_natural as in the grid step.  q = exp(log q) of the new
// state is written next to it, so that neighbours read q without
// recomputing exponentials.  Free-energy partials are FP64 per block and
// reduced in a fixed order by the last block of each instance.
#include <cmath>

#include "dfloat.cuh"
#include "internal.h"

namespace proxmf {

namespace {

constexpr int kSW = 8;               // warps per block
constexpr int kST = kSW * 32;
// Variables per warp: more per warp for large graphs (fewer blocks, so fewer
// FP64 block partials for the last block to sum: FP64 is the narrow pipe of
// this part), one per warp for small ones (enough warps to fill the SMs).
__host__ __device__ inline int sparse_vpw(int N) { return N >= 131072 ? 8 : (N >= 8192 ? 4 : 1); }

// sum_e w_e q[col_e][lane] over one adjacency list, four entries in flight
__device__ __forceinline__ float gather(const int *__restrict__ ptr, const int *__restrict__ col,
                                        const float *__restrict__ wt, const float *__restrict__ q, size_t base,
                                        int i, int lane, int LP) {
    const int e0 = ptr[i], e1 = ptr[i + 1];
    float acc = 0.f;
    int e = e0;
    for (; e + 4 <= e1; e += 4) {
        const int c0 = col[e], c1 = col[e + 1], c2 = col[e + 2], c3 = col[e + 3];
        const float w0 = wt[e], w1 = wt[e + 1], w2 = wt[e + 2], w3 = wt[e + 3];
        if (lane < LP) {
            const float q0 = __ldg(q + (base + c0) * LP + lane), q1 = __ldg(q + (base + c1) * LP + lane);
            const float q2 = __ldg(q + (base + c2) * LP + lane), q3 = __ldg(q + (base + c3) * LP + lane);
            acc = fmaf(w0, q0, acc);
            acc = fmaf(w1, q1, acc);
            acc = fmaf(w2, q2, acc);
            acc = fmaf(w3, q3, acc);
        }
    }
    for (; e < e1; ++e) {
        const float qj = lane < LP ? __ldg(q + (base + col[e]) * LP + lane) : 0.f;
        acc = fmaf(wt[e], qj, acc);
    }
    return acc;
}

// The same sums for few labels (L <= LM): the lanes split the adjacency
// list instead (lane j takes entries j, j + 32, ...), each keeping the L
// partial sums, which a fixed-shape tree brings to lane 0 and a broadcast
// hands to every lane.  Returns lane's own label sum (0 past L).
template <int LM>
__device__ __forceinline__ float gather_edges(const int *__restrict__ ptr, const int *__restrict__ col,
                                              const float *__restrict__ wt, const float *__restrict__ q,
                                              size_t base, int i, int lane, int L, int LP) {
    float S[LM];
#pragma unroll
    for (int l = 0; l < LM; ++l) S[l] = 0.f;
    const int e0 = ptr[i], e1 = ptr[i + 1];
#pragma unroll 4
    for (int e = e0 + lane; e < e1; e += 32) {
        const float w = wt[e];
        const float *qr = q + (base + col[e]) * LP;
#pragma unroll
        for (int l = 0; l < LM; ++l)
            if (l < L) S[l] = fmaf(w, __ldg(qr + l), S[l]);
    }
    float mine = 0.f;
#pragma unroll
    for (int l = 0; l < LM; ++l) {
        if (l >= L) break;   // warp-uniform
        float v = S[l];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        v = __shfl_sync(0xffffffffu, v, 0);
        if (lane == l) mine = v;
    }
    return mine;
}

// Neighbour sums of variable i for lane's label: label-parallel for many
// labels, edge-parallel for few (LM > 0).
template <int LM>
__device__ __forceinline__ float neighbour_sum(const int *ptr, const int *col, const float *wt, const float *q,
                                               size_t base, int i, int lane, int L, int LP) {
    if constexpr (LM > 0)
        return gather_edges<LM>(ptr, col, wt, q, base, i, lane, L, LP);
    else
        return gather(ptr, col, wt, q, base, i, lane, LP);
}

template <bool SYM, int LM>
__global__ void __launch_bounds__(kST) sparse_step_kernel(const SparseStepLaunch a) {
    __shared__ double red[kSW];
    __shared__ int is_last;
    const int b = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int N = a.N, L = a.L, LP = a.LP;
    const size_t base = (size_t)b * N;
    const int vpw = sparse_vpw(N);
    const int i0 = (blockIdx.x * kSW + warp) * vpw;

    if (a.done != nullptr && a.done[b] != 0) {
        // stopping rule met: carry the state through unchanged
        for (int v = 0; v < vpw; ++v) {
            const int i = i0 + v;
            if (a.update && i < N && lane < LP) {
                const size_t o = (base + i) * LP + lane;
                a.s_out[o] = a.s_in[o];
                a.q_out[o] = a.q_in[o];
            }
        }
        return;
    }

    const bool live = lane < L;
    __shared__ float mus[kMaxLabels * kMaxLabels];
    for (int e = threadIdx.x; e < L * L; e += kST) mus[e] = a.mu[e];
    __syncthreads();
    const float eta = a.eta[b];
    float fh = 0.f, fl = 0.f;   // compensated sum of this lane's F terms
    for (int v = 0; v < vpw; ++v) {
        const int i = i0 + v;
        if (i >= N) break;
        const size_t o = (base + i) * LP + lane;
        // a1: neighbour sums and m_l = sum_k mu[l][k] S_k (+ sum_k mu[k][l] T_k)
        const float S = neighbour_sum<LM>(a.out_ptr, a.out_col, a.out_w, a.q_in, base, i, lane, L, LP);
        float m = 0.f;
        if constexpr (SYM) {
            for (int k = 0; k < L; ++k) {
                const float Sk = __shfl_sync(0xffffffffu, S, k);
                if (live) m = fmaf(mus[lane * L + k], Sk, m);
            }
        } else {
            const float T = neighbour_sum<LM>(a.in_ptr, a.in_col, a.in_w, a.q_in, base, i, lane, L, LP);
            for (int k = 0; k < L; ++k) {
                const float Sk = __shfl_sync(0xffffffffu, S, k);
                const float Tk = __shfl_sync(0xffffffffu, T, k);
                if (live) m = fmaf(mus[lane * L + k], Sk, fmaf(mus[k * L + lane], Tk, m));
            }
        }
        // a2-a4
        const float s = live ? a.s_in[o] : 0.f;
        const float u = live ? a.U[o] : 0.f;
        const float q = live ? a.q_in[o] : 0.f;
        {
            float se, ee;
            two_sum(fh, live ? q * (u + 0.5f * m + s) : 0.f, se, ee);
            fh = se;
            fl = __fadd_rn(fl, ee);
        }
        const float av = live ? fmaf(-eta, u + m, (1.f - eta) * s) : -INFINITY;
        float mx = av;
#pragma unroll
        for (int w = 16; w > 0; w >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, w));
        float z = live ? __expf(av - mx) : 0.f;
#pragma unroll
        for (int w = 16; w > 0; w >>= 1) z += __shfl_xor_sync(0xffffffffu, z, w);
        const float sn = av - mx - __logf(z);
        if (a.update && lane < LP) {
            a.s_out[o] = live ? sn : kPadLogQ;
            a.q_out[o] = live ? __expf(sn) : 0.f;
        }
    }
    // a5: F partial of the block, FP64, fixed order
    // double-float warp tree (FP64 is the narrow pipe), one FP64 value per warp
    const df fw = warp_sum_df(df_fast_two_sum(fh, fl));
    if (lane == 0) red[warp] = df_to(fw);
    __syncthreads();
    if (threadIdx.x == 0) {
        double bs = 0.0;
        for (int k = 0; k < kSW; ++k) bs += red[k];
        a.partial[(size_t)b * a.nblk + blockIdx.x] = bs;
        __threadfence();
        is_last = atomicAdd(a.counter + b, 1u) == (unsigned)(a.nblk - 1);
    }
    __syncthreads();
    if (!is_last) return;
    // last block of the instance: all threads reduce the partials, each a
    // fixed strided subset, then a fixed-shape tree
    __threadfence();
    double acc = 0.0;
    for (int k = threadIdx.x; k < a.nblk; k += kST) acc += __ldcg(a.partial + (size_t)b * a.nblk + k);
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, w);
    __syncthreads();   // red is reused
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double F = 0.0;
    for (int k = 0; k < kSW; ++k) F += red[k];
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

// max over variables of the summed |w| of the adjacency lists (for the
// step bound); scratch word as float bits (non-negative floats order as uints)
__global__ void sparse_degree_kernel(const int *ptr, const float *w, int N, unsigned *out_bits) {
    float best = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        float d = 0.f;
        for (int e = ptr[i]; e < ptr[i + 1]; ++e) d += fabsf(w[e]);
        best = fmaxf(best, d);
    }
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(best));
}

}  // namespace

int sparse_blocks(int N) { return (N + kSW * sparse_vpw(N) - 1) / (kSW * sparse_vpw(N)); }

cudaError_t launch_sparse_step(const SparseStepLaunch &a, cudaStream_t st) {
    dim3 grid(sparse_blocks(a.N), a.B);
    // up to 8 labels the lanes split the adjacency lists instead of the labels
    if (a.L <= 8) {
        if (a.sym)
            sparse_step_kernel<true, 8><<<grid, kST, 0, st>>>(a);
        else
            sparse_step_kernel<false, 8><<<grid, kST, 0, st>>>(a);
    } else {
        if (a.sym)
            sparse_step_kernel<true, 0><<<grid, kST, 0, st>>>(a);
        else
            sparse_step_kernel<false, 0><<<grid, kST, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_sparse_degree(const int *ptr, const float *w, int N, unsigned *out_bits, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out_bits, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    sparse_degree_kernel<<<std::min((N + 255) / 256, 1024), 256, 0, st>>>(ptr, w, N, out_bits);
    return cudaGetLastError();
}

}  // namespace proxmf
