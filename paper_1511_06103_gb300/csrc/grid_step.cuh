// grid_step.cuh -- the fused parallel proximal mean-field step on a grid CRF.
//
// One launch performs one iteration of Eq. method:update_natural for every
// pixel of every instance, and the free energy of the state it reads:
//   a1  S_i = sum_{i->j} w_ij q_j ,  T_i = sum_{k->i} w_ki q_k        (neighbour sums)
//       m_i = mu S_i + mu^T T_i     (= mu (S_i + T_i) for symmetric mu)
//   a2  g_i = U_i + m_i  = grad E(q^t)_i                                  (Sec. 3.1)
//   a3  a_i = -eta g_i + (1 - eta) log q^t_i                             (Eq. fixedStepSize)
//   a4  log q^{t+1}_i = a_i - logsumexp(a_i)
//   a5  F(q^t) = sum_i q_i . (U_i + m_i / 2 + log q_i)                   (Eq. related:mf-objective)
// The identity in a5 holds because E is quadratic: the pairwise energy is
// half of sum_i q_i . m_i, each edge being seen from both ends.
//
// Layout: label-planar [B][L][H][P] FP32, so a warp (32 consecutive x of one
// row) reads one 128-byte line per label.  Each CTA stages exp(log q) of a
// (GY+2) x (GX+2) tile (one-pixel halo) and the weights it needs into shared
// memory; mu lives in the kernel's parameter space (constant bank), so the
// L x L product issues no loads.  Free-energy partials are reduced per tile in
// FP64 and finished by the last tile of each instance in a fixed order, so F
// does not depend on scheduling or on the other instances of the batch.
#pragma once

#include <cmath>

#include "internal.h"

namespace proxmf {

template <int LP>
struct GridStepArgs {
    const float *s_in;
    float *s_out;
    const float *U;
    const float *w;
    const float *eta;
    double *partial;
    unsigned int *counter;
    double *f_trace;
    double *f_cur;
    int *done;
    int *status;
    int L, H, W, P;
    int nbx, nblk;
    int t, trace_cap, update;
    double rel_tol;
    float mu[LP * LP];       // row-major, zero padded to LP x LP
};

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int LP, int CONN, bool SYM>
__global__ void __launch_bounds__(GT, (LP >= 24 || !SYM) ? 1 : 2)
grid_prox_step_kernel(const __grid_constant__ GridStepArgs<LP> a) {
    constexpr int ND = CONN == 8 ? 4 : 2;
    constexpr int HALO = 2 * (GX + 2) + 2 * GY;
    __shared__ float qs[LP][GY + 2][GX + 2];
    __shared__ float ws[ND][GY + 1][GX + 2];
    __shared__ double red[GT / 32];
    __shared__ int is_last;

    const int b = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * GX + tx;
    const int x0 = blockIdx.x * GX, y0 = blockIdx.y * GY;
    const int x = x0 + tx, y = y0 + ty;
    const int H = a.H, W = a.W, P = a.P, L = a.L;
    const bool inside = (x < W) && (y < H);
    const size_t plane = (size_t)H * P;
    const float *sin = a.s_in + (size_t)b * L * plane;
    const float *Ub = a.U + (size_t)b * L * plane;
    const float *wb = a.w + (size_t)b * ND * plane;
    const size_t pix = (size_t)y * P + x;

    if (a.done != nullptr && a.done[b] != 0) {
        // This instance has met its stopping rule: carry the state through
        // unchanged so that the ping-pong parity stays the same for all.
        if (a.update && inside)
            for (int l = 0; l < L; ++l) a.s_out[(size_t)b * L * plane + l * plane + pix] = sin[l * plane + pix];
        return;
    }

    // own state and unaries: coalesced, all loads issued before first use
    float s[LP], u[LP];
#pragma unroll
    for (int l = 0; l < LP; ++l) {
        if (l < L && inside) {
            s[l] = __ldg(sin + l * plane + pix);
            u[l] = __ldg(Ub + l * plane + pix);
        } else {
            s[l] = -1e30f;
            u[l] = 0.f;
        }
    }

    // halo of q = exp(log q); cells outside the image hold 0
    for (int idx = tid; idx < HALO * L; idx += GT) {
        const int l = idx / HALO;
        const int h = idx - l * HALO;
        int hy, hx;
        if (h < GX + 2) {
            hy = 0;
            hx = h;
        } else if (h < 2 * (GX + 2)) {
            hy = GY + 1;
            hx = h - (GX + 2);
        } else {
            const int k = h - 2 * (GX + 2);
            hy = 1 + (k >> 1);
            hx = (k & 1) ? GX + 1 : 0;
        }
        const int gy = y0 - 1 + hy, gx = x0 - 1 + hx;
        float v = 0.f;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = expf(__ldg(sin + l * plane + (size_t)gy * P + gx));
        qs[l][hy][hx] = v;
    }
    // weights of the edges leaving and entering this tile's pixels
    for (int idx = tid; idx < ND * (GY + 1) * (GX + 2); idx += GT) {
        const int k = idx / ((GY + 1) * (GX + 2));
        const int r = idx - k * ((GY + 1) * (GX + 2));
        const int hy = r / (GX + 2), hx = r - hy * (GX + 2);
        const int gy = y0 - 1 + hy, gx = x0 - 1 + hx;
        float v = 0.f;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = __ldg(wb + k * plane + (size_t)gy * P + gx);
        ws[k][hy][hx] = v;
    }
#pragma unroll
    for (int l = 0; l < LP; ++l) qs[l][ty + 1][tx + 1] = (l < L && inside) ? expf(s[l]) : 0.f;
    __syncthreads();

    // a1: weighted neighbour sums (out-going edges S, in-coming edges T)
    const float w_r = ws[0][ty + 1][tx + 1], w_d = ws[1][ty + 1][tx + 1];
    const float w_l = ws[0][ty + 1][tx], w_u = ws[1][ty][tx + 1];
    float w_dr = 0.f, w_dl = 0.f, w_ul = 0.f, w_ur = 0.f;
    if (CONN == 8) {
        w_dr = ws[2][ty + 1][tx + 1];
        w_dl = ws[3][ty + 1][tx + 1];
        w_ul = ws[2][ty][tx];
        w_ur = ws[3][ty][tx + 2];
    }
    float So[LP];
    float Si[SYM ? 1 : LP];
#pragma unroll
    for (int l = 0; l < LP; ++l) {
        float o = w_r * qs[l][ty + 1][tx + 2];
        o = fmaf(w_d, qs[l][ty + 2][tx + 1], o);
        float i = w_l * qs[l][ty + 1][tx];
        i = fmaf(w_u, qs[l][ty][tx + 1], i);
        if (CONN == 8) {
            o = fmaf(w_dr, qs[l][ty + 2][tx + 2], o);
            o = fmaf(w_dl, qs[l][ty + 2][tx], o);
            i = fmaf(w_ul, qs[l][ty][tx], i);
            i = fmaf(w_ur, qs[l][ty][tx + 2], i);
        }
        if (SYM) {
            So[l] = o + i;
        } else {
            So[l] = o;
            Si[SYM ? 0 : l] = i;
        }
    }

    // a2-a3 and the free-energy term of this pixel
    const float eta = a.eta[b];
    const float ome = 1.f - eta;
    float f = 0.f;
    float mx = -INFINITY;
#pragma unroll
    for (int l = 0; l < LP; ++l) {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < LP; ++k) {
            m = fmaf(a.mu[l * LP + k], So[k], m);
            if (!SYM) m = fmaf(a.mu[k * LP + l], Si[SYM ? 0 : k], m);
        }
        const float g = u[l] + m;
        const float ql = qs[l][ty + 1][tx + 1];
        if (l < L) f = fmaf(ql, u[l] + 0.5f * m + s[l], f);
        float av = fmaf(-eta, g, ome * s[l]);
        if (l >= L) av = -INFINITY;
        s[l] = av;
        mx = fmaxf(mx, av);
    }
    // a4: renormalise (log-sum-exp over labels held by this thread)
    float z = 0.f;
#pragma unroll
    for (int l = 0; l < LP; ++l)
        if (l < L) z += expf(s[l] - mx);
    const float lse = mx + logf(z);
    if (a.update && inside) {
        float *so = a.s_out + (size_t)b * L * plane;
#pragma unroll
        for (int l = 0; l < LP; ++l)
            if (l < L) so[l * plane + pix] = s[l] - lse;
    }

    // a5: F partial of this tile, FP64
    double fd = inside ? (double)f : 0.0;
    fd = warp_sum_f64(fd);
    if ((tid & 31) == 0) red[tid >> 5] = fd;
    __syncthreads();
    const int blk = blockIdx.y * a.nbx + blockIdx.x;
    if (tid == 0) {
        double bs = 0.0;
#pragma unroll
        for (int k = 0; k < GT / 32; ++k) bs += red[k];
        a.partial[(size_t)b * a.nblk + blk] = bs;
        __threadfence();
        const unsigned prev = atomicAdd(a.counter + b, 1u);
        is_last = (prev == (unsigned)(a.nblk - 1));
    }
    __syncthreads();
    if (!is_last) return;
    // last tile of instance b: reduce all partials in a fixed order
    __threadfence();
    double acc = 0.0;
    for (int k = tid; k < a.nblk; k += GT) acc += __ldcg(a.partial + (size_t)b * a.nblk + k);
    acc = warp_sum_f64(acc);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        double F = 0.0;
#pragma unroll
        for (int k = 0; k < GT / 32; ++k) F += red[k];
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

template <int LP>
cudaError_t launch_grid_step_bucket(const GridStepLaunch &l, cudaStream_t st) {
    GridStepArgs<LP> a;
    a.s_in = l.s_in;
    a.s_out = l.s_out;
    a.U = l.U;
    a.w = l.w;
    a.eta = l.eta;
    a.partial = l.partial;
    a.counter = l.counter;
    a.f_trace = l.f_trace;
    a.f_cur = l.f_cur;
    a.done = l.done;
    a.status = l.status;
    a.L = l.L;
    a.H = l.H;
    a.W = l.W;
    a.P = l.P;
    int nbx, nby;
    grid_tiles(l.H, l.W, &nbx, &nby);
    a.nbx = nbx;
    a.nblk = nbx * nby;
    a.t = l.t;
    a.trace_cap = l.trace_cap;
    a.update = l.update;
    a.rel_tol = l.rel_tol;
    for (int i = 0; i < LP * LP; ++i) a.mu[i] = 0.f;
    for (int i = 0; i < l.L; ++i)
        for (int k = 0; k < l.L; ++k) a.mu[i * LP + k] = l.mu_host[i * l.L + k];
    dim3 grid(nbx, nby, l.B), block(GX, GY, 1);
    if (l.conn == 8) {
        if (l.mu_sym)
            grid_prox_step_kernel<LP, 8, true><<<grid, block, 0, st>>>(a);
        else
            grid_prox_step_kernel<LP, 8, false><<<grid, block, 0, st>>>(a);
    } else {
        if (l.mu_sym)
            grid_prox_step_kernel<LP, 4, true><<<grid, block, 0, st>>>(a);
        else
            grid_prox_step_kernel<LP, 4, false><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace proxmf
