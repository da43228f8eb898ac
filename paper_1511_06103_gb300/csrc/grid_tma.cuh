// grid_tma.cuh -- the FP32 grid step (fixed step size) with its tiles staged
// by the Tensor Memory Accelerator.
//
// Same iteration and free energy as grid_prox_step_kernel (grid_step.cuh):
//   a1  S_i = sum_{i->j} w_ij q_j , T_i = sum_{k->i} w_ki q_k ,  m_i = mu S_i + mu^T T_i
//   a2  g_i = U_i + m_i                                             (Sec. 3.1)
//   a3  a_i = -eta g_i + (1 - eta) log q_i                          (Eq. fixedStepSize)
//   a4  log q'_i = a_i - logsumexp(a_i)
//   a5  F(q) = sum_i q_i . (U_i + m_i / 2 + log q_i)                (Eq. related:mf-objective)
// with a3 and a5 regrouped around the only term that needs the neighbours:
//   c_i = -eta U_i + (1 - eta) log q_i ,  a_i = -eta m_i + c_i ,
//   F_i = q_i . (U_i + log q_i) + q_i . m_i / 2 .
// c_i and the first part of F_i are formed while the tile is converted to q,
// so the step after the L x L product is one FMA per label.
//
// Data movement (GB300): a pixel is LP floats (96 bytes at 21 labels) in
// HBM, so one thread per pixel reading its own 16-byte vectors makes every
// warp-wide load touch 24 cache lines for 512 useful bytes; that, not the
// arithmetic, bounded the per-thread-load form of the step.  Here one thread
// asks the TMA for two boxes of a 4-D view [B][H][W][LP]:
//   - log q of the 32 x 8 tile and its one-pixel halo (34 x 10 cells),
//   - U of the tile (32 x 8 cells),
// each cell widened to CS = tile_stride(LP) floats (the TMA fills the labels
// past LP with zeros), so that eight threads reading 16 bytes at consecutive
// cells hit disjoint shared-memory banks.  The TMA zero-fills cells outside
// the image: log q = 0 there gives q = 1, which only ever meets edge weights
// that are zero (edges leaving the image do not exist).  The tile's new log q
// is written over its U cells and leaves with one TMA store, which clips the
// cells and labels outside the image.  Edge weights are read directly: one
// 16-byte vector per pixel is already a coalesced warp load.
#pragma once

#include <cuda.h>

namespace proxmf {

struct GridTmaMaps {
    CUtensorMap s_in;    // log q^t, box {CS, GX + 2, GY + 2, 1}
    CUtensorMap U;       // unaries, box {CS, GX, GY, 1}
    CUtensorMap s_out;   // log q^{t+1}, box {CS, GX, GY, 1}
};

template <int LT>
struct GridTmaGeom {
    static constexpr int LP = storage_labels(LT);
    static constexpr int CS = tile_stride(LP);
    static constexpr int QW = GX + 2, QH = GY + 2;
    static constexpr int QBYTES = QH * QW * CS * 4;            // log q / q tile with halo
    static constexpr int COFF = (QBYTES + 127) / 128 * 128;
    static constexpr int CBYTES = GY * GX * CS * 4;            // U, then c, then log q'
    static constexpr int bytes = COFF + CBYTES + 128;          // + alignment slack
    // three CTAs per SM while they fit next to each other (21 labels and below)
    static constexpr int ctas = (3 * (bytes + 1024 + 8 * 1024) <= 227 * 1024) ? 3 : 2;
};

namespace tma {

__device__ __forceinline__ void load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                        int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];" ::"r"(tc::smem_u32(dst)),
        "l"((uint64_t)map), "r"(tc::smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

__device__ __forceinline__ void store_4d(const CUtensorMap *map, const void *src, int c0, int c1, int c2, int c3) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                     (uint64_t)map),
                 "r"(tc::smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}

__device__ __forceinline__ void commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until the committed bulk stores have finished reading shared memory.
__device__ __forceinline__ void wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

}  // namespace tma

// LP floats of one cell as pairs.
template <int LP>
__device__ __forceinline__ void get_cell(float2 (&v)[LP / 2], const float *c) {
#pragma unroll
    for (int i = 0; i < LP / 4; ++i) {
        const float4 t = reinterpret_cast<const float4 *>(c)[i];
        v[2 * i] = make_float2(t.x, t.y);
        v[2 * i + 1] = make_float2(t.z, t.w);
    }
}

template <int LP>
__device__ __forceinline__ void set_cell(float *c, const float2 (&v)[LP / 2]) {
#pragma unroll
    for (int i = 0; i < LP / 4; ++i)
        reinterpret_cast<float4 *>(c)[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
}

template <int LT, int CONN, bool SYM>
__global__ void __launch_bounds__(GT, GridTmaGeom<LT>::ctas)
grid_tma_step_kernel(const __grid_constant__ GridTmaMaps maps, const __grid_constant__ GridStepArgs a) {
    using G = GridTmaGeom<LT>;
    constexpr int LP = G::LP, CS = G::CS, TW = G::QW;
    constexpr int NP = (LT + 1) / 2;                 // label pairs in the arithmetic
    constexpr int NPP = (NP + 1) / 2 * 2;            // pair slots per mu column
    constexpr int ND = CONN == 8 ? 4 : 2;
    constexpr int HALO = 2 * TW + 2 * GY;
    constexpr bool MASK = (LT == LP);                // runtime L may be < LT
    constexpr bool kParamMu = mu_in_params<LT, SYM, false, 0>();
    static_assert(LP >= 4 && LP % 4 == 0, "cells are whole 16-byte vectors");
    static_assert(HALO <= GT, "one halo cell per thread");
    extern __shared__ __align__(128) uint8_t tsm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(16) float2 mus[SYM ? 1 : 2][kParamMu ? 2 : LT * NPP];
    __shared__ double red[GT / 32];
    __shared__ int is_last;

    const int b = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * GX + tx;
    const int x0 = blockIdx.x * GX, y0 = blockIdx.y * GY;
    const int x = x0 + tx, y = y0 + ty;
    const int H = a.H, W = a.W, L = a.L;
    const size_t N = (size_t)H * W;
    const bool inside = (x < W) && (y < H);
    const size_t p = (size_t)y * W + x;
    // 128-byte aligned start, by pointer arithmetic on the shared array (so
    // the compiler keeps shared-memory loads and stores)
    uint8_t *base = tsm + ((128u - (tc::smem_u32(tsm) & 127u)) & 127u);
    float *qt = reinterpret_cast<float *>(base);              // [QH][QW][CS]: log q, then q
    float *ct = reinterpret_cast<float *>(base + G::COFF);   // [GY][GX][CS]: U, then c, then log q'

    // The next step may be launched now (programmatic dependent launch): its
    // tiles take the SMs that this launch frees and wait below.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_init_fence();
    }
    __syncthreads();
    // U and the edge weights do not change between steps: they are fetched
    // before the wait for the previous step
    if (tid == 0) {
        tc::mbar_expect_tx(&bar, (uint32_t)(G::QH * G::QW * CS * 4 + G::CBYTES));
        tma::load_4d(ct, &maps.U, &bar, 0, x0, y0, b);
    }
    for (int i = tid; !kParamMu && i < LT * NPP; i += GT) {
        mus[0][i] = a.mu_out[i];
        if (!SYM) mus[SYM ? 0 : 1][i] = a.mu_in[i];
    }
    // edge weights leaving this pixel, and entering it (stored at the pixel
    // that owns the edge)
    float wo[4] = {0.f, 0.f, 0.f, 0.f}, wi[4] = {0.f, 0.f, 0.f, 0.f};
    if (inside) {
        const float *wb = a.w + (size_t)b * N * ND;
        if (ND == 4) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(wb + p * ND));
            wo[0] = t.x;
            wo[1] = t.y;
            wo[2] = t.z;
            wo[3] = t.w;
        } else {
            const float2 t = __ldg(reinterpret_cast<const float2 *>(wb + p * ND));
            wo[0] = t.x;
            wo[1] = t.y;
        }
        if (x > 0) wi[0] = __ldg(wb + (p - 1) * ND + 0);
        if (y > 0) wi[1] = __ldg(wb + (p - W) * ND + 1);
        if (CONN == 8) {
            if (x > 0 && y > 0) wi[2] = __ldg(wb + (p - W - 1) * ND + 2);
            if (x + 1 < W && y > 0) wi[3] = __ldg(wb + (p - W + 1) * ND + 3);
        }
    }
    // the previous step (when it was launched as a programmatic dependency)
    // has finished and its writes are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (a.done != nullptr && a.done[b] != 0) {
        // stopped instance: carry the state through (keeps the ping-pong parity)
        if (a.update && inside) {
            float2 v[LP / 2];
            load_px<LP>(v, a.s_in + ((size_t)b * N + p) * LP);
            store_px<LP>(a.s_out + ((size_t)b * N + p) * LP, v);
        }
        if (tid == 0) {
            // complete the barrier's transaction before the tile leaves
            tma::load_4d(qt, &maps.s_in, &bar, 0, x0 - 1, y0 - 1, b);
            tc::mbar_wait(&bar, 0, a.status);
        }
        return;
    }
    if (tid == 0) tma::load_4d(qt, &maps.s_in, &bar, 0, x0 - 1, y0 - 1, b);
    const float eta = a.eta[b];
    const float2 neta = splat2(-eta), ome = splat2(1.f - eta);
    const bool ok = tc::mbar_wait(&bar, 0, a.status);

    // conversion: halo cells to q; the own cell to q, c and its unary-entropy
    // part of F
    if (tid < HALO) {
        int hr, hc;
        if (tid < TW) {
            hr = 0;
            hc = tid;
        } else if (tid < 2 * TW) {
            hr = GY + 1;
            hc = tid - TW;
        } else {
            const int k = tid - 2 * TW;
            hr = 1 + (k >> 1);
            hc = (k & 1) ? TW - 1 : 0;
        }
        float *c = qt + (hr * TW + hc) * CS;
        float2 h[LP / 2];
        get_cell<LP>(h, c);
#pragma unroll
        for (int k = 0; k < LP / 2; ++k) h[k] = exp2v(h[k]);
        set_cell<LP>(c, h);
    }
    float *qown = qt + ((ty + 1) * TW + tx + 1) * CS;
    float *cown = ct + (ty * GX + tx) * CS;
    float f0;
    {
        float2 s[LP / 2], u[LP / 2], q[LP / 2], c[LP / 2];
        get_cell<LP>(s, qown);
        get_cell<LP>(u, cown);
        float2 acc = splat2(0.f);
#pragma unroll
        for (int k = 0; k < LP / 2; ++k) {
            q[k] = exp2v(s[k]);
            c[k] = fma2(neta, u[k], mul2(ome, s[k]));
            if (k < NP) acc = fma2(q[k], add2(u[k], s[k]), acc);
        }
        set_cell<LP>(qown, q);
        set_cell<LP>(cown, c);
        f0 = acc.x + acc.y;
    }
    __syncthreads();

    const float *c_r = qt + ((ty + 1) * TW + tx + 2) * CS;
    const float *c_d = qt + ((ty + 2) * TW + tx + 1) * CS;
    const float *c_dr = qt + ((ty + 2) * TW + tx + 2) * CS;
    const float *c_dl = qt + ((ty + 2) * TW + tx) * CS;
    const float *c_l = qt + ((ty + 1) * TW + tx) * CS;
    const float *c_u = qt + (ty * TW + tx + 1) * CS;
    const float *c_ul = qt + (ty * TW + tx) * CS;
    const float *c_ur = qt + (ty * TW + tx + 2) * CS;

    // a1: neighbour sums and the L x L product
    float2 m[NP], S[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        m[k] = splat2(0.f);
        S[k] = splat2(0.f);
    }
    acc_cell<NP>(S, c_r, wo[0]);
    acc_cell<NP>(S, c_d, wo[1]);
    if (CONN == 8) {
        acc_cell<NP>(S, c_dr, wo[2]);
        acc_cell<NP>(S, c_dl, wo[3]);
    }
    if (SYM) {
        acc_cell<NP>(S, c_l, wi[0]);
        acc_cell<NP>(S, c_u, wi[1]);
        if (CONN == 8) {
            acc_cell<NP>(S, c_ul, wi[2]);
            acc_cell<NP>(S, c_ur, wi[3]);
        }
    }
    if constexpr (kParamMu)
        pair_matvec<LT, NP, NPP>(m, a.mu_p, S);
    else
        pair_matvec<LT, NP, NPP>(m, mus[0], S);
    if (!SYM) {
#pragma unroll
        for (int k = 0; k < NP; ++k) S[k] = splat2(0.f);
        acc_cell<NP>(S, c_l, wi[0]);
        acc_cell<NP>(S, c_u, wi[1]);
        if (CONN == 8) {
            acc_cell<NP>(S, c_ul, wi[2]);
            acc_cell<NP>(S, c_ur, wi[3]);
        }
        pair_matvec<LT, NP, NPP>(m, mus[SYM ? 0 : 1], S);
    }

    // a3 with the pairwise half of F, a4, log q' over the U cell
    float2 fm = splat2(0.f);
    float mx = -INFINITY;
    {
        float2 q[LP / 2], c[LP / 2];
        get_cell<LP>(q, qown);
        get_cell<LP>(c, cown);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            fm = fma2(q[k], m[k], fm);
            float2 av = fma2(neta, m[k], c[k]);
            const int l0 = 2 * k, l1 = 2 * k + 1;
            if ((MASK && l0 >= L)) av.x = -INFINITY;
            if ((MASK && l1 >= L) || l1 >= LT) av.y = -INFINITY;
            m[k] = av;
            mx = fmaxf(mx, fmaxf(av.x, av.y));
        }
    }
    float2 z2 = splat2(0.f);
#pragma unroll
    for (int k = 0; k < NP; ++k) z2 = add2(z2, exp2v(add2(m[k], splat2(-mx))));
    const float2 nlse = splat2(-(mx + lg2_ftz(z2.x + z2.y) * kLn2));
    {
        float2 o[LP / 2];
#pragma unroll
        for (int k = 0; k < LP / 2; ++k) {
            if (k < NP) {
                o[k] = add2(m[k], nlse);
                const int l0 = 2 * k, l1 = 2 * k + 1;
                if ((MASK && l0 >= L)) o[k].x = kPadLogQ;
                if ((MASK && l1 >= L) || l1 >= LT) o[k].y = kPadLogQ;
            } else {
                o[k] = splat2(kPadLogQ);
            }
        }
        set_cell<LP>(cown, o);
    }
    tc::fence_async_smem();   // the TMA store reads these cells
    const df fw = warp_sum_df(df{inside ? f0 + 0.5f * (fm.x + fm.y) : 0.f, 0.f});
    if ((tid & 31) == 0) red[tid >> 5] = df_to(fw);
    __syncthreads();
    double bs = 0.0;
    if (tid == 0) {
        if (a.update && ok) {
            tma::store_4d(&maps.s_out, ct, 0, x0, y0, b);
            tma::commit();
        }
#pragma unroll
        for (int k = 0; k < GT / 32; ++k) bs += red[k];
    }
    grid_step_finish(a, b, bs, red, &is_last);
    if (tid == 0 && a.update && ok) tma::wait_read();
}

// Host side: the three tensor maps of one launch.  The state is read as a 4-D
// view [B][H][W][LP] (FP32); each box widens a cell to CS floats.
cudaError_t encode_grid_maps(GridTmaMaps *m, const GridStepLaunch &l, int LP, int CS);

template <int LT, int CONN, bool SYM>
cudaError_t launch_grid_tma(const GridTmaMaps &maps, const GridStepArgs &a, dim3 grid, dim3 block, cudaStream_t st) {
    constexpr int bytes = GridTmaGeom<LT>::bytes;
    static SmemOptIn optin;   // once per device
    const cudaError_t attr = smem_optin(optin, grid_tma_step_kernel<LT, CONN, SYM>, bytes);
    if (attr != cudaSuccess) return attr;
    // programmatic dependent launch: the step may start while the previous
    // kernel on the stream drains (the kernel waits before it reads the state)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = st;
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, grid_tma_step_kernel<LT, CONN, SYM>, maps, a);
}

}  // namespace proxmf
