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
    CUtensorMap s_out2;  // log q^{t+1}, box {CS, GX, 2, 1}: the two rows of one warp
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
    extern __shared__ __align__(1024) uint8_t tsm[];
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
    // U and the edge weights do not change between steps: they are fetched
    // before the wait for the previous step; thread 0 requests both boxes
    // before anything else
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_init_fence();
        tc::mbar_expect_tx(&bar, (uint32_t)(G::QH * G::QW * CS * 4 + G::CBYTES));
        tma::load_4d(ct, &maps.U, &bar, 0, x0, y0, b);
        asm volatile("griddepcontrol.wait;" ::: "memory");
        tma::load_4d(qt, &maps.s_in, &bar, 0, x0 - 1, y0 - 1, b);
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
    // the pending F of the previous step is summed while the tile is in flight
    // (the prologue's barrier also publishes the mbarrier initialisation)
    if (grid_step_prologue<GT>(a, b, red)) {
        // stopped instance: carry the state through (keeps the ping-pong parity)
        if (a.update && inside) {
            float2 v[LP / 2];
            load_px<LP>(v, a.s_in + ((size_t)b * N + p) * LP);
            store_px<LP>(a.s_out + ((size_t)b * N + p) * LP, v);
        }
        // complete the barrier's transaction before the tile leaves
        if (tid == 0) tc::mbar_wait(&bar, 0, a.status);
        return;
    }
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

// m1 += A S1 and m2 += A S2 with A given as pair columns (see pair_matvec):
// every pair of A is loaded once for both pixels.
template <int LT, int NP, int NPP>
__device__ __forceinline__ void pair_matvec2(float2 (&m1)[NP], float2 (&m2)[NP], const float2 *A,
                                             const float2 (&S1)[NP], const float2 (&S2)[NP]) {
#pragma unroll
    for (int k = 0; k < LT; ++k) {
        const float2 s1 = splat2((k & 1) ? S1[k >> 1].y : S1[k >> 1].x);
        const float2 s2 = splat2((k & 1) ? S2[k >> 1].y : S2[k >> 1].x);
        const float4 *col = reinterpret_cast<const float4 *>(A + k * NPP);
#pragma unroll
        for (int i = 0; i < (NP + 1) / 2; ++i) {
            const float4 t = col[i];
            const float2 lo = make_float2(t.x, t.y), hi = make_float2(t.z, t.w);
            m1[2 * i] = fma2(lo, s1, m1[2 * i]);
            m2[2 * i] = fma2(lo, s2, m2[2 * i]);
            if (2 * i + 1 < NP) {
                m1[2 * i + 1] = fma2(hi, s1, m1[2 * i + 1]);
                m2[2 * i + 1] = fma2(hi, s2, m2[2 * i + 1]);
            }
        }
    }
}

// acc1 += w1 q(cell), acc2 += w2 q(cell): one cell read for two pixels.
template <int NP>
__device__ __forceinline__ void acc_cell2(float2 (&acc1)[NP], float2 (&acc2)[NP], const float *c, float w1,
                                          float w2) {
    const float2 a = splat2(w1), b = splat2(w2);
#pragma unroll
    for (int i = 0; i < (NP + 1) / 2; ++i) {
        const float4 t = reinterpret_cast<const float4 *>(c)[i];
        const float2 lo = make_float2(t.x, t.y), hi = make_float2(t.z, t.w);
        acc1[2 * i] = fma2(a, lo, acc1[2 * i]);
        acc2[2 * i] = fma2(b, lo, acc2[2 * i]);
        if (2 * i + 1 < NP) {
            acc1[2 * i + 1] = fma2(a, hi, acc1[2 * i + 1]);
            acc2[2 * i + 1] = fma2(b, hi, acc2[2 * i + 1]);
        }
    }
}

// acc += w v over pairs held in registers.
template <int NP>
__device__ __forceinline__ void acc_regs(float2 (&acc)[NP], const float2 (&v)[NP], float w) {
    const float2 ww = splat2(w);
#pragma unroll
    for (int i = 0; i < NP; ++i) acc[i] = fma2(ww, v[i], acc[i]);
}

// The same step with two vertically adjacent pixels per thread (symmetric mu):
// 128 threads per 32 x 8 tile.  Of the twelve cells around a pixel pair, the
// pair's own two are in registers and the other ten are read once for both
// (instead of sixteen reads), every pair of mu is fetched once for both
// products, and the tile's 84 halo cells are converted 21 per warp, so no warp
// waits on another at the barrier that follows the conversion.
constexpr int GT2 = GX * GY / 2;   // threads of the two-pixel tile

template <int LT, int CONN>
__global__ void __launch_bounds__(GT2, GridTmaGeom<LT>::ctas)
grid_tma2_step_kernel(const __grid_constant__ GridTmaMaps maps, const __grid_constant__ GridStepArgs a) {
    using G = GridTmaGeom<LT>;
    constexpr int LP = G::LP, CS = G::CS, TW = G::QW;
    constexpr int NP = (LT + 1) / 2;
    constexpr int NPP = (NP + 1) / 2 * 2;
    constexpr int ND = CONN == 8 ? 4 : 2;
    constexpr int HALO = 2 * TW + 2 * GY;             // 84 cells
    constexpr int HPW = (HALO + 3) / 4;               // halo cells per warp
    constexpr bool MASK = (LT == LP);
    constexpr bool kParamMu = mu_in_params<LT, true, false, 0>();
    static_assert(LP >= 4 && LP % 4 == 0, "cells are whole 16-byte vectors");
    static_assert(HPW <= 32, "one halo cell per lane");
    extern __shared__ __align__(1024) uint8_t tsm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(16) float2 mus[kParamMu ? 2 : LT * NPP];
    __shared__ double red[GT2 / 32];
    __shared__ int is_last;

    const int b = blockIdx.z;
    const int tx = threadIdx.x, tw = threadIdx.y, tid = tw * GX + tx;
    const int x0 = blockIdx.x * GX, y0 = blockIdx.y * GY;
    const int x = x0 + tx, y1 = y0 + 2 * tw, y2 = y1 + 1;
    const int H = a.H, W = a.W, L = a.L;
    const size_t N = (size_t)H * W;
    const bool in1 = (x < W) && (y1 < H), in2 = (x < W) && (y2 < H);
    const size_t p1 = (size_t)y1 * W + x, p2 = p1 + W;
    uint8_t *base = tsm + ((128u - (tc::smem_u32(tsm) & 127u)) & 127u);
    float *qt = reinterpret_cast<float *>(base);              // [QH][QW][CS]: log q, then q
    float *ct = reinterpret_cast<float *>(base + G::COFF);   // [GY][GX][CS]: U, then c, then log q'

    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) {
        // both boxes are requested before anything else: U at once, log q as
        // soon as the previous step has finished
        tc::mbar_init(&bar, 1);
        tc::mbar_init_fence();
        tc::mbar_expect_tx(&bar, (uint32_t)(G::QH * G::QW * CS * 4 + G::CBYTES));
        tma::load_4d(ct, &maps.U, &bar, 0, x0, y0, b);
        asm volatile("griddepcontrol.wait;" ::: "memory");
        tma::load_4d(qt, &maps.s_in, &bar, 0, x0 - 1, y0 - 1, b);
    }
    for (int i = tid; !kParamMu && i < LT * NPP; i += GT2) mus[i] = a.mu_out[i];
    // weights of the edges leaving each pixel and entering it
    float wo1[4] = {0.f, 0.f, 0.f, 0.f}, wi1[4] = {0.f, 0.f, 0.f, 0.f};
    float wo2[4] = {0.f, 0.f, 0.f, 0.f}, wi2[4] = {0.f, 0.f, 0.f, 0.f};
    {
        const float *wb = a.w + (size_t)b * N * ND;
        if (in1) {
            if (ND == 4) {
                const float4 t = __ldg(reinterpret_cast<const float4 *>(wb + p1 * ND));
                wo1[0] = t.x;
                wo1[1] = t.y;
                wo1[2] = t.z;
                wo1[3] = t.w;
            } else {
                const float2 t = __ldg(reinterpret_cast<const float2 *>(wb + p1 * ND));
                wo1[0] = t.x;
                wo1[1] = t.y;
            }
            if (x > 0) wi1[0] = __ldg(wb + (p1 - 1) * ND + 0);
            if (y1 > 0) wi1[1] = __ldg(wb + (p1 - W) * ND + 1);
            if (CONN == 8) {
                if (x > 0 && y1 > 0) wi1[2] = __ldg(wb + (p1 - W - 1) * ND + 2);
                if (x + 1 < W && y1 > 0) wi1[3] = __ldg(wb + (p1 - W + 1) * ND + 3);
            }
        }
        if (in2) {
            if (ND == 4) {
                const float4 t = __ldg(reinterpret_cast<const float4 *>(wb + p2 * ND));
                wo2[0] = t.x;
                wo2[1] = t.y;
                wo2[2] = t.z;
                wo2[3] = t.w;
            } else {
                const float2 t = __ldg(reinterpret_cast<const float2 *>(wb + p2 * ND));
                wo2[0] = t.x;
                wo2[1] = t.y;
            }
            if (x > 0) wi2[0] = __ldg(wb + (p2 - 1) * ND + 0);
            wi2[1] = wo1[1];   // the edge (x, y1) -> (x, y2)
            if (CONN == 8) {
                if (x > 0) wi2[2] = __ldg(wb + (p2 - W - 1) * ND + 2);
                if (x + 1 < W) wi2[3] = __ldg(wb + (p2 - W + 1) * ND + 3);
            }
        }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // the pending F of the previous step is summed while the tile is in flight
    // (the prologue's barrier also publishes the mbarrier initialisation)
    if (grid_step_prologue<GT2>(a, b, red)) {
        if (a.update) {
            float2 v[LP / 2];
            if (in1) {
                load_px<LP>(v, a.s_in + ((size_t)b * N + p1) * LP);
                store_px<LP>(a.s_out + ((size_t)b * N + p1) * LP, v);
            }
            if (in2) {
                load_px<LP>(v, a.s_in + ((size_t)b * N + p2) * LP);
                store_px<LP>(a.s_out + ((size_t)b * N + p2) * LP, v);
            }
        }
        if (tid == 0) tc::mbar_wait(&bar, 0, a.status);
        return;
    }
    const float eta = a.eta[b];
    const float2 neta = splat2(-eta), ome = splat2(1.f - eta);
    const bool ok = tc::mbar_wait(&bar, 0, a.status);

    // halo cells, HPW consecutive ones per warp
    if (tx < HPW && tw * HPW + tx < HALO) {
        const int h = tw * HPW + tx;
        int hr, hc;
        if (h < TW) {
            hr = 0;
            hc = h;
        } else if (h < 2 * TW) {
            hr = GY + 1;
            hc = h - TW;
        } else {
            const int k = h - 2 * TW;
            hr = 1 + (k >> 1);
            hc = (k & 1) ? TW - 1 : 0;
        }
        float *c = qt + (hr * TW + hc) * CS;
        float2 v[LP / 2];
        get_cell<LP>(v, c);
#pragma unroll
        for (int k = 0; k < LP / 2; ++k) v[k] = exp2v(v[k]);
        set_cell<LP>(c, v);
    }
    // the two own cells: q (kept in registers), c and the unary-entropy part of F
    float *q1c = qt + ((2 * tw + 1) * TW + tx + 1) * CS;
    float *q2c = q1c + TW * CS;
    float *c1c = ct + (2 * tw * GX + tx) * CS;
    float *c2c = c1c + GX * CS;
    float2 q1[NP], q2[NP];
    float f01, f02;
    {
        float2 s[LP / 2], u[LP / 2], q[LP / 2], c[LP / 2];
        float2 acc = splat2(0.f);
        get_cell<LP>(s, q1c);
        get_cell<LP>(u, c1c);
#pragma unroll
        for (int k = 0; k < LP / 2; ++k) {
            q[k] = exp2v(s[k]);
            c[k] = fma2(neta, u[k], mul2(ome, s[k]));
            if (k < NP) {
                acc = fma2(q[k], add2(u[k], s[k]), acc);
                q1[k] = q[k];
            }
        }
        set_cell<LP>(q1c, q);
        set_cell<LP>(c1c, c);
        f01 = acc.x + acc.y;
        acc = splat2(0.f);
        get_cell<LP>(s, q2c);
        get_cell<LP>(u, c2c);
#pragma unroll
        for (int k = 0; k < LP / 2; ++k) {
            q[k] = exp2v(s[k]);
            c[k] = fma2(neta, u[k], mul2(ome, s[k]));
            if (k < NP) {
                acc = fma2(q[k], add2(u[k], s[k]), acc);
                q2[k] = q[k];
            }
        }
        set_cell<LP>(q2c, q);
        set_cell<LP>(c2c, c);
        f02 = acc.x + acc.y;
    }
    __syncthreads();

    // a1: neighbour sums (ten cells read, each once) and the two L x L products
    float2 m1[NP], m2[NP];
    {
        float2 S1[NP], S2[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            S1[k] = splat2(0.f);
            S2[k] = splat2(0.f);
        }
        const float *r1 = qt + ((2 * tw + 1) * TW + tx + 1) * CS;   // (x, y1)
        const float *r0 = r1 - TW * CS;                             // (x, y1 - 1)
        const float *r2 = r1 + TW * CS;                             // (x, y2)
        const float *r3 = r2 + TW * CS;                             // (x, y2 + 1)
        acc_regs<NP>(S1, q2, wo1[1]);                               // down of 1
        acc_regs<NP>(S2, q1, wi2[1]);                               // up of 2
        acc_cell2<NP>(S1, S2, r1 + CS, wo1[0], CONN == 8 ? wi2[3] : 0.f);   // (x+1, y1)
        acc_cell2<NP>(S1, S2, r1 - CS, wi1[0], CONN == 8 ? wi2[2] : 0.f);   // (x-1, y1)
        acc_cell2<NP>(S2, S1, r2 + CS, wo2[0], CONN == 8 ? wo1[2] : 0.f);   // (x+1, y2)
        acc_cell2<NP>(S2, S1, r2 - CS, wi2[0], CONN == 8 ? wo1[3] : 0.f);   // (x-1, y2)
        acc_cell<NP>(S1, r0, wi1[1]);                               // (x, y1-1)
        acc_cell<NP>(S2, r3, wo2[1]);                               // (x, y2+1)
        if (CONN == 8) {
            acc_cell<NP>(S1, r0 - CS, wi1[2]);                      // (x-1, y1-1)
            acc_cell<NP>(S1, r0 + CS, wi1[3]);                      // (x+1, y1-1)
            acc_cell<NP>(S2, r3 + CS, wo2[2]);                      // (x+1, y2+1)
            acc_cell<NP>(S2, r3 - CS, wo2[3]);                      // (x-1, y2+1)
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            m1[k] = splat2(0.f);
            m2[k] = splat2(0.f);
        }
        if constexpr (kParamMu)
            pair_matvec2<LT, NP, NPP>(m1, m2, a.mu_p, S1, S2);
        else
            pair_matvec2<LT, NP, NPP>(m1, m2, mus, S1, S2);
    }

    // a3-a4 per pixel, log q' over the unary cells; F of the pair
    float fpair = 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        float2 (&m)[NP] = r == 0 ? m1 : m2;
        const float2 (&q)[NP] = r == 0 ? q1 : q2;
        float *cc = r == 0 ? c1c : c2c;
        float2 c[LP / 2];
        get_cell<LP>(c, cc);
        float2 fm = splat2(0.f);
        float mx = -INFINITY;
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
        float2 z2 = splat2(0.f);
#pragma unroll
        for (int k = 0; k < NP; ++k) z2 = add2(z2, exp2v(add2(m[k], splat2(-mx))));
        const float2 nlse = splat2(-(mx + lg2_ftz(z2.x + z2.y) * kLn2));
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
        set_cell<LP>(cc, o);
        const bool in = r == 0 ? in1 : in2;
        if (in) fpair += (r == 0 ? f01 : f02) + 0.5f * (fm.x + fm.y);
    }
    tc::fence_async_smem();   // the TMA store reads these cells
    const df fw = warp_sum_df(df{fpair, 0.f});
    if (a.defer) {
        // in a step loop each warp leaves on its own: its two rows by one TMA
        // store, its F partial (summed by the next step), no block barrier
        __syncwarp();
        if (tx == 0) {
            if (a.update && ok) {
                tma::store_4d(&maps.s_out2, ct + 2 * tw * GX * CS, 0, x0, y0 + 2 * tw, b);
                tma::commit();
            }
            const size_t blk = (size_t)blockIdx.y * a.nbx + blockIdx.x;
            a.partial[(size_t)(a.t & 1) * a.pslot + ((size_t)b * a.nblk + blk) * a.defer + tw] = df_to(fw);
            if (a.update && ok) tma::wait_read();
        }
        return;
    }
    if ((tid & 31) == 0) red[tid >> 5] = df_to(fw);
    __syncthreads();
    double bs = 0.0;
    if (tid == 0) {
        if (a.update && ok) {
            tma::store_4d(&maps.s_out, ct, 0, x0, y0, b);
            tma::commit();
        }
#pragma unroll
        for (int k = 0; k < GT2 / 32; ++k) bs += red[k];
    }
    grid_step_finish<GT2>(a, b, bs, red, &is_last);
    if (tid == 0 && a.update && ok) tma::wait_read();
}

// Host side: the three tensor maps of one launch.  The state is read as a 4-D
// view [B][H][W][LP] (FP32); each box widens a cell to CS floats.
cudaError_t encode_grid_maps(GridTmaMaps *m, const GridStepLaunch &l, int LP, int CS);

template <int LT, int CONN, bool SYM>
cudaError_t launch_grid_tma(const GridTmaMaps &maps, const GridStepArgs &a, dim3 grid, dim3 block, cudaStream_t st) {
    constexpr int bytes = GridTmaGeom<LT>::bytes;
    // symmetric mu: two pixels per thread
    auto kern = SYM ? grid_tma2_step_kernel<LT, CONN> : grid_tma_step_kernel<LT, CONN, SYM>;
    if (SYM) block = dim3(GX, GY / 2, 1);
    static SmemOptIn optin;   // once per device
    const cudaError_t attr = smem_optin(optin, kern, bytes);
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
    return cudaLaunchKernelEx(&cfg, kern, maps, a);
}

}  // namespace proxmf
