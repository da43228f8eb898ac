// grid_tma_tc.cuh -- the BF16 tensor-core grid step with TMA-staged tiles.
// Shares the staging helpers of the FP32 form (grid_tma.cuh).
#pragma once

#include <cuda.h>

namespace proxmf {

// ---------------------------------------------------------------------------
// BF16 tensor-core form with TMA-staged tiles (symmetric mu).
//
// Same step; the neighbour gather and the L x L product run on BF16 copies:
//   - U is held in BF16 (2 bytes per label instead of 4), state, update and
//     softmax stay FP32;
//   - each cell of the tile is converted once to a BF16 q cell, so the eight
//     neighbour reads of a pixel move half the bytes of the FP32 form;
//   - S (FP32 neighbour sums) is rounded to BF16 into the A operand of
//     tcgen05.mma (kind::f16, FP32 accumulation in TMEM); mu (BF16) is the B
//     operand; each thread reads its row of D = (mu S)^T back with tcgen05.ld.
// The log-q tile arrives as five FP32 boxes (the 32 x 8 interior, dense, and
// the two halo rows and two halo columns), so that the interior can take c and
// then log q' in place and leave with one TMA store.  The BF16 q tile is
// reused for the A operand once every neighbour read is done.

// BF16 cell of the tile: an odd number of 16-byte chunks (so eight threads
// reading 16 bytes at consecutive cells hit disjoint banks), >= LP labels.
__host__ __device__ constexpr int bf16_cell(int LP) {
    return ((LP + 7) / 8 % 2 == 1 ? (LP + 7) / 8 : (LP + 7) / 8 + 1) * 8;
}

template <int LT>
struct GridTmaTcGeom {
    static constexpr int LP = storage_labels(LT);
    static constexpr int CS = tile_stride(LP);
    static constexpr int C16 = bf16_cell(LP);
    static constexpr int UP = u16_pitch(LP);
    static constexpr int KP = tc_k(LT), SBO = tc_sbo(KP);
    static constexpr int AHALF = 128 * KP * 2;
    static constexpr int TW = GX + 2;
    static constexpr int al(int v, int a) { return (v + a - 1) / a * a; }
    static constexpr int INT_B = GY * GX * CS * 4;
    static constexpr int ROW_B = TW * CS * 4;
    static constexpr int COL_B = GY * CS * 4;
    static constexpr int U16_B = GY * GX * C16 * 2;
    static constexpr int Q16_B = (GY + 2) * TW * C16 * 2;
    static constexpr int INT = 0;
    static constexpr int TOP = al(INT + INT_B, 128);
    static constexpr int BOT = al(TOP + ROW_B, 128);
    static constexpr int LEFT = al(BOT + ROW_B, 128);
    static constexpr int RIGHT = al(LEFT + COL_B, 128);
    static constexpr int U16 = al(RIGHT + COL_B, 128);
    static constexpr int Q16 = al(U16 + U16_B, 1024);
    // the A operand lives over the halo and unary boxes, which the conversion
    // consumes, where it fits (else after the q tile)
    static constexpr bool A_OVER = U16 + U16_B - TOP >= 2 * AHALF;
    static constexpr int AOP = A_OVER ? TOP : al(Q16 + Q16_B, 1024);
    static constexpr int BOP = al(A_OVER ? Q16 + Q16_B : AOP + 2 * AHALF, 1024);
    static constexpr int B_B = KP * KP * 2;
    static constexpr int bytes = BOP + B_B + 1024;                          // + alignment slack
    static constexpr uint32_t TX = INT_B + 2 * ROW_B + 2 * COL_B + U16_B + B_B;   // copy bytes per tile
    static constexpr int NCOL = 2 * KP < 32 ? 32 : 2 * KP;                  // TMEM columns
    static constexpr int ctas = (3 * (bytes + 1024 + 1024) <= 227 * 1024) ? 3 : 2;
};

struct GridTmaTcMaps {
    CUtensorMap s_int;   // log q^t, box {CS, GX, GY, 1}
    CUtensorMap s_row;   // log q^t, box {CS, GX + 2, 1, 1}
    CUtensorMap s_col;   // log q^t, box {CS, 1, GY, 1}
    CUtensorMap U16;     // BF16 unaries [B][H][W][UP], box {C16, GX, GY, 1}
    CUtensorMap s_out;   // log q^{t+1}, box {CS, GX, GY, 1}
};

__device__ __forceinline__ float2 bf2_to_f2(uint32_t v) {
    return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
}

__device__ __forceinline__ uint32_t f2_to_bf2(float2 v) {
    const __nv_bfloat162 t = __floats2bfloat162_rn(v.x, v.y);
    return *reinterpret_cast<const uint32_t *>(&t);
}

// A BF16 cell of C16 labels from FP32 pairs (zero past NP2 pairs).
template <int NP2, int C16>
__device__ __forceinline__ void put_cell16(uint8_t *c, const float2 *v) {
#pragma unroll
    for (int i = 0; i < C16 / 8; ++i) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = (4 * i + j < NP2) ? f2_to_bf2(v[4 * i + j]) : 0u;
        reinterpret_cast<uint4 *>(c)[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// acc += w q(cell) over the first NP pairs of a BF16 cell.
template <int NP>
__device__ __forceinline__ void acc_cell16(float2 (&acc)[NP], const uint8_t *c, float w) {
    const float2 ww = splat2(w);
#pragma unroll
    for (int i = 0; i < (NP + 3) / 4; ++i) {
        const uint4 t = reinterpret_cast<const uint4 *>(c)[i];
        const uint32_t v[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (4 * i + j < NP) acc[4 * i + j] = fma2(ww, bf2_to_f2(v[j]), acc[4 * i + j]);
    }
}

// acc1 += w1 q(cell), acc2 += w2 q(cell) from one BF16 cell read.
template <int NP>
__device__ __forceinline__ void acc_cell16x2(float2 (&acc1)[NP], float2 (&acc2)[NP], const uint8_t *c, float w1,
                                             float w2) {
    const float2 a1 = splat2(w1), a2 = splat2(w2);
#pragma unroll
    for (int i = 0; i < (NP + 3) / 4; ++i) {
        const uint4 t = reinterpret_cast<const uint4 *>(c)[i];
        const uint32_t v[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (4 * i + j < NP) {
                const float2 f = bf2_to_f2(v[j]);
                acc1[4 * i + j] = fma2(a1, f, acc1[4 * i + j]);
                acc2[4 * i + j] = fma2(a2, f, acc2[4 * i + j]);
            }
    }
}

// The BF16 tensor-core step with two vertically adjacent pixels per thread
// (128 threads per 32 x 8 tile), as the FP32 two-pixel kernel does it: the
// pair's own q stay in registers (FP32) and serve as each other's vertical
// neighbour, the other ten cells are read once for both pixels, the halo is
// converted 21 cells per warp.  The pair's two rows of the A operand are
// placed so that both come back in the thread's own TMEM lane: row
// k * 128 + 32 * warp + lane for pixel k of the pair.
template <int LT, int CONN>
__global__ void __launch_bounds__(GT2, GridTmaTcGeom<LT>::ctas)
grid_tma2_tc_step_kernel(const __grid_constant__ GridTmaTcMaps maps, const __grid_constant__ GridStepArgs a) {
    using G = GridTmaTcGeom<LT>;
    constexpr int LP = G::LP, CS = G::CS, C16 = G::C16, KP = G::KP, TW = G::TW;
    constexpr int NP = (LT + 1) / 2;
    constexpr int ND = CONN == 8 ? 4 : 2;
    constexpr int HALO = 2 * TW + 2 * GY;             // 84 cells
    constexpr int HPW = (HALO + 3) / 4;               // 21 halo cells per warp
    constexpr bool MASK = (LT == LP);
    static_assert(LP >= 4 && LP % 4 == 0, "cells are whole 16-byte vectors");
    extern __shared__ __align__(1024) uint8_t tsm[];
    __shared__ __align__(8) uint64_t bars[2];         // TMA loads, MMA completion
    __shared__ uint32_t tmem_slot;
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
    uint8_t *base = tsm + ((1024u - (tc::smem_u32(tsm) & 1023u)) & 1023u);
    float *rint = reinterpret_cast<float *>(base + G::INT);
    float *rtop = reinterpret_cast<float *>(base + G::TOP);
    float *rbot = reinterpret_cast<float *>(base + G::BOT);
    float *rleft = reinterpret_cast<float *>(base + G::LEFT);
    float *rright = reinterpret_cast<float *>(base + G::RIGHT);
    uint8_t *u16 = base + G::U16;
    uint8_t *q16 = base + G::Q16;
    uint8_t *Aop = base + G::AOP;
    uint8_t *Bop = base + G::BOP;

    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::mbar_init_fence();
    }
    if (tid < 32) tc::tmem_alloc(&tmem_slot, G::NCOL);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    if (tid == 0) {
        // U and the BF16 image of mu (the B operand) do not depend on the previous step
        tc::mbar_expect_tx(&bars[0], G::TX);
        tma::load_4d(u16, &maps.U16, &bars[0], 0, x0, y0, b);
        tc::bulk_load(Bop, a.mu_tc, (uint32_t)G::B_B, &bars[0]);
    }
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
    if (tid == 0) {
        tma::load_4d(rint, &maps.s_int, &bars[0], 0, x0, y0, b);
        tma::load_4d(rtop, &maps.s_row, &bars[0], 0, x0 - 1, y0 - 1, b);
        tma::load_4d(rbot, &maps.s_row, &bars[0], 0, x0 - 1, y0 + GY, b);
        tma::load_4d(rleft, &maps.s_col, &bars[0], 0, x0 - 1, y0, b);
        tma::load_4d(rright, &maps.s_col, &bars[0], 0, x0 + GX, y0, b);
    }
    // the pending F of the previous step is summed while the tile is in flight
    const bool stopped = grid_step_prologue<GT2>(a, b, red);
    if (stopped) {
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
        if (tid == 0) tc::mbar_wait(&bars[0], 0, a.status);   // no copy into this CTA's memory outlives it
        __syncthreads();
        if (tid < 32) tc::tmem_dealloc(tmem, G::NCOL);
        return;
    }
    const float eta = a.eta[b];
    const float2 neta = splat2(-eta), ome = splat2(1.f - eta);
    const bool ok = tc::mbar_wait(&bars[0], 0, a.status);

    // halo cells -> BF16 q, HPW consecutive ones per warp
    if (tx < HPW && tw * HPW + tx < HALO) {
        const int h = tw * HPW + tx;
        const float *src;
        int hr, hc;
        if (h < TW) {
            hr = 0;
            hc = h;
            src = rtop + hc * CS;
        } else if (h < 2 * TW) {
            hr = GY + 1;
            hc = h - TW;
            src = rbot + hc * CS;
        } else {
            const int k = h - 2 * TW;
            hr = 1 + (k >> 1);
            hc = (k & 1) ? TW - 1 : 0;
            src = ((k & 1) ? rright : rleft) + (hr - 1) * CS;
        }
        float2 v[LP / 2];
        get_cell<LP>(v, src);
#pragma unroll
        for (int k = 0; k < LP / 2; ++k) v[k] = exp2v(v[k]);
        put_cell16<LP / 2, C16>(q16 + (hr * TW + hc) * C16 * 2, v);
    }
    // the two own cells: BF16 q for the neighbours, c in place, FP32 q kept
    float *c1c = rint + (2 * tw * GX + tx) * CS;
    float *c2c = c1c + GX * CS;
    float2 q1[NP], q2[NP];
    float f01, f02;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        float *cown = r == 0 ? c1c : c2c;
        float2 s[LP / 2], u[LP / 2], q[LP / 2], c[LP / 2];
        get_cell<LP>(s, cown);
        const uint4 *uc = reinterpret_cast<const uint4 *>(u16 + ((2 * tw + r) * GX + tx) * C16 * 2);
#pragma unroll
        for (int i = 0; i < LP / 8; ++i) {
            const uint4 t = uc[i];
            u[4 * i] = bf2_to_f2(t.x);
            u[4 * i + 1] = bf2_to_f2(t.y);
            u[4 * i + 2] = bf2_to_f2(t.z);
            u[4 * i + 3] = bf2_to_f2(t.w);
        }
        if constexpr (LP % 8 != 0) {
            const uint2 t = reinterpret_cast<const uint2 *>(uc)[LP / 4 - 1];
            u[LP / 2 - 2] = bf2_to_f2(t.x);
            u[LP / 2 - 1] = bf2_to_f2(t.y);
        }
        float2 acc = splat2(0.f);
#pragma unroll
        for (int k = 0; k < LP / 2; ++k) {
            q[k] = exp2v(s[k]);
            c[k] = fma2(neta, u[k], mul2(ome, s[k]));
            if (k < NP) {
                acc = fma2(q[k], add2(u[k], s[k]), acc);
                if (r == 0)
                    q1[k] = q[k];
                else
                    q2[k] = q[k];
            }
        }
        put_cell16<LP / 2, C16>(q16 + ((2 * tw + r + 1) * TW + tx + 1) * C16 * 2, q);
        set_cell<LP>(cown, c);
        if (r == 0)
            f01 = acc.x + acc.y;
        else
            f02 = acc.x + acc.y;
    }
    __syncthreads();

    // a1: neighbour sums (ten BF16 cells, each read once; the pair's own q in
    // FP32 registers), FP32 accumulation
    float2 S1[NP], S2[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        S1[k] = splat2(0.f);
        S2[k] = splat2(0.f);
    }
    {
        constexpr int R = TW * C16 * 2, C = C16 * 2;
        const uint8_t *r1 = q16 + ((2 * tw + 1) * TW + tx + 1) * C;   // (x, y1)
        const uint8_t *r0 = r1 - R, *r2 = r1 + R, *r3 = r2 + R;
        acc_regs<NP>(S1, q2, wo1[1]);
        acc_regs<NP>(S2, q1, wi2[1]);
        acc_cell16x2<NP>(S1, S2, r1 + C, wo1[0], CONN == 8 ? wi2[3] : 0.f);
        acc_cell16x2<NP>(S1, S2, r1 - C, wi1[0], CONN == 8 ? wi2[2] : 0.f);
        acc_cell16x2<NP>(S2, S1, r2 + C, wo2[0], CONN == 8 ? wo1[2] : 0.f);
        acc_cell16x2<NP>(S2, S1, r2 - C, wi2[0], CONN == 8 ? wo1[3] : 0.f);
        acc_cell16<NP>(S1, r0, wi1[1]);
        acc_cell16<NP>(S2, r3, wo2[1]);
        if (CONN == 8) {
            acc_cell16<NP>(S1, r0 - C, wi1[2]);
            acc_cell16<NP>(S1, r0 + C, wi1[3]);
            acc_cell16<NP>(S2, r3 + C, wo2[2]);
            acc_cell16<NP>(S2, r3 - C, wo2[3]);
        }
    }
    {
        const int lane_row = 32 * tw + tx;   // this thread's TMEM lane
        uint8_t *arow = Aop + (lane_row >> 3) * G::SBO + (lane_row & 7) * 16;
        put_a_row<NP, KP>(arow, S1);
        put_a_row<NP, KP>(arow + G::AHALF, S2);
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(Aop), b0 = tc::smem_u32(Bop);
        constexpr uint32_t idesc = tc::idesc_bf16(128, KP);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
#pragma unroll
            for (int ks = 0; ks < KP / 16; ++ks)
                tc::mma_bf16(tmem + hh * KP, tc::smem_desc(a0 + hh * G::AHALF + ks * 256, 128, G::SBO, 0),
                             tc::smem_desc(b0 + ks * 256, 128, G::SBO, 0), idesc, ks > 0 ? 1u : 0u);
        tc::mma_commit(&bars[1]);
    }
    __syncwarp();
    const bool okm = tc::mbar_wait(&bars[1], 0, a.status);
    tc::fence_after_sync();

    // a3-a4 per pixel from its row of D, log q' over the interior cells
    float fpair = 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        float2 m[NP];
        {
            float mm[KP];
            const uint32_t taddr = tmem + ((uint32_t)(32 * tw) << 16) + (uint32_t)(r * KP);
            if (okm) {
                if constexpr (KP == 32)
                    tc::tmem_ld32(taddr, mm);
                else
                    tc::tmem_ld16(taddr, mm);
            } else {
#pragma unroll
                for (int i = 0; i < KP; ++i) mm[i] = 0.f;
            }
#pragma unroll
            for (int k = 0; k < NP; ++k) m[k] = make_float2(mm[2 * k], mm[2 * k + 1]);
        }
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
    tc::fence_before_sync();   // TMEM reads done before the block syncs
    tc::fence_async_smem();    // the TMA store reads the interior cells
    const df fw = warp_sum_df(df{fpair, 0.f});
    if ((tid & 31) == 0) red[tid >> 5] = df_to(fw);
    __syncthreads();
    if (tid < 32) {
        // a wait that ran out: the copies and MMAs in flight get a second
        // bounded wait before the TMEM columns are freed
        if (tid == 0) {
            if (!ok) tc::mbar_wait(&bars[0], 0, a.status);
            if (!okm) tc::mbar_wait(&bars[1], 0, a.status);
        }
        __syncwarp();
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, G::NCOL);
    }
    double bs = 0.0;
    if (tid == 0) {
        if (a.update && ok && okm) {
            tma::store_4d(&maps.s_out, rint, 0, x0, y0, b);
            tma::commit();
        }
#pragma unroll
        for (int k = 0; k < GT2 / 32; ++k) bs += red[k];
    }
    grid_step_finish<GT2>(a, b, bs, red, &is_last);
    if (tid == 0 && a.update && ok && okm) tma::wait_read();
}

cudaError_t encode_grid_tc_maps(GridTmaTcMaps *m, const GridStepLaunch &l, int LP, int CS, int C16, int UP);

template <int LT, int CONN>
cudaError_t launch_grid_tma_tc(const GridTmaTcMaps &maps, const GridStepArgs &a, dim3 grid, cudaStream_t st) {
    constexpr int bytes = GridTmaTcGeom<LT>::bytes;
    static SmemOptIn optin;   // once per device
    const cudaError_t attr = smem_optin(optin, grid_tma2_tc_step_kernel<LT, CONN>, bytes);
    if (attr != cudaSuccess) return attr;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(GX, GY / 2, 1);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = st;
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, grid_tma2_tc_step_kernel<LT, CONN>, maps, a);
}

}  // namespace proxmf
