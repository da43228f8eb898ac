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
// Layout and work split (GB300):
//  - HBM: pixel-major [B][N][LP] FP32, labels innermost and padded to LP (a
//    multiple of 4, or 2), so a pixel's state or unaries come in LP/4 128-bit
//    loads with immediate offsets and a warp covers one contiguous span;
//    weights [B][N][n_dirs] come in one vector load plus the entering edges.
//  - One thread per pixel, CTA tile of 32 x 8 pixels.  q = exp(log q) of the
//    tile plus a one-pixel halo (one halo pixel per thread) is staged in
//    shared memory with a per-pixel stride == 4 (mod 8) floats, so neighbour
//    reads are conflict-free 128-bit loads.
//  - mu is staged in shared memory as column pairs and read with broadcast
//    128-bit loads (keeping it in the parameter space, read through uniform
//    registers, is faster to run but makes ptxas take minutes per label
//    count); the L x L product, the neighbour sums and the element-wise update
//    use packed f32x2 FMAs (one instruction per two labels), with ceil(L/2)
//    independent accumulators.
//  - The FP32 form keeps the pixel's own log q in shared memory and loads
//    the unaries after the L x L product, so that three CTAs fit per SM
//    (measured 4.5 % faster than two CTAs holding both in registers).
//  - Free-energy partials are reduced per tile in FP64 and summed in a fixed
//    order -- by the next step of a loop (the deferred form below) or by the
//    last tile of each instance -- so F does not depend on scheduling or on
//    the other instances of the batch.
#pragma once

#include <cmath>

#include <cuda_bf16.h>

#include "f32x2.cuh"
#include "dfloat.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace proxmf {

// Symmetric mu with up to 21 labels travels in the kernel's parameter bank:
// the L x L product then takes mu as constant-bank operands of its FMAs
// instead of broadcast shared-memory loads, which the shared-memory pipe
// (the step's bottleneck) does not see (measured 14 % faster at L = 21).
constexpr int kMuParamLT = 21;
constexpr int kMuParam = kMuParamLT * 12;   // column pairs of LT = 21 (mu_pair_slots(21) = 12)
template <int LT, bool SYM, bool TC, int RULE>
__host__ __device__ constexpr bool mu_in_params() {
    return SYM && !TC && RULE == 0 && LT <= kMuParamLT;
}

struct GridStepArgs {
    float2 mu_p[kMuParam];   // symmetric mu column pairs (see mu_in_params)
    const float *adapt_d;    // [B] adaptive binary step (null: fixed eta); Adam: d0 per instance
    float *mom, *vv;         // momentum / Adam state [B][N][LP]
    float gamma1, gamma2, eps;
    int rule_first;
    const uint4 *mu_tc;      // tensor-core form: BF16 images of mu (and mu^T), see tc_k
    const float *s_in;
    float *s_out;
    const float *U;
    const float *w;
    const float *eta;
    const float2 *mu_out;    // device [LT][NPP] column pairs
    const float2 *mu_in;     // device [LT][NPP] row pairs
    double *partial;
    unsigned int *counter;
    double *f_trace;
    double *f_cur;
    int *done;
    int *status;
    int L, H, W;
    int nbx, nblk;
    int t, trace_cap, update;
    double rel_tol;
    size_t pslot;            // B * nblk * kMaxFParts: offset of the second slot of partial
    int defer, prev_pending; // deferred free energy: partials per tile (see GridStepLaunch)
};

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Shared-memory pixel stride: >= LP floats and == 4 (mod 8), so that eight
// threads reading 16 bytes each at consecutive pixels hit disjoint banks
// (LP = 2 uses 8-byte accesses and a dense stride).
__host__ __device__ constexpr int tile_stride(int LP) { return LP == 2 ? 2 : LP + ((4 - LP % 8) + 8) % 8; }

// Load LP floats of one pixel from HBM as float2 pairs.
template <int LP>
__device__ __forceinline__ void load_px(float2 (&v)[LP / 2], const float *p) {
    if constexpr (LP == 2) {
        v[0] = __ldg(reinterpret_cast<const float2 *>(p));
    } else {
#pragma unroll
        for (int i = 0; i < LP / 4; ++i) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(p) + i);
            v[2 * i] = make_float2(t.x, t.y);
            v[2 * i + 1] = make_float2(t.z, t.w);
        }
    }
}

template <int LP>
__device__ __forceinline__ void store_px(float *p, const float2 (&v)[LP / 2]) {
    if constexpr (LP == 2) {
        *reinterpret_cast<float2 *>(p) = v[0];
    } else {
#pragma unroll
        for (int i = 0; i < LP / 4; ++i)
            reinterpret_cast<float4 *>(p)[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
    }
}

// Write q = exp(s) of one pixel into its tile cell.
template <int LP>
__device__ __forceinline__ void put_cell(float *c, const float2 (&s)[LP / 2]) {
    if constexpr (LP == 2) {
        *reinterpret_cast<float2 *>(c) = make_float2(__expf(s[0].x), __expf(s[0].y));
    } else {
#pragma unroll
        for (int i = 0; i < LP / 4; ++i)
            reinterpret_cast<float4 *>(c)[i] = make_float4(__expf(s[2 * i].x), __expf(s[2 * i].y),
                                                           __expf(s[2 * i + 1].x), __expf(s[2 * i + 1].y));
    }
}

// acc += w * q(cell) over the first NP label pairs of a staged pixel.
template <int NP>
__device__ __forceinline__ void acc_cell(float2 (&acc)[NP], const float *c, float w) {
    const float2 ww = splat2(w);
    if constexpr (NP == 1) {
        acc[0] = fma2(ww, *reinterpret_cast<const float2 *>(c), acc[0]);
    } else {
#pragma unroll
        for (int i = 0; i < (NP + 1) / 2; ++i) {
            const float4 t = reinterpret_cast<const float4 *>(c)[i];
            acc[2 * i] = fma2(ww, make_float2(t.x, t.y), acc[2 * i]);
            if (2 * i + 1 < NP) acc[2 * i + 1] = fma2(ww, make_float2(t.z, t.w), acc[2 * i + 1]);
        }
    }
}

// m += A S with A given as shared-memory pair columns: for every k,
// (m[2j], m[2j+1]) += A[k][j] * S_k, two pairs per broadcast 128-bit load.
template <int LT, int NP, int NPP>
__device__ __forceinline__ void pair_matvec(float2 (&m)[NP], const float2 *A, const float2 (&S)[NP]) {
#pragma unroll
    for (int k = 0; k < LT; ++k) {
        const float sk = (k & 1) ? S[k >> 1].y : S[k >> 1].x;
        const float2 ss = splat2(sk);
        const float4 *col = reinterpret_cast<const float4 *>(A + k * NPP);
#pragma unroll
        for (int i = 0; i < (NP + 1) / 2; ++i) {
            const float4 t = col[i];
            m[2 * i] = fma2(make_float2(t.x, t.y), ss, m[2 * i]);
            if (2 * i + 1 < NP) m[2 * i + 1] = fma2(make_float2(t.z, t.w), ss, m[2 * i + 1]);
        }
    }
}

// Tensor-core form of the L x L product (BF16 operands, FP32 accumulation):
// the neighbour sums S of a tile's 256 pixels form the A operand (two
// M = 128 halves, K = tc_k labels), mu the B operand (N = tc_k labels), and
// D = A B^T = (mu S)^T lands in TMEM, one pixel per lane.
// (tc_k, tc_sbo and the operand layout: internal.h)

struct TcTile {
    float *qt;               // q tile with halo (dynamic shared memory)
    uint8_t *A;              // [SYM ? 1 : 2][2 halves][128 x KP] BF16 operands
    const uint8_t *B;        // [SYM ? 1 : 2][KP x KP] BF16 mu, mu^T
    uint32_t tmem;           // 2 x KP FP32 columns
    uint64_t *bar;           // MMA completion
    int *status;
};

// One pixel's row of A (a tc_k-label BF16 vector) from FP32 label pairs.
template <int NP, int KP>
__device__ __forceinline__ void put_a_row(uint8_t *row, const float2 (&S)[NP]) {
#pragma unroll
    for (int c = 0; c < KP / 8; ++c) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int p = 4 * c + i;
            if (p < NP) {
                const __nv_bfloat162 v = __floats2bfloat162_rn(S[p].x, S[p].y);
                w[i] = *reinterpret_cast<const uint32_t *>(&v);
            } else {
                w[i] = 0u;
            }
        }
        *reinterpret_cast<uint4 *>(row + c * 128) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// One instance as seen by one tile: pointers already offset to the instance.
struct TileJob {
    const float *s_in;
    float *s_out;
    const float *U;
    const float *w;
    const float2 *mu_out;
    const float2 *mu_in;
    const float2 *mu_p;      // column pairs read by the L x L product when mu_in_params (parameter bank or global)
    float eta;
    float adapt_d;           // adaptive binary step parameter d (when adaptive)
    bool adaptive;
    // momentum / Adam state (RULE 1, 2): pixel-major like the log q
    float *mom, *vv;
    float gamma1, gamma2, eps, d0;
    bool first;              // first step of a run: no history yet
    int L, H, W;
    int update;
};

// One 32 x 8 tile of one instance: a1-a4 for its pixels (state written when
// j.update), and the tile's free-energy partial, returned in thread 0.
// All threads of the block must call it; it may be called repeatedly by a
// persistent block (shared memory is reused).
// With mu_in_params the L x L product reads mu from j.mu_p (the launch's
// parameter bank, or global memory for the serving step) instead of shared
// memory.
template <int LT, int CONN, bool SYM, bool TC = false, int RULE = 0>
__device__ __forceinline__ double grid_tile(const TileJob &j, int bx, int by, const TcTile *tcx = nullptr) {
    constexpr int LP = storage_labels(LT);           // floats per pixel in HBM
    constexpr int NP = (LT + 1) / 2;                 // label pairs in the arithmetic
    constexpr int NPP = (NP + 1) / 2 * 2;            // pair slots per mu column
    constexpr int ND = CONN == 8 ? 4 : 2;
    constexpr int LS = tile_stride(LP);
    constexpr int TW = GX + 2;                       // tile width with halo
    constexpr int HALO = 2 * TW + 2 * GY;            // halo pixels of a tile
    constexpr bool MASK = (LT == LP);                // runtime L may be < LT
    static_assert(HALO <= GT, "one halo pixel per thread");
    static_assert(2 * NP <= LP, "pairs fit in the stored labels");
    __shared__ __align__(16) float qt_s[TC ? 4 : (GY + 2) * TW * LS];
    __shared__ __align__(16) float sown[TC ? 4 : GT * LS];
    __shared__ __align__(16) float2 mus[SYM ? 1 : 2][TC ? 2 : LT * NPP];
    float *qt = TC ? tcx->qt : qt_s;
    __shared__ double red[GT / 32];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * GX + tx;
    const int x0 = bx * GX, y0 = by * GY;
    const int x = x0 + tx, y = y0 + ty;
    const int H = j.H, W = j.W, L = j.L;
    const bool inside = (x < W) && (y < H);
    const size_t p = (size_t)y * W + x;
    const float *sin = j.s_in;
    __syncthreads();   // shared memory of a previous tile is no longer read

    constexpr bool kParamMu = mu_in_params<LT, SYM, TC, RULE>();
    // mu pairs into shared memory
    for (int i = tid; !TC && !kParamMu && i < LT * NPP; i += GT) {
        mus[0][i] = j.mu_out[i];
        if (!SYM) mus[SYM ? 0 : 1][i] = j.mu_in[i];
    }

    // own log q
    float2 s[LP / 2];
    if (inside) {
        load_px<LP>(s, sin + p * LP);
    } else {
#pragma unroll
        for (int i = 0; i < LP / 2; ++i) s[i] = splat2(kPadLogQ);
    }

    // one halo pixel per thread for the first HALO threads; 0 off the image
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
        const int gy = y0 - 1 + hr, gx = x0 - 1 + hc;
        float2 h[LP / 2];
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            load_px<LP>(h, sin + ((size_t)gy * W + gx) * LP);
        } else {
#pragma unroll
            for (int i = 0; i < LP / 2; ++i) h[i] = splat2(kPadLogQ);
        }
        put_cell<LP>(qt + (hr * TW + hc) * LS, h);
    }
    put_cell<LP>(qt + ((ty + 1) * TW + tx + 1) * LS, s);
    if constexpr (!TC) store_px<LP>(sown + tid * LS, s);

    // edge weights leaving this pixel, and entering it (stored at the pixel
    // that owns the edge)
    float wo[4] = {0.f, 0.f, 0.f, 0.f}, wi[4] = {0.f, 0.f, 0.f, 0.f};
    if (inside) {
        const float *wb = j.w;
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
    __syncthreads();

    // unaries: the FP32 form loads them after the L x L product
    float2 u[LP / 2];
    if (TC) {
        if (inside) {
            load_px<LP>(u, j.U + p * LP);
        } else {
#pragma unroll
            for (int i = 0; i < LP / 2; ++i) u[i] = splat2(0.f);
        }
    }

    const float *c_r = qt + ((ty + 1) * TW + tx + 2) * LS;
    const float *c_d = qt + ((ty + 2) * TW + tx + 1) * LS;
    const float *c_dr = qt + ((ty + 2) * TW + tx + 2) * LS;
    const float *c_dl = qt + ((ty + 2) * TW + tx) * LS;
    const float *c_l = qt + ((ty + 1) * TW + tx) * LS;
    const float *c_u = qt + (ty * TW + tx + 1) * LS;
    const float *c_ul = qt + (ty * TW + tx) * LS;
    const float *c_ur = qt + (ty * TW + tx + 2) * LS;

    // a1: neighbour sums and the L x L product, m = mu S_out + mu^T S_in
    float2 m[NP], S[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        m[j] = splat2(0.f);
        S[j] = splat2(0.f);
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
    if constexpr (!TC) {
        if constexpr (kParamMu)
            pair_matvec<LT, NP, NPP>(m, j.mu_p, S);
        else
            pair_matvec<LT, NP, NPP>(m, mus[0], S);
        if (!SYM) {
#pragma unroll
            for (int j = 0; j < NP; ++j) S[j] = splat2(0.f);
            acc_cell<NP>(S, c_l, wi[0]);
            acc_cell<NP>(S, c_u, wi[1]);
            if (CONN == 8) {
                acc_cell<NP>(S, c_ul, wi[2]);
                acc_cell<NP>(S, c_ur, wi[3]);
            }
            pair_matvec<LT, NP, NPP>(m, mus[SYM ? 0 : 1], S);
        }
    } else {
        constexpr int KP = tc_k(LT), SBO = tc_sbo(KP);
        constexpr int AHALF = 128 * KP * 2;        // bytes of one M = 128 operand
        const int half = tid >> 7, hrow = tid & 127;
        uint8_t *arow = tcx->A + half * AHALF + (hrow >> 3) * SBO + (hrow & 7) * 16;
        put_a_row<NP, KP>(arow, S);
        if (!SYM) {
#pragma unroll
            for (int j = 0; j < NP; ++j) S[j] = splat2(0.f);
            acc_cell<NP>(S, c_l, wi[0]);
            acc_cell<NP>(S, c_u, wi[1]);
            if (CONN == 8) {
                acc_cell<NP>(S, c_ul, wi[2]);
                acc_cell<NP>(S, c_ur, wi[3]);
            }
            put_a_row<NP, KP>(arow + 2 * AHALF, S);
        }
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_u32(tcx->A), b0 = tc::smem_u32(tcx->B);
            constexpr uint32_t idesc = tc::idesc_bf16(128, KP);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int ks = 0; ks < KP / 16; ++ks)
                    tc::mma_bf16(tcx->tmem + h * KP, tc::smem_desc(a0 + h * AHALF + ks * 256, 128, SBO, 0),
                                 tc::smem_desc(b0 + ks * 256, 128, SBO, 0), idesc, ks > 0 ? 1u : 0u);
                if (!SYM) {
#pragma unroll
                    for (int ks = 0; ks < KP / 16; ++ks)
                        tc::mma_bf16(tcx->tmem + h * KP,
                                     tc::smem_desc(a0 + 2 * AHALF + h * AHALF + ks * 256, 128, SBO, 0),
                                     tc::smem_desc(b0 + KP * KP * 2 + ks * 256, 128, SBO, 0), idesc, 1u);
                }
            }
            tc::mma_commit(tcx->bar);
        }
        __syncwarp();
        const bool ok = tc::mbar_wait(tcx->bar, 0, tcx->status);
        tc::fence_after_sync();
        float mm[KP];
        const uint32_t taddr = tcx->tmem + ((uint32_t)(((tid >> 5) & 3) * 32) << 16) + (uint32_t)(half * KP);
        if (ok) {
            if constexpr (KP == 32)
                tc::tmem_ld32(taddr, mm);
            else
                tc::tmem_ld16(taddr, mm);
        } else {
#pragma unroll
            for (int i = 0; i < KP; ++i) mm[i] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < NP; ++j) m[j] = make_float2(mm[2 * j], mm[2 * j + 1]);
    }

    if constexpr (!TC) {
        if (inside) {
            load_px<LP>(u, j.U + p * LP);
        } else {
#pragma unroll
            for (int i = 0; i < LP / 2; ++i) u[i] = splat2(0.f);
        }
        if constexpr (LP == 2) {
            s[0] = *reinterpret_cast<const float2 *>(sown + tid * LS);
        } else {
#pragma unroll
            for (int i = 0; i < LP / 4; ++i) {
                const float4 v = reinterpret_cast<const float4 *>(sown + tid * LS)[i];
                s[2 * i] = make_float2(v.x, v.y);
                s[2 * i + 1] = make_float2(v.z, v.w);
            }
        }
    }
    // a2-a3 and this pixel's free-energy term (q read back from the tile)
    float2 qc[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) qc[j] = splat2(0.f);
    acc_cell<NP>(qc, qt + ((ty + 1) * TW + tx + 1) * LS, 1.f);
    float eta = j.eta;
    if constexpr (LT == 2) {
        // adaptive binary step (Sec. 3.3, Eq. hessian): d_i = d q_i0 q_i1
        if (j.adaptive) eta = 1.f / fmaf(j.adapt_d * qc[0].x, qc[0].y, 1.f);
    }
    const float2 neta = splat2(-eta), ome = splat2(1.f - eta), half = splat2(0.5f);
    float2 f2 = splat2(0.f);
    float mx = -INFINITY;
    if constexpr (RULE == 0) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float2 g = add2(u[k], m[k]);
            const float2 h = add2(fma2(half, m[k], u[k]), s[k]);
            f2 = fma2(qc[k], h, f2);
            float2 av = fma2(neta, g, mul2(ome, s[k]));
            const int l0 = 2 * k, l1 = 2 * k + 1;
            if ((MASK && l0 >= L)) av.x = -INFINITY;
            if ((MASK && l1 >= L) || l1 >= LT) av.y = -INFINITY;
            s[k] = av;
            mx = fmaxf(mx, fmaxf(av.x, av.y));
        }
    } else if constexpr (RULE == 3) {
        // ADHOC (Sec. 2.2.2, Eq. related:parallel-update): damping of the mean
        // parameters, q' = (1 - eta) q + eta softmax(-g)
        float gmx = -INFINITY;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float2 g = add2(u[k], m[k]);
            const int l0 = 2 * k, l1 = 2 * k + 1;
            if (!(MASK && l0 >= L)) gmx = fmaxf(gmx, -g.x);
            if (!((MASK && l1 >= L) || l1 >= LT)) gmx = fmaxf(gmx, -g.y);
        }
        float zs = 0.f;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float2 g = add2(u[k], m[k]);
            const int l0 = 2 * k, l1 = 2 * k + 1;
            if (!(MASK && l0 >= L)) zs += __expf(-g.x - gmx);
            if (!((MASK && l1 >= L) || l1 >= LT)) zs += __expf(-g.y - gmx);
        }
        const float izs = 1.f / zs;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float2 g = add2(u[k], m[k]);
            const float2 h = add2(fma2(half, m[k], u[k]), s[k]);
            f2 = fma2(qc[k], h, f2);
            const int l0 = 2 * k, l1 = 2 * k + 1;
            float2 av = make_float2(__logf(fmaf(1.f - eta, qc[k].x, eta * __expf(-g.x - gmx) * izs)),
                                    __logf(fmaf(1.f - eta, qc[k].y, eta * __expf(-g.y - gmx) * izs)));
            if ((MASK && l0 >= L)) av.x = -INFINITY;
            if ((MASK && l1 >= L) || l1 >= LT) av.y = -INFINITY;
            s[k] = av;
            mx = fmaxf(mx, fmaxf(av.x, av.y));
        }
    } else {
        // OURS-MOMENTUM (RULE 1, Sec. 3.4): the gradient is replaced by its
        // running average mo' = g1 mo + (1 - g1) g (mo' = g on the first step).
        // OURS-ADAM (RULE 2, Sec. 3.5): in addition eta per label from the
        // second moment v' = g2 v + (1 - g2) r^2 of the centred natural
        // gradient r = g + log q - mean(g + log q) (v = 1 at the start):
        // d = max(sqrt(v') d0 + eps - 1, 0), eta = 1/(1 + d).
        float2 mo[LP / 2], vo[LP / 2];
#pragma unroll
        for (int k = 0; k < LP / 2; ++k) {
            mo[k] = splat2(0.f);
            vo[k] = splat2(1.f);
        }
        if (inside && !j.first) {
            load_px<LP>(mo, j.mom + p * LP);
            if (RULE == 2) load_px<LP>(vo, j.vv + p * LP);
        }
        float mean = 0.f;
        if constexpr (RULE == 2) {
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float2 t = add2(add2(u[k], m[k]), s[k]);
                const int l0 = 2 * k, l1 = 2 * k + 1;
                if (!(MASK && l0 >= L)) mean += t.x;
                if (!((MASK && l1 >= L) || l1 >= LT)) mean += t.y;
            }
            mean /= (float)L;
        }
        const float2 g1 = splat2(j.gamma1), og1 = splat2(1.f - j.gamma1);
        const float2 g2 = splat2(j.gamma2), og2 = splat2(1.f - j.gamma2);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float2 g = add2(u[k], m[k]);
            const float2 h = add2(fma2(half, m[k], u[k]), s[k]);
            f2 = fma2(qc[k], h, f2);
            const float2 mn = j.first ? g : fma2(g1, mo[k], mul2(og1, g));
            const int l0 = 2 * k, l1 = 2 * k + 1;
            const bool dead0 = (MASK && l0 >= L), dead1 = (MASK && l1 >= L) || l1 >= LT;
            float2 av;
            if constexpr (RULE == 1) {
                av = fma2(neta, mn, mul2(ome, s[k]));
            } else {
                float2 r = add2(add2(g, s[k]), splat2(-mean));
                if (dead0) r.x = 0.f;
                if (dead1) r.y = 0.f;
                const float2 vn = fma2(g2, vo[k], mul2(og2, mul2(r, r)));
                const float d0 = fmaxf(fmaf(sqrtf(vn.x), j.d0, j.eps - 1.f), 0.f);
                const float d1 = fmaxf(fmaf(sqrtf(vn.y), j.d0, j.eps - 1.f), 0.f);
                const float e0 = 1.f / (1.f + d0), e1 = 1.f / (1.f + d1);
                av = make_float2(fmaf(-e0, mn.x, (1.f - e0) * s[k].x), fmaf(-e1, mn.y, (1.f - e1) * s[k].y));
                vo[k] = make_float2(dead0 ? 0.f : vn.x, dead1 ? 0.f : vn.y);
            }
            mo[k] = make_float2(dead0 ? 0.f : mn.x, dead1 ? 0.f : mn.y);
            if (dead0) av.x = -INFINITY;
            if (dead1) av.y = -INFINITY;
            s[k] = av;
            mx = fmaxf(mx, fmaxf(av.x, av.y));
        }
        if (j.update && inside) {
#pragma unroll
            for (int k = NP; k < LP / 2; ++k) mo[k] = vo[k] = splat2(0.f);
            store_px<LP>(j.mom + p * LP, mo);
            if (RULE == 2) store_px<LP>(j.vv + p * LP, vo);
        }
    }
    // a4: renormalise
    float z = 0.f;
#pragma unroll
    for (int k = 0; k < NP; ++k) z += __expf(s[k].x - mx) + __expf(s[k].y - mx);
    const float2 nlse = splat2(-(mx + __logf(z)));
    if (j.update && inside) {
        float2 o[LP / 2];
#pragma unroll
        for (int k = 0; k < LP / 2; ++k) {
            if (k < NP) {
                o[k] = add2(s[k], nlse);
                const int l0 = 2 * k, l1 = 2 * k + 1;
                if ((MASK && l0 >= L)) o[k].x = kPadLogQ;
                if ((MASK && l1 >= L) || l1 >= LT) o[k].y = kPadLogQ;
            } else {
                o[k] = splat2(kPadLogQ);
            }
        }
        store_px<LP>(j.s_out + p * LP, o);
    }

    // a5: F partial of this tile: double-float warp trees (FP64 is the narrow
    // pipe of this part), one FP64 value per warp, the warps in FP64
    const df fw = warp_sum_df(df{inside ? f2.x + f2.y : 0.f, 0.f});
    if ((tid & 31) == 0) red[tid >> 5] = df_to(fw);
    if constexpr (TC) tc::fence_before_sync();   // TMEM reads done before the block syncs
    __syncthreads();
    double bs = 0.0;
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < GT / 32; ++k) bs += red[k];
    }
    return bs;
}

// Dynamic shared memory of the tensor-core form: q tile, A and B operands.
template <int LT, bool SYM>
struct GridTcSmem {
    static constexpr int LP = storage_labels(LT), LS = tile_stride(LP), KP = tc_k(LT);
    static constexpr int QT = ((GY + 2) * (GX + 2) * LS * 4 + 1023) / 1024 * 1024;
    static constexpr int A = (SYM ? 1 : 2) * 2 * 128 * KP * 2;
    static constexpr int B = (SYM ? 1 : 2) * KP * KP * 2;
    static constexpr int NCOL = 2 * KP < 32 ? 32 : 2 * KP;   // TMEM columns (power of two)
    static constexpr int bytes = QT + A + B + 1024;           // + alignment slack
};

// a5, per instance: thread 0 of every tile publishes its tile's partial bs.
// In a loop (a.defer) that is all: the next step sums the slot.  Otherwise
// the last tile of instance b to arrive sums all partials in a fixed order
// (the result does not depend on scheduling), stores F, appends it to the
// trace and applies the stopping rule |F^t - F^{t-1}| <= rel_tol |F^t|
// (Sec. 3.1).  All NT threads of the block call it; red holds NT / 32 doubles.
template <int NT = GT>
__device__ __forceinline__ void grid_step_finish(const GridStepArgs &a, int b, double bs, double *red, int *is_last) {
    const int tid = threadIdx.y * GX + threadIdx.x;
    const int blk = blockIdx.y * a.nbx + blockIdx.x;
    if (a.defer) {
        // the next step (or the flush kernel) reduces this slot (one partial per tile)
        if (tid == 0) a.partial[(size_t)(a.t & 1) * a.pslot + (size_t)b * a.nblk + blk] = bs;
        return;
    }
    if (tid == 0) {
        a.partial[(size_t)b * a.nblk + blk] = bs;
        __threadfence();
        const unsigned prev = atomicAdd(a.counter + b, 1u);
        *is_last = (prev == (unsigned)(a.nblk - 1));
    }
    __syncthreads();
    if (!*is_last) return;
    // last tile of instance b: reduce all partials in a fixed order
    __threadfence();
    double acc = 0.0;
    for (int k = tid; k < a.nblk; k += NT) acc += __ldcg(a.partial + (size_t)b * a.nblk + k);
    acc = warp_sum_f64(acc);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        double F = 0.0;
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) F += red[k];
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

// Sum of the n partials of one instance by the whole block, in a fixed order
// (thread k takes k, k + NT, ...; warps in order), so that every block that
// sums them gets the same value.
template <int NT>
__device__ __forceinline__ double sum_partials(const double *p, int n, double *red) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    double acc = 0.0;
    for (int k = tid; k < n; k += NT) acc += __ldcg(p + k);
    acc = warp_sum_f64(acc);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    double F = 0.0;
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) F += red[k];
    __syncthreads();   // red is reused
    return F;
}

// F of step t_prev from its deferred partials: trace entry and F_cur (by the
// writer block), and the stopping rule |F - F_prev| <= rel_tol |F|, which
// every block that asks evaluates identically.
// Returns true when instance b stops after step t_prev.
template <int NT>
__device__ __forceinline__ bool deferred_f(const GridStepArgs &a, int b, int t_prev, int parts, bool writer,
                                           double *red) {
    const size_t n = (size_t)a.nblk * parts;   // partials of one instance, [nblk][parts]
    const double F = sum_partials<NT>(a.partial + (size_t)(t_prev & 1) * a.pslot + (size_t)b * n, (int)n, red);
    bool stop = false;
    if (a.done != nullptr && a.rel_tol > 0.0 && t_prev > 0 && t_prev - 1 < a.trace_cap) {
        const double Fp = a.f_trace[(size_t)b * a.trace_cap + t_prev - 1];
        stop = fabs(F - Fp) <= a.rel_tol * fabs(F);
    }
    if (writer && threadIdx.x == 0 && threadIdx.y == 0) {
        a.f_cur[b] = F;
        if (!isfinite(F)) atomicExch(a.status, -6);
        if (t_prev < a.trace_cap) a.f_trace[(size_t)b * a.trace_cap + t_prev] = F;
        if (stop) a.done[b] = t_prev + 1;
    }
    return stop;
}

// Start of a step after griddepcontrol.wait: true when instance b no longer
// updates (stopped before, or the pending F of step t - 1 meets the rule).
// The pending F is summed by tile (0, 0) alone when no stopping rule runs,
// else by every tile, each of which needs the decision.
// The block reads done[b] once (tile (0, 0) of this very launch may set it
// while other tiles read it), so every thread takes the same branch; the
// barrier also publishes the block's mbarrier initialisation.
template <int NT>
__device__ __forceinline__ bool grid_step_prologue(const GridStepArgs &a, int b, double *red) {
    __shared__ int done_b;
    if (threadIdx.x == 0 && threadIdx.y == 0) done_b = a.done != nullptr ? a.done[b] : 0;
    __syncthreads();
    if (done_b != 0) return true;
    if (!a.prev_pending) return false;
    const bool writer = blockIdx.x == 0 && blockIdx.y == 0;
    const bool decide = a.done != nullptr && a.rel_tol > 0.0;
    if (!writer && !decide) return false;
    return deferred_f<NT>(a, b, a.t - 1, a.prev_pending, writer, red);
}

// The pending F of the last step of a loop (block b: instance b).
__global__ void grid_f_flush_kernel(const __grid_constant__ GridStepArgs a);

template <int LT, int CONN, bool SYM, bool TC, int RULE = 0>
__global__ void __launch_bounds__(GT, (RULE == 2) ? 1 : ((LT >= 24 || RULE) ? 2 : 3))
grid_prox_step_kernel(const __grid_constant__ GridStepArgs a) {
    constexpr int LP = storage_labels(LT);
    __shared__ double red[GT / 32];
    __shared__ int is_last;
    const int b = blockIdx.z;
    const int tid = threadIdx.y * GX + threadIdx.x;
    const size_t N = (size_t)a.H * a.W;
    if (a.done != nullptr && a.done[b] != 0) {
        // This instance has met its stopping rule: carry the state through
        // unchanged so that the ping-pong parity stays the same for all.
        const int x = blockIdx.x * GX + threadIdx.x, y = blockIdx.y * GY + threadIdx.y;
        if (a.update && x < a.W && y < a.H) {
            const size_t p = (size_t)y * a.W + x;
            float2 v[LP / 2];
            load_px<LP>(v, a.s_in + ((size_t)b * N + p) * LP);
            store_px<LP>(a.s_out + ((size_t)b * N + p) * LP, v);
        }
        return;
    }
    TcTile tct{};
    if constexpr (TC) {
        using SM = GridTcSmem<LT, SYM>;
        extern __shared__ __align__(1024) uint8_t gsm[];
        __shared__ __align__(8) uint64_t bar;
        __shared__ uint32_t tmem_slot;
        uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gsm) + 1023) & ~(uintptr_t)1023);
        tct.qt = reinterpret_cast<float *>(base);
        tct.A = base + SM::QT;
        tct.B = tct.A + SM::A;
        for (int i = tid; i < SM::B / 16; i += GT) reinterpret_cast<uint4 *>(tct.A + SM::A)[i] = a.mu_tc[i];
        if (tid == 0) {
            tc::mbar_init(&bar, 1);
            tc::mbar_init_fence();
        }
        if (tid < 32) tc::tmem_alloc(&tmem_slot, SM::NCOL);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        tct.tmem = tmem_slot;
        tct.bar = &bar;
        tct.status = a.status;
    }
    TileJob j;
    j.s_in = a.s_in + (size_t)b * N * LP;
    j.s_out = a.s_out + (size_t)b * N * LP;
    j.U = a.U + (size_t)b * N * LP;
    j.w = a.w + (size_t)b * N * (CONN == 8 ? 4 : 2);
    j.mu_out = a.mu_out;
    j.mu_in = a.mu_in;
    j.eta = a.eta[b];
    j.mu_p = a.mu_p;
    j.adaptive = RULE == 0 && a.adapt_d != nullptr;
    j.adapt_d = j.adaptive ? a.adapt_d[b] : 0.f;
    j.mom = (RULE == 1 || RULE == 2) ? a.mom + (size_t)b * N * LP : nullptr;
    j.vv = RULE == 2 ? a.vv + (size_t)b * N * LP : nullptr;
    j.gamma1 = a.gamma1;
    j.gamma2 = a.gamma2;
    j.eps = a.eps;
    j.d0 = RULE == 2 ? a.adapt_d[b] : 0.f;
    j.first = a.rule_first != 0;
    j.L = a.L;
    j.H = a.H;
    j.W = a.W;
    j.update = a.update;
    const double bs = grid_tile<LT, CONN, SYM, TC, RULE>(j, blockIdx.x, blockIdx.y, &tct);
    if constexpr (TC) {
        // every thread's TMEM reads finished before the block sync inside grid_tile
        tc::fence_after_sync();
        if (tid < 32) tc::tmem_dealloc(tct.tmem, GridTcSmem<LT, SYM>::NCOL);
    }

    grid_step_finish(a, b, bs, red, &is_last);
}

}  // namespace proxmf

#include "grid_tma.cuh"
#include "grid_tma_tc.cuh"

namespace proxmf {

template <int LT, int CONN, bool SYM>
cudaError_t launch_grid_tc(const GridStepArgs &a, dim3 grid, dim3 block, cudaStream_t st) {
    constexpr int bytes = GridTcSmem<LT, SYM>::bytes;
    static SmemOptIn optin;   // once per device
    const cudaError_t attr = smem_optin(optin, grid_prox_step_kernel<LT, CONN, SYM, true>, bytes);
    if (attr != cudaSuccess) return attr;
    grid_prox_step_kernel<LT, CONN, SYM, true><<<grid, block, bytes, st>>>(a);
    return cudaGetLastError();
}

template <int LT, int CONN, bool SYM, int RULE>
cudaError_t launch_grid_rule(const GridStepArgs &a, dim3 grid, dim3 block, cudaStream_t st) {
    grid_prox_step_kernel<LT, CONN, SYM, false, RULE><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <int LT>
cudaError_t launch_grid_step_lt(const GridStepLaunch &l, cudaStream_t st) {
    GridStepArgs a;
    a.mu_out = l.mu_out;
    a.mu_in = l.mu_in;
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
    int nbx, nby;
    grid_tiles(l.H, l.W, &nbx, &nby);
    a.nbx = nbx;
    a.nblk = nbx * nby;
    a.t = l.t;
    a.trace_cap = l.trace_cap;
    a.update = l.update;
    a.rel_tol = l.rel_tol;
    a.pslot = (size_t)l.B * a.nblk * kMaxFParts;
    a.defer = l.defer;
    a.prev_pending = l.prev_pending;
    // only the TMA-staged kernels take the deferred free energy, each with
    // its own number of partials per tile
    if ((l.defer || l.prev_pending) && !(storage_labels(LT) >= 4 && grid_step_uses_tma(l)))
        return cudaErrorInvalidValue;
    if (l.defer && l.defer != grid_step_fparts(l)) return cudaErrorInvalidValue;
    if (l.prev_pending < 0 || l.prev_pending > kMaxFParts) return cudaErrorInvalidValue;
    a.mu_tc = l.mu_tc;
    a.adapt_d = l.adapt_d;
    if (l.mu_sym && LT <= kMuParamLT) {
        if (!l.mu_host) return cudaErrorInvalidValue;
        const int n = LT * mu_pair_slots(LT);
        for (int i = 0; i < kMuParam; ++i) a.mu_p[i] = i < n ? l.mu_host[i] : make_float2(0.f, 0.f);
    }
    a.mom = l.mom;
    a.vv = l.vv;
    a.gamma1 = l.gamma1;
    a.gamma2 = l.gamma2;
    a.eps = l.eps;
    a.rule_first = l.rule_first;
    dim3 grid(nbx, nby, l.B), block(GX, GY, 1);
    if (l.rule == 3) {
        if (l.conn == 8)
            return l.mu_sym ? launch_grid_rule<LT, 8, true, 3>(a, grid, block, st)
                            : launch_grid_rule<LT, 8, false, 3>(a, grid, block, st);
        return l.mu_sym ? launch_grid_rule<LT, 4, true, 3>(a, grid, block, st)
                        : launch_grid_rule<LT, 4, false, 3>(a, grid, block, st);
    }
    if (l.rule == 1 || l.rule == 2) {
        if (l.conn == 8) {
            if (l.rule == 1)
                return l.mu_sym ? launch_grid_rule<LT, 8, true, 1>(a, grid, block, st)
                                : launch_grid_rule<LT, 8, false, 1>(a, grid, block, st);
            return l.mu_sym ? launch_grid_rule<LT, 8, true, 2>(a, grid, block, st)
                            : launch_grid_rule<LT, 8, false, 2>(a, grid, block, st);
        }
        if (l.rule == 1)
            return l.mu_sym ? launch_grid_rule<LT, 4, true, 1>(a, grid, block, st)
                            : launch_grid_rule<LT, 4, false, 1>(a, grid, block, st);
        return l.mu_sym ? launch_grid_rule<LT, 4, true, 2>(a, grid, block, st)
                        : launch_grid_rule<LT, 4, false, 2>(a, grid, block, st);
    }
    if constexpr (storage_labels(LT) >= 4) {
        // BF16 form, symmetric mu: TMA-staged tiles with BF16 gather and unaries
        if (l.tc && l.mu_sym && l.U16 != nullptr && l.rule == 0 && l.adapt_d == nullptr) {
            using TG = GridTmaTcGeom<LT>;
            GridTmaTcMaps maps;
            const cudaError_t e = encode_grid_tc_maps(&maps, l, TG::LP, TG::CS, TG::C16, TG::UP);
            if (e != cudaSuccess) return e;
            return l.conn == 8 ? launch_grid_tma_tc<LT, 8>(maps, a, grid, st)
                               : launch_grid_tma_tc<LT, 4>(maps, a, grid, st);
        }
    }
    if (l.tc) {
        if (l.conn == 8)
            return l.mu_sym ? launch_grid_tc<LT, 8, true>(a, grid, block, st) : launch_grid_tc<LT, 8, false>(a, grid, block, st);
        return l.mu_sym ? launch_grid_tc<LT, 4, true>(a, grid, block, st) : launch_grid_tc<LT, 4, false>(a, grid, block, st);
    }
    if constexpr (storage_labels(LT) >= 4) {
        // fixed step, FP32: the TMA-staged tile (grid_tma.cuh)
        if (a.adapt_d == nullptr) {
            GridTmaMaps maps;
            const cudaError_t e = encode_grid_maps(&maps, l, storage_labels(LT), GridTmaGeom<LT>::CS);
            if (e != cudaSuccess) return e;
            if (l.conn == 8)
                return l.mu_sym ? launch_grid_tma<LT, 8, true>(maps, a, grid, block, st)
                                : launch_grid_tma<LT, 8, false>(maps, a, grid, block, st);
            return l.mu_sym ? launch_grid_tma<LT, 4, true>(maps, a, grid, block, st)
                            : launch_grid_tma<LT, 4, false>(maps, a, grid, block, st);
        }
    }
    if (l.conn == 8) {
        if (l.mu_sym)
            grid_prox_step_kernel<LT, 8, true, false><<<grid, block, 0, st>>>(a);
        else
            grid_prox_step_kernel<LT, 8, false, false><<<grid, block, 0, st>>>(a);
    } else {
        if (l.mu_sym)
            grid_prox_step_kernel<LT, 4, true, false><<<grid, block, 0, st>>>(a);
        else
            grid_prox_step_kernel<LT, 4, false, false><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace proxmf
