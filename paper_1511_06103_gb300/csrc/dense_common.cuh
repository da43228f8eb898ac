// dense_common.cuh -- pieces shared by the FP32 and tensor-core dense steps.
#pragma once

#include <cuda_bf16.h>

#include "f32x2.cuh"
#include "internal.h"

namespace proxmf {

// mu^T in shared memory for dense_row_update: musT[k * kMaxLabels + l] =
// mu[l][k], zero outside L x L.  All threads of the block call it.
__device__ __forceinline__ void load_mu_transposed(float *musT, const float *mu, int L, int tid, int nthreads) {
    for (int i = tid; i < kMaxLabels * kMaxLabels; i += nthreads) {
        const int k = i / kMaxLabels, l = i % kMaxLabels;
        musT[i] = (k < L && l < L) ? mu[l * L + k] : 0.f;
    }
}

// LP floats of a row (16-byte vectors; 8-byte for LP = 2).
template <int LP>
__device__ __forceinline__ void load_row(float (&v)[LP], const float *p) {
    if constexpr (LP % 4 == 0) {
#pragma unroll
        for (int i = 0; i < LP / 4; ++i) {
            const float4 t = reinterpret_cast<const float4 *>(p)[i];
            v[4 * i] = t.x;
            v[4 * i + 1] = t.y;
            v[4 * i + 2] = t.z;
            v[4 * i + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < LP / 2; ++i) {
            const float2 t = reinterpret_cast<const float2 *>(p)[i];
            v[2 * i] = t.x;
            v[2 * i + 1] = t.y;
        }
    }
}

template <int LP>
__device__ __forceinline__ void store_row(float *p, const float (&v)[LP]) {
    if constexpr (LP % 4 == 0) {
#pragma unroll
        for (int i = 0; i < LP / 4; ++i)
            reinterpret_cast<float4 *>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < LP / 2; ++i) reinterpret_cast<float2 *>(p)[i] = make_float2(v[2 * i], v[2 * i + 1]);
    }
}

// Epilogue shared by the FP32 and tensor-core dense steps: S_i (LP label
// sums of row i, FP32; zero for labels >= L) -> m_i = mu S_i, update,
// renormalise, store, F term.  musT is mu^T (load_mu_transposed); m is summed
// over k in ascending order with one fused multiply-add per term, the padding
// labels adding exact zeros.  Returns this row's free-energy term.
template <int LP>
__device__ __forceinline__ float dense_row_update(const float *S, const float *musT, int L, float eta,
                                                  const float *s_row, const float *u_row, float *so_row,
                                                  float *qo_row, __nv_bfloat16 *qt_col, size_t qt_stride,
                                                  bool update) {
    constexpr int LQ = (LP + 3) / 4 * 4;   // label slots covered by 16-byte reads of musT
    float2 m2[LQ / 2];
#pragma unroll
    for (int j = 0; j < LQ / 2; ++j) m2[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < LP; ++k) {
        const float2 sk = splat2(S[k]);
        const float4 *col = reinterpret_cast<const float4 *>(musT + k * kMaxLabels);
#pragma unroll
        for (int i = 0; i < LQ / 4; ++i) {
            const float4 t = col[i];
            m2[2 * i] = fma2(make_float2(t.x, t.y), sk, m2[2 * i]);
            m2[2 * i + 1] = fma2(make_float2(t.z, t.w), sk, m2[2 * i + 1]);
        }
    }
    float s[LP], u[LP];
    load_row<LP>(s, s_row);
    load_row<LP>(u, u_row);
    float f = 0.f, mx = -INFINITY;
    const float ome = 1.f - eta;
#pragma unroll
    for (int l = 0; l < LP; ++l) {
        if (l >= L) continue;
        const float ml = (l & 1) ? m2[l >> 1].y : m2[l >> 1].x;
        const float q = __expf(s[l]);
        f = fmaf(q, fmaf(0.5f, ml, u[l]) + s[l], f);
        const float av = fmaf(-eta, u[l] + ml, ome * s[l]);
        s[l] = av;
        mx = fmaxf(mx, av);
    }
    float z = 0.f;
#pragma unroll
    for (int l = 0; l < LP; ++l)
        if (l < L) z += __expf(s[l] - mx);
    const float lse = mx + __logf(z);
    if (update) {
        float o[LP], qv[LP];
#pragma unroll
        for (int l = 0; l < LP; ++l) {
            o[l] = l < L ? s[l] - lse : kPadLogQ;
            qv[l] = l < L ? __expf(o[l]) : 0.f;
        }
        store_row<LP>(so_row, o);
        if (qo_row) store_row<LP>(qo_row, qv);
        if (qt_col) {
#pragma unroll
            for (int l = 0; l < LP && l < 32; ++l) qt_col[(size_t)l * qt_stride] = __float2bfloat16_rn(qv[l]);
        }
    }
    return f;
}

}  // namespace proxmf
