// dense_common.cuh -- pieces shared by the FP32 and tensor-core dense steps.
#pragma once

#include <cuda_bf16.h>

#include "internal.h"

namespace proxmf {

// Epilogue shared by the FP32 and tensor-core dense steps: S_i (LP label
// sums of row i, FP32) -> m_i = mu S_i, update, renormalise, store, F term.
// Returns this row's free-energy term (0 for rows >= N).
template <int LP>
__device__ __forceinline__ float dense_row_update(const float *S, const float *mus, int L, float eta,
                                                  const float *s_row, const float *u_row, float *so_row,
                                                  float *qo_row, __nv_bfloat16 *qt_col, size_t qt_stride,
                                                  bool update) {
    float m[LP], s[LP];
#pragma unroll
    for (int l = 0; l < LP; ++l) {
        float acc = 0.f;
        for (int k = 0; k < L; ++k) acc = fmaf(mus[l * kMaxLabels + k], S[k], acc);
        m[l] = acc;
        s[l] = l < L ? s_row[l] : kPadLogQ;
    }
    float f = 0.f, mx = -INFINITY;
    const float ome = 1.f - eta;
#pragma unroll
    for (int l = 0; l < LP; ++l) {
        if (l >= L) continue;
        const float u = u_row[l];
        const float q = __expf(s[l]);
        f = fmaf(q, fmaf(0.5f, m[l], u) + s[l], f);
        const float av = fmaf(-eta, u + m[l], ome * s[l]);
        s[l] = av;
        mx = fmaxf(mx, av);
    }
    float z = 0.f;
#pragma unroll
    for (int l = 0; l < LP; ++l)
        if (l < L) z += __expf(s[l] - mx);
    const float lse = mx + __logf(z);
    if (update) {
#pragma unroll
        for (int l = 0; l < LP; ++l) {
            const float o = l < L ? s[l] - lse : kPadLogQ;
            so_row[l] = o;
            const float q = l < L ? __expf(o) : 0.f;
            if (qo_row) qo_row[l] = q;
            if (qt_col && l < 32) qt_col[(size_t)l * qt_stride] = __float2bfloat16_rn(q);
        }
    }
    return f;
}

}  // namespace proxmf
