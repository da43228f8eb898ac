#pragma once

// dfloat.cuh -- double-float arithmetic on the FP32 pipe.
//
// FP64 issues at 2 lanes per clock per SM on this part against 128 for FP32,
// so sums and recurrences that need more than FP32 (the scalar Lanczos steps,
// the Sturm sequences, the free energy of the one-launch grid loop) are
// carried in double-float: a value is the unevaluated sum h + l of two floats
// with |l| <= ulp(h) / 2, about 48 significant bits.  The error-free
// transformations are Knuth's two-sum, Dekker's fast two-sum (|a| >= |b|)
// and the FMA form of Dekker's exact product; sums of products accumulate
// the rounding errors of the running sum in a second float (the compensated
// dot product of Ogita, Rump and Oishi, 2005).  The _rn intrinsics keep the
// compiler from contracting or reassociating these sequences.

namespace proxmf {

struct df {
    float h, l;
};

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// (s, e) with s = fl(a + b) and a + b = s + e exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ df df_from(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double df_to(df x) { return (double)x.h + (double)x.l; }

__device__ __forceinline__ df df_add(df x, df y) {
    float s, e;
    two_sum(x.h, y.h, s, e);
    return df_fast_two_sum(s, __fadd_rn(e, __fadd_rn(x.l, y.l)));
}

__device__ __forceinline__ df df_mul(df x, df y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return df_fast_two_sum(p, e);
}

// running compensated sum (sh, sl) += a * b
__device__ __forceinline__ void acc_prod(float &sh, float &sl, df a, df b) {
    const float p = __fmul_rn(a.h, b.h);
    float pe = __fmaf_rn(a.h, b.h, -p);
    pe = __fmaf_rn(a.h, b.l, pe);
    pe = __fmaf_rn(a.l, b.h, pe);
    float s, e;
    two_sum(sh, p, s, e);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(e, pe));
}

// running compensated sum (sh, sl) += w * b, w a float
__device__ __forceinline__ void acc_prod_f(float &sh, float &sl, float w, df b) {
    const float p = __fmul_rn(w, b.h);
    const float pe = __fmaf_rn(w, b.l, __fmaf_rn(w, b.h, -p));
    float s, e;
    two_sum(sh, p, s, e);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(e, pe));
}

__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const df u = {__shfl_down_sync(0xffffffffu, v.h, o), __shfl_down_sync(0xffffffffu, v.l, o)};
        v = df_add(v, u);
    }
    return v;
}

}  // namespace proxmf
