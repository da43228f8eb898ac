// f32x2.cuh -- packed FP32 pair arithmetic (PTX add/mul/fma .rn.f32x2, sm_100+).
// Each operation rounds every lane exactly like its scalar counterpart, so
// results are bit-identical to fmaf / __fadd_rn / __fmul_rn per component;
// the pair form halves the issued instructions of the element-wise work.
#pragma once

#include <cuda_runtime.h>

namespace proxmf {

__device__ __forceinline__ unsigned long long pk(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}

__device__ __forceinline__ float2 upk(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}

// a * b + c per lane
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(d);
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}

__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }

// Base-2 exponential and logarithm of the special-function unit, with
// subnormal results flushed to zero.  e^x = 2^(x log2 e) and
// ln z = log2(z) ln 2 are the change-of-base identities; the callers form
// x log2 e (or its packed pair) themselves.
constexpr float kLog2e = 1.44269504088896340736f;
constexpr float kLn2 = 0.69314718055994530942f;

__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_ftz(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// e^v per lane: one packed multiply, two base-2 exponentials.
__device__ __forceinline__ float2 exp2v(float2 v) {
    const float2 t = mul2(v, splat2(kLog2e));
    return make_float2(ex2_ftz(t.x), ex2_ftz(t.y));
}

}  // namespace proxmf
