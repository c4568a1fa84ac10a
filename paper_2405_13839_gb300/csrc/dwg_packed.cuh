// dwg_packed.cuh -- device helpers shared by the evaluation kernels: packed
// FP32x2 arithmetic (two queries per instruction), MUFU rsqrt/ex2, two-sum.
#pragma once

#include "dwg_internal.cuh"

namespace dwg {

// ---------------------------------------------------------------------------
// packed FP32x2 arithmetic (PTX ISA 8.6, sm_100 family and later)
// ---------------------------------------------------------------------------
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float rsqrt_mufu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_mufu(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ f2 rsqrt2(f2 v)
{
    float a, b;
    upk(v, a, b);
    return pk(rsqrt_mufu(a), rsqrt_mufu(b));
}
__device__ __forceinline__ f2 ex22(f2 v)
{
    float a, b;
    upk(v, a, b);
    return pk(ex2_mufu(a), ex2_mufu(b));
}
// lane-wise max (the clamp of the modified kernel: rho^2 = max(r^2, delta^2))
__device__ __forceinline__ f2 max2(f2 a, f2 b)
{
    float a0, a1, b0, b1;
    upk(a, a0, a1);
    upk(b, b0, b1);
    return pk(fmaxf(a0, b0), fmaxf(a1, b1));
}
// lane-wise: v where x >= t, else 0
__device__ __forceinline__ f2 keep_ge(f2 v, f2 x, f2 t)
{
    float v0, v1, x0, x1, t0, t1;
    upk(v, v0, v1);
    upk(x, x0, x1);
    upk(t, t0, t1);
    return pk(x0 >= t0 ? v0 : 0.f, x1 >= t1 ? v1 : 0.f);
}
// (hi, lo) += t with Knuth's two-sum, both lanes at once
__device__ __forceinline__ void two_sum_acc(f2 &hi, f2 &lo, f2 t)
{
    f2 s = add2(hi, t);
    f2 bb = sub2(s, hi);
    f2 e = add2(sub2(hi, sub2(s, bb)), sub2(t, bb));
    lo = add2(lo, e);
    hi = s;
}
__device__ __forceinline__ void two_sum1(float &hi, float &lo, float t)
{
    float s = __fadd_rn(hi, t);
    float bb = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(t, bb));
    lo = __fadd_rn(lo, e);
    hi = s;
}

}  // namespace dwg
