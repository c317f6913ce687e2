// Double-float ("df32") arithmetic: a value is an unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi)/2, about 48 significant bits.  Built from
// the error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and
// FMA-based TwoProd (the product's rounding error is fma(a, b, -a*b)).
// Every operation runs on the FP32 pipe.  Intrinsics with explicit rounding
// keep the compiler from contracting or reordering the error terms.
#pragma once

#include <cuda_runtime.h>

namespace rbffd {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) {
    df r;
    r.hi = hi;
    r.lo = lo;
    return r;
}

// s + e = a + b exactly.
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df_make(s, e);
}

// s + e = a + b exactly, given |a| >= |b| (or a == 0).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df_make(s, e);
}

// p + e = a * b exactly.
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return df_make(p, e);
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    float e = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, e);
    e = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df a) { return df_make(-a.hi, -a.lo); }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, e);
}

// a (double-float) times f (float).
__device__ __forceinline__ df df_mul_f(df a, float f) {
    df p = two_prod(a.hi, f);
    const float e = __fmaf_rn(a.lo, f, p.lo);
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }

// Compensated accumulator: sum of df terms kept as (s, c) with TwoSum on the
// leading parts; cheaper than df_add per term and as accurate for sums.
struct DfAcc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(df t) {
        const df u = two_sum(s, t.hi);
        s = u.hi;
        c = __fadd_rn(c, __fadd_rn(u.lo, t.lo));
    }
    __device__ __forceinline__ df value() const { return fast_two_sum(s, c); }
};

__device__ __forceinline__ df df_from_double(double v) {
    const float hi = __double2float_rn(v);
    const float lo = __double2float_rn(v - (double)hi);
    return df_make(hi, lo);
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// float2 storage of a df value (hi in .x, lo in .y): 8 bytes, like a double.
__device__ __forceinline__ df df_load(const float2* p) {
    const float2 v = *p;
    return df_make(v.x, v.y);
}
__device__ __forceinline__ df df_ldg(const float2* p) {
    const float2 v = __ldg(p);
    return df_make(v.x, v.y);
}
__device__ __forceinline__ void df_store(float2* p, df a) { *p = make_float2(a.hi, a.lo); }

__device__ __forceinline__ df df_shfl_xor(df a, int o, int width) {
    return df_make(__shfl_xor_sync(0xffffffffu, a.hi, o, width), __shfl_xor_sync(0xffffffffu, a.lo, o, width));
}

}  // namespace rbffd
