// df32.cuh -- a value held as an unevaluated sum hi + lo of two FP32 numbers,
// with arithmetic built only from FP32 operations through error-free
// transformations:
//   two_sum       Knuth (TAOCP vol. 2, 4.2.2): s + e == a + b exactly
//   fast_two_sum  Dekker (1971): same, when |a| >= |b|
//   two_prod      with a fused multiply-add: p + e == a * b exactly
// The compound operations below are the "sloppy" Dekker forms: their error is
// a small multiple of 2^-48 times the larger operand, which is what the inner
// sweeps of the mixed-precision solver need (FP32 storage alone cannot carry
// the partial products of high SRJ levels).  Compile without fast-math: the
// transformations rely on IEEE rounding and on the compiler not re-associating.
#pragma once

struct df32 {
    float hi, lo;
};

__device__ __forceinline__ df32 df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df32 df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ df32 df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
    const df32 s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df32 df_sub(df32 a, df32 b) {
    return df_add(a, df32{-b.hi, -b.lo});
}

__device__ __forceinline__ df32 df_add_f(df32 a, float b) {
    const df32 s = df_two_sum(a.hi, b);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df32 df_mul_f(df32 a, float b) {
    const df32 p = df_two_prod(a.hi, b);
    return df_fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

__device__ __forceinline__ double df_to_double(df32 a) {
    return (double)a.hi + (double)a.lo;
}
