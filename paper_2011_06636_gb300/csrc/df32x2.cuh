// df32x2.cuh -- two FP32 pairs side by side (df32.cuh's arithmetic on two
// values at once) for the packed FP32 instructions of sm_100 and later.
#pragma once

#include <cuda_runtime.h>

// Two FP32 pairs side by side (components x and y) for the packed FP32
// instructions of sm_100 and later: __fadd2_rn, __fmul2_rn and __ffma2_rn do
// one operation on both components in one instruction, each component
// rounded exactly as the scalar operation (a negated operand costs nothing).
// Every function below performs the operations of its scalar counterpart in
// the same order, so each component equals the scalar result bit for bit.
struct df2 {
    float2 hi, lo;
};

__device__ __forceinline__ float2 f2_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2_bcast(float a) { return make_float2(a, a); }

__device__ __forceinline__ df2 df2_two_sum(float2 a, float2 b) {
    const float2 s = __fadd2_rn(a, b);
    const float2 bb = __fadd2_rn(s, f2_neg(a));
    const float2 e = __fadd2_rn(__fadd2_rn(a, f2_neg(__fadd2_rn(s, f2_neg(bb)))),
                                __fadd2_rn(b, f2_neg(bb)));
    return df2{s, e};
}

// as df_q_vark, per component
template <int NQ>
__device__ __forceinline__ df2 df2_q_vark(const df2 *nb, const float2 *w, float2 invd, float2 f) {
    float2 sh = f, sl = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const float2 ph = __fmul2_rn(nb[q].hi, w[q]);
        const float2 pe = __ffma2_rn(nb[q].hi, w[q], f2_neg(ph));
        const float2 pl = __ffma2_rn(nb[q].lo, w[q], pe);
        const df2 sq = df2_two_sum(sh, ph);
        sh = sq.hi;
        sl = __fadd2_rn(sl, __fadd2_rn(sq.lo, pl));
    }
    const float2 mh = __fmul2_rn(sh, invd);
    const float2 me = __ffma2_rn(sh, invd, f2_neg(mh));
    return df2{mh, __ffma2_rn(sl, invd, me)};
}

// as df_q_axes, per component (a: the axis coefficients, the same for both)
template <int NA>
__device__ __forceinline__ df2 df2_q_axes(const df2 *nb, const float *a, float2 g) {
    float2 sh = g, sl = make_float2(0.f, 0.f);
#pragma unroll
    for (int ax = 0; ax < NA; ++ax) {
        const float2 aa = f2_bcast(a[ax]);
        const df2 s = df2_two_sum(nb[2 * ax].hi, nb[2 * ax + 1].hi);
        const float2 slo = __fadd2_rn(s.lo, __fadd2_rn(nb[2 * ax].lo, nb[2 * ax + 1].lo));
        const float2 ph = __fmul2_rn(s.hi, aa);
        const float2 pe = __ffma2_rn(s.hi, aa, f2_neg(ph));
        const float2 pl = __ffma2_rn(slo, aa, pe);
        const df2 q = df2_two_sum(sh, ph);
        sh = q.hi;
        sl = __fadd2_rn(sl, __fadd2_rn(q.lo, pl));
    }
    return df2{sh, sl};
}

// as df_relax_to, per component: u' = (1 - omega) u + omega q
__device__ __forceinline__ df2 df2_relax_to(const df2 &u, const df2 &q, float omega,
                                            float one_minus_omega) {
    const float2 om = f2_bcast(omega), om1m = f2_bcast(one_minus_omega);
    const float2 p1 = __fmul2_rn(om1m, u.hi);
    const float2 e1 = __ffma2_rn(om1m, u.lo, __ffma2_rn(om1m, u.hi, f2_neg(p1)));
    const float2 p2 = __fmul2_rn(om, q.hi);
    const float2 e2 = __ffma2_rn(om, q.lo, __ffma2_rn(om, q.hi, f2_neg(p2)));
    const df2 z = df2_two_sum(p1, p2);
    const float2 lo = __fadd2_rn(z.lo, __fadd2_rn(e1, e2));
    const float2 h = __fadd2_rn(z.hi, lo);
    return df2{h, __fadd2_rn(lo, f2_neg(__fadd2_rn(h, f2_neg(z.hi))))};
}
