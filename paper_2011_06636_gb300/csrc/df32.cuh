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

__device__ __forceinline__ double df_to_double(df32 a) {
    return (double)a.hi + (double)a.lo;
}

// 2D constant-coefficient sweep residual in FP32-pair arithmetic:
//   t = ax (w + e) + ay (s + n) + g - u,   g = D^-1 f (scaled right-hand side)
// Each pair sum and scaling keeps its rounding error in a low part and the
// low parts are summed plainly.  The result is left unnormalised (|lo| may
// exceed half an ulp of hi when hi cancels): df_axpy consumes lo through an
// FMA and renormalises its own result, and residual norms use hi + lo.
// 45 FP32 operations.
__device__ __forceinline__ df32 df_t2d(df32 w, df32 e, df32 s, df32 n, float ax, float ay,
                                       float g, df32 u) {
    const df32 sx = df_two_sum(w.hi, e.hi);
    const float sxl = __fadd_rn(sx.lo, __fadd_rn(w.lo, e.lo));
    const df32 sy = df_two_sum(s.hi, n.hi);
    const float syl = __fadd_rn(sy.lo, __fadd_rn(s.lo, n.lo));
    const df32 px = df_two_prod(sx.hi, ax);
    const float pxl = __fmaf_rn(sxl, ax, px.lo);
    const df32 py = df_two_prod(sy.hi, ay);
    const float pyl = __fmaf_rn(syl, ay, py.lo);
    const df32 q = df_two_sum(px.hi, py.hi);
    const df32 r1 = df_two_sum(q.hi, g);
    const df32 r2 = df_two_sum(r1.hi, -u.hi);
    const float lo =
        __fsub_rn(__fadd_rn(__fadd_rn(q.lo, __fadd_rn(pxl, pyl)), __fadd_rn(r1.lo, r2.lo)), u.lo);
    return df32{r2.hi, lo};
}

// Sum of two FP32 pairs with an unnormalised result: the high parts by an
// error-free sum, the low parts and its error added plainly.  8 FP32
// operations.
__device__ __forceinline__ df32 df_pair_sum(df32 a, df32 b) {
    const df32 s = df_two_sum(a.hi, b.hi);
    return df32{s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}

// The isotropic case ax = ay = 1/4 (equal spacing and coefficients) from two
// pair sums p and q that together hold the four neighbours: the scaling by
// 1/4 is exact, so no product error terms arise.  24 FP32 operations.
__device__ __forceinline__ df32 df_t2d_iso_pairs(df32 p, df32 q, float g, df32 u) {
    const df32 s = df_pair_sum(p, q);
    const df32 r1 = df_two_sum(__fmul_rn(s.hi, 0.25f), g);
    const df32 r2 = df_two_sum(r1.hi, -u.hi);
    const float lo = __fsub_rn(__fadd_rn(__fmaf_rn(s.lo, 0.25f, r1.lo), r2.lo), u.lo);
    return df32{r2.hi, lo};
}

// The isotropic case from the four neighbours: 40 FP32 operations (the pass
// kernels share each diagonal pair sum between two points instead, 32 per
// point: see wave_item.cuh).
__device__ __forceinline__ df32 df_t2d_iso(df32 w, df32 e, df32 s, df32 n, float g, df32 u) {
    return df_t2d_iso_pairs(df_pair_sum(w, e), df_pair_sum(s, n), g, u);
}

// Variable-coefficient sweep residual in FP32-pair arithmetic:
//   t = invd (f + sum_q w_q n_q) - u
// Every product and pair sum keeps its rounding error; the errors are summed
// plainly into one low part that is never renormalised on the way (the
// result is left unnormalised as in df_t2d).  11 FP32 operations per
// neighbour, 11 more for the scaling and the subtraction.
template <int NQ>
__device__ __forceinline__ df32 df_t_vark(const df32 *nb, const float *w, float invd, float f,
                                          df32 u) {
    float sh = f, sl = 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const df32 pq = df_two_prod(nb[q].hi, w[q]);
        const float pl = __fmaf_rn(nb[q].lo, w[q], pq.lo);
        const df32 sq = df_two_sum(sh, pq.hi);
        sh = sq.hi;
        sl = __fadd_rn(sl, __fadd_rn(sq.lo, pl));
    }
    const df32 m = df_two_prod(sh, invd);
    const float ml = __fmaf_rn(sl, invd, m.lo);
    const df32 r = df_two_sum(m.hi, -u.hi);
    return df32{r.hi, __fsub_rn(__fadd_rn(ml, r.lo), u.lo)};
}

// Constant-coefficient sweep residual on NA axes in FP32-pair arithmetic:
//   t = sum_a a_a (n_2a + n_2a+1) + g - u,   g = D^-1 f (scaled right-hand side)
// with the same single unnormalised low part.  19 FP32 operations per axis,
// 8 for the subtraction.
template <int NA>
__device__ __forceinline__ df32 df_t_axes(const df32 *nb, const float *a, float g, df32 u) {
    float sh = g, sl = 0.f;
#pragma unroll
    for (int ax = 0; ax < NA; ++ax) {
        const df32 s = df_two_sum(nb[2 * ax].hi, nb[2 * ax + 1].hi);
        const float slo = __fadd_rn(s.lo, __fadd_rn(nb[2 * ax].lo, nb[2 * ax + 1].lo));
        const df32 p = df_two_prod(s.hi, a[ax]);
        const float pl = __fmaf_rn(slo, a[ax], p.lo);
        const df32 q = df_two_sum(sh, p.hi);
        sh = q.hi;
        sl = __fadd_rn(sl, __fadd_rn(q.lo, pl));
    }
    const df32 r = df_two_sum(sh, -u.hi);
    return df32{r.hi, __fsub_rn(__fadd_rn(sl, r.lo), u.lo)};
}

// One relaxed sweep at a point of the isotropic case, fused:
//   u' = (1 - omega) u + omega q,   q = (p + q2) / 4 + g,
// the same value as u + omega (q - u).  1 - omega is exact in FP32 for every
// factor of the scheme tables (omega lies in (0.5, 2^24): for omega <= 2 by
// Sterbenz's lemma, above 2 because 1 is a multiple of omega's last place).
// Both products keep their rounding errors (two_prod) and meet in one
// error-free sum, so no difference q - u is formed first: 40 FP32 operations
// with the shared pair sum, against 46 for df_t2d_iso_pairs + df_axpy, in the
// same accuracy class (every rounding left is of order eps^2 omega |u|).
template <bool RENORM = true>
__device__ __forceinline__ df32 df_relax_iso_pairs(df32 p, df32 q2, float g, df32 u, float omega,
                                                   float one_minus_omega) {
    const df32 s = df_two_sum(p.hi, q2.hi);
    const float slo = __fadd_rn(s.lo, __fadd_rn(p.lo, q2.lo));
    // q = s / 4 + g: Knuth's two-sum of a = s / 4 (exact) and g with the
    // quarter folded into FMAs (fl(a + g), fl(q - a) and fl(a - t) each round
    // once, as the two-sum's own steps do): 6 operations for scale and sum
    const float qh = __fmaf_rn(s.hi, 0.25f, g);
    const float bb = __fmaf_rn(s.hi, -0.25f, qh);
    const float t1 = __fsub_rn(qh, bb);
    const float qe = __fadd_rn(__fmaf_rn(s.hi, 0.25f, -t1), __fsub_rn(g, bb));
    const df32 qs{qh, qe};
    const float qlo = __fmaf_rn(slo, 0.25f, qs.lo);
    const df32 p1 = df_two_prod(one_minus_omega, u.hi);
    const float e1 = __fmaf_rn(one_minus_omega, u.lo, p1.lo);
    const df32 p2 = df_two_prod(omega, qs.hi);
    const float e2 = __fmaf_rn(omega, qlo, p2.lo);
    const df32 z = df_two_sum(p1.hi, p2.hi);
    const float lo = __fadd_rn(z.lo, __fadd_rn(e1, e2));
    // without the renormalisation the pair stays an unevaluated sum whose low
    // part may exceed half an ulp of the high part; every later use takes the
    // high parts through error-free sums and adds the low parts plainly, so
    // the roundings stay of the same order (used for the levels of a pass
    // that are not stored)
    if constexpr (!RENORM) return df32{z.hi, lo};
    return df_fast_two_sum(z.hi, lo);
}

// The value q a sweep relaxes towards, u' = u + omega (q - u), as an
// unnormalised FP32 pair (its low part carries every rounding error):
//   variable coefficients   q = invd (f + sum_q w_q n_q)        11 NQ + 3 ops
//   constant, NA axes       q = sum_a a_a (n_2a + n_2a+1) + g   19 NA ops
//   2D constant (general)   q = ax (w + e) + ay (s + n) + g     38 ops
template <int NQ>
__device__ __forceinline__ df32 df_q_vark(const df32 *nb, const float *w, float invd, float f) {
    float sh = f, sl = 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const df32 pq = df_two_prod(nb[q].hi, w[q]);
        const float pl = __fmaf_rn(nb[q].lo, w[q], pq.lo);
        const df32 sq = df_two_sum(sh, pq.hi);
        sh = sq.hi;
        sl = __fadd_rn(sl, __fadd_rn(sq.lo, pl));
    }
    const df32 m = df_two_prod(sh, invd);
    return df32{m.hi, __fmaf_rn(sl, invd, m.lo)};
}

template <int NA>
__device__ __forceinline__ df32 df_q_axes(const df32 *nb, const float *a, float g) {
    float sh = g, sl = 0.f;
#pragma unroll
    for (int ax = 0; ax < NA; ++ax) {
        const df32 s = df_two_sum(nb[2 * ax].hi, nb[2 * ax + 1].hi);
        const float slo = __fadd_rn(s.lo, __fadd_rn(nb[2 * ax].lo, nb[2 * ax + 1].lo));
        const df32 p = df_two_prod(s.hi, a[ax]);
        const float pl = __fmaf_rn(slo, a[ax], p.lo);
        const df32 q = df_two_sum(sh, p.hi);
        sh = q.hi;
        sl = __fadd_rn(sl, __fadd_rn(q.lo, pl));
    }
    return df32{sh, sl};
}

__device__ __forceinline__ df32 df_q_2d(df32 w, df32 e, df32 s, df32 n, float ax, float ay,
                                        float g) {
    const df32 sx = df_two_sum(w.hi, e.hi);
    const float sxl = __fadd_rn(sx.lo, __fadd_rn(w.lo, e.lo));
    const df32 sy = df_two_sum(s.hi, n.hi);
    const float syl = __fadd_rn(sy.lo, __fadd_rn(s.lo, n.lo));
    const df32 px = df_two_prod(sx.hi, ax);
    const float pxl = __fmaf_rn(sxl, ax, px.lo);
    const df32 py = df_two_prod(sy.hi, ay);
    const float pyl = __fmaf_rn(syl, ay, py.lo);
    const df32 q = df_two_sum(px.hi, py.hi);
    const df32 r1 = df_two_sum(q.hi, g);
    return df32{r1.hi, __fadd_rn(__fadd_rn(q.lo, __fadd_rn(pxl, pyl)), r1.lo)};
}

// u' = (1 - omega) u + omega q with both products' rounding errors kept and
// one renormalisation: the same value as u + omega (q - u) without forming
// the difference (1 - omega is exact in FP32 for the scheme's factors; see
// df_relax_iso_pairs).  17 FP32 operations.
__device__ __forceinline__ df32 df_relax_to(df32 u, df32 q, float omega, float one_minus_omega) {
    const df32 p1 = df_two_prod(one_minus_omega, u.hi);
    const float e1 = __fmaf_rn(one_minus_omega, u.lo, p1.lo);
    const df32 p2 = df_two_prod(omega, q.hi);
    const float e2 = __fmaf_rn(omega, q.lo, p2.lo);
    const df32 z = df_two_sum(p1.hi, p2.hi);
    return df_fast_two_sum(z.hi, __fadd_rn(z.lo, __fadd_rn(e1, e2)));
}

// u + omega t with one renormalisation (about 14 FP32 operations).
__device__ __forceinline__ df32 df_axpy(df32 u, df32 t, float omega) {
    const df32 d = df_two_prod(t.hi, omega);
    const float dl = __fmaf_rn(t.lo, omega, d.lo);
    const df32 z = df_two_sum(u.hi, d.hi);
    return df_fast_two_sum(z.hi, __fadd_rn(z.lo, __fadd_rn(u.lo, dl)));
}
