// stencil_point.cuh -- per-point arithmetic of the relaxed Jacobi sweep
// (Sec. 2, Eq. relaxed-jacobi) and of the residual, for the three state
// representations: FP64, FP32 and the FP32 pair (df32.cuh).  Shared by the
// pass kernels (file-local copies per translation unit).
#pragma once

#include "df32.cuh"
#include "srj_internal.h"

namespace srj {
namespace {

// ------------------------------------------------------------- element access
template <int PREC>
struct Elem;
template <>
struct Elem<PREC_F64> {
    using T = double;   // state
    using C = double;   // coefficients / rhs
};
template <>
struct Elem<PREC_F32> {
    using T = float;
    using C = float;
};
template <>
struct Elem<PREC_DF> {
    using T = df32;
    using C = float;
};

// The source iterate of a pass is never written during that pass (the pass
// writes the other buffer of the pair), so it is read through the read-only
// data path: that also tells the compiler the loads cannot alias the stores,
// so loads of later points can be issued ahead of earlier stores.
template <int PREC>
__device__ __forceinline__ typename Elem<PREC>::T load_u(const IterBufs &b, int which,
                                                        long long i) {
    if constexpr (PREC == PREC_DF) {
        const float *hi = (const float *)b.u[which];
        const float *lo = (const float *)b.ulo[which];
        return df32{__ldg(hi + i), __ldg(lo + i)};
    } else {
        return __ldg((const typename Elem<PREC>::T *)b.u[which] + i);
    }
}

template <int PREC>
__device__ __forceinline__ void store_u(const IterBufs &b, int which, long long i,
                                        typename Elem<PREC>::T v) {
    if constexpr (PREC == PREC_DF) {
        ((float *)b.u[which])[i] = v.hi;
        ((float *)b.ulo[which])[i] = v.lo;
    } else {
        ((typename Elem<PREC>::T *)b.u[which])[i] = v;
    }
}

template <int PREC>
__device__ __forceinline__ typename Elem<PREC>::T zero_u() {
    if constexpr (PREC == PREC_DF) return df32{0.f, 0.f};
    else return typename Elem<PREC>::T(0);
}

// ---------------------------------------------- relaxation, residual at a point
// Neighbour values nb[0..5] = -x, +x, -y, +y, -z, +z (zero outside);
// weights wgt[0..5] the matching face weights (variable k) or the axis
// coefficients c_a (constant); invd = 1/D; f the right-hand side.
//
// SWEEP:  t = D^-1 (f + sum_q w_q u_q) - u_c;  u' = u_c + omega t
// RESID:  r = D t
template <int PREC, int DIM>
struct Point {
    using T = typename Elem<PREC>::T;
    using C = typename Elem<PREC>::C;

    // t = D^-1 (f + sum w u_nb) - u_c
    __device__ __forceinline__ static T t_of(const T *nb, const C *wgt, C invd, C f,
                                             T uc) {
        if constexpr (PREC == PREC_DF) {
            return df_t_vark<2 * DIM>(nb, wgt, invd, f, uc);
        } else {
            T s = f + wgt[0] * nb[0] + wgt[1] * nb[1];
            if (DIM > 1) s += wgt[2] * nb[2] + wgt[3] * nb[3];
            if (DIM > 2) s += wgt[4] * nb[4] + wgt[5] * nb[5];
            return s * invd - uc;
        }
    }

    // constant coefficients: t = a_x (u_-x + u_+x) + ... + D^-1 f - u_c with
    // a = c / D, written as the cheaper sum-then-scale form.  The FP32-pair
    // state takes its right-hand side already scaled, f = D^-1 f (the
    // mixed-precision outer residual stores it so; invd is then unused).
    __device__ __forceinline__ static T t_const(const T *nb, const C *a, C invd, C f, T uc) {
        if constexpr (PREC == PREC_DF) {
            (void)invd;
            if constexpr (DIM == 2) {
                return df_t2d(nb[0], nb[1], nb[2], nb[3], a[0], a[1], f, uc);
            } else {
                return df_t_axes<DIM>(nb, a, f, uc);
            }
        } else {
            T s = a[0] * (nb[0] + nb[1]);
            if (DIM > 1) s += a[1] * (nb[2] + nb[3]);
            if (DIM > 2) s += a[2] * (nb[4] + nb[5]);
            return s + invd * f - uc;
        }
    }

    // 2D isotropic FP32-pair case a_x = a_y = 1/4 (scaled right-hand side)
    __device__ __forceinline__ static T t_const_iso(const T *nb, C f, T uc) {
        static_assert(PREC == PREC_DF && DIM == 2, "isotropic form: 2D FP32 pair only");
        return df_t2d_iso(nb[0], nb[1], nb[2], nb[3], f, uc);
    }

    // 2D isotropic case a_x = a_y = 1/4 from two pair sums p, q that together
    // hold the four neighbours (the wave kernel shares each pair sum between
    // two points): FP32 pair 8 + 24 operations with the scaled right-hand
    // side (invd unused); FP64 t = fma(1/4, p + q, fma(invd, f, -u_c)), with
    // the pair sum 4 FP64 instructions instead of 6.
    __device__ __forceinline__ static T pair_sum(T a, T b) {
        if constexpr (PREC == PREC_DF) return df_pair_sum(a, b);
        else return a + b;
    }
    __device__ __forceinline__ static T t_iso_pairs(T p, T q, C invd, C f, T uc) {
        static_assert(DIM == 2, "isotropic form: 2D only");
        if constexpr (PREC == PREC_DF) {
            (void)invd;
            return df_t2d_iso_pairs(p, q, f, uc);
        } else {
            return fma(C(0.25), p + q, fma(invd, f, -uc));
        }
    }

    // One sweep at the point, u_c + omega t: for the FP32 pair in the fused
    // form (1 - omega) u_c + omega q (df_relax_to), 5 to 6 operations fewer
    // than forming t first; otherwise relax(t).
    __device__ __forceinline__ static T sweep_of(const T *nb, const C *wgt, C invd, C f, T uc,
                                                 double omega) {
        if constexpr (PREC == PREC_DF) {
            const float om = (float)omega;
            return df_relax_to(uc, df_q_vark<2 * DIM>(nb, wgt, invd, f), om, 1.f - om);
        } else {
            return relax(uc, t_of(nb, wgt, invd, f, uc), omega);
        }
    }
    __device__ __forceinline__ static T sweep_const(const T *nb, const C *a, C invd, C f, T uc,
                                                    double omega) {
        if constexpr (PREC == PREC_DF) {
            const float om = (float)omega;
            df32 q;
            if constexpr (DIM == 2) q = df_q_2d(nb[0], nb[1], nb[2], nb[3], a[0], a[1], f);
            else q = df_q_axes<DIM>(nb, a, f);
            return df_relax_to(uc, q, om, 1.f - om);
        } else {
            return relax(uc, t_const(nb, a, invd, f, uc), omega);
        }
    }

    __device__ __forceinline__ static T relax(T uc, T t, double omega) {
        if constexpr (PREC == PREC_DF) return df_axpy(uc, t, (float)omega);
        else return uc + (C)omega * t;
    }

    __device__ __forceinline__ static double resid2(T t, C diag) {
        double r;
        if constexpr (PREC == PREC_DF) r = (double)diag * df_to_double(t);
        else r = (double)(diag * t);
        return r * r;
    }
};

}  // namespace
}  // namespace srj
