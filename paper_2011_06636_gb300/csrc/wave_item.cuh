// wave_item.cuh -- one work item of the temporally blocked 2D SRJ pass: a
// warp streams a strip of 32*V columns down (or up) a segment of rows, doing
// up to T relaxed Jacobi sweeps (Sec. 2, Eq. relaxed-jacobi) of the current
// cycle as a wavefront, and optionally the residual of the final state
// (Sec. 3, Eq. relative-residual) for the cycle-end norm.
//
// Shared by the single-grid pass kernel (kernels_wave2d.cu) and the batched
// persistent kernel (kernels_batched.cu); everything here is file-local.
//
//  * lane l of the warp holds V consecutive columns; horizontal neighbours move
//    by warp shuffles, so the outer H >= T columns of a strip lose validity one
//    per sweep and only the inner 32V - 2H columns are written;
//  * at step t the warp loads row j(t) into level 0 and computes level s at
//    row j(t) -+ 2s, keeping the last three rows of every level in registers.
//    With this two-row lag per level, level s at step t reads only rows that
//    level s-1 produced at steps t-1, t-2, t-3, so the T levels of one step
//    are independent (T*V independent updates per lane instead of V); levels
//    run in descending order so that each ring slot is read before it is
//    overwritten;
//  * rows of the iterate and of f arrive through per-warp shared-memory rings
//    filled by cp.async with zero fill outside the grid (Dirichlet ghosts);
//    each lane reads back only what it copied, so a per-thread wait suffices.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "stencil_point.cuh"
#include "srj_internal.h"

// The FP32-pair isotropic levels use the fused relaxation df_relax_iso_pairs
// (define SRJ_DF_RELAX_FUSED=0 for the two-step form).
#ifndef SRJ_DF_RELAX_FUSED
#define SRJ_DF_RELAX_FUSED 1
#endif
#ifndef SRJ_DF_SKIP_RENORM
#define SRJ_DF_SKIP_RENORM 1
#endif

namespace srj {
namespace {

constexpr int kWaveWarps = 8;  // warps per CTA of the wave kernels

// V: columns per lane; ES: bytes per element; LO: FP32-pair iterate; PD:
// cp.async prefetch distance in steps (3: measured enough for every
// precision; 6 did not help the FP32 kernel).
template <int PREC>
struct WaveTraits;
template <>
struct WaveTraits<PREC_F32> {
    static constexpr int V = 4;
    static constexpr int ES = 4;
    static constexpr bool LO = false;
    static constexpr int PD = 3;
    // separate unchecked steady-state loop: fewer tests per step, three
    // copies of the step body (measured: +2 % for FP32, -15 % for the much
    // larger FP32-pair body, whose three copies overflow the instruction cache)
    static constexpr bool SPLIT = true;
};
template <>
struct WaveTraits<PREC_DF> {
    static constexpr int V = 4;
    static constexpr int ES = 4;
    static constexpr bool LO = true;
    static constexpr int PD = 3;
    static constexpr bool SPLIT = false;
};
template <>
struct WaveTraits<PREC_F64> {
    static constexpr int V = 2;
    static constexpr int ES = 8;
    static constexpr bool LO = false;
    static constexpr int PD = 3;
    static constexpr bool SPLIT = false;
};

__host__ __device__ constexpr int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p *= 2;
    return p;
}

__host__ __device__ constexpr int wave_halo(int T, int V, int ES) {
    // multiple of V, and of 16 bytes when the chunks are 16 bytes wide
    return ES == 8 ? T : ((T + V - 1) / V) * V;
}

__device__ __forceinline__ void cp_async(void *smem, const void *gmem, int bytes, bool valid,
                                         const void *safe) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const void *g = valid ? gmem : safe;
    const int n = valid ? bytes : 0;
    if (bytes == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(g), "r"(n));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(g), "r"(n));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <int PREC, int T>
struct Wave {
    using Tr = WaveTraits<PREC>;
    static constexpr int V = Tr::V;
    static constexpr int WC = 32 * V;                  // strip width (columns)
    static constexpr int H = wave_halo(T, V, Tr::ES);  // halo columns per side
    static constexpr int OUTW = WC - 2 * H;            // written columns per strip
    static constexpr int PD = Tr::PD;                  // prefetch distance
    // ring slot counts are powers of two so that slot = step & (count - 1)
    static constexpr int UR = pow2_at_least(PD + 1);          // iterate ring slots
    static constexpr int FR = pow2_at_least(2 * T + 3 + PD);  // rhs ring slots
    static constexpr bool VEC_OUT = (H % V) == 0;      // whole lanes are written
    static constexpr int CHUNK = (Tr::ES == 8 && (H % 2)) ? 8 : 16;
    static constexpr int ROWB = WC * Tr::ES;           // bytes per ring row
    static constexpr int SMEM_WARP = (UR * (Tr::LO ? 2 : 1) + FR) * ROWB;
};

// Everything one item needs: geometry, the source / destination iterates,
// the right-hand side and this pass's factors.
template <int PREC, int T>
struct ItemCtx {
    using E = typename Elem<PREC>::T;
    using C = typename Elem<PREC>::C;
    int nx, ny;
    long long pitch;
    const unsigned char *src, *src_lo, *fsrc;
    E *dst;
    float *dst_hi, *dst_lo;
    C omega[T];
    C omega1m[T];  // 1 - omega, exact in FP32 for the scheme's factors
    int nsw;     // sweeps of this pass (levels beyond nsw are identities)
    int resid;   // 1: accumulate the residual of the final state
    int iso;     // FP32 pair or FP64 with acoef = {1/4, 1/4}: the isotropic stencil form
    C diag, invd, acoef[3];
};

// Process the item (strip, segment [y0, y1)) and return this lane's sum of
// squared residuals (0 unless c.resid).  The caller owns the warp's ring
// memory wbase (Wave<PREC,T>::SMEM_WARP bytes).
template <int PREC, int T, bool RESID, bool ISO>
__device__ __forceinline__ double wave_item_impl(const ItemCtx<PREC, T> &c, int strip, int y0,
                                                 int y1, int dir, unsigned char *wbase, int lane) {
    using W = Wave<PREC, T>;
    using E = typename Elem<PREC>::T;
    using C = typename Elem<PREC>::C;
    constexpr int V = W::V;
    constexpr int ES = WaveTraits<PREC>::ES;
    constexpr bool LO = WaveTraits<PREC>::LO;

    unsigned char *uring = wbase;
    unsigned char *uring_lo = wbase + W::UR * W::ROWB;
    unsigned char *fring = wbase + W::UR * W::ROWB * (LO ? 2 : 1);
    const long long pitchB = c.pitch * ES;

    const int xs = strip * W::OUTW - W::H;  // first column of the strip
    // level s at step t holds row j(t) - 2 s dir; the residual at step t is
    // that of row j(t) - (2T + 2) dir.  Rows loaded: [y0 - T - 1, y1 + T].
    const int nsteps = (y1 - y0) + 3 * T + 3;
    const int nload = (y1 - y0) + 2 * T + 2;          // steps that load a row
    const int jbase = dir > 0 ? y0 - T - 1 : y1 + T;  // j(t) = jbase + dir * t
    const int col0 = xs + lane * V;                   // this lane's first column
    const bool edge = (xs < 0) || (xs + W::WC > c.nx);
    bool colok[V];
#pragma unroll
    for (int v = 0; v < V; ++v) colok[v] = (col0 + v >= 0) && (col0 + v < c.nx);
    bool outcol[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int cc = lane * V + v;
        outcol[v] = (cc >= W::H) && (cc < W::WC - W::H) && colok[v];
    }
    bool whole_lane = true;  // every column of this lane is written
#pragma unroll
    for (int v = 0; v < V; ++v) whole_lane = whole_lane && outcol[v];

    // issue the copies of step t (row j(t) of the iterate and of f)
    auto issue = [&](int t) {
        const int row = jbase + dir * t;
        const bool rok = (row >= 0) && (row < c.ny) && (t < nload);
        const int us = t & (W::UR - 1), fs = t & (W::FR - 1);
#pragma unroll
        for (int k = 0; k < (V * ES) / W::CHUNK; ++k) {
            const int colc = col0 + k * (W::CHUNK / ES);
            const bool ok = rok && colc >= 0 && colc < c.pitch;
            const long long off = (long long)row * pitchB + (long long)colc * ES;
            const int so = us * W::ROWB + lane * V * ES + k * W::CHUNK;
            const int fo = fs * W::ROWB + lane * V * ES + k * W::CHUNK;
            cp_async(uring + so, c.src + off, W::CHUNK, ok, c.src);
            if constexpr (LO) cp_async(uring_lo + so, c.src_lo + off, W::CHUNK, ok, c.src_lo);
            cp_async(fring + fo, c.fsrc + off, W::CHUNK, ok, c.fsrc);
        }
    };

    // registers: last three rows of every level 0..T
    E ring[T + 1][3][V];
#pragma unroll
    for (int s = 0; s <= T; ++s)
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int v = 0; v < V; ++v) ring[s][q][v] = zero_u<PREC>();
    // isotropic form: each level's diagonal pair sums of the row it computed
    // at the previous step (see the level loop)
    E pprev[ISO ? T : 1][V];
#pragma unroll
    for (int s = 0; s < (ISO ? T : 1); ++s)
#pragma unroll
        for (int v = 0; v < V; ++v) pprev[s][v] = zero_u<PREC>();
    float kahan_s = 0.f, kahan_c = 0.f;  // FP32 paths: compensated r^2 sum
    double dsum = 0.0;                   // FP64 path

    __syncwarp();
    for (int t = 0; t < W::PD; ++t) {
        if (t < nsteps) issue(t);
        cp_commit();
    }

    // one 16-byte shared-memory load of this lane's V values of a ring row
    auto load_vec = [&](const unsigned char *ringb, int slot, C *out) {
        const unsigned char *p = ringb + slot * W::ROWB + lane * V * ES;
        if constexpr (PREC == PREC_F64) {
            const double2 q = *(const double2 *)p;
            out[0] = q.x;
            out[1] = q.y;
        } else {
            const float4 q = *(const float4 *)p;
            out[0] = q.x;
            out[1] = q.y;
            out[2] = q.z;
            out[3] = q.w;
        }
    };
    auto shfl_left = [&](const E &x) -> E {
        if constexpr (LO)
            return df32{__shfl_up_sync(0xffffffffu, x.hi, 1), __shfl_up_sync(0xffffffffu, x.lo, 1)};
        else
            return __shfl_up_sync(0xffffffffu, x, 1);
    };
    auto shfl_right = [&](const E &x) -> E {
        if constexpr (LO)
            return df32{__shfl_down_sync(0xffffffffu, x.hi, 1),
                        __shfl_down_sync(0xffffffffu, x.lo, 1)};
        else
            return __shfl_down_sync(0xffffffffu, x, 1);
    };

    // CHK: this step may lie in the warm-up or drain range, where some levels
    // have no needed row; steady steps skip those tests
    auto step = [&](int t, auto phase_tag, auto chk_tag) {
        constexpr int PH = decltype(phase_tag)::value;
        constexpr bool CHK = decltype(chk_tag)::value;
        // ring slots of the rows produced at steps t-1, t-2, t-3 (and t = t-3's)
        constexpr int S1 = (PH + 2) % 3, S2 = (PH + 1) % 3, S3 = PH;
        if (t + W::PD < nsteps) issue(t + W::PD);
        cp_commit();
        cp_wait<W::PD>();
        const int jt = jbase + dir * t;
        // residual of the final state at row j(t) - (2T+2) dir, from level T's
        // rows of steps t-1, t-2 (centre), t-3 -- before level T overwrites S3
        if (RESID && t >= 3 * T + 3) {
            const int row = jt - dir * (2 * T + 2);
            const int fs = (t - 2 * T - 2) & (W::FR - 1);
            const E left = shfl_left(ring[T][S2][V - 1]);
            const E right = shfl_right(ring[T][S2][0]);
            if (row >= y0 && row < y1) {
                C fr[V];
                load_vec(fring, fs, fr);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if (!outcol[v]) continue;
                    const C fvv = fr[v];
                    E nb[6];
                    nb[0] = v > 0 ? ring[T][S2][v - 1] : left;
                    nb[1] = v < V - 1 ? ring[T][S2][v + 1] : right;
                    nb[2] = ring[T][S3][v];
                    nb[3] = ring[T][S1][v];
                    E tt;
                    if constexpr (ISO && LO) tt = Point<PREC, 2>::t_const_iso(nb, fvv, ring[T][S2][v]);
                    else tt = Point<PREC, 2>::t_const(nb, c.acoef, c.invd, fvv, ring[T][S2][v]);
                    if constexpr (PREC == PREC_F64) {
                        const double r = c.diag * tt;
                        dsum = fma(r, r, dsum);
                    } else {
                        float r;
                        if constexpr (LO) r = c.diag * (tt.hi + tt.lo);
                        else r = c.diag * tt;
                        // Kahan: sum += r^2
                        const float y = fmaf(r, r, -kahan_c);
                        const float sum = kahan_s + y;
                        kahan_c = (sum - kahan_s) - y;
                        kahan_s = sum;
                    }
                }
            }
        }
        // levels T..1 (descending): level s reads level s-1's rows of steps
        // t-1, t-2, t-3 and writes its row of step t into slot S3
#pragma unroll
        for (int s = T; s >= 1; --s) {
            // above every needed row (the isotropic form starts one step early:
            // the first needed row takes the pair sums of the row before it)
            if (CHK && t < 3 * s - (ISO ? 1 : 0)) continue;
            if (CHK && t > nload - 1 + s) continue;   // below every needed row
            const int row = jt - dir * (2 * s);
            // identity level: only in the last pass of a cycle (a pass without
            // the residual always runs all T sweeps)
            if (RESID && s > c.nsw) {
#pragma unroll
                for (int v = 0; v < V; ++v) ring[s][S3][v] = ring[s - 1][S2][v];
                continue;
            }
            const int fs = (t - 2 * s) & (W::FR - 1);
            C fv[V];
            load_vec(fring, fs, fv);
            if constexpr (ISO) {
                // Row r = j(t) - 2 s dir with the four neighbours grouped in
                // diagonal pairs: p(x) = u(x+1, r) + u(x, r + dir) from the rows
                // of steps t-2 and t-1, and the partner pair u(x-1, r) +
                // u(x, r - dir), which is p(x-1) of row r - dir: this level's
                // pair sums of the previous step.  One pair sum per point
                // instead of two.
                const E right = shfl_right(ring[s - 1][S2][0]);
                const E pleft = shfl_left(pprev[s - 1][V - 1]);
                E pc[V];
#pragma unroll
                for (int v = 0; v < V; ++v)
                    pc[v] = Point<PREC, 2>::pair_sum(v < V - 1 ? ring[s - 1][S2][v + 1] : right,
                                                     ring[s - 1][S1][v]);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const E uc = ring[s - 1][S2][v];
                    const E pl = v > 0 ? pprev[s - 1][v - 1] : pleft;
#if SRJ_DF_RELAX_FUSED
                    if constexpr (LO) {
                        // only the level that is stored renormalises its pair
                        if (SRJ_DF_SKIP_RENORM && s < T)
                            ring[s][S3][v] = df_relax_iso_pairs<false>(
                                pc[v], pl, fv[v], uc, c.omega[s - 1], c.omega1m[s - 1]);
                        else
                            ring[s][S3][v] = df_relax_iso_pairs<true>(
                                pc[v], pl, fv[v], uc, c.omega[s - 1], c.omega1m[s - 1]);
                        continue;
                    }
#endif
                    const E tt = Point<PREC, 2>::t_iso_pairs(pc[v], pl, c.invd, fv[v], uc);
                    ring[s][S3][v] = Point<PREC, 2>::relax(uc, tt, (double)c.omega[s - 1]);
                }
#pragma unroll
                for (int v = 0; v < V; ++v) pprev[s - 1][v] = pc[v];
            } else {
                const E left = shfl_left(ring[s - 1][S2][V - 1]);
                const E right = shfl_right(ring[s - 1][S2][0]);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    E nb[6];
                    nb[0] = v > 0 ? ring[s - 1][S2][v - 1] : left;
                    nb[1] = v < V - 1 ? ring[s - 1][S2][v + 1] : right;
                    nb[2] = ring[s - 1][S3][v];
                    nb[3] = ring[s - 1][S1][v];
                    const E uc = ring[s - 1][S2][v];
                    ring[s][S3][v] = Point<PREC, 2>::sweep_const(nb, c.acoef, c.invd, fv[v], uc,
                                                                 (double)c.omega[s - 1]);
                }
            }
            // Dirichlet ghosts stay zero (a warp-uniform test: the row is the
            // same for every lane and `edge` is per strip)
            if (edge || row < 0 || row >= c.ny) {
                const bool rok = (row >= 0) && (row < c.ny);
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (!rok || !colok[v]) ring[s][S3][v] = zero_u<PREC>();
            }
        }
        // output: level T's new row j(t) - 2T dir
        {
            const int row = jt - dir * (2 * T);
            if ((!RESID || c.nsw > 0) && row >= y0 && row < y1) {
                const long long base = (long long)row * c.pitch + col0;
                if (W::VEC_OUT && whole_lane) {  // one 16-byte store per array
                    if constexpr (LO) {
                        *(float4 *)(c.dst_hi + base) = make_float4(
                            ring[T][S3][0].hi, ring[T][S3][1].hi, ring[T][S3][2].hi, ring[T][S3][3].hi);
                        *(float4 *)(c.dst_lo + base) = make_float4(
                            ring[T][S3][0].lo, ring[T][S3][1].lo, ring[T][S3][2].lo, ring[T][S3][3].lo);
                    } else if constexpr (PREC == PREC_F64) {
                        *(double2 *)(c.dst + base) = make_double2(ring[T][S3][0], ring[T][S3][1]);
                    } else {
                        *(float4 *)(c.dst + base) = make_float4(ring[T][S3][0], ring[T][S3][1],
                                                                ring[T][S3][2], ring[T][S3][3]);
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        if (!outcol[v]) continue;
                        if constexpr (LO) {
                            c.dst_hi[base + v] = ring[T][S3][v].hi;
                            c.dst_lo[base + v] = ring[T][S3][v].lo;
                        } else {
                            c.dst[base + v] = ring[T][S3][v];
                        }
                    }
                }
            }
        }
        // level 0: row j(t), after every level has read slot S3 of level 0
        {
            const int us = t & (W::UR - 1);
            C hi[V];
            load_vec(uring, us, hi);
            if constexpr (LO) {
                C lo[V];
                load_vec(uring_lo, us, lo);
#pragma unroll
                for (int v = 0; v < V; ++v) ring[0][S3][v] = df32{hi[v], lo[v]};
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) ring[0][S3][v] = hi[v];
            }
        }
    };

    using P0 = std::integral_constant<int, 0>;
    using P1 = std::integral_constant<int, 1>;
    using P2 = std::integral_constant<int, 2>;
    using Y = std::true_type;
    using N = std::false_type;
    // steps [3T, nload] compute every level; the ranges before and after are
    // run with the per-level tests (boundaries kept on multiples of 3 so the
    // register-ring phase stays a compile-time constant)
    int t = 0;
    if constexpr (WaveTraits<PREC>::SPLIT) {
        const int t_steady = 3 * T;
        int t_drain = ((nload + 1) / 3) * 3;
        if (t_drain < t_steady) t_drain = t_steady;
        if (t_drain > nsteps) t_drain = nsteps;
        for (; t < t_steady && t < nsteps; t += 3) {
            step(t, P0{}, Y{});
            if (t + 1 < nsteps) step(t + 1, P1{}, Y{});
            if (t + 2 < nsteps) step(t + 2, P2{}, Y{});
        }
        for (; t + 3 <= t_drain; t += 3) {
            step(t, P0{}, N{});
            step(t + 1, P1{}, N{});
            step(t + 2, P2{}, N{});
        }
    }
    for (; t < nsteps; t += 3) {
        step(t, P0{}, Y{});
        if (t + 1 < nsteps) step(t + 1, P1{}, Y{});
        if (t + 2 < nsteps) step(t + 2, P2{}, Y{});
    }
    cp_wait<0>();
    __syncwarp();
    if constexpr (PREC == PREC_F64) return dsum;
    else return (double)kahan_s - (double)kahan_c;
}

// The residual level is compiled only into the variant for the last pass of
// a cycle, the isotropic form only into the FP32-pair and FP64 variants (the
// FP32 pass is bound by memory, not arithmetic).
template <int PREC, int T>
__device__ __forceinline__ double wave_item(const ItemCtx<PREC, T> &c, int strip, int y0, int y1,
                                            int dir, unsigned char *wbase, int lane) {
    if constexpr (PREC == PREC_DF || PREC == PREC_F64) {
        if (c.iso) {
            if (c.resid) return wave_item_impl<PREC, T, true, true>(c, strip, y0, y1, dir, wbase, lane);
            return wave_item_impl<PREC, T, false, true>(c, strip, y0, y1, dir, wbase, lane);
        }
    }
    if (c.resid) return wave_item_impl<PREC, T, true, false>(c, strip, y0, y1, dir, wbase, lane);
    return wave_item_impl<PREC, T, false, false>(c, strip, y0, y1, dir, wbase, lane);
}

// Factors, coefficients and buffers of one pass of one grid.
template <int PREC, int T>
__device__ __forceinline__ void fill_ctx(ItemCtx<PREC, T> &c, const GridGeo &g,
                                         const IterBufs &b, int cur, int nsw, int resid,
                                         const double *w64, int woff) {
    using E = typename Elem<PREC>::T;
    using C = typename Elem<PREC>::C;
    c.nx = g.nx;
    c.ny = g.ny;
    c.pitch = g.pitch;
    c.src = (const unsigned char *)b.u[cur];
    c.src_lo = WaveTraits<PREC>::LO ? (const unsigned char *)b.ulo[cur] : nullptr;
    c.fsrc = (const unsigned char *)b.f;
    c.dst = (E *)b.u[cur ^ 1];
    c.dst_hi = (float *)b.u[cur ^ 1];
    c.dst_lo = (float *)b.ulo[cur ^ 1];
#pragma unroll
    for (int s = 0; s < T; ++s) {
        c.omega[s] = (s < nsw) ? (C)w64[woff + s] : C(0);
        c.omega1m[s] = C(1) - c.omega[s];
    }
    c.nsw = nsw;
    c.resid = resid;
    c.diag = C(g.diag);
    c.invd = C(g.invdiag);
    c.acoef[0] = C(g.acx);
    c.acoef[1] = C(g.acy);
    c.acoef[2] = C(0);
    c.iso = (PREC == PREC_DF || PREC == PREC_F64) && c.acoef[0] == C(0.25) &&
            c.acoef[1] == C(0.25);
}

}  // namespace
}  // namespace srj
