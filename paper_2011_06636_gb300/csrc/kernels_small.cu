// kernels_small.cu -- a whole SRJ solve of a small grid in one CTA.
//
// For grids whose iterate pair, right-hand side (and face weights) fit in
// shared memory, one CTA of 1024 threads runs every pass of the solve: the
// same pass plan and state machine as the pass kernels (plan_pass /
// advance_state: cycle position, residual ratio, Alg. 1 of Sec. 3 or the
// other selectors, convergence test, trace), with one block barrier per sweep
// instead of one kernel launch.  A small solve is bound by launch latency
// otherwise (a few microseconds per pass for a few microseconds of work).
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "df32.cuh"
#include "pass_common.cuh"
#include "stencil_point.cuh"
#include "srj_internal.h"

namespace srj {
namespace {

constexpr int kSmallThreads = 1024;

template <int PREC>
struct SmallElem {
    static constexpr int ES = PREC == PREC_F64 ? 8 : 4;  // bytes of one state / coefficient word
    static constexpr int UW = PREC == PREC_DF ? 2 : 1;   // state words per point
};

// Shared-memory bytes for n points.
template <int PREC, bool VARK>
constexpr long long small_bytes(long long n) {
    return n * SmallElem<PREC>::ES * (2 * SmallElem<PREC>::UW + 1 + (VARK ? 4 : 0));
}

template <int PREC, int DIM, bool VARK>
__global__ void __launch_bounds__(kSmallThreads) small_solve_kernel(PassLaunch a) {
    using T = typename Elem<PREC>::T;
    using C = typename Elem<PREC>::C;
    using P = Point<PREC, DIM>;
    constexpr bool LO = PREC == PREC_DF;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PassPlan s_plan;
    __shared__ double s_omega;

    const GridGeo &g = a.geo;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int n = nx * ny * nz;
    const int tid = threadIdx.x;
    // layout: state hi [2][n], (lo [2][n]), f [n], (wx, wy, wz, invd [n])
    using H = typename std::conditional<PREC == PREC_F64, double, float>::type;
    H *s_hi[2] = {(H *)smem, (H *)smem + n};
    float *s_lo[2] = {nullptr, nullptr};
    C *base = (C *)((H *)smem + 2 * n);
    if constexpr (LO) {
        s_lo[0] = (float *)base;
        s_lo[1] = (float *)base + n;
        base = (C *)((float *)base + 2 * n);
    }
    C *sf = base;
    C *swx = sf + n, *swy = swx + n, *swz = swy + n, *sid = swz + n;

    const int cur0 = a.st->cur;
    auto gidx = [&](int i) -> long long {
        const int x = i % nx, yz = i / nx;
        const int y = yz % ny, z = yz / ny;
        return (long long)x + g.pitch * y + g.plane * z;
    };
    for (int i = tid; i < n; i += kSmallThreads) {
        const long long q = gidx(i);
        s_hi[cur0][i] = ((const H *)a.bufs.u[cur0])[q];
        if constexpr (LO) s_lo[cur0][i] = ((const float *)a.bufs.ulo[cur0])[q];
        sf[i] = ((const C *)a.bufs.f)[q];
        if constexpr (VARK) {
            swx[i] = ((const C *)a.bufs.wx)[q];
            swy[i] = ((const C *)a.bufs.wy)[q];
            swz[i] = ((const C *)a.bufs.wz)[q];
            sid[i] = ((const C *)a.bufs.invd)[q];
        }
    }
    C cconst[3], invd_c = C(g.invdiag), diag_c = C(g.diag);
    cconst[0] = C(g.acx);
    cconst[1] = C(g.acy);
    cconst[2] = C(g.acz);
    const bool nx_ = g.neu & 1, ny_ = g.neu & 2, nz_ = g.neu & 4;
    __syncthreads();

    for (;;) {
        if (tid == 0) {
            s_plan = plan_pass(a, 1);
            s_omega = (s_plan.run && s_plan.nsw) ? a.w64[s_plan.woff] : 0.0;
        }
        __syncthreads();
        const PassPlan p = s_plan;
        if (!p.run) break;
        const double omega = s_omega;
        const int src = p.cur, dst = p.cur ^ 1;
        const bool dinf = a.dinf && p.nsw;
        auto ld = [&](int j) -> T {
            if constexpr (LO) return df32{s_hi[src][j], s_lo[src][j]};
            else return s_hi[src][j];
        };
        double part = 0.0;  // residual sum (resid pass)
        long long dbits = 0;  // largest |u' - u| of the sweep (abs_diff_bits)
        for (int i = tid; i < n; i += kSmallThreads) {
            const int x = i % nx, yz = i / nx;
            const int y = yz % ny, z = yz / ny;
            const T zero = zero_u<PREC>();
            T nb[6];
            nb[0] = x > 0 ? ld(i - 1) : (nx_ ? ld(i + 1) : zero);
            nb[1] = x + 1 < nx ? ld(i + 1) : (nx_ ? ld(i - 1) : zero);
            if (DIM > 1) {
                nb[2] = y > 0 ? ld(i - nx) : (ny_ ? ld(i + nx) : zero);
                nb[3] = y + 1 < ny ? ld(i + nx) : (ny_ ? ld(i - nx) : zero);
            }
            if (DIM > 2) {
                const int pl = nx * ny;
                nb[4] = z > 0 ? ld(i - pl) : (nz_ ? ld(i + pl) : zero);
                nb[5] = z + 1 < nz ? ld(i + pl) : (nz_ ? ld(i - pl) : zero);
            }
            const T uc = ld(i);
            T t = zero_u<PREC>(), un_v = zero_u<PREC>();
            C diag_i = diag_c;
            if constexpr (VARK) {
                C w[6];
                w[0] = x > 0 ? swx[i - 1] : C(0);
                w[1] = swx[i];
                if (DIM > 1) {
                    w[2] = y > 0 ? swy[i - nx] : C(0);
                    w[3] = swy[i];
                }
                if (DIM > 2) {
                    w[4] = z > 0 ? swz[i - nx * ny] : C(0);
                    w[5] = swz[i];
                }
                if (p.nsw) {
                    un_v = P::sweep_of(nb, w, sid[i], sf[i], uc, omega);
                } else {
                    t = P::t_of(nb, w, sid[i], sf[i], uc);
                    diag_i = C(1) / sid[i];
                }
            } else if (p.nsw) {
                un_v = P::sweep_const(nb, cconst, invd_c, sf[i], uc, omega);
            } else {
                t = P::t_const(nb, cconst, invd_c, sf[i], uc);
            }
            if (p.nsw) {
                const T un = un_v;
                if constexpr (LO) {
                    s_hi[dst][i] = un.hi;
                    s_lo[dst][i] = un.lo;
                } else {
                    s_hi[dst][i] = un;
                }
                if constexpr (PREC != PREC_DF)
                    if (dinf) dbits = max_bits(dbits, abs_diff_bits((double)un, (double)uc));
            } else {
                part += P::resid2(t, diag_i);
            }
        }
        // (the other threads keep to their copy of the plan, so thread 0 may
        // advance the state while they finish the sweep; the barrier at the
        // end of the iteration orders the sweep before the next one)
        double tot = 0.0;
        if (p.resid) tot = block_sum(part);
        else if (dinf) tot = block_max_bits(dbits);
        int pick = -1;
        if (tid < 32) {  // the reductions leave the total in thread 0 only
            const double t0 = __shfl_sync(0xffffffffu, tot, 0);
            pick = mlp_pick_at_cycle_end(a.st, a.cfg, p, t0, a.lvl_m, tid);
        }
        if (tid == 0) advance_state(a.st, a.cfg, p, p.resid ? tot : 0.0, pick, dinf ? tot : -1.0);
        __syncthreads();
    }
    // the final iterate back into the padded buffer the state points at
    const int fin = a.st->cur;
    for (int i = tid; i < n; i += kSmallThreads) {
        const long long q = gidx(i);
        ((H *)a.bufs.u[fin])[q] = s_hi[fin][i];
        if constexpr (LO) ((float *)a.bufs.ulo[fin])[q] = s_lo[fin][i];
    }
}

template <int PREC, int DIM, bool VARK>
void *small_entry() {
    return (void *)&small_solve_kernel<PREC, DIM, VARK>;
}

template <int PREC>
void *small_pick(int dim, bool vark) {
    if (dim == 1) return vark ? small_entry<PREC, 1, true>() : small_entry<PREC, 1, false>();
    if (dim == 2) return vark ? small_entry<PREC, 2, true>() : small_entry<PREC, 2, false>();
    return vark ? small_entry<PREC, 3, true>() : small_entry<PREC, 3, false>();
}

long long small_need(int prec, bool vark, long long n) {
    if (prec == PREC_F64) return vark ? small_bytes<PREC_F64, true>(n) : small_bytes<PREC_F64, false>(n);
    if (prec == PREC_F32) return vark ? small_bytes<PREC_F32, true>(n) : small_bytes<PREC_F32, false>(n);
    return vark ? small_bytes<PREC_DF, true>(n) : small_bytes<PREC_DF, false>(n);
}

}  // namespace

// Dynamic shared memory of the one-CTA solve, or 0 when the grid is too large
// for it (the limit leaves room for the block's own reduction arrays).
int small_solve_smem(int prec, bool vark, const GridGeo &g) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long need = small_need(prec, vark, n);
    return need <= 200 * 1024 ? (int)need : 0;
}

cudaError_t small_solve_launch(int prec, bool vark, const PassLaunch &a, cudaStream_t s) {
    const int smem = small_solve_smem(prec, vark, a.geo);
    void *k = prec == PREC_F64 ? small_pick<PREC_F64>(a.geo.dim, vark)
              : prec == PREC_F32 ? small_pick<PREC_F32>(a.geo.dim, vark)
                                 : small_pick<PREC_DF>(a.geo.dim, vark);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(k, dim3(1), dim3(kSmallThreads), args, smem, s);
}

}  // namespace srj
