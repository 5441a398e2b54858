// kernels_wave2d.cu -- temporally blocked SRJ pass for 2D constant-coefficient
// grids (Poisson and the anisotropic -eps_x u_xx - eps_y u_yy).
//
// One pass applies up to T consecutive relaxation factors of the current
// cycle (Sec. 2, Eq. relaxed-jacobi) while reading the iterate and f from HBM
// once and writing the iterate once.  The last pass of a cycle (fewer than T
// sweeps) also forms the residual of the cycle's final state, so the norm
// that drives Alg. 1 costs no extra pass over memory.
//
// Work decomposition (no CTA-wide synchronisation at all):
//  * a warp owns a strip of 32*V columns; lane l holds V consecutive columns.
//    Horizontal neighbours move by warp shuffles, so the outer H columns of a
//    strip lose validity one per sweep and only the inner 32V - 2H columns are
//    written (H >= T, aligned to 16 bytes).
//  * the warp streams down (or up) a segment of rows as a wavefront: at step
//    t it loads row j(t) into level 0 and computes level s (sweep s) at row
//    j(t) -+ s, keeping the last three rows of every level in registers.
//    Neighbouring segments stream in opposite directions so that the rows
//    they share are read at about the same time (L2 hits).
//  * rows and f arrive through per-warp shared-memory rings filled by
//    cp.async with zero fill outside the grid (the Dirichlet ghosts); each
//    lane reads back only what it copied, so a per-thread wait suffices.
#include <cuda_runtime.h>

#include <type_traits>

#include "pass_common.cuh"
#include "stencil_point.cuh"
#include "srj_internal.h"

namespace srj {
namespace {

constexpr int kWarps = 8;  // warps per CTA
constexpr int kPD = 3;     // prefetch distance (steps)

template <int PREC>
struct WaveTraits;
template <>
struct WaveTraits<PREC_F32> {
    static constexpr int V = 4;
    static constexpr int ES = 4;  // bytes per element of the iterate / f
    static constexpr bool LO = false;
};
template <>
struct WaveTraits<PREC_DF> {
    static constexpr int V = 4;
    static constexpr int ES = 4;
    static constexpr bool LO = true;
};
template <>
struct WaveTraits<PREC_F64> {
    static constexpr int V = 2;
    static constexpr int ES = 8;
    static constexpr bool LO = false;
};

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
    static constexpr int WC = 32 * V;                 // strip width (columns)
    static constexpr int H = wave_halo(T, V, Tr::ES);  // halo columns per side
    static constexpr int OUTW = WC - 2 * H;           // written columns per strip
    static constexpr int UR = kPD + 1;                // iterate ring slots
    static constexpr int FR = T + 2 + kPD;            // rhs ring slots
    static constexpr int CHUNK = (Tr::ES == 8 && (H % 2)) ? 8 : 16;
    static constexpr int ROWB = WC * Tr::ES;          // bytes per ring row
    static constexpr int SMEM_WARP = (UR * (Tr::LO ? 2 : 1) + FR) * ROWB;
};

struct WaveDims {
    int nstrips, nsegs, R, nitems;
};

// CTAs per SM the register budget is sized for: the deep FP32 and the
// FP32-pair instantiations keep more rows of levels in registers than the
// 128 registers of a two-CTA budget allow without spilling.
template <int PREC, int T>
constexpr int wave_min_blocks() {
    return ((PREC == PREC_F32 && T >= 8) || (PREC == PREC_DF && T >= 4)) ? 1 : 2;
}

template <int PREC, int T>
__global__ void __launch_bounds__(32 * kWarps, (wave_min_blocks<PREC, T>()))
    wave2d_kernel(PassLaunch a, WaveDims wd) {
    using W = Wave<PREC, T>;
    using E = typename Elem<PREC>::T;  // state element
    using C = typename Elem<PREC>::C;  // rhs / coefficient element
    constexpr int V = W::V;
    constexpr int ES = WaveTraits<PREC>::ES;
    constexpr bool LO = WaveTraits<PREC>::LO;

    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PassPlan s_plan;
    __shared__ double s_omega[T];
    __shared__ double s_wsum[kWarps];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_plan = plan_pass(a, T);
        for (int s = 0; s < T; ++s) s_omega[s] = (s < s_plan.nsw) ? a.w64[s_plan.woff + s] : 0.0;
        if (!s_plan.run && a.cfg.use_cond && blockIdx.x == 0)
            cudaGraphSetConditional(a.cfg.cond, 0);
    }
    __syncthreads();
    const PassPlan p = s_plan;
    if (!p.run) return;

    const GridGeo &g = a.geo;
    const int nsw = p.nsw;
    C omega[T];
#pragma unroll
    for (int s = 0; s < T; ++s) omega[s] = (C)s_omega[s];
    const C diag = C(g.diag), invd = C(1.0 / g.diag);
    C acoef[3] = {C(g.cx / g.diag), C(g.cy / g.diag), C(0)};

    unsigned char *wbase = smem + warp * W::SMEM_WARP;
    unsigned char *uring = wbase;
    unsigned char *uring_lo = wbase + W::UR * W::ROWB;
    unsigned char *fring = wbase + W::UR * W::ROWB * (LO ? 2 : 1);

    const unsigned char *src = (const unsigned char *)a.bufs.u[p.cur];
    const unsigned char *src_lo = LO ? (const unsigned char *)a.bufs.ulo[p.cur] : nullptr;
    E *dst = nullptr;
    float *dst_hi = nullptr, *dst_lo = nullptr;
    if constexpr (LO) {
        dst_hi = (float *)a.bufs.u[p.cur ^ 1];
        dst_lo = (float *)a.bufs.ulo[p.cur ^ 1];
    } else {
        dst = (E *)a.bufs.u[p.cur ^ 1];
    }
    const unsigned char *fsrc = (const unsigned char *)a.bufs.f;
    const long long pitchB = g.pitch * ES;

    double acc_resid = 0.0;  // this lane's sum of r^2
    const int gwarp = blockIdx.x * kWarps + warp;
    const int nwarps = gridDim.x * kWarps;

    for (int item = gwarp; item < wd.nitems; item += nwarps) {
        const int strip = item % wd.nstrips, seg = item / wd.nstrips;
        const int xs = strip * W::OUTW - W::H;  // first column of the strip
        const int y0 = seg * wd.R;
        const int y1 = min(y0 + wd.R, g.ny);
        const int dir = (seg & 1) ? -1 : 1;
        const int nsteps = (y1 - y0) + 2 * T + 2;
        const int jbase = dir > 0 ? y0 - T - 1 : y1 + T;  // j(t) = jbase + dir * t
        const int col0 = xs + lane * V;                   // this lane's first column
        const bool edge = (xs < 0) || (xs + W::WC > g.nx);
        bool colok[V];
#pragma unroll
        for (int v = 0; v < V; ++v) colok[v] = (col0 + v >= 0) && (col0 + v < g.nx);
        bool outcol[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int c = lane * V + v;
            outcol[v] = (c >= W::H) && (c < W::WC - W::H) && colok[v];
        }

        // issue the copies of step t (row j(t) of the iterate and of f)
        auto issue = [&](int t) {
            const int row = jbase + dir * t;
            const bool rok = (row >= 0) && (row < g.ny);
            const int us = t % W::UR, fs = t % W::FR;
#pragma unroll
            for (int c = 0; c < (V * ES) / W::CHUNK; ++c) {
                const int colc = col0 + c * (W::CHUNK / ES);
                const bool ok = rok && colc >= 0 && colc < g.pitch;
                const long long off = (long long)row * pitchB + (long long)colc * ES;
                const int so = us * W::ROWB + lane * V * ES + c * W::CHUNK;
                const int fo = fs * W::ROWB + lane * V * ES + c * W::CHUNK;
                cp_async(uring + so, src + off, W::CHUNK, ok, src);
                if constexpr (LO) cp_async(uring_lo + so, src_lo + off, W::CHUNK, ok, src_lo);
                cp_async(fring + fo, fsrc + off, W::CHUNK, ok, fsrc);
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
        float kahan_s = 0.f, kahan_c = 0.f;  // FP32 paths: compensated r^2 sum
        double dsum = 0.0;                   // FP64 path

        __syncwarp();
        for (int t = 0; t < kPD; ++t) {
            if (t < nsteps) issue(t);
            cp_commit();
        }

        auto load_row = [&](unsigned char *ringb, int slot, int v) -> float {
            return ((const float *)(ringb + slot * W::ROWB))[lane * V + v];
        };

        auto step = [&](int t, auto phase_tag) {
            constexpr int PH = decltype(phase_tag)::value;
            constexpr int CUR = PH, CEN = (PH + 2) % 3, BEH = (PH + 1) % 3;
            if (t + kPD < nsteps) issue(t + kPD);
            cp_commit();
            cp_wait<kPD>();
            const int jt = jbase + dir * t;
            // level 0: row j(t)
            {
                const int us = t % W::UR;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if constexpr (PREC == PREC_F64) {
                        ring[0][CUR][v] = ((const double *)(uring + us * W::ROWB))[lane * V + v];
                    } else if constexpr (LO) {
                        ring[0][CUR][v] = df32{load_row(uring, us, v), load_row(uring_lo, us, v)};
                    } else {
                        ring[0][CUR][v] = load_row(uring, us, v);
                    }
                }
            }
            // levels 1..T
#pragma unroll
            for (int s = 1; s <= T; ++s) {
                if (t < 2 * s) continue;  // row not needed by any output
                const int row = jt - dir * s;
                if (s > nsw) {  // identity level (last pass of a cycle)
#pragma unroll
                    for (int v = 0; v < V; ++v) ring[s][CUR][v] = ring[s - 1][CEN][v];
                    continue;
                }
                const int fs = (t - s) % W::FR;
                C fv[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if constexpr (PREC == PREC_F64)
                        fv[v] = ((const double *)(fring + fs * W::ROWB))[lane * V + v];
                    else
                        fv[v] = load_row(fring, fs, v);
                }
                E left, right;
                if constexpr (LO) {
                    left = df32{__shfl_up_sync(0xffffffffu, ring[s - 1][CEN][V - 1].hi, 1),
                                __shfl_up_sync(0xffffffffu, ring[s - 1][CEN][V - 1].lo, 1)};
                    right = df32{__shfl_down_sync(0xffffffffu, ring[s - 1][CEN][0].hi, 1),
                                 __shfl_down_sync(0xffffffffu, ring[s - 1][CEN][0].lo, 1)};
                } else {
                    left = __shfl_up_sync(0xffffffffu, ring[s - 1][CEN][V - 1], 1);
                    right = __shfl_down_sync(0xffffffffu, ring[s - 1][CEN][0], 1);
                }
                const bool rok = (row >= 0) && (row < g.ny);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    E nb[6];
                    nb[0] = v > 0 ? ring[s - 1][CEN][v - 1] : left;
                    nb[1] = v < V - 1 ? ring[s - 1][CEN][v + 1] : right;
                    nb[2] = ring[s - 1][BEH][v];
                    nb[3] = ring[s - 1][CUR][v];
                    const E uc = ring[s - 1][CEN][v];
                    const E tt = Point<PREC, 2>::t_const(nb, acoef, invd, fv[v], uc);
                    E un = Point<PREC, 2>::relax(uc, tt, (double)omega[s - 1]);
                    if (!rok || (edge && !colok[v])) un = zero_u<PREC>();
                    ring[s][CUR][v] = un;
                }
            }
            // output: level T at row j(t) - dir*T
            {
                const int row = jt - dir * T;
                if (p.nsw > 0 && row >= y0 && row < y1) {
                    const long long base = (long long)row * g.pitch + col0;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        if (!outcol[v]) continue;
                        if constexpr (LO) {
                            dst_hi[base + v] = ring[T][CUR][v].hi;
                            dst_lo[base + v] = ring[T][CUR][v].lo;
                        } else {
                            dst[base + v] = ring[T][CUR][v];
                        }
                    }
                }
            }
            // residual of the final state at row j(t) - dir*(T+1)
            if (p.resid && t >= 2 * T + 2) {
                const int row = jt - dir * (T + 1);
                const int fs = (t - T - 1) % W::FR;
                E left, right;
                if constexpr (LO) {
                    left = df32{__shfl_up_sync(0xffffffffu, ring[T][CEN][V - 1].hi, 1),
                                __shfl_up_sync(0xffffffffu, ring[T][CEN][V - 1].lo, 1)};
                    right = df32{__shfl_down_sync(0xffffffffu, ring[T][CEN][0].hi, 1),
                                 __shfl_down_sync(0xffffffffu, ring[T][CEN][0].lo, 1)};
                } else {
                    left = __shfl_up_sync(0xffffffffu, ring[T][CEN][V - 1], 1);
                    right = __shfl_down_sync(0xffffffffu, ring[T][CEN][0], 1);
                }
                if (row >= y0 && row < y1) {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        if (!outcol[v]) continue;
                        C fvv;
                        if constexpr (PREC == PREC_F64)
                            fvv = ((const double *)(fring + fs * W::ROWB))[lane * V + v];
                        else
                            fvv = load_row(fring, fs, v);
                        E nb[6];
                        nb[0] = v > 0 ? ring[T][CEN][v - 1] : left;
                        nb[1] = v < V - 1 ? ring[T][CEN][v + 1] : right;
                        nb[2] = ring[T][BEH][v];
                        nb[3] = ring[T][CUR][v];
                        const E tt = Point<PREC, 2>::t_const(nb, acoef, invd, fvv, ring[T][CEN][v]);
                        if constexpr (PREC == PREC_F64) {
                            const double r = diag * tt;
                            dsum = fma(r, r, dsum);
                        } else {
                            float r;
                            if constexpr (LO) r = diag * tt.hi;
                            else r = diag * tt;
                            // Kahan: sum += r^2
                            const float y = fmaf(r, r, -kahan_c);
                            const float sum = kahan_s + y;
                            kahan_c = (sum - kahan_s) - y;
                            kahan_s = sum;
                        }
                    }
                }
            }
        };

        using P0 = std::integral_constant<int, 0>;
        using P1 = std::integral_constant<int, 1>;
        using P2 = std::integral_constant<int, 2>;
        int t = 0;
        for (; t + 3 <= nsteps; t += 3) {
            step(t, P0{});
            step(t + 1, P1{});
            step(t + 2, P2{});
        }
        if (t < nsteps) step(t, P0{});
        if (t + 1 < nsteps) step(t + 1, P1{});
        cp_wait<0>();
        __syncwarp();
        if constexpr (PREC == PREC_F64) acc_resid += dsum;
        else acc_resid += (double)kahan_s - (double)kahan_c;
    }

    // CTA partial: lanes in a fixed butterfly, warps in order
    double tot = 0.0;
    if (p.resid) {
        double v = acc_resid;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_wsum[warp] = v;
        __syncthreads();
        if (tid == 0)
            for (int w = 0; w < kWarps; ++w) tot += s_wsum[w];
    }
    finish_pass(a, p, tot);
}

template <int PREC, int T>
struct WaveLaunch {
    static void *entry() { return (void *)&wave2d_kernel<PREC, T>; }
    static int smem() { return kWarps * Wave<PREC, T>::SMEM_WARP; }
    static int outw() { return Wave<PREC, T>::OUTW; }
    static int per_sm() { return wave_min_blocks<PREC, T>(); }
};

struct WaveCfg {
    void *entry;
    int smem;
    int outw;
    int per_sm;
};

WaveCfg wave_cfg(int prec, int T) {
#define WC_(P, TT) \
    WaveCfg{WaveLaunch<P, TT>::entry(), WaveLaunch<P, TT>::smem(), WaveLaunch<P, TT>::outw(), \
            WaveLaunch<P, TT>::per_sm()}
    if (prec == PREC_F32) {
        if (T == 4) return WC_(PREC_F32, 4);
        return WC_(PREC_F32, 8);
    }
    if (prec == PREC_DF) {
        if (T == 2) return WC_(PREC_DF, 2);
        return WC_(PREC_DF, 4);
    }
    if (T == 2) return WC_(PREC_F64, 2);
    return WC_(PREC_F64, 1);
#undef WC_
}

}  // namespace

int wave2d_depth(int prec, int requested) {
    if (prec == PREC_F32) return requested == 4 ? 4 : 8;
    if (prec == PREC_DF) return requested == 2 ? 2 : 4;
    return requested == 2 ? 2 : 1;
}

Wave2dPlan wave2d_plan(int prec, int T, const GridGeo &g, int num_sms) {
    WaveCfg c = wave_cfg(prec, T);
    Wave2dPlan p{};
    p.T = T;
    p.entry = c.entry;
    p.smem = c.smem;
    p.block = 32 * kWarps;
    p.nstrips = (g.nx + c.outw - 1) / c.outw;
    // aim at about one item per resident warp, but keep segments tall enough
    // that the wavefront warm-up (2T + 2 rows) stays a small fraction of the
    // work
    const int warps = num_sms * c.per_sm * kWarps;
    int nsegs = (warps + p.nstrips - 1) / p.nstrips;
    int R = (g.ny + nsegs - 1) / nsegs;
    const int rmin = 8 * T + 16;
    if (R < rmin) R = rmin;
    if (R > g.ny) R = g.ny;
    p.R = R;
    p.nsegs = (g.ny + R - 1) / R;
    p.nitems = p.nstrips * p.nsegs;
    const int ctas = (p.nitems + kWarps - 1) / kWarps;
    p.grid = ctas < num_sms * c.per_sm ? ctas : num_sms * c.per_sm;
    return p;
}

cudaError_t wave2d_prepare(int prec, int T) {
    WaveCfg c = wave_cfg(prec, T);
    return cudaFuncSetAttribute(c.entry, cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
}

cudaError_t wave2d_launch(const Wave2dPlan &p, const PassLaunch &a, cudaStream_t s) {
    WaveDims wd{p.nstrips, p.nsegs, p.R, p.nitems};
    void *args[] = {(void *)&a, (void *)&wd};
    return cudaLaunchKernel(p.entry, dim3(p.grid), dim3(p.block), args, p.smem, s);
}

cudaError_t add_wave2d_node(const Wave2dPlan &p, const PassLaunch &a, cudaGraph_t body) {
    WaveDims wd{p.nstrips, p.nsegs, p.R, p.nitems};
    void *args[] = {(void *)&a, (void *)&wd};
    cudaKernelNodeParams kp{};
    kp.func = p.entry;
    kp.gridDim = dim3(p.grid);
    kp.blockDim = dim3(p.block);
    kp.sharedMemBytes = p.smem;
    kp.kernelParams = args;
    cudaGraphNode_t node;
    return cudaGraphAddKernelNode(&node, body, nullptr, 0, &kp);
}

}  // namespace srj
