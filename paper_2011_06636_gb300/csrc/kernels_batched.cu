// kernels_batched.cu -- one persistent kernel that advances many independent
// 2D constant-coefficient problems of uneven sizes at once, each through its
// own mixed-precision SRJ solve:
//
//   OUTER   FP64 r = f - A u on the user's arrays, ||r||, convergence test,
//           then r is stored (FP32) as the right-hand side of an inner solve;
//   INNER   SRJ on A e = r (Sec. 2 scheme family, Alg. 1 selection) with FP32
//           arithmetic on an FP32-pair iterate, temporally blocked passes
//           (wave_item.cuh), residual fused into each cycle's last pass;
//   UPDATE  FP64 u += e, and e is cleared for the next inner solve.
//
// Each launch does one step of every unfinished problem: the grid-stride warp
// loop walks a list of items (strip x segment of some problem), and the warp
// that completes the last item of a problem in this launch (per-problem
// ticket) folds that problem's partials in a fixed order and advances its
// state machine.  When the last problem finishes, that warp clears the loop
// condition of the CUDA graph (WHILE node around this kernel).  No warp ever
// waits for another.
#include <cuda_runtime.h>

#include "pass_common.cuh"
#include "srj_internal.h"
#include "wave_item.cuh"

namespace srj {
namespace {

// Warps per CTA: 6 for T = 2 (the FP32-pair item needs about 160 registers
// to keep its update chains without recomputation; see kernels_wave2d.cu).
template <int T>
__host__ __device__ constexpr int batch_warps() {
    return T == 2 ? 6 : kWaveWarps;
}

enum BatchPhase : int32_t { BPH_OUTER = 0, BPH_INNER = 1, BPH_UPDATE = 2, BPH_DONE = 3 };

template <int T>
constexpr int batch_min_blocks() {
    return T >= 4 ? 1 : 2;
}

// FP64 residual over the item's region of the user's dense arrays; writes the
// FP32 inner right-hand side and returns this lane's sum of r^2.
__device__ double outer_item(const BatchProb &P, int x0, int x1, int y0, int y1, int lane) {
    const GridGeo &g = P.geo;
    double acc = 0.0;
    for (int y = y0; y < y1; ++y) {
        for (int x = x0 + lane; x < x1; x += 32) {
            const long long i = (long long)y * g.nx + x;
            const double uc = P.u[i];
            const double uxm = x > 0 ? P.u[i - 1] : 0.0;
            const double uxp = x + 1 < g.nx ? P.u[i + 1] : 0.0;
            const double uym = y > 0 ? P.u[i - g.nx] : 0.0;
            const double uyp = y + 1 < g.ny ? P.u[i + g.nx] : 0.0;
            const double Au = g.cx * ((uc - uxm) + (uc - uxp)) + g.cy * ((uc - uym) + (uc - uyp));
            const double r = P.f[i] - Au;
            // scaled by D^-1: the FP32-pair sweeps read D^-1 f
            ((float *)P.inner.f)[(long long)y * g.pitch + x] = (float)(r / g.diag);
            acc = fma(r, r, acc);
        }
    }
    return acc;
}

// u += e[cur] over the item's region; e[cur] is cleared for the next solve.
__device__ void update_item(const BatchProb &P, int cur, int x0, int x1, int y0, int y1,
                            int lane) {
    const GridGeo &g = P.geo;
    float *eh = (float *)P.inner.u[cur];
    float *el = (float *)P.inner.ulo[cur];
    for (int y = y0; y < y1; ++y) {
        for (int x = x0 + lane; x < x1; x += 32) {
            const long long pp = (long long)y * g.pitch + x;
            P.u[(long long)y * g.nx + x] += (double)eh[pp] + (double)el[pp];
            eh[pp] = 0.f;
            el[pp] = 0.f;
        }
    }
}

// Advance problem p after all its items of this launch finished (lane 0).
__device__ void finalize_problem(const BatchLaunch &b, int p, const PassPlan &plan,
                                 double norm2, int pick) {
    BatchState &S = b.states[p];
    bool done = false;
    if (S.phase == BPH_OUTER) {
        const double rn = sqrt(norm2);
        S.rn = rn;
        if (S.outer == 0) S.r0 = rn;
        const double test = b.tol_kind == SRJ_TOL_ABS ? rn : (S.r0 > 0 ? rn / S.r0 : 0.0);
        if (!isfinite(rn)) {
            S.result = DST_DIVERGED;
            done = true;
        } else if (rn == 0.0 || test < b.tol) {
            S.result = DST_CONVERGED;
            done = true;
        } else if (S.outer >= b.max_outer || S.sweeps >= b.max_sweeps) {
            S.result = DST_NOTCONV;
            done = true;
        } else {
            DevState &in = S.in;
            const int cur = in.cur;  // the cleared buffer
            const long long left = b.max_sweeps - S.sweeps;
            // aim at the reduction still needed (margin 2), not below the
            // FP32-pair accuracy floor b.inner_tol
            const double target = b.tol_kind == SRJ_TOL_ABS ? b.tol : b.tol * S.r0;
            double eta = 0.5 * target / rn;
            if (eta < b.inner_tol) eta = b.inner_tol;
            if (eta > 0.5) eta = 0.5;
            in = DevState{};
            in.tol = eta;
            in.tol_kind = SRJ_TOL_REL;
            in.selector = b.selector;
            in.max_level = b.max_level;
            in.fixed_level = b.fixed_level;
            in.max_sweeps = left < 200000 ? left : 200000;
            in.stall_stop = b.stall_stop;
            in.level = S.carry;
            in.cur = cur;
            in.status = DST_RUNNING;
            in.dim = 2;
            in.npoints = (double)b.probs[p].geo.nx * (double)b.probs[p].geo.ny;
            S.phase = BPH_INNER;
        }
    } else if (S.phase == BPH_INNER) {
        DevState &in = S.in;
        advance_state(&in, b.cfg, plan, norm2, pick);
        if (in.status != DST_RUNNING) {
            S.sweeps += in.sweeps;
            S.cycles += in.cycles;
            S.passes += in.passes;
            S.final_level = in.level;
            if (in.status == DST_DIVERGED) {
                S.result = DST_DIVERGED;
                done = true;
            } else {
                S.carry = in.level - kInnerCarry > 0 ? in.level - kInnerCarry : 0;
                S.phase = BPH_UPDATE;
            }
        }
    } else if (S.phase == BPH_UPDATE) {
        S.outer += 1;
        S.phase = BPH_OUTER;
    }
    if (done) {
        S.phase = BPH_DONE;
        // its items leave the counts that choose the next launches' layout
        const BatchProb &P = b.probs[p];
        for (int l = 0; l < kBatchLayouts; ++l)
            atomicAdd((unsigned long long *)&b.active[l],
                      (unsigned long long)(-(long long)P.nitems[l]));
    }
    S.ticket = 0;
    __threadfence();
    if (done) {
        const unsigned int nd = atomicAdd(b.ndone, 1u);
        if (nd + 1 == (unsigned int)b.nprob && b.cfg.use_cond)
            cudaGraphSetConditional(b.cfg.cond, 0);
    }
}

template <int T>
__global__ void __launch_bounds__(32 * batch_warps<T>(), (batch_min_blocks<T>()))
    batched_kernel(BatchLaunch b) {
    using W = Wave<PREC_DF, T>;
    constexpr int kBW = batch_warps<T>();
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0 && *(volatile unsigned int *)b.ndone >=
                                                   (unsigned int)b.nprob && b.cfg.use_cond)
        cudaGraphSetConditional(b.cfg.cond, 0);
    unsigned char *wbase = smem + warp * W::SMEM_WARP;
    const int gwarp = blockIdx.x * kBW + warp;
    const int nwarps = gridDim.x * kBW;
    // this launch's layout: written only by the previous launch's last CTA
    const int lay = b.fixed_layout >= 0 ? b.fixed_layout : *(volatile const int32_t *)b.ctl;
    const int32_t *item_prob = b.item_prob[lay];

    for (int item = gwarp; item < b.total_items[lay]; item += nwarps) {
        const int p = item_prob[item];
        const BatchProb &P = b.probs[p];
        BatchState &S = b.states[p];
        const int phase = S.phase;  // uniform: same address for every lane
        if (phase == BPH_DONE) continue;
        const int li = item - P.item_base[lay];
        const int strip = li % P.nstrips, seg = li / P.nstrips;
        const int y0 = seg * P.R[lay];
        const int y1 = min(y0 + P.R[lay], P.geo.ny);
        const int x0 = strip * W::OUTW;
        const int x1 = min(x0 + W::OUTW, P.geo.nx);
        PassPlan plan{};
        double part = 0.0;
        if (phase == BPH_OUTER) {
            part = outer_item(P, x0, x1, y0, y1, lane);
        } else if (phase == BPH_INNER) {
            plan = plan_pass(&S.in, b.lvl_m, b.lvl_off, T);
            ItemCtx<PREC_DF, T> c;
            fill_ctx<PREC_DF, T>(c, P.geo, P.inner, plan.cur, plan.nsw, plan.resid, b.w64,
                                 plan.woff);
            const int dir = (seg & 1) ? -1 : 1;
            part = wave_item<PREC_DF, T>(c, strip, y0, y1, dir, wbase, lane);
        } else {
            update_item(P, S.in.cur, x0, x1, y0, y1, lane);
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        int last = 0;
        if (lane == 0) {
            b.partials[item] = part;
            __threadfence();
            last = atomicAdd(&S.ticket, 1u) == (unsigned int)(P.nitems[lay] - 1);
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            __threadfence();
            double acc = 0.0;
            const volatile double *pv = b.partials + P.item_base[lay];
            for (int i = lane; i < P.nitems[lay]; i += 32) acc += pv[i];
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            int pick = -1;
            if (phase == BPH_INNER) pick = mlp_pick_at_cycle_end(&S.in, b.cfg, plan, acc, b.lvl_m, lane);
            if (lane == 0) finalize_problem(b, p, plan, acc, pick);
        }
        __syncwarp();
    }
    // the launch's last CTA picks the next launch's layout: the tallest
    // segments whose items still cover the resident warps, else the shortest
    __syncthreads();
    if (threadIdx.x == 0 && b.fixed_layout < 0) {
        __threadfence();
        if (atomicAdd((unsigned int *)&b.ctl[1], 1u) == gridDim.x - 1) {
            __threadfence();
            int next = kBatchLayouts - 1;
            for (int l = 0; l < kBatchLayouts; ++l) {
                const long long act =
                    (long long)atomicAdd((unsigned long long *)&b.active[l], 0ull);
                if (act >= b.resident_warps) {
                    next = l;
                    break;
                }
            }
            b.ctl[0] = next;
            b.ctl[1] = 0;
            __threadfence();
        }
    }
}

}  // namespace

int batched_outw(int T) { return T >= 4 ? Wave<PREC_DF, 4>::OUTW : Wave<PREC_DF, 2>::OUTW; }

static void *batched_entry(int T) {
    return T >= 4 ? (void *)&batched_kernel<4> : (void *)&batched_kernel<2>;
}

static int batched_warps(int T) { return T >= 4 ? batch_warps<4>() : batch_warps<2>(); }

int batched_smem(int T) {
    return batched_warps(T) * (T >= 4 ? Wave<PREC_DF, 4>::SMEM_WARP : Wave<PREC_DF, 2>::SMEM_WARP);
}

int batched_grid(int T, int num_sms) { return num_sms * (T >= 4 ? 1 : 2); }

cudaError_t batched_prepare(int T) {
    return cudaFuncSetAttribute(batched_entry(T), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                batched_smem(T));
}

cudaError_t batched_launch(int T, int num_sms, const BatchLaunch &b, cudaStream_t s) {
    void *args[] = {(void *)&b};
    return cudaLaunchKernel(batched_entry(T), dim3(batched_grid(T, num_sms)),
                            dim3(32 * batched_warps(T)),
                            args, batched_smem(T), s);
}

cudaError_t add_batched_node(int T, int num_sms, const BatchLaunch &b, cudaGraph_t body) {
    void *args[] = {(void *)&b};
    cudaKernelNodeParams kp{};
    kp.func = batched_entry(T);
    kp.gridDim = dim3(batched_grid(T, num_sms));
    kp.blockDim = dim3(32 * batched_warps(T));
    kp.sharedMemBytes = batched_smem(T);
    kp.kernelParams = args;
    cudaGraphNode_t node;
    return cudaGraphAddKernelNode(&node, body, nullptr, 0, &kp);
}

}  // namespace srj
