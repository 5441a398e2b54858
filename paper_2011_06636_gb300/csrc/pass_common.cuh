// pass_common.cuh -- device-side cycle bookkeeping shared by every SRJ pass
// kernel (included by each kernel translation unit; everything is
// file-local).
//
// Each pass reads the solve state at its start (plan_pass), does its sweeps
// and/or residual, and the last CTA to take a ticket folds the per-CTA
// residual partials in a fixed order and advances the state (advance_state):
// cycle bookkeeping, ratio = r_after / r_before, convergence test and the
// next level by Sec. 3, Alg. 1.  No CTA ever waits for another.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "mlp.cuh"
#include "srj_internal.h"

namespace srj {
namespace {

// ----------------------------------------------------------- state decisions
struct PassPlan {
    int run;     // 0: solve finished, nothing to do
    int resid;   // 1: this pass computes the residual norm
    int nsw;     // sweeps done by this pass (0 or 1 here)
    int cur;     // source buffer
    int woff;    // index of this sweep's factor in the tables
};

__device__ __forceinline__ PassPlan plan_pass(const DevState *st, const int *lvl_m,
                                              const int *lvl_off, int depth) {
    PassPlan p{};
    if (st->status != DST_RUNNING) return p;
    p.run = 1;
    p.cur = st->cur;
    if (st->phase == 0) {
        p.resid = 1;
        return p;
    }
    // plain Jacobi (Sec. 2, Eq. jacobi): cycles of M(fixed_level) sweeps
    // with omega = 1, read from the ones at the end of the factor tables
    const bool jac = st->selector == DSEL_JACOBI;
    const int M = lvl_m[jac ? st->fixed_level : st->level];
    const int rem = M - st->k;
    // A cycle of M sweeps takes floor(M / depth) + 1 passes; the last one does
    // rem < depth sweeps and then the residual of the cycle's final state.
    p.nsw = rem >= depth ? depth : rem;
    p.resid = rem < depth ? 1 : 0;
    p.woff = jac ? kTotalOmegas : lvl_off[st->level] + st->k;
    return p;
}

// With a two-sweep kernel beside it, a one-sweep kernel runs only the tail of
// a cycle: the initial residual, a single remaining sweep, the residual.
__device__ __forceinline__ bool pass_is_tail(const DevState *st, const int *lvl_m) {
    if (st->phase == 0) return true;
    const bool jac = st->selector == DSEL_JACOBI;
    return lvl_m[jac ? st->fixed_level : st->level] - st->k < 2;
}

__device__ __forceinline__ PassPlan plan_pass(const PassLaunch &a, int depth) {
    return plan_pass(a.st, a.lvl_m, a.lvl_off, depth);
}

__device__ __forceinline__ int next_level(DevState *st, const SolveCfg &cfg, double ratio,
                                          int level, int mlp_pick) {
    const int top = st->max_level;
    if (st->selector == DSEL_MLP) {
        // the network picks; Alg. 1 judges.  The finished cycle's average
        // convergence rate (Sec. 3, Eq. average-convergence-rate; st->k is
        // its M) is compared with that of the latest cycle Alg. 1 chose: a
        // picked cycle that did not shrink the residual, or shrank it more
        // slowly per sweep than Alg. 1's did, hands the next decision back to
        // Alg. 1.  The first cycle counts as Alg. 1's.
        const double rate = -log(ratio) / (double)(st->k > 0 ? st->k : 1);
        bool take = mlp_pick >= 0;
        if (st->mlp_last) take = take && ratio < 1.0 && rate >= st->alg1_rate;
        else st->alg1_rate = rate;
        if (take) {
            st->mlp_last = 1;
            return mlp_pick < top ? mlp_pick : top;
        }
        if (st->mlp_last) st->mlp_fallbacks += 1;
        st->mlp_last = 0;
    }
    switch (st->selector) {
        case DSEL_INCREASING:
            return level < top ? level + 1 : level;
        case DSEL_FIXED:
            return st->fixed_level;
        case DSEL_JACOBI:  // no scheme level: every cycle is M(fixed_level) plain sweeps
            return level;
        case DSEL_SCHEDULE:
            return (st->cycles < st->nsched) ? cfg.sched[st->cycles] : level;
        default:  // Alg. 1 (also the fallback of the learned selector)
            if (ratio > 0.4) return level < top ? level + 1 : level;
            if (ratio < 0.4 && ratio > 0.2) return level > 0 ? level - 1 : level;
            return level;
    }
}

// log of a residual ratio as the selector's features use it
__device__ __forceinline__ float hist_log(double ratio) {
    const double l = ratio > 0 ? log(ratio) : -20.0;
    return (float)(l < -20.0 ? -20.0 : (l > 5.0 ? 5.0 : l));
}

// Executed by one thread of the last CTA of a pass.  mlp_pick is the learned
// selector's choice for the next cycle (-1 when not evaluated); dmax is the
// largest |u' - u| of this pass's sweep (negative when not measured).
__device__ void advance_state(DevState *st, const SolveCfg &cfg, const PassPlan &p,
                              double norm2, int mlp_pick = -1, double dmax = -1.0) {
    st->passes += 1;
    if (st->status != DST_RUNNING) return;  // a CTA of this pass recorded a failure
    if (p.nsw > 0) {
        st->cur ^= 1;
        st->k += p.nsw;
        st->sweeps += p.nsw;
        if (dmax >= 0.0 || dmax != dmax) {
            // Sec. 4.2.2: stop after the first sweep whose largest change is
            // below tol, inside the cycle if need be (NaN never is)
            st->dlast = dmax;
            if (dmax < st->tol) {
                st->status = DST_CONVERGED;
                return;
            }
        }
    }
    if (!p.resid) return;
    const double rn = sqrt(norm2);
    if (st->phase == 0) {
        st->phase = 1;
        st->r0 = rn;
        st->rprev = rn;
        st->rn = rn;
        if (!isfinite(rn)) st->status = DST_DIVERGED;
        else if (st->tol_kind != SRJ_TOL_DINF &&
                 (rn == 0.0 || (st->tol_kind == SRJ_TOL_ABS && rn < st->tol)))
            st->status = DST_CONVERGED;
        return;
    }
    const double ratio = rn / st->rprev;
    st->rprev = rn;
    st->rn = rn;
    for (int i = 7; i > 0; --i) st->hist[i] = st->hist[i - 1];
    st->hist[0] = hist_log(ratio);
    st->nhist = st->nhist < 8 ? st->nhist + 1 : 8;
    const long long c = st->cycles;
    const long long ti = c + st->trace_base;
    if (ti < cfg.trace_cap) {
        cfg.trace_level[ti] = st->level;
        cfg.trace_rn[ti] = rn;
    }
    st->cycles = c + 1;
    const double test = (st->tol_kind == SRJ_TOL_ABS) ? rn : rn / st->r0;
    if (!isfinite(rn)) {
        st->status = DST_DIVERGED;
    } else if (st->tol_kind != SRJ_TOL_DINF && test < st->tol) {
        st->status = DST_CONVERGED;
    } else if (st->selector == DSEL_SCHEDULE && st->cycles >= st->nsched) {
        st->status = DST_DONE;
    } else if (st->stall_stop && ratio >= 1.0) {
        st->status = DST_STALLED;
    } else if (st->sweeps >= st->max_sweeps) {
        st->status = DST_NOTCONV;
    } else {
        st->level = next_level(st, cfg, ratio, st->level, mlp_pick);
        st->k = 0;
    }
}

// The learned selector's pick for the cycle after the one whose residual this
// pass completed, evaluated by one full warp (every lane returns it); -1 when
// the selector is not the network or no cycle ended.
__device__ __forceinline__ int mlp_pick_at_cycle_end(const DevState *st, const SolveCfg &cfg,
                                                     const PassPlan &p, double norm2,
                                                     const int *lvl_m, int lane) {
    if (!p.resid || st->phase == 0 || st->selector != DSEL_MLP || cfg.mlp_w == nullptr)
        return -1;
    const double ratio = sqrt(norm2) / st->rprev;
    float hist[8];
    hist[0] = hist_log(ratio);
    for (int i = 1; i < 8; ++i) hist[i] = st->hist[i - 1];
    const int nh = st->nhist < 8 ? st->nhist + 1 : 8;
    float x[kMlpIn];
    mlp_features(x, hist, nh, st->npoints, st->dim, st->level, lvl_m[st->level]);
    return mlp_pick_warp(cfg.mlp_w, x, lane, nullptr, st->level, st->max_level);
}

// Deterministic block sum: butterfly within warps, then warps in order.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double s_warp[32];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthreads = blockDim.x * blockDim.y;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) s_warp[tid >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (tid == 0)
        for (int w = 0; w < (nthreads + 31) / 32; ++w) t += s_warp[w];
    return t;  // valid in thread 0
}

// |a - b| as the bit pattern of a non-negative double.  Such patterns order
// like the values they encode, and a NaN (exponent all ones, mantissa not
// zero) lies above +inf, so an integer max of them is the largest change with
// a NaN kept, taken on the integer units instead of FP64 compares (FP64 issues
// at a small fraction of the FP32 rate on this part).
__device__ __forceinline__ long long abs_diff_bits(double a, double b) {
    return __double_as_longlong(a - b) & 0x7fffffffffffffffLL;
}

__device__ __forceinline__ long long max_bits(long long a, long long b) { return a > b ? a : b; }

// Block max of abs_diff_bits values, returned as the double (valid in thread 0).
__device__ __forceinline__ double block_max_bits(long long v) {
    __shared__ long long s_wbits[32];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthreads = blockDim.x * blockDim.y;
    for (int o = 16; o > 0; o >>= 1) v = max_bits(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((tid & 31) == 0) s_wbits[tid >> 5] = v;
    __syncthreads();
    long long t = 0;
    if (tid == 0)
        for (int w = 0; w < (nthreads + 31) / 32; ++w) t = max_bits(t, s_wbits[w]);
    return __longlong_as_double(t);
}

// Ticket + last-CTA finish, shared by all pass kernels.  block_total is the
// CTA's partial (valid in thread 0): the residual sum of a residual pass, or,
// with dinf set, the largest |u' - u| of a sweep pass.  Returns after the
// bookkeeping.
__device__ void finish_pass(const PassLaunch &a, const PassPlan &p, double block_total,
                            bool dinf = false) {
    __shared__ int s_last;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const unsigned int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const bool dpass = dinf && p.nsw > 0;
    if (tid == 0) {
        if (p.resid || dpass) a.partials[bid] = block_total;
        __threadfence();
        const unsigned int t = atomicAdd(&a.st->ticket, 1u);
        s_last = (t == nblocks - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the whole CTA folds the partials (written by other CTAs: read from L2),
    // each thread a fixed stride of them, then the block in a fixed order:
    // deterministic for a given grid
    const int nthreads = blockDim.x * blockDim.y;
    double norm2 = 0.0, dmax = -1.0;
    if (p.resid) {
        double acc = 0.0;
#pragma unroll 4
        for (unsigned int i = tid; i < nblocks; i += nthreads) acc += __ldcg(a.partials + i);
        norm2 = block_sum(acc);
    } else if (dpass) {
        long long acc = 0;
#pragma unroll 4
        for (unsigned int i = tid; i < nblocks; i += nthreads)
            acc = max_bits(acc, __double_as_longlong(__ldcg(a.partials + i)));
        dmax = block_max_bits(acc);
    }
    if (tid < 32) norm2 = __shfl_sync(0xffffffffu, norm2, 0);  // block totals sit in thread 0
    int pick = -1;
    if (tid < 32) pick = mlp_pick_at_cycle_end(a.st, a.cfg, p, norm2, a.lvl_m, tid);
    if (tid == 0) {
        DevState *st = a.st;
        advance_state(st, a.cfg, p, norm2, pick, dmax);
        st->ticket = 0;
        __threadfence();
        if (a.cfg.use_cond && st->status != DST_RUNNING)
            cudaGraphSetConditional(a.cfg.cond, 0);
    }
}

}  // namespace
}  // namespace srj
