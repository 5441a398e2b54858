// kernels_wave2d.cu -- temporally blocked SRJ pass for 2D constant-coefficient
// grids (Poisson and the anisotropic -eps_x u_xx - eps_y u_yy).
//
// One pass applies up to T consecutive relaxation factors of the current
// cycle (Sec. 2, Eq. relaxed-jacobi) while reading the iterate and f from HBM
// once and writing the iterate once.  The last pass of a cycle (fewer than T
// sweeps) also forms the residual of the cycle's final state, so the norm
// that drives Alg. 1 costs no extra pass over memory.
//
// Work decomposition (no CTA-wide synchronisation inside a pass): the grid
// is cut into items = (strip of 32*V columns, segment of rows); each warp
// takes items in a fixed grid-stride order and runs wave_item() on each (see
// wave_item.cuh).  Neighbouring segments stream in opposite directions so
// that the rows they share are read at about the same time (L2 hits).
#include <cuda_runtime.h>

#include "pass_common.cuh"
#include "srj_internal.h"
#include "wave_item.cuh"

namespace srj {
namespace {

// Warps per CTA.  The FP32-pair T = 2 pass needs about 160 registers per
// thread for all its independent update chains: at 8 warps x 2 CTAs (128
// registers) the compiler recomputes values instead of keeping them (8 % more
// instructions); 6 warps x 2 CTAs keep everything in registers and ran 6 %
// faster per pass on GB300.
template <int PREC, int T>
__host__ __device__ constexpr int wave_warps() {
    return (PREC == PREC_DF && T == 2) ? 6 : kWaveWarps;
}

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
__global__ void __launch_bounds__(32 * wave_warps<PREC, T>(), (wave_min_blocks<PREC, T>()))
    wave2d_kernel(PassLaunch a, WaveDims wd) {
    using W = Wave<PREC, T>;
    constexpr int kWarps = wave_warps<PREC, T>();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PassPlan s_plan;
    __shared__ double s_wsum[kWarps];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_plan = plan_pass(a, T);
        if (!s_plan.run && a.cfg.use_cond && blockIdx.x == 0)
            cudaGraphSetConditional(a.cfg.cond, 0);
    }
    __syncthreads();
    const PassPlan p = s_plan;
    if (!p.run) return;

    ItemCtx<PREC, T> c;
    fill_ctx<PREC, T>(c, a.geo, a.bufs, p.cur, p.nsw, p.resid, a.w64, p.woff);
    unsigned char *wbase = smem + warp * W::SMEM_WARP;

    double acc_resid = 0.0;  // this lane's sum of r^2
    const int gwarp = blockIdx.x * kWarps + warp;
    const int nwarps = gridDim.x * kWarps;
    for (int item = gwarp; item < wd.nitems; item += nwarps) {
        const int strip = item % wd.nstrips, seg = item / wd.nstrips;
        const int y0 = seg * wd.R;
        const int y1 = min(y0 + wd.R, a.geo.ny);
        // neighbouring segments stream in opposite directions
        const int dir = (seg & 1) ? -1 : 1;
        acc_resid += wave_item<PREC, T>(c, strip, y0, y1, dir, wbase, lane);
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
    static int smem() { return wave_warps<PREC, T>() * Wave<PREC, T>::SMEM_WARP; }
    static int outw() { return Wave<PREC, T>::OUTW; }
    static int per_sm() { return wave_min_blocks<PREC, T>(); }
    static int warps() { return wave_warps<PREC, T>(); }
};

struct WaveCfg {
    void *entry;
    int smem;
    int outw;
    int per_sm;
    int warps;
};

WaveCfg wave_cfg(int prec, int T) {
#define WC_(P, TT) \
    WaveCfg{WaveLaunch<P, TT>::entry(), WaveLaunch<P, TT>::smem(), WaveLaunch<P, TT>::outw(), \
            WaveLaunch<P, TT>::per_sm(), WaveLaunch<P, TT>::warps()}
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

// Default depths measured on GB300 at 4096^2 (mixed solve / FP32 leg): FP32
// pair 2 (1559 ms per solve vs 1710 ms at 4), FP32 4 (1074 vs 976 GLUP/s at
// 8): the shallower instantiations fit two CTAs per SM, and occupancy wins
// over fewer HBM passes.
int wave2d_depth(int prec, int requested) {
    if (prec == PREC_F32) return requested == 8 ? 8 : 4;
    if (prec == PREC_DF) return requested == 4 ? 4 : 2;
    return requested == 2 ? 2 : 1;
}

Wave2dPlan wave2d_plan(int prec, int T, const GridGeo &g, int num_sms) {
    WaveCfg c = wave_cfg(prec, T);
    Wave2dPlan p{};
    p.T = T;
    p.entry = c.entry;
    p.smem = c.smem;
    p.block = 32 * c.warps;
    p.nstrips = (g.nx + c.outw - 1) / c.outw;
    // at most one item per resident warp (an uneven split would leave a few
    // warps with two items and double the pass time), with segments tall
    // enough that the wavefront warm-up (about 3T rows) stays small
    const int warps = num_sms * c.per_sm * c.warps;
    int nsegs = warps / p.nstrips;
    if (nsegs < 1) nsegs = 1;
    int R = (g.ny + nsegs - 1) / nsegs;
    const int rmin = 8 * T + 16;
    if (R < rmin) R = rmin;
    if (R > g.ny) R = g.ny;
    p.R = R;
    p.nsegs = (g.ny + R - 1) / R;
    p.nitems = p.nstrips * p.nsegs;
    const int ctas = (p.nitems + c.warps - 1) / c.warps;
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
