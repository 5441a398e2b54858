// kernels_collect.cu -- the data collection of Sec. 3, the procedure the
// heuristic of Alg. 1 was read from, on the 1D Poisson systems the paper
// collects on (Sec. 3, Eq. poisson: -u'' = f, N interior points, h = 1/(N+1),
// zero Dirichlet values, b = 1 and x = 0 by default).
//
// One CTA runs one trial entirely in shared memory: a first cycle at level 0,
// then steps.  At each step every allowed move (decrease, keep, increase the
// level inside [0, max_level]) is tried from the current iterate, one cycle
// each, and recorded with the state (residual ratio of the previous cycle,
// current level) and the residual norms before and after its cycle -- the
// average convergence rate of Eq. average-convergence-rate follows from
// them.  One tried move is then taken at random, and its iterate, level and
// ratio become the next state.  A trial ends once the taken residual norm is
// below tol (the paper: 1e-8) or after max_steps steps.
//
// The random move is drawn by a counter-based generator, the output function
// of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) applied to
// seed + (index + 1) * 0x9E3779B97F4A7C15 with index = trial * 2^32 + step;
// the move is candidate floor(u * ncand), u = (output >> 11) * 2^-53, in
// integer arithmetic.  Each trial writes its records to its own slice of the
// output, so trials never touch each other's memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "srj_internal.h"

namespace srj {
namespace {

constexpr int kCollectThreads = 128;
constexpr int kCollectMaxN = 4096;  // 6 FP64 arrays of N in shared memory

struct CollectArgs {
    int n;
    double a_off;  // 1 / h^2: the off-diagonal magnitude of A
    double diag;   // 2 / h^2
    double invd;   // h^2 / 2
    const double *f;  // device array of n values, or null for b = 1
    double tol;
    int max_level;
    uint64_t seed;
    long long trial0;
    int max_steps;
    srj_move_record *out;  // ntrials slices of 3 * max_steps records
    int32_t *counts;       // records written per trial
    const double *w64;     // factor tables (Leja order), kTableOmegas
    int lvl_m[kNumLevels];
    int lvl_off[kNumLevels];
};

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t index) {
    uint64_t z = seed + (index + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int draw_move(uint64_t seed, long long trial, int step, int ncand) {
    const uint64_t index = ((uint64_t)trial << 32) + (uint64_t)step;
    const uint64_t bits = splitmix64(seed, index) >> 11;
    return (int)((bits * (uint64_t)ncand) >> 53);
}

// ||f - A x||_2 over the block: per-thread strided sums, a fixed butterfly in
// each warp, warps added in order by thread 0; every thread returns it.
__device__ double resid_norm(const CollectArgs &a, const double *x, const double *f) {
    __shared__ double s_w[kCollectThreads / 32];
    __shared__ double s_tot;
    const int tid = threadIdx.x;
    double acc = 0.0;
    for (int i = tid; i < a.n; i += kCollectThreads) {
        const double xm = i > 0 ? x[i - 1] : 0.0;
        const double xp = i + 1 < a.n ? x[i + 1] : 0.0;
        const double r = f[i] - (a.diag * x[i] - a.a_off * (xm + xp));
        acc = fma(r, r, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((tid & 31) == 0) s_w[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kCollectThreads / 32; ++w) t += s_w[w];
        s_tot = sqrt(t);
    }
    __syncthreads();
    return s_tot;
}

// One cycle of scheme level `level` (Sec. 2, Eq. relaxed-jacobi, the level's
// M factors in the table's order) on *x, ping-ponging with *tmp; on return
// *x holds the result (the two pointers may have been exchanged).
__device__ void run_cycle(const CollectArgs &a, int level, double *&x, double *&tmp,
                          const double *f) {
    const int M = a.lvl_m[level];
    const double *w = a.w64 + a.lvl_off[level];
    for (int j = 0; j < M; ++j) {
        const double om = w[j];
        for (int i = threadIdx.x; i < a.n; i += kCollectThreads) {
            const double xm = i > 0 ? x[i - 1] : 0.0;
            const double xp = i + 1 < a.n ? x[i + 1] : 0.0;
            const double r = f[i] - (a.diag * x[i] - a.a_off * (xm + xp));
            tmp[i] = x[i] + om * (r * a.invd);
        }
        __syncthreads();
        double *t = x;
        x = tmp;
        tmp = t;
    }
}

__global__ void __launch_bounds__(kCollectThreads) collect_kernel(CollectArgs a) {
    extern __shared__ __align__(16) double sm[];
    const int n = a.n, tid = threadIdx.x;
    double *u = sm, *f = sm + n, *tmp = sm + 2 * n;
    double *cand[3] = {sm + 3 * n, sm + 4 * n, sm + 5 * n};
    const long long trial = a.trial0 + blockIdx.x;
    srj_move_record *out = a.out + (long long)blockIdx.x * 3 * a.max_steps;

    for (int i = tid; i < n; i += kCollectThreads) {
        u[i] = 0.0;
        f[i] = a.f ? a.f[i] : 1.0;
    }
    __syncthreads();
    const double r0 = resid_norm(a, u, f);
    run_cycle(a, 0, u, tmp, f);  // the first cycle, at level 0
    double rcur = resid_norm(a, u, f);
    double prev = r0 > 0.0 ? rcur / r0 : 0.0;
    int L = 0;
    int nrec = 0;
    for (int step = 0; step < a.max_steps && !(rcur < a.tol); ++step) {
        int ncand = 0, clevel[3];
        double rc[3];
        for (int mv = -1; mv <= 1; ++mv) {
            const int c = L + mv;
            if (c < 0 || c > a.max_level) continue;
            double *x = cand[ncand];
            for (int i = tid; i < n; i += kCollectThreads) x[i] = u[i];
            __syncthreads();
            run_cycle(a, c, x, tmp, f);
            cand[ncand] = x;  // the buffer holding the result
            rc[ncand] = resid_norm(a, x, f);
            clevel[ncand] = c;
            if (tid == 0) {
                srj_move_record &r = out[nrec];
                r.prev_ratio = prev;
                r.r_before = rcur;
                r.r_after = rc[ncand];
                r.level = L;
                r.action = mv;
            }
            ++nrec;
            ++ncand;
        }
        const int k = draw_move(a.seed, trial, step, ncand);
        // the taken candidate's buffer becomes the iterate; the old iterate's
        // buffer takes its place among the candidate buffers
        double *t = u;
        u = cand[k];
        cand[k] = t;
        prev = rc[k] / rcur;
        rcur = rc[k];
        L = clevel[k];
    }
    if (tid == 0) a.counts[blockIdx.x] = nrec;
}

}  // namespace
}  // namespace srj

using namespace srj;

extern "C" srj_status srj_collect_moves(int64_t n, const double *f, double tol, int32_t max_level,
                                        uint64_t seed, int64_t trial0, int32_t ntrials,
                                        int32_t max_steps, srj_move_record *out, int32_t *counts,
                                        void *stream) {
    if (n < 1 || n > kCollectMaxN || !out || !counts || ntrials < 1 || max_steps < 1 ||
        max_level < 0 || max_level > kMaxLevel || trial0 < 0 || !(tol > 0) || !std::isfinite(tol))
        return SRJ_EINVAL;
    if ((long long)trial0 + ntrials > (1LL << 31)) return SRJ_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> w(kTableOmegas, 1.0);
    build_omega_table(w.data());
    double *dw = nullptr;
    if (cudaMalloc(&dw, kTableOmegas * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return SRJ_ENOMEM;
    }
    srj_status rc = SRJ_OK;
    CollectArgs a{};
    const double h = 1.0 / (double)(n + 1);
    a.n = (int)n;
    a.a_off = 1.0 / (h * h);
    a.diag = 2.0 * a.a_off;
    a.invd = 1.0 / a.diag;
    a.f = f;
    a.tol = tol;
    a.max_level = max_level;
    a.seed = seed;
    a.trial0 = trial0;
    a.max_steps = max_steps;
    a.out = out;
    a.counts = counts;
    a.w64 = dw;
    for (int l = 0; l < kNumLevels; ++l) {
        a.lvl_m[l] = kLevelM[l];
        a.lvl_off[l] = level_offset(l);
    }
    const int smem = 6 * (int)n * (int)sizeof(double);
    if (cudaMemcpyAsync(dw, w.data(), kTableOmegas * sizeof(double), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaFuncSetAttribute(collect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess)
        rc = SRJ_ECUDA;
    if (rc == SRJ_OK) {
        collect_kernel<<<(unsigned)ntrials, kCollectThreads, smem, s>>>(a);
        if (cudaGetLastError() != cudaSuccess) rc = SRJ_ECUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = SRJ_ECUDA;
    cudaFree(dw);
    return rc;
}
