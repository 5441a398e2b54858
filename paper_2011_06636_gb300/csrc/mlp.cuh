// mlp.cuh -- the learned scheme selector evaluated by one warp on the device.
//
// Not in the paper: it replaces the hand-derived rule of Alg. 1 (Sec. 3) with
// a small network over the solver state the paper's data collection records
// (recent residual ratios, current level) plus the problem size and
// dimension.  Alg. 1 stays as fallback and judge: a pick whose cycle did not
// shrink the residual hands the next decision back to Alg. 1.
//
//   x (12): log of the last 8 ratios (most recent first, 0 if absent, clipped
//           to [-20, 5]), log10(#points)/10, dim/3, level/24,
//           log(M(level))/log(2362)
//   h1 = relu(W1 x + b1) (64), h2 = relu(W2 h1 + b2) (64), z = W3 h2 + b3 (25)
//   pick = argmax z over the levels the paper's selector can move to from the
//          current level L, {L-1, L, L+1} within [0, top] (ties to the lower
//          level); without a current level (L < 0) over all 25 levels
// Weights are BF16 (parameter order W1, b1, W2, b2, W3, b3, row-major), every
// dot product is accumulated in FP32 in index order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace srj {
namespace {

constexpr int kMlpIn = 12, kMlpH = 64, kMlpOut = 25;
constexpr int kMlpW1 = 0, kMlpB1 = kMlpW1 + kMlpH * kMlpIn, kMlpW2 = kMlpB1 + kMlpH,
              kMlpB2 = kMlpW2 + kMlpH * kMlpH, kMlpW3 = kMlpB2 + kMlpH,
              kMlpB3 = kMlpW3 + kMlpOut * kMlpH, kMlpParams = kMlpB3 + kMlpOut;  // 6617

__device__ __forceinline__ float bf16_to_f32(uint16_t b) {
    return __uint_as_float(((uint32_t)b) << 16);
}

// Feature vector of the selector from the ratio history (hist[0] = most
// recent log ratio), the number of recorded ratios, problem size and level.
__device__ __forceinline__ void mlp_features(float *x, const float *hist, int nhist,
                                             double npoints, int dim, int level, int M) {
    for (int i = 0; i < 8; ++i) x[i] = i < nhist ? hist[i] : 0.f;
    x[8] = (float)(log10(npoints) / 10.0);
    x[9] = (float)dim / 3.f;
    x[10] = (float)level / 24.f;
    x[11] = (float)(log((double)M) / log(2362.0));
}

// Warp-cooperative forward pass; every lane passes the same x and receives
// the argmax (restricted to the moves from `level` when level >= 0).  logits
// (optional, lane-indexed) receives z[lane] for lane < 25.
__device__ __forceinline__ int mlp_pick_warp(const uint16_t *w, const float *x, int lane,
                                             float *logit_out, int level = -1, int top = 24) {
    // layer 1: lane owns units lane and lane + 32
    float h1[2];
    for (int q = 0; q < 2; ++q) {
        const int u = lane + 32 * q;
        float acc = bf16_to_f32(w[kMlpB1 + u]);
        for (int k = 0; k < kMlpIn; ++k) acc = fmaf(bf16_to_f32(w[kMlpW1 + u * kMlpIn + k]), x[k], acc);
        h1[q] = fmaxf(acc, 0.f);
    }
    // layer 2
    float h2[2];
    for (int q = 0; q < 2; ++q) {
        const int v = lane + 32 * q;
        float acc = bf16_to_f32(w[kMlpB2 + v]);
        for (int u = 0; u < kMlpH; ++u) {
            const float hu = __shfl_sync(0xffffffffu, h1[u >> 5], u & 31);
            acc = fmaf(bf16_to_f32(w[kMlpW2 + v * kMlpH + u]), hu, acc);
        }
        h2[q] = fmaxf(acc, 0.f);
    }
    // layer 3: lane < 25 owns logit lane
    const int j = lane < kMlpOut ? lane : kMlpOut - 1;
    float z = bf16_to_f32(w[kMlpB3 + j]);
    for (int u = 0; u < kMlpH; ++u) {
        const float hu = __shfl_sync(0xffffffffu, h2[u >> 5], u & 31);
        z = fmaf(bf16_to_f32(w[kMlpW3 + j * kMlpH + u]), hu, z);
    }
    if (logit_out && lane < kMlpOut) logit_out[lane] = z;
    // argmax, ties to the lower index
    bool allowed = lane < kMlpOut;
    if (level >= 0) allowed = allowed && lane >= level - 1 && lane <= level + 1 && lane <= top;
    float best = allowed ? z : -INFINITY;
    int arg = allowed ? lane : kMlpOut;
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ob > best || (ob == best && oa < arg)) {
            best = ob;
            arg = oa;
        }
    }
    return arg;
}

}  // namespace
}  // namespace srj
