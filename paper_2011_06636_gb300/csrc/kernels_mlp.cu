// kernels_mlp.cu -- training and batch inference of the learned scheme
// selector (mlp.cuh).  Not in the paper; see mlp.cuh for the network.
//
// Training: one persistent CTA runs every Adam step (Kingma & Ba) of
// softmax cross-entropy on minibatches whose sample order the caller passes
// in.  Parameters, gradients and activations live in shared memory; every sum
// runs in a fixed order, so training is deterministic.  FP32 master weights;
// the solver uses their BF16 rounding.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp.cuh"
#include "srj_internal.h"

namespace srj {
namespace {

constexpr int kTrainThreads = 256;
constexpr int kMaxBatch = 64;

struct TrainArgs {
    const float *X;        // n x 12
    const int32_t *y;      // n labels in [0, 25)
    const int32_t *order;  // steps * batch sample indices
    long long n, steps;
    int batch;
    float lr, beta1, beta2, eps;
    float *theta;          // 6617 FP32 (in / out)
    float *m, *v;          // Adam moments (zero on entry)
    float *loss;           // per step (may be null)
};

__global__ void __launch_bounds__(kTrainThreads) mlp_train_kernel(TrainArgs a) {
    extern __shared__ float sm[];
    float *th = sm;                                  // kMlpParams
    float *g = th + kMlpParams;                      // kMlpParams
    float *xb = g + kMlpParams;                      // B x 12
    float *a1 = xb + kMaxBatch * kMlpIn;             // B x 64 (pre-activation)
    float *a2 = a1 + kMaxBatch * kMlpH;              // B x 64
    float *dz = a2 + kMaxBatch * kMlpH;              // B x 25 (logits, then dL/dz)
    float *d2 = dz + kMaxBatch * kMlpOut;            // B x 64 (dL/da2)
    float *d1 = d2 + kMaxBatch * kMlpH;              // B x 64 (dL/da1)
    __shared__ int yb[kMaxBatch];
    __shared__ float lossb[kMaxBatch];
    const int tid = threadIdx.x;
    const int B = a.batch;
    for (int i = tid; i < kMlpParams; i += kTrainThreads) th[i] = a.theta[i];
    __syncthreads();

    for (long long step = 0; step < a.steps; ++step) {
        for (int i = tid; i < B * kMlpIn; i += kTrainThreads) {
            const int b = i / kMlpIn, k = i % kMlpIn;
            xb[i] = a.X[(long long)a.order[step * B + b] * kMlpIn + k];
        }
        if (tid < B) yb[tid] = a.y[a.order[step * B + tid]];
        __syncthreads();
        // forward
        for (int i = tid; i < B * kMlpH; i += kTrainThreads) {
            const int b = i / kMlpH, u = i % kMlpH;
            float acc = th[kMlpB1 + u];
            for (int k = 0; k < kMlpIn; ++k) acc = fmaf(th[kMlpW1 + u * kMlpIn + k], xb[b * kMlpIn + k], acc);
            a1[i] = acc;
        }
        __syncthreads();
        for (int i = tid; i < B * kMlpH; i += kTrainThreads) {
            const int b = i / kMlpH, v = i % kMlpH;
            float acc = th[kMlpB2 + v];
            for (int u = 0; u < kMlpH; ++u)
                acc = fmaf(th[kMlpW2 + v * kMlpH + u], fmaxf(a1[b * kMlpH + u], 0.f), acc);
            a2[i] = acc;
        }
        __syncthreads();
        for (int i = tid; i < B * kMlpOut; i += kTrainThreads) {
            const int b = i / kMlpOut, j = i % kMlpOut;
            float acc = th[kMlpB3 + j];
            for (int u = 0; u < kMlpH; ++u)
                acc = fmaf(th[kMlpW3 + j * kMlpH + u], fmaxf(a2[b * kMlpH + u], 0.f), acc);
            dz[i] = acc;
        }
        __syncthreads();
        // softmax cross-entropy; dz <- (p - onehot) / B
        if (tid < B) {
            float *z = dz + tid * kMlpOut;
            float zmax = z[0];
            for (int j = 1; j < kMlpOut; ++j) zmax = fmaxf(zmax, z[j]);
            float se = 0.f;
            for (int j = 0; j < kMlpOut; ++j) se += expf(z[j] - zmax);
            const float lse = zmax + logf(se);
            lossb[tid] = lse - z[yb[tid]];
            for (int j = 0; j < kMlpOut; ++j) {
                const float pj = expf(z[j] - lse);
                z[j] = (pj - (j == yb[tid] ? 1.f : 0.f)) / (float)B;
            }
        }
        __syncthreads();
        if (tid == 0 && a.loss) {
            float l = 0.f;
            for (int b = 0; b < B; ++b) l += lossb[b];
            a.loss[step] = l / (float)B;
        }
        // backward: layer 3
        for (int i = tid; i < kMlpOut * kMlpH; i += kTrainThreads) {
            const int j = i / kMlpH, u = i % kMlpH;
            float acc = 0.f;
            for (int b = 0; b < B; ++b) acc = fmaf(dz[b * kMlpOut + j], fmaxf(a2[b * kMlpH + u], 0.f), acc);
            g[kMlpW3 + i] = acc;
        }
        for (int j = tid; j < kMlpOut; j += kTrainThreads) {
            float acc = 0.f;
            for (int b = 0; b < B; ++b) acc += dz[b * kMlpOut + j];
            g[kMlpB3 + j] = acc;
        }
        for (int i = tid; i < B * kMlpH; i += kTrainThreads) {
            const int b = i / kMlpH, u = i % kMlpH;
            float acc = 0.f;
            for (int j = 0; j < kMlpOut; ++j) acc = fmaf(dz[b * kMlpOut + j], th[kMlpW3 + j * kMlpH + u], acc);
            d2[i] = a2[i] > 0.f ? acc : 0.f;
        }
        __syncthreads();
        // layer 2
        for (int i = tid; i < kMlpH * kMlpH; i += kTrainThreads) {
            const int v = i / kMlpH, u = i % kMlpH;
            float acc = 0.f;
            for (int b = 0; b < B; ++b) acc = fmaf(d2[b * kMlpH + v], fmaxf(a1[b * kMlpH + u], 0.f), acc);
            g[kMlpW2 + i] = acc;
        }
        for (int v = tid; v < kMlpH; v += kTrainThreads) {
            float acc = 0.f;
            for (int b = 0; b < B; ++b) acc += d2[b * kMlpH + v];
            g[kMlpB2 + v] = acc;
        }
        for (int i = tid; i < B * kMlpH; i += kTrainThreads) {
            const int b = i / kMlpH, u = i % kMlpH;
            float acc = 0.f;
            for (int v = 0; v < kMlpH; ++v) acc = fmaf(d2[b * kMlpH + v], th[kMlpW2 + v * kMlpH + u], acc);
            d1[i] = a1[i] > 0.f ? acc : 0.f;
        }
        __syncthreads();
        // layer 1
        for (int i = tid; i < kMlpH * kMlpIn; i += kTrainThreads) {
            const int u = i / kMlpIn, k = i % kMlpIn;
            float acc = 0.f;
            for (int b = 0; b < B; ++b) acc = fmaf(d1[b * kMlpH + u], xb[b * kMlpIn + k], acc);
            g[kMlpW1 + i] = acc;
        }
        for (int u = tid; u < kMlpH; u += kTrainThreads) {
            float acc = 0.f;
            for (int b = 0; b < B; ++b) acc += d1[b * kMlpH + u];
            g[kMlpB1 + u] = acc;
        }
        __syncthreads();
        // Adam
        const float t = (float)(step + 1);
        const float c1 = 1.f - powf(a.beta1, t), c2 = 1.f - powf(a.beta2, t);
        for (int i = tid; i < kMlpParams; i += kTrainThreads) {
            const float gi = g[i];
            const float mi = a.beta1 * a.m[i] + (1.f - a.beta1) * gi;
            const float vi = a.beta2 * a.v[i] + (1.f - a.beta2) * gi * gi;
            a.m[i] = mi;
            a.v[i] = vi;
            th[i] -= a.lr * (mi / c1) / (sqrtf(vi / c2) + a.eps);
        }
        __syncthreads();
    }
    for (int i = tid; i < kMlpParams; i += kTrainThreads) a.theta[i] = th[i];
}

__global__ void mlp_forward_kernel(const uint16_t *w, const float *X, long long n, int32_t *pick,
                                   float *logits) {
    const int lane = threadIdx.x & 31;
    const long long s = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (s >= n) return;
    float x[kMlpIn];
    for (int k = 0; k < kMlpIn; ++k) x[k] = X[s * kMlpIn + k];
    __shared__ float lg[8][32];
    const int wi = threadIdx.x >> 5;
    const int arg = mlp_pick_warp(w, x, lane, lg[wi]);
    __syncwarp();
    if (lane == 0) pick[s] = arg;
    if (logits && lane < kMlpOut) logits[s * kMlpOut + lane] = lg[wi][lane];
}

size_t train_smem() {
    return sizeof(float) * (2 * kMlpParams + kMaxBatch * (kMlpIn + 4 * kMlpH + kMlpOut));
}

}  // namespace
}  // namespace srj

using namespace srj;

extern "C" {

srj_status srj_mlp_forward(const uint16_t *w_host, const float *x_host, int64_t n,
                           int32_t *pick_host, float *logits_host) {
    if (!w_host || !x_host || !pick_host || n < 1) return SRJ_EINVAL;
    uint16_t *dw = nullptr;
    float *dx = nullptr, *dl = nullptr;
    int32_t *dp = nullptr;
    srj_status rc = SRJ_OK;
    if (cudaMalloc(&dw, kMlpParams * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc(&dx, n * kMlpIn * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&dp, n * sizeof(int32_t)) != cudaSuccess ||
        (logits_host && cudaMalloc(&dl, n * kMlpOut * sizeof(float)) != cudaSuccess)) {
        cudaGetLastError();  // the failure is returned; clear the runtime's last error
        rc = SRJ_ENOMEM;
    } else if (cudaMemcpy(dw, w_host, kMlpParams * sizeof(uint16_t), cudaMemcpyHostToDevice) !=
                   cudaSuccess ||
               cudaMemcpy(dx, x_host, n * kMlpIn * sizeof(float), cudaMemcpyHostToDevice) !=
                   cudaSuccess) {
        rc = SRJ_ECUDA;
    } else {
        const int blocks = (int)((n + 7) / 8);
        mlp_forward_kernel<<<blocks, 256>>>(dw, dx, n, dp, dl);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(pick_host, dp, n * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
            (logits_host && cudaMemcpy(logits_host, dl, n * kMlpOut * sizeof(float),
                                       cudaMemcpyDeviceToHost) != cudaSuccess))
            rc = SRJ_ECUDA;
    }
    cudaFree(dw);
    cudaFree(dx);
    cudaFree(dp);
    cudaFree(dl);
    return rc;
}

srj_status srj_mlp_train(const float *x_dev, const int32_t *y_dev, int64_t n,
                         const int32_t *order_dev, int64_t steps, int32_t batch, float lr,
                         float *theta_dev, float *loss_host, void *stream) {
    if (!x_dev || !y_dev || !order_dev || !theta_dev || n < 1 || steps < 0 || batch < 1 ||
        batch > kMaxBatch || !(lr > 0))
        return SRJ_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    float *m = nullptr, *v = nullptr, *loss = nullptr;
    srj_status rc = SRJ_OK;
    if (cudaMalloc(&m, kMlpParams * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&v, kMlpParams * sizeof(float)) != cudaSuccess ||
        (loss_host && steps > 0 && cudaMalloc(&loss, steps * sizeof(float)) != cudaSuccess)) {
        cudaGetLastError();  // the failure is returned; clear the runtime's last error
        rc = SRJ_ENOMEM;
    } else {
        TrainArgs a{x_dev, y_dev, order_dev, n, steps, batch, lr, 0.9f, 0.999f, 1e-8f,
                    theta_dev, m, v, loss};
        const size_t smem = train_smem();
        if (cudaMemsetAsync(m, 0, kMlpParams * sizeof(float), s) != cudaSuccess ||
            cudaMemsetAsync(v, 0, kMlpParams * sizeof(float), s) != cudaSuccess ||
            cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess) {
            rc = SRJ_ECUDA;
        } else {
            mlp_train_kernel<<<1, kTrainThreads, smem, s>>>(a);
            if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
                rc = SRJ_ECUDA;
            else if (loss_host && steps > 0 &&
                     cudaMemcpy(loss_host, loss, steps * sizeof(float), cudaMemcpyDeviceToHost) !=
                         cudaSuccess)
                rc = SRJ_ECUDA;
        }
    }
    cudaFree(m);
    cudaFree(v);
    cudaFree(loss);
    return rc;
}

}  // extern "C"
