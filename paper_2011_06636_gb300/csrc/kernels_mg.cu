// kernels_mg.cu -- geometric multigrid with SRJ smoothing: an adjacent use of
// the method (Sec. 1 names Jacobi iteration as the usual multigrid smoother,
// Sec. 5 names SRJ schemes as smoothers that accelerate multigrid).  FP64
// kernels on dense x-fastest arrays of the constant-coefficient operator with
// zero Dirichlet values:
//   sweep      u' = u + omega D^-1 (f - A u)            (Sec. 2, Eq. relaxed-jacobi)
//   residual   r = f - A u, optionally with per-CTA partial sums of r^2
//   restrict   full weighting onto the grid with (n - 1) / 2 points per axis
//              (coarse point c sits on fine point 2c + 1; weights prod_a 1/2
//              on the axis, 1/4 one step off)
//   prolong    linear interpolation per axis (fine 2c + 1 takes coarse c,
//              fine 2c half of coarse c - 1 and c), added to the fine iterate
// The V-cycle that strings them together is host code in api.cu.
#include <cuda_runtime.h>

#include "srj_internal.h"

namespace srj {
namespace {

constexpr int kMgBlock = 256;
constexpr int kMgMaxCtas = 152 * 8;

__device__ __forceinline__ void mg_coords(const MgGeo &g, long long i, int &x, int &y, int &z) {
    x = (int)(i % g.nx);
    const long long yz = i / g.nx;
    y = (int)(yz % g.ny);
    z = (int)(yz / g.ny);
}

// (A u)_i with zero Dirichlet values outside the grid
template <int DIM>
__device__ __forceinline__ double mg_Au(const MgGeo &g, const double *u, long long i, int x, int y,
                                        int z) {
    const double uc = u[i];
    const double xm = x > 0 ? u[i - 1] : 0.0, xp = x + 1 < g.nx ? u[i + 1] : 0.0;
    double a = g.cx * ((uc - xm) + (uc - xp));
    if (DIM > 1) {
        const long long sy = g.nx;
        const double ym = y > 0 ? u[i - sy] : 0.0, yp = y + 1 < g.ny ? u[i + sy] : 0.0;
        a += g.cy * ((uc - ym) + (uc - yp));
    }
    if (DIM > 2) {
        const long long sz = (long long)g.nx * g.ny;
        const double zm = z > 0 ? u[i - sz] : 0.0, zp = z + 1 < g.nz ? u[i + sz] : 0.0;
        a += g.cz * ((uc - zm) + (uc - zp));
    }
    return a;
}

template <int DIM>
__global__ void __launch_bounds__(kMgBlock) mg_sweep_kernel(MgGeo g, const double *u, double *uo,
                                                            const double *f, double omega) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    const double invd = 1.0 / g.diag;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        mg_coords(g, i, x, y, z);
        uo[i] = u[i] + omega * ((f[i] - mg_Au<DIM>(g, u, i, x, y, z)) * invd);
    }
}

template <int DIM>
__global__ void __launch_bounds__(kMgBlock) mg_residual_kernel(MgGeo g, const double *u,
                                                               const double *f, double *r,
                                                               double *partials) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        mg_coords(g, i, x, y, z);
        const double ri = f[i] - mg_Au<DIM>(g, u, i, x, y, z);
        if (r) r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    if (!partials) return;
    // deterministic CTA sum: fixed butterfly, warps in order
    __shared__ double s_w[kMgBlock / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kMgBlock / 32; ++w) t += s_w[w];
        partials[blockIdx.x] = t;
    }
}

// one CTA: fixed assignment of partials to lanes, fixed butterfly
__global__ void mg_sum_kernel(const double *partials, int n, double *out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) acc += partials[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) *out = acc;
}

template <int DIM>
__global__ void __launch_bounds__(kMgBlock) mg_restrict_kernel(MgGeo gf, const double *r, MgGeo gc,
                                                               double *fc) {
    const long long n = (long long)gc.nx * gc.ny * gc.nz;
    const long long sy = gf.nx, sz = (long long)gf.nx * gf.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        mg_coords(gc, i, x, y, z);
        const long long fx = 2 * x + 1, fy = DIM > 1 ? 2 * y + 1 : 0, fz = DIM > 2 ? 2 * z + 1 : 0;
        const long long c = fx + sy * fy + sz * fz;
        double acc = 0.0;
#pragma unroll
        for (int dz = (DIM > 2 ? -1 : 0); dz <= (DIM > 2 ? 1 : 0); ++dz)
#pragma unroll
            for (int dy = (DIM > 1 ? -1 : 0); dy <= (DIM > 1 ? 1 : 0); ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    double w = dx == 0 ? 0.5 : 0.25;
                    if (DIM > 1) w *= dy == 0 ? 0.5 : 0.25;
                    if (DIM > 2) w *= dz == 0 ? 0.5 : 0.25;
                    acc += w * r[c + dx + sy * dy + sz * dz];
                }
        fc[i] = acc;
    }
}

template <int DIM>
__global__ void __launch_bounds__(kMgBlock) mg_prolong_kernel(MgGeo gc, const double *ec, MgGeo gf,
                                                              double *u) {
    const long long n = (long long)gf.nx * gf.ny * gf.nz;
    const long long sy = gc.nx, sz = (long long)gc.nx * gc.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        mg_coords(gf, i, x, y, z);
        // per axis: up to two coarse neighbours (index, weight)
        int cxa[2], cya[2], cza[2];
        double wxa[2], wya[2], wza[2];
        int mx, my = 1, mz = 1;
        if (x & 1) { cxa[0] = x >> 1; wxa[0] = 1.0; mx = 1; }
        else { cxa[0] = (x >> 1) - 1; cxa[1] = x >> 1; wxa[0] = wxa[1] = 0.5; mx = 2; }
        cya[0] = 0; wya[0] = 1.0;
        if (DIM > 1) {
            if (y & 1) { cya[0] = y >> 1; my = 1; }
            else { cya[0] = (y >> 1) - 1; cya[1] = y >> 1; wya[0] = wya[1] = 0.5; my = 2; }
        }
        cza[0] = 0; wza[0] = 1.0;
        if (DIM > 2) {
            if (z & 1) { cza[0] = z >> 1; mz = 1; }
            else { cza[0] = (z >> 1) - 1; cza[1] = z >> 1; wza[0] = wza[1] = 0.5; mz = 2; }
        }
        double acc = 0.0;
        for (int c = 0; c < mz; ++c)
            for (int b = 0; b < my; ++b)
                for (int a = 0; a < mx; ++a) {
                    if (cxa[a] < 0 || cxa[a] >= gc.nx) continue;
                    if (DIM > 1 && (cya[b] < 0 || cya[b] >= gc.ny)) continue;
                    if (DIM > 2 && (cza[c] < 0 || cza[c] >= gc.nz)) continue;
                    acc += wxa[a] * wya[b] * wza[c] * ec[cxa[a] + sy * cya[b] + sz * cza[c]];
                }
        u[i] += acc;
    }
}

int mg_blocks(long long n) {
    long long b = (n + kMgBlock - 1) / kMgBlock;
    if (b < 1) b = 1;
    return (int)(b < kMgMaxCtas ? b : kMgMaxCtas);
}

}  // namespace

int mg_partials_needed() { return kMgMaxCtas; }

cudaError_t mg_sweep_launch(const MgGeo &g, const double *u, double *uo, const double *f,
                            double omega, cudaStream_t s) {
    const int nb = mg_blocks((long long)g.nx * g.ny * g.nz);
    if (g.dim == 1) mg_sweep_kernel<1><<<nb, kMgBlock, 0, s>>>(g, u, uo, f, omega);
    else if (g.dim == 2) mg_sweep_kernel<2><<<nb, kMgBlock, 0, s>>>(g, u, uo, f, omega);
    else mg_sweep_kernel<3><<<nb, kMgBlock, 0, s>>>(g, u, uo, f, omega);
    return cudaGetLastError();
}

cudaError_t mg_residual_launch(const MgGeo &g, const double *u, const double *f, double *r,
                               double *partials, int *nparts, cudaStream_t s) {
    const int nb = mg_blocks((long long)g.nx * g.ny * g.nz);
    if (nparts) *nparts = nb;
    if (g.dim == 1) mg_residual_kernel<1><<<nb, kMgBlock, 0, s>>>(g, u, f, r, partials);
    else if (g.dim == 2) mg_residual_kernel<2><<<nb, kMgBlock, 0, s>>>(g, u, f, r, partials);
    else mg_residual_kernel<3><<<nb, kMgBlock, 0, s>>>(g, u, f, r, partials);
    return cudaGetLastError();
}

cudaError_t mg_sum_launch(const double *partials, int n, double *out, cudaStream_t s) {
    mg_sum_kernel<<<1, 32, 0, s>>>(partials, n, out);
    return cudaGetLastError();
}

cudaError_t mg_restrict_launch(const MgGeo &gf, const double *r, const MgGeo &gc, double *fc,
                               cudaStream_t s) {
    const int nb = mg_blocks((long long)gc.nx * gc.ny * gc.nz);
    if (gf.dim == 1) mg_restrict_kernel<1><<<nb, kMgBlock, 0, s>>>(gf, r, gc, fc);
    else if (gf.dim == 2) mg_restrict_kernel<2><<<nb, kMgBlock, 0, s>>>(gf, r, gc, fc);
    else mg_restrict_kernel<3><<<nb, kMgBlock, 0, s>>>(gf, r, gc, fc);
    return cudaGetLastError();
}

cudaError_t mg_prolong_launch(const MgGeo &gc, const double *ec, const MgGeo &gf, double *u,
                              cudaStream_t s) {
    const int nb = mg_blocks((long long)gf.nx * gf.ny * gf.nz);
    if (gf.dim == 1) mg_prolong_kernel<1><<<nb, kMgBlock, 0, s>>>(gc, ec, gf, u);
    else if (gf.dim == 2) mg_prolong_kernel<2><<<nb, kMgBlock, 0, s>>>(gc, ec, gf, u);
    else mg_prolong_kernel<3><<<nb, kMgBlock, 0, s>>>(gc, ec, gf, u);
    return cudaGetLastError();
}

}  // namespace srj
