// kernels_generic.cu -- the general SRJ pass kernel (one sweep or one residual
// per pass, any dimension, constant or variable coefficients, FP64 / FP32 /
// FP32-pair state), the device-side cycle bookkeeping shared by every pass
// kernel, and the FP64 outer kernels of mixed-precision refinement.
//
// A pass of the SRJ cycle (Sec. 3) is either
//   SWEEP: u' = u + omega_k D^-1 (f - A u)           (Sec. 2, Eq. relaxed-jacobi)
//   RESID: ||f - A u||_2^2, per-CTA partials          (Sec. 3, Eq. relative-residual)
// and the last CTA to finish a pass (ticket counter) advances the cycle state:
// after a RESID at the end of a cycle it forms ratio = r_after / r_before,
// tests convergence and picks the next level with Alg. 1.  No CTA ever waits
// for another: the only cross-CTA communication is that ticket.
#include <cuda_runtime.h>
#include <math.h>

#include "df32.cuh"
#include "pass_common.cuh"
#include "stencil_point.cuh"
#include "srj_internal.h"

namespace srj {

namespace {

constexpr int kBlock = 256;

// ---------------------------------------------------------- the pass kernel
// Thread (tx, ty) of a CTA owns grid column (x, y) and walks z through
// [z0, z0 + chunk); the z neighbours rotate through registers, the x and y
// neighbours come through L1.  On 2D grids the thread instead takes rows
// y0 + ty, y0 + ty + 8, ... of a band of 8 * chunk rows (fewer CTAs, so fewer
// partials for the last CTA to fold).  1D grids use 256x1 blocks.
template <int PREC, int DIM, bool VARK>
__global__ void __launch_bounds__(kBlock) generic_pass_kernel(PassLaunch a, int chunk) {
    using T = typename Elem<PREC>::T;
    using C = typename Elem<PREC>::C;
    using P = Point<PREC, DIM>;

    __shared__ PassPlan s_plan;
    __shared__ double s_omega;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (tid == 0) {
        s_plan = plan_pass(a, 1);
        s_omega = (s_plan.run && s_plan.nsw) ? a.w64[s_plan.woff] : 0.0;
        if (!s_plan.run && a.cfg.use_cond && blockIdx.x == 0 && blockIdx.y == 0 &&
            blockIdx.z == 0)
            cudaGraphSetConditional(a.cfg.cond, 0);
    }
    __syncthreads();
    const PassPlan p = s_plan;
    if (!p.run) return;
    const double omega = s_omega;

    const GridGeo &g = a.geo;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int zchunk = DIM > 2 ? chunk : 1;
    const int rows = DIM == 2 ? chunk : 1;  // rows per thread
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    const int src = p.cur, dst = p.cur ^ 1;
    const C *f = (const C *)a.bufs.f;

    C cconst[3], invd_c = C(g.invdiag), diag_c = C(g.diag);
    cconst[0] = C(g.acx);
    cconst[1] = C(g.acy);
    cconst[2] = C(g.acz);

    double part = 0.0;  // residual sum (resid pass)
    long long dbits = 0;  // largest |u' - u| of the sweep (abs_diff_bits)
    // Neumann axes (Sec. 4.2.2): the ghost node one step outside mirrors the
    // node one step inside; Dirichlet axes read zero there
    const bool nx_ = g.neu & 1, ny_ = g.neu & 2, nz_ = g.neu & 4;
    const bool dinf = a.dinf && p.nsw;
    for (int r = 0; r < rows; ++r) {
        const int y = (blockIdx.y * rows + r) * blockDim.y + threadIdx.y;
        if (x >= g.nx || y >= g.ny) break;
        const long long col = (long long)x + g.pitch * y;
        T u_zm = (DIM > 2 && z0 > 0) ? load_u<PREC>(a.bufs, src, col + g.plane * (z0 - 1))
                                     : zero_u<PREC>();
        T u_c = (z0 < z1) ? load_u<PREC>(a.bufs, src, col + g.plane * z0) : zero_u<PREC>();
        // the updates of successive z planes are independent; unrolling lets
        // their long dependent chains (FP32-pair arithmetic) overlap
#pragma unroll 4
        for (int z = z0; z < z1; ++z) {
            const long long i = col + g.plane * z;
            T u_zp = (DIM > 2 && z + 1 < g.nz) ? load_u<PREC>(a.bufs, src, i + g.plane)
                                               : zero_u<PREC>();
            T nb[6];
            nb[0] = x > 0 ? load_u<PREC>(a.bufs, src, i - 1)
                          : (nx_ ? load_u<PREC>(a.bufs, src, i + 1) : zero_u<PREC>());
            nb[1] = x + 1 < g.nx ? load_u<PREC>(a.bufs, src, i + 1)
                                 : (nx_ ? load_u<PREC>(a.bufs, src, i - 1) : zero_u<PREC>());
            if (DIM > 1) {
                nb[2] = y > 0 ? load_u<PREC>(a.bufs, src, i - g.pitch)
                              : (ny_ ? load_u<PREC>(a.bufs, src, i + g.pitch) : zero_u<PREC>());
                nb[3] = y + 1 < g.ny
                            ? load_u<PREC>(a.bufs, src, i + g.pitch)
                            : (ny_ ? load_u<PREC>(a.bufs, src, i - g.pitch) : zero_u<PREC>());
            }
            nb[4] = (DIM > 2 && nz_ && z == 0) ? u_zp : u_zm;
            nb[5] = (DIM > 2 && nz_ && z + 1 == g.nz) ? u_zm : u_zp;
            // f and the face weights are read-only for the whole solve
            const C fi = __ldg(f + i);
            T t;
            C diag_i = diag_c;
            if constexpr (VARK) {
                const C *wx = (const C *)a.bufs.wx;
                const C *wy = (const C *)a.bufs.wy;
                const C *wz = (const C *)a.bufs.wz;
                const C invd_i = __ldg((const C *)a.bufs.invd + i);
                C wgt[6];
                wgt[0] = x > 0 ? __ldg(wx + i - 1) : C(0);
                wgt[1] = __ldg(wx + i);
                if (DIM > 1) {
                    wgt[2] = y > 0 ? __ldg(wy + i - g.pitch) : C(0);
                    wgt[3] = __ldg(wy + i);
                }
                if (DIM > 2) {
                    wgt[4] = z > 0 ? __ldg(wz + i - g.plane) : C(0);
                    wgt[5] = __ldg(wz + i);
                }
                if (p.nsw) {
                    const T un = P::sweep_of(nb, wgt, invd_i, fi, u_c, omega);
                    store_u<PREC>(a.bufs, dst, i, un);
                    if constexpr (PREC != PREC_DF)
                        if (dinf) dbits = max_bits(dbits, abs_diff_bits((double)un, (double)u_c));
                } else {
                    t = P::t_of(nb, wgt, invd_i, fi, u_c);
                    diag_i = C(1) / invd_i;
                    part += P::resid2(t, diag_i);
                }
            } else if (p.nsw) {
                const T un = P::sweep_const(nb, cconst, invd_c, fi, u_c, omega);
                store_u<PREC>(a.bufs, dst, i, un);
                if constexpr (PREC != PREC_DF)
                    if (dinf) dbits = max_bits(dbits, abs_diff_bits((double)un, (double)u_c));
            } else {
                t = P::t_const(nb, cconst, invd_c, fi, u_c);
                part += P::resid2(t, diag_i);
            }
            u_zm = u_c;
            u_c = u_zp;
        }
    }
    double tot = 0.0;
    if (p.resid) tot = block_sum(part);
    else if (dinf) tot = block_max_bits(dbits);
    finish_pass(a, p, tot, dinf);
}

template <int PREC, int DIM, bool VARK>
void *generic_entry() {
    return (void *)&generic_pass_kernel<PREC, DIM, VARK>;
}

template <int PREC>
void *pick_entry(int dim, bool vark) {
    if (dim == 1) return vark ? generic_entry<PREC, 1, true>() : generic_entry<PREC, 1, false>();
    if (dim == 2) return vark ? generic_entry<PREC, 2, true>() : generic_entry<PREC, 2, false>();
    return vark ? generic_entry<PREC, 3, true>() : generic_entry<PREC, 3, false>();
}

void *entry_for(int prec, int dim, bool vark) {
    if (prec == PREC_F64) return pick_entry<PREC_F64>(dim, vark);
    if (prec == PREC_F32) return pick_entry<PREC_F32>(dim, vark);
    return pick_entry<PREC_DF>(dim, vark);
}

}  // namespace

// ------------------------------------------------------------------ host side
GenericPlan generic_plan(int prec, const GridGeo &g, bool vark) {
    GenericPlan p{};
    if (g.dim == 3 && g.neu == 0) {  // plane-streaming 3D pass
        const Plane3dPlan q = plane3d_plan(prec, g, vark);
        p.grid = q.grid;
        p.block = q.block;
        p.zchunk = q.zchunk;
        p.kernel = q.kernel;
        p.smem = q.smem;
        p.plane3d = 1;
        return p;
    }
    if (g.dim == 1) {
        p.block = dim3(kBlock, 1, 1);
        p.zchunk = 1;
        p.grid = dim3((g.nx + kBlock - 1) / kBlock, 1, 1);
    } else if (g.dim == 2) {
        // bands of 8 * rows rows, rows chosen so that the grid stays within
        // 16 CTAs per SM
        p.block = dim3(32, kBlock / 32, 1);
        const long long bx = (g.nx + 31) / 32, by = (g.ny + p.block.y - 1) / p.block.y;
        const long long cap = 152 * 16;
        long long rows = (bx * by + cap - 1) / cap;
        if (rows < 1) rows = 1;
        p.zchunk = (int)rows;
        p.grid = dim3((unsigned)bx, (unsigned)((by + rows - 1) / rows), 1);
    } else {
        p.block = dim3(32, kBlock / 32, 1);
        p.zchunk = g.nz < 32 ? g.nz : 32;
        p.grid = dim3((g.nx + 31) / 32, (g.ny + p.block.y - 1) / p.block.y,
                      (g.nz + p.zchunk - 1) / p.zchunk);
    }
    p.kernel = entry_for(prec, g.dim, vark);
    return p;
}

int generic_partials_needed(const GridGeo &g) {
    GenericPlan p = generic_plan(PREC_F64, g, false);
    return (int)(p.grid.x * p.grid.y * p.grid.z);
}

cudaError_t generic_pass_launch(int prec, bool vark, const PassLaunch &a, cudaStream_t s,
                                const Plane3dMaps *maps) {
    GenericPlan p = generic_plan(prec, a.geo, vark);
    if (p.plane3d) {
        if (!maps) return cudaErrorInvalidValue;
        const cudaError_t e = plane3d_prepare(prec, vark);
        if (e != cudaSuccess) return e;
    }
    void *args[] = {(void *)&a, (void *)&p.zchunk, (void *)maps};
    return cudaLaunchKernel(p.kernel, p.grid, p.block, args, p.smem, s);
}

cudaError_t add_generic_pass_node(int prec, bool vark, const PassLaunch &a, cudaGraph_t body,
                                  const Plane3dMaps *maps) {
    GenericPlan p = generic_plan(prec, a.geo, vark);
    if (p.plane3d) {
        if (!maps) return cudaErrorInvalidValue;
        const cudaError_t e = plane3d_prepare(prec, vark);
        if (e != cudaSuccess) return e;
    }
    void *args[] = {(void *)&a, (void *)&p.zchunk, (void *)maps};
    cudaKernelNodeParams kp{};
    kp.func = p.kernel;
    kp.gridDim = p.grid;
    kp.blockDim = p.block;
    kp.sharedMemBytes = p.smem;
    kp.kernelParams = args;
    cudaGraphNode_t node;
    return cudaGraphAddKernelNode(&node, body, nullptr, 0, &kp);
}

// --------------------------------------------- dense <-> padded iterate copies
namespace {

template <typename T>
__global__ void copy_in_kernel(GridGeo g, const T *dense, T *padded) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long x = i % g.nx, yz = i / g.nx;
        const long long y = yz % g.ny, z = yz / g.ny;
        padded[x + g.pitch * y + g.plane * z] = dense[i];
    }
}

template <typename T>
__global__ void copy_out_kernel(GridGeo g, const DevState *st, const T *p0, const T *p1,
                                T *dense) {
    const T *src = st->cur ? p1 : p0;
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long x = i % g.nx, yz = i / g.nx;
        const long long y = yz % g.ny, z = yz / g.ny;
        dense[i] = src[x + g.pitch * y + g.plane * z];
    }
}

int stream_blocks(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

cudaError_t copy_in_launch(int prec, const GridGeo &g, const void *dense, void *padded,
                           cudaStream_t s) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    if (prec == PREC_F64)
        copy_in_kernel<double><<<stream_blocks(n), 256, 0, s>>>(g, (const double *)dense,
                                                                (double *)padded);
    else
        copy_in_kernel<float><<<stream_blocks(n), 256, 0, s>>>(g, (const float *)dense,
                                                               (float *)padded);
    return cudaGetLastError();
}

cudaError_t copy_out_launch(int prec, const GridGeo &g, const DevState *st, void *const *pads,
                            void *dense, cudaStream_t s) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    if (prec == PREC_F64)
        copy_out_kernel<double><<<stream_blocks(n), 256, 0, s>>>(
            g, st, (const double *)pads[0], (const double *)pads[1], (double *)dense);
    else
        copy_out_kernel<float><<<stream_blocks(n), 256, 0, s>>>(
            g, st, (const float *)pads[0], (const float *)pads[1], (float *)dense);
    return cudaGetLastError();
}

// ------------------------------------------- variable-coefficient face weights
namespace {

__global__ void vark_faces_kernel(GridGeo g, const double *k, double *wx, double *wy,
                                  double *wz, double *invd, float *wx32, float *wy32,
                                  float *wz32, float *invd32) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long kp = g.nx + 2;
    const long long kq = kp * (g.dim > 1 ? g.ny + 2 : 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long x = i % g.nx, yz = i / g.nx;
        const long long y = yz % g.ny, z = yz / g.ny;
        const long long kc = (x + 1) + kp * (g.dim > 1 ? y + 1 : 0) + kq * (g.dim > 2 ? z + 1 : 0);
        const double k0 = k[kc];
        auto hm = [&](double k1) { return 2.0 * k0 * k1 / (k0 + k1); };
        const double fxm = g.cx * hm(k[kc - 1]), fxp = g.cx * hm(k[kc + 1]);
        double d = fxm + fxp, fyp = 0.0, fzp = 0.0;
        if (g.dim > 1) {
            fyp = g.cy * hm(k[kc + kp]);
            d += g.cy * hm(k[kc - kp]) + fyp;
        }
        if (g.dim > 2) {
            fzp = g.cz * hm(k[kc + kq]);
            d += g.cz * hm(k[kc - kq]) + fzp;
        }
        const long long p = x + g.pitch * y + g.plane * z;
        wx[p] = fxp;
        wy[p] = fyp;
        wz[p] = fzp;
        invd[p] = 1.0 / d;
        wx32[p] = (float)fxp;
        wy32[p] = (float)fyp;
        wz32[p] = (float)fzp;
        invd32[p] = (float)(1.0 / d);
    }
}

// Explicit symmetric operator: the sweep and residual kernels read it in
// the same form as face weights (A u)_p = u_p / invd_p - sum_q w_q u_q.
__global__ void explicit_faces_kernel(GridGeo g, const double *adiag, const double *ax,
                                      const double *ay, const double *az, double *wx,
                                      double *wy, double *wz, double *invd, float *wx32,
                                      float *wy32, float *wz32, float *invd32) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long x = i % g.nx, yz = i / g.nx;
        const long long y = yz % g.ny, z = yz / g.ny;
        const double fx = x + 1 < g.nx ? -ax[i] : 0.0;
        const double fy = (g.dim > 1 && y + 1 < g.ny) ? -ay[i] : 0.0;
        const double fz = (g.dim > 2 && z + 1 < g.nz) ? -az[i] : 0.0;
        const double id = 1.0 / adiag[i];
        const long long p = x + g.pitch * y + g.plane * z;
        wx[p] = fx;
        wy[p] = fy;
        wz[p] = fz;
        invd[p] = id;
        wx32[p] = (float)fx;
        wy32[p] = (float)fy;
        wz32[p] = (float)fz;
        invd32[p] = (float)id;
    }
}

}  // namespace

cudaError_t explicit_faces_launch(const GridGeo &g, const double *adiag,
                                  const double *const *aoff, double *wx, double *wy,
                                  double *wz, double *invd, float *wx32, float *wy32,
                                  float *wz32, float *invd32, cudaStream_t s) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    explicit_faces_kernel<<<stream_blocks(n), 256, 0, s>>>(g, adiag, aoff[0], aoff[1], aoff[2],
                                                           wx, wy, wz, invd, wx32, wy32, wz32,
                                                           invd32);
    return cudaGetLastError();
}

cudaError_t vark_faces_launch(const GridGeo &g, const double *k, double *wx, double *wy,
                              double *wz, double *invd, float *wx32, float *wy32, float *wz32,
                              float *invd32, cudaStream_t s) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    vark_faces_kernel<<<stream_blocks(n), 256, 0, s>>>(g, k, wx, wy, wz, invd, wx32, wy32, wz32,
                                                       invd32);
    return cudaGetLastError();
}

// ------------------------------------------------ mixed-precision outer kernels
namespace {

// r = f - A u in FP64 on the dense user arrays; r is stored (FP32) into the
// padded inner right-hand side and ||r||^2 is reduced to *out_norm2.
template <int DIM, bool VARK>
__global__ void __launch_bounds__(kBlock) outer_residual_kernel(OuterArgs a) {
    const GridGeo &g = a.geo;
    const long long n = (long long)g.nx * g.ny * g.nz;
    double part = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long x = i % g.nx, yz = i / g.nx;
        const long long y = yz % g.ny, z = yz / g.ny;
        const long long sy = g.nx, sz = (long long)g.nx * g.ny;
        const double uc = a.u[i];
        const double uxm = x > 0 ? a.u[i - 1] : 0.0, uxp = x + 1 < g.nx ? a.u[i + 1] : 0.0;
        double uym = 0, uyp = 0, uzm = 0, uzp = 0;
        if (DIM > 1) {
            uym = y > 0 ? a.u[i - sy] : 0.0;
            uyp = y + 1 < g.ny ? a.u[i + sy] : 0.0;
        }
        if (DIM > 2) {
            uzm = z > 0 ? a.u[i - sz] : 0.0;
            uzp = z + 1 < g.nz ? a.u[i + sz] : 0.0;
        }
        double Au;
        const long long pp = x + g.pitch * y + g.plane * z;
        if constexpr (VARK) {
            const double wxp = a.wx[pp], wxm = x > 0 ? a.wx[pp - 1] : 0.0;
            double s = wxm * uxm + wxp * uxp;
            if (DIM > 1) s += (y > 0 ? a.wy[pp - g.pitch] : 0.0) * uym + a.wy[pp] * uyp;
            if (DIM > 2) s += (z > 0 ? a.wz[pp - g.plane] : 0.0) * uzm + a.wz[pp] * uzp;
            Au = uc / a.invd[pp] - s;
        } else {
            Au = g.cx * ((uc - uxm) + (uc - uxp));
            if (DIM > 1) Au += g.cy * ((uc - uym) + (uc - uyp));
            if (DIM > 2) Au += g.cz * ((uc - uzm) + (uc - uzp));
        }
        const double r = a.f[i] - Au;
        // the FP32-pair sweeps read a constant-coefficient right-hand side
        // scaled by D^-1 (one rounding either way)
        a.r32[pp] = VARK ? (float)r : (float)(r / g.diag);
        part += r * r;
    }
    const double tot = block_sum(part);
    __shared__ int s_last;
    const int tid = threadIdx.x;
    if (tid == 0) {
        a.partials[blockIdx.x] = tot;
        __threadfence();
        s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last && tid < 32) {
        __threadfence();
        double acc = 0.0;
        const volatile double *part_v = a.partials;
        for (unsigned int b = tid; b < gridDim.x; b += 32) acc += part_v[b];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (tid == 0) {
            *a.out_norm2 = acc;
            *a.ticket = 0;
        }
    }
}

__global__ void outer_update_kernel(OuterArgs a) {
    const GridGeo &g = a.geo;
    const long long n = (long long)g.nx * g.ny * g.nz;
    const int cur = a.inner->cur;
    const float *eh = a.ehi[cur], *el = a.elo[cur];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long x = i % g.nx, yz = i / g.nx;
        const long long y = yz % g.ny, z = yz / g.ny;
        const long long pp = x + g.pitch * y + g.plane * z;
        a.u_out[i] = a.u[i] + ((double)eh[pp] + (double)el[pp]);
    }
}

}  // namespace

int outer_partials_needed(const GridGeo &g) {
    (void)g;
    return 152 * 8;
}

cudaError_t outer_residual_launch(const OuterArgs &a, cudaStream_t s) {
    const long long n = (long long)a.geo.nx * a.geo.ny * a.geo.nz;
    long long b = (n + kBlock - 1) / kBlock;
    const int blocks = (int)(b < 152 * 8 ? (b < 1 ? 1 : b) : 152 * 8);
    const bool vark = a.wx != nullptr;
    if (a.geo.dim == 1)
        vark ? outer_residual_kernel<1, true><<<blocks, kBlock, 0, s>>>(a)
             : outer_residual_kernel<1, false><<<blocks, kBlock, 0, s>>>(a);
    else if (a.geo.dim == 2)
        vark ? outer_residual_kernel<2, true><<<blocks, kBlock, 0, s>>>(a)
             : outer_residual_kernel<2, false><<<blocks, kBlock, 0, s>>>(a);
    else
        vark ? outer_residual_kernel<3, true><<<blocks, kBlock, 0, s>>>(a)
             : outer_residual_kernel<3, false><<<blocks, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t outer_update_launch(const OuterArgs &a, cudaStream_t s) {
    const long long n = (long long)a.geo.nx * a.geo.ny * a.geo.nz;
    outer_update_kernel<<<stream_blocks(n), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace srj
