// noalloc.cu -- srj_residual_norm_noalloc: the FP64 residual norm
// ||f - A u||_2 of a constant-coefficient grid computed without allocating any
// memory, for callers that cannot call cudaMalloc or cudaFree.  Examples: code
// that runs under a memory pool or a fixed device-memory budget it does not
// own (a framework's caching allocator, a service sharing the GPU), and code
// on a latency-critical path where cudaFree's implicit device-wide
// synchronisation is not acceptable.
//
// The reduction scratch of the kernel (one partial sum per grid row, a
// completion counter and the total) lives in the file-scope device array
// g_na_scratch below.  Every GPU that loads the library holds this array
// (about 512 KB) until the process exits.  Host code cannot use the array's
// name as a device address, so the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and caches
// it; later calls on that device reuse it.  A cudaDeviceReset tears down the
// module that holds the array, so the cached address is not valid across a
// reset: this entry point must not be used after the device was reset.
//
// All calls on a device share the one array: the counter is cleared at the
// start of each call, and calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on the array and must be
// serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "srj_internal.h"

namespace {

constexpr long long kNaMaxRows = 65536;  // rows (ny * nz) the scratch can hold
constexpr int kNaMaxDevices = 64;

struct NaScratch {
    double row_sum[kNaMaxRows];  // sum of r^2 over each grid row
    unsigned int ticket;         // CTAs finished in the current call
    unsigned int pad;
    double total;                // sum of r^2 over the grid
};

static __device__ __align__(256) NaScratch g_na_scratch;

NaScratch *g_na_ptr[kNaMaxDevices] = {};
std::mutex g_na_mutex;

// r = f - A u on dense arrays (x fastest), zero Dirichlet values outside;
// one warp per grid row, rows summed by the last CTA in row order.
__global__ void na_residual_kernel(NaScratch *sc, const double *f, const double *u, int dim,
                                   int nx, int ny, int nz, double cx, double cy, double cz) {
    const int lane = threadIdx.x & 31;
    const long long rows = (long long)ny * nz;
    const long long gwarp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long sy = nx, sz = (long long)nx * ny;
    for (long long row = gwarp; row < rows; row += nwarps) {
        const int y = (int)(row % ny), z = (int)(row / ny);
        double acc = 0.0;
        for (int x = lane; x < nx; x += 32) {
            const long long i = row * nx + x;
            const double uc = u[i];
            const double uxm = x > 0 ? u[i - 1] : 0.0, uxp = x + 1 < nx ? u[i + 1] : 0.0;
            double Au = cx * ((uc - uxm) + (uc - uxp));
            if (dim > 1) {
                const double uym = y > 0 ? u[i - sy] : 0.0, uyp = y + 1 < ny ? u[i + sy] : 0.0;
                Au += cy * ((uc - uym) + (uc - uyp));
            }
            if (dim > 2) {
                const double uzm = z > 0 ? u[i - sz] : 0.0, uzp = z + 1 < nz ? u[i + sz] : 0.0;
                Au += cz * ((uc - uzm) + (uc - uzp));
            }
            const double r = f[i] - Au;
            acc = fma(r, r, acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) sc->row_sum[row] = acc;
    }
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x < 32) {
        __threadfence();
        const volatile double *rs = sc->row_sum;
        double acc = 0.0;
        for (long long i = lane; i < rows; i += 32) acc += rs[i];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) sc->total = acc;
    }
}

}  // namespace

extern "C" srj_status srj_residual_norm_noalloc(const srj_grid *grid, const srj_stencil *stencil,
                                                const double *f, const double *u, double *out,
                                                void *stream) {
    if (!grid || !f || !u || !out) return SRJ_EINVAL;
    if (grid->dim < 1 || grid->dim > 3) return SRJ_EINVAL;
    if (stencil && (stencil->k || stencil->a_diag)) return SRJ_EUNSUPPORTED;
    for (int a = 0; a < grid->dim; ++a)
        if (grid->bc[a] != SRJ_BC_DIRICHLET) return SRJ_EUNSUPPORTED;
    long long n[3] = {1, 1, 1};
    double c[3] = {0, 0, 0};
    for (int a = 0; a < grid->dim; ++a) {
        // the same argument checks as srj_create: a negative or non-finite
        // spacing or coefficient is an error, zero means the default
        if (grid->n[a] < 1 || grid->n[a] > (1LL << 30)) return SRJ_EINVAL;
        if (grid->h[a] < 0 || !std::isfinite(grid->h[a])) return SRJ_EINVAL;
        const double ea = stencil ? stencil->eps[a] : 0.0;
        if (ea < 0 || !std::isfinite(ea)) return SRJ_EINVAL;
        n[a] = grid->n[a];
        const double h = grid->h[a] > 0 ? grid->h[a] : 1.0 / (double)(n[a] + 1);
        const double e = ea > 0 ? ea : 1.0;
        c[a] = e / (h * h);
    }
    if (n[1] * n[2] > kNaMaxRows) return SRJ_EINVAL;  // beyond the scratch: ny * nz > 65536
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return SRJ_ECUDA;
    NaScratch *sc = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return SRJ_ECUDA;
            g_na_ptr[dev] = (NaScratch *)p;
        }
        sc = g_na_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) return SRJ_ECUDA;
    const long long rows = n[1] * n[2];
    long long blocks = (rows + 7) / 8;  // 8 warps per CTA, one row per warp
    if (blocks > 152 * 8) blocks = 152 * 8;
    na_residual_kernel<<<(unsigned)blocks, 256, 0, s>>>(sc, f, u, grid->dim, (int)n[0], (int)n[1],
                                                        (int)n[2], c[0], c[1], c[2]);
    if (cudaGetLastError() != cudaSuccess) return SRJ_ECUDA;
    double total = 0.0;
    if (cudaMemcpyAsync(&total, &sc->total, sizeof(double), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SRJ_ECUDA;
    *out = std::sqrt(total);
    return SRJ_OK;
}
