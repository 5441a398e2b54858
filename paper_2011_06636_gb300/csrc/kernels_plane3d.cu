// kernels_plane3d.cu -- the 3D SRJ pass (one relaxed sweep or one residual per
// pass, Sec. 2 Eq. relaxed-jacobi and Sec. 3 Eq. relative-residual) as a
// plane-streaming kernel: a CTA owns a 32 x 8 column tile and walks a chunk of
// z planes.  Every plane it needs -- the iterate with a one-cell halo, the
// right-hand side and, for variable coefficients, the face weights and 1/D --
// is brought into a five-slot shared-memory ring by TMA tensor copies
// (cp.async.bulk.tensor, one elected thread, one mbarrier per slot), three
// planes ahead of the plane computed.  The tensor maps bound every array to
// the grid, so the copies zero-fill the ghost rows, columns and planes: the
// zero Dirichlet values and zero boundary faces.  Same pass protocol as the
// generic kernel: plan_pass / finish_pass.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cstring>

#include "df32.cuh"
#include "pass_common.cuh"
#include "stencil_point.cuh"
#include "srj_internal.h"

namespace srj {
namespace {

constexpr int kTX = 32, kTY = 8;    // column tile (threads)
constexpr int kHX = 4;              // columns staged left of the tile: x0 - 4 is 16-byte aligned
constexpr int kSX = kTX + 2 * kHX;  // staged row width: x0 - 4 .. x0 + 35
constexpr int kPD = 3;              // planes in flight ahead of the one computed
constexpr int kNS = kPD + 2;        // ring slots: planes z-1 .. z+PD

__host__ __device__ constexpr int al128(int b) { return (b + 127) / 128 * 128; }

// One ring slot: every array at a 128-byte aligned offset.  Boxes (elements):
// iterate {40, 10} from (x0-4, y0-1); x faces {40, 8} from (x0-4, y0);
// y faces {32, 9} from (x0, y0-1); rhs, z faces, 1/D {32, 8} from (x0, y0).
template <int PREC, bool VARK>
struct Plane {
    static constexpr bool LO = PREC == PREC_DF;
    static constexpr int ES = PREC == PREC_F64 ? 8 : 4;
    static constexpr int BU = kSX * (kTY + 2) * ES, BF = kTX * kTY * ES;
    static constexpr int BWX = kSX * kTY * ES, BWY = kTX * (kTY + 1) * ES;
    static constexpr int o_hi = 0, o_lo = o_hi + al128(BU), o_f = o_lo + (LO ? al128(BU) : 0);
    static constexpr int o_wx = o_f + al128(BF), o_wy = o_wx + (VARK ? al128(BWX) : 0);
    static constexpr int o_wz = o_wy + (VARK ? al128(BWY) : 0), o_id = o_wz + (VARK ? al128(BF) : 0);
    static constexpr int BYTES = o_id + (VARK ? al128(BF) : 0);
    static constexpr int SMEM = kNS * BYTES;
    // bytes one plane's copies deliver (the transaction count of its barrier)
    static constexpr unsigned TX = BU * (LO ? 2 : 1) + BF + (VARK ? BWX + BWY + 2 * BF : 0);
};

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// true once the phase with the given parity has completed; false after
// `limit` polls (at once for limit 0)
__device__ __forceinline__ bool bar_wait(uint64_t *bar, unsigned parity, long long limit) {
    const unsigned a = smem_u32(bar);
    for (long long it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma3(void *dst, const CUtensorMap *map, int x, int y, int z,
                                     uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

template <int PREC, bool VARK>
__global__ void __launch_bounds__(kTX * kTY)
    plane3d_kernel(PassLaunch a, int zchunk, const __grid_constant__ Plane3dMaps maps) {
    using T = typename Elem<PREC>::T;
    using C = typename Elem<PREC>::C;
    using P = Point<PREC, 3>;
    using L = Plane<PREC, VARK>;
    constexpr int ES = L::ES;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_bar[kNS];
    __shared__ PassPlan s_plan;
    __shared__ double s_omega;
    __shared__ long long s_wlim;
    __shared__ int s_err;

    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kTX * ty;
    if (tid == 0) {
        s_plan = plan_pass(a, 1);
        s_omega = (s_plan.run && s_plan.nsw) ? a.w64[s_plan.woff] : 0.0;
        s_wlim = a.st->wait_limit;
        s_err = 0;
        if (!s_plan.run && a.cfg.use_cond && blockIdx.x == 0 && blockIdx.y == 0 &&
            blockIdx.z == 0)
            cudaGraphSetConditional(a.cfg.cond, 0);
        if (s_plan.run) {
            for (int k = 0; k < kNS; ++k) bar_init(&s_bar[k]);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
    }
    __syncthreads();
    const PassPlan p = s_plan;
    if (!p.run) return;
    const double omega = s_omega;
    const long long wlim = s_wlim;

    const GridGeo &g = a.geo;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    const int src = p.cur, dst = p.cur ^ 1;
    const bool dinf = a.dinf && p.nsw;

    // plane zz (>= z0 - 1) lives in slot (zz - z0 + 1) mod NS; the n-th plane
    // of a slot completes its barrier's phase n, parity n & 1
    auto rel = [&](int zz) { return zz - (z0 - 1); };
    auto slot = [&](int zz) -> unsigned char * { return smem + (rel(zz) % kNS) * L::BYTES; };
    auto issue = [&](int zz) {  // one thread
        unsigned char *s = slot(zz);
        uint64_t *bar = &s_bar[rel(zz) % kNS];
        // order the block's earlier reads of this slot before the async writes
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        bar_expect(bar, L::TX);
        tma3(s + L::o_hi, &maps.u[src], x0 - kHX, y0 - 1, zz, bar);
        if constexpr (L::LO) tma3(s + L::o_lo, &maps.ulo[src], x0 - kHX, y0 - 1, zz, bar);
        tma3(s + L::o_f, &maps.f, x0, y0, zz, bar);
        if constexpr (VARK) {
            tma3(s + L::o_wx, &maps.wx, x0 - kHX, y0, zz, bar);
            tma3(s + L::o_wy, &maps.wy, x0, y0 - 1, zz, bar);
            tma3(s + L::o_wz, &maps.wz, x0, y0, zz, bar);
            tma3(s + L::o_id, &maps.invd, x0, y0, zz, bar);
        }
    };
    auto wait = [&](int zz, long long limit) -> bool {
        return bar_wait(&s_bar[rel(zz) % kNS], (unsigned)((rel(zz) / kNS) & 1), limit);
    };
    auto ld = [&](const unsigned char *s, int off, int idx) -> C {
        return *(const C *)(s + off + idx * ES);
    };
    // iterate at tile column cx (-1 .. 32) and row cy (-1 .. 8)
    auto ldu = [&](const unsigned char *s, int cx, int cy) -> T {
        const int c = (cx + kHX) + kSX * (cy + 1);
        if constexpr (L::LO)
            return df32{*(const float *)(s + L::o_hi + c * 4), *(const float *)(s + L::o_lo + c * 4)};
        else
            return *(const T *)(s + L::o_hi + c * ES);
    };

    C cconst[3], invd_c = C(g.invdiag), diag_c = C(g.diag);
    cconst[0] = C(g.acx);
    cconst[1] = C(g.acy);
    cconst[2] = C(g.acz);

    if (tid == 0)
        for (int zz = z0 - 1; zz < z0 + kPD; ++zz) issue(zz);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = gx < g.nx && gy < g.ny;
    const long long col = (long long)gx + g.pitch * gy;
    double part = 0.0;  // residual sum (resid pass)
    long long dbits = 0;  // largest |u' - u| of the sweep (abs_diff_bits)
    int last_issued = z0 + kPD - 1;  // planes issued so far: z0 - 1 .. last_issued
    int next_wait = z0 - 1;          // first plane this thread has not seen land
    bool ok = true;
    // ring slots of planes z - 1, z, z + 1 (advanced with z, no modulo)
    int im = 0, i0 = 1 % kNS, ip = 2 % kNS;
    // the column's iterate at z - 1 and z and its -z face weight carry over
    // in registers from the previous plane
    T u_m = zero_u<PREC>(), u_c = zero_u<PREC>();
    C wz_m = C(0);
    for (int z = z0; z < z1; ++z) {
        // a wait that runs out leaves next_wait at its plane, so the drain
        // below waits for that plane and every later one
        while (ok && next_wait <= z + 1) {
            if (wait(next_wait, wlim)) ++next_wait;
            else ok = false;
        }
        // one decision for the whole block (a bounded wait may run out in one
        // thread and not in another); the barrier also means every thread is
        // done with plane z - 2's slot
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (tid == 0) issue(z + kPD);
        last_issued = z + kPD;
        const unsigned char *sm = smem + im * L::BYTES, *s0 = smem + i0 * L::BYTES,
                            *sp = smem + ip * L::BYTES;
        if (active) {
            if (z == z0) {
                u_m = ldu(sm, tx, ty);
                u_c = ldu(s0, tx, ty);
                if constexpr (VARK) wz_m = ld(sm, L::o_wz, tid);
            }
            T nb[6];
            nb[0] = ldu(s0, tx - 1, ty);
            nb[1] = ldu(s0, tx + 1, ty);
            nb[2] = ldu(s0, tx, ty - 1);
            nb[3] = ldu(s0, tx, ty + 1);
            nb[4] = u_m;
            nb[5] = ldu(sp, tx, ty);
            const C fi = ld(s0, L::o_f, tid);
            T t;
            C invd_i = invd_c;
            if constexpr (VARK) {
                C wgt[6];
                wgt[0] = ld(s0, L::o_wx, ty * kSX + kHX + tx - 1);
                wgt[1] = ld(s0, L::o_wx, ty * kSX + kHX + tx);
                wgt[2] = ld(s0, L::o_wy, ty * kTX + tx);
                wgt[3] = ld(s0, L::o_wy, (ty + 1) * kTX + tx);
                wgt[4] = wz_m;
                wgt[5] = ld(s0, L::o_wz, tid);
                wz_m = wgt[5];
                invd_i = ld(s0, L::o_id, tid);
                t = P::t_of(nb, wgt, invd_i, fi, u_c);
            } else {
                t = P::t_const(nb, cconst, invd_c, fi, u_c);
            }
            const long long i = col + (long long)g.plane * z;
            if (p.nsw) {
                const T un = P::relax(u_c, t, omega);
                store_u<PREC>(a.bufs, dst, i, un);
                if constexpr (PREC != PREC_DF)
                    if (dinf) dbits = max_bits(dbits, abs_diff_bits((double)un, (double)u_c));
            } else {
                part += P::resid2(t, VARK ? C(1) / invd_i : diag_c);
            }
            u_m = u_c;
            u_c = nb[5];
        }
        im = i0;
        i0 = ip;
        ip = ip + 1 == kNS ? 0 : ip + 1;
    }
    // every copy still in flight lands before the CTA's shared memory goes
    // away: after a wait that ran out too (this drain uses the default limit,
    // so a solve with a short limit still exits cleanly); a wait that ran out
    // marks the solve
    for (; next_wait <= last_issued; ++next_wait) ok = wait(next_wait, kDefaultWaitLimit) && ok;
    if (!ok) atomicOr(&s_err, 1);
    __syncthreads();
    if (s_err && tid == 0) atomicExch(&a.st->status, (int)DST_TIMEOUT);
    double tot = 0.0;
    if (p.resid) tot = block_sum(part);
    else if (dinf) tot = block_max_bits(dbits);
    finish_pass(a, p, tot, dinf);
}

template <int PREC, bool VARK>
void *plane_entry() {
    return (void *)&plane3d_kernel<PREC, VARK>;
}

template <int PREC, bool VARK>
cudaError_t plane_prepare() {
    static bool done = false;  // idempotent; a repeated call is harmless
    if (done) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(plane_entry<PREC, VARK>(),
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               Plane<PREC, VARK>::SMEM);
    if (e == cudaSuccess) done = true;
    return e;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

int plane3d_zchunk(const GridGeo &g) { return g.nz < 32 ? g.nz : 32; }

Plane3dPlan plane3d_plan(int prec, const GridGeo &g, bool vark) {
    Plane3dPlan p{};
    p.block = dim3(kTX, kTY, 1);
    p.zchunk = plane3d_zchunk(g);
    p.grid = dim3((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, (g.nz + p.zchunk - 1) / p.zchunk);
    if (prec == PREC_F64) {
        p.kernel = vark ? plane_entry<PREC_F64, true>() : plane_entry<PREC_F64, false>();
        p.smem = vark ? Plane<PREC_F64, true>::SMEM : Plane<PREC_F64, false>::SMEM;
    } else if (prec == PREC_F32) {
        p.kernel = vark ? plane_entry<PREC_F32, true>() : plane_entry<PREC_F32, false>();
        p.smem = vark ? Plane<PREC_F32, true>::SMEM : Plane<PREC_F32, false>::SMEM;
    } else {
        p.kernel = vark ? plane_entry<PREC_DF, true>() : plane_entry<PREC_DF, false>();
        p.smem = vark ? Plane<PREC_DF, true>::SMEM : Plane<PREC_DF, false>::SMEM;
    }
    return p;
}

cudaError_t plane3d_prepare(int prec, bool vark) {
    if (prec == PREC_F64) return vark ? plane_prepare<PREC_F64, true>() : plane_prepare<PREC_F64, false>();
    if (prec == PREC_F32) return vark ? plane_prepare<PREC_F32, true>() : plane_prepare<PREC_F32, false>();
    return vark ? plane_prepare<PREC_DF, true>() : plane_prepare<PREC_DF, false>();
}

// Tensor maps of the staged arrays: 3D {nx, ny, nz} over the padded layout
// (row stride pitch, plane stride pitch * ny elements), boxes as in Plane.
// Coordinates outside {nx, ny, nz} read as zero.
cudaError_t plane3d_encode(int prec, bool vark, const GridGeo &g, const IterBufs &b,
                           Plane3dMaps *m) {
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                               cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return e != cudaSuccess ? e : cudaErrorNotSupported;
        encode = (EncodeTiledFn)fn;
    }
    const int es = prec == PREC_F64 ? 8 : 4;
    const CUtensorMapDataType dt =
        prec == PREC_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * es, (cuuint64_t)g.plane * es};
    const cuuint32_t estr[3] = {1, 1, 1};
    auto enc = [&](CUtensorMap *map, const void *base, cuuint32_t bx, cuuint32_t by) -> cudaError_t {
        const cuuint32_t box[3] = {bx, by, 1};
        const CUresult r = encode(map, dt, 3, const_cast<void *>(base), dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
    };
    std::memset((void *)m, 0, sizeof(*m));
    cudaError_t e = cudaSuccess;
    auto ck = [&](cudaError_t x) {
        if (x != cudaSuccess && e == cudaSuccess) e = x;
    };
    for (int k = 0; k < 2; ++k) {
        ck(enc(&m->u[k], b.u[k], kSX, kTY + 2));
        if (prec == PREC_DF) ck(enc(&m->ulo[k], b.ulo[k], kSX, kTY + 2));
    }
    ck(enc(&m->f, b.f, kTX, kTY));
    if (vark) {
        ck(enc(&m->wx, b.wx, kSX, kTY));
        ck(enc(&m->wy, b.wy, kTX, kTY + 1));
        ck(enc(&m->wz, b.wz, kTX, kTY));
        ck(enc(&m->invd, b.invd, kTX, kTY));
    }
    return e;
}

}  // namespace srj
