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
#include <type_traits>

#include "df32.cuh"
#include "df32x2.cuh"
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
    __shared__ int s_skip;
    if (tid == 0) {
        s_plan = plan_pass(a, 1);
        // beside the two-sweep kernel this one runs only a cycle's tail
        s_skip = s_plan.run && a.tail_only && !pass_is_tail(a.st, a.lvl_m);
        s_omega = (s_plan.run && s_plan.nsw) ? a.w64[s_plan.woff] : 0.0;
        s_wlim = a.st->wait_limit;
        s_err = 0;
        if (!s_plan.run && a.cfg.use_cond && blockIdx.x == 0 && blockIdx.y == 0 &&
            blockIdx.z == 0)
            cudaGraphSetConditional(a.cfg.cond, 0);
        if (s_plan.run && !s_skip) {
            for (int k = 0; k < kNS; ++k) bar_init(&s_bar[k]);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
    }
    __syncthreads();
    const PassPlan p = s_plan;
    if (!p.run || s_skip) return;
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
            T t = zero_u<PREC>(), un = zero_u<PREC>();
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
                if (p.nsw) un = P::sweep_of(nb, wgt, invd_i, fi, u_c, omega);
                else t = P::t_of(nb, wgt, invd_i, fi, u_c);
            } else {
                if (p.nsw) un = P::sweep_const(nb, cconst, invd_c, fi, u_c, omega);
                else t = P::t_const(nb, cconst, invd_c, fi, u_c);
            }
            const long long i = col + (long long)g.plane * z;
            if (p.nsw) {
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

// ---------------------------------------------------------------------------
// Two sweeps per pass (temporal blocking along z, 2.5D).  A CTA of 32 x 8
// threads owns a 32 x 16 output tile and walks a chunk of z planes.  Input
// planes (iterate, rhs and, for variable coefficients, the face weights and
// 1/D) arrive by TMA in one box shape {40, 20} from (x0 - 4, y0 - 2): four
// ring slots, planes issued up to three ahead.  At step z, level 1 (the first
// sweep of the pass) computes plane z on the tile plus a one-cell halo (34 x
// 18 points) into a two-plane ring of level-1 values; after a block barrier,
// level 2 (the second sweep) computes plane z - 1 of the tile from the
// level-1 ring and stores it.  Thread (tx, ty) owns the tile points (tx, ty)
// and (tx, ty + 8) at both levels; the 100 points of the halo ring belong to
// threads 0 .. 99.  A thread's two points therefore pass from level 1 to
// level 2 in registers: the level-1 value (level 2's +z neighbour) and every
// coefficient level 1 read for the plane (level 2 uses them one step later);
// only the four in-plane neighbours come from the level-1 ring.  The z
// neighbours and the -z face weights are carried from plane to plane.  In
// the FP32-pair form the two points of a thread are the two components of
// packed FP32 instructions (df2).  Level-1 values outside the grid are zero
// (the Dirichlet ghosts).  Only passes of two sweeps run here; the last pass
// of a cycle (fewer sweeps, the residual) runs in plane3d_kernel.
constexpr int kT2Y = 16;              // output rows per tile (two per thread)
constexpr int kBW = 40, kBH = 20;     // staged box: columns x0-4 .., rows y0-2 ..
constexpr int kL1W = 34, kL1H = 18;   // level-1 region: columns x0-1 .., rows y0-1 ..
constexpr int kL1N = kL1W * kL1H;     // 612 points
constexpr int kNS2 = 4;               // input ring slots
constexpr int kT2Threads = kTX * kTY;  // 256
constexpr int kL1Lo = al128(kL1N * 4);  // FP32 pair: offset of a level-1 plane's low part

template <int PREC, bool VARK>
struct Plane2 {
    using T = typename Elem<PREC>::T;
    static constexpr bool LO = PREC == PREC_DF;
    static constexpr int ES = PREC == PREC_F64 ? 8 : 4;
    static constexpr int BOX = kBW * kBH * ES;  // bytes of one staged array (multiple of 128)
    static constexpr int o_hi = 0, o_lo = BOX, o_f = o_lo + (LO ? BOX : 0);
    static constexpr int o_wx = o_f + BOX, o_wy = o_wx + (VARK ? BOX : 0);
    static constexpr int o_wz = o_wy + (VARK ? BOX : 0), o_id = o_wz + (VARK ? BOX : 0);
    static constexpr int BYTES = o_id + (VARK ? BOX : 0);    // one ring slot
    static constexpr unsigned TX = (unsigned)BYTES;          // bytes a plane's copies deliver
    // one level-1 plane (the FP32 pair as separate high and low planes)
    static constexpr int L1B = LO ? 2 * kL1Lo : al128(kL1N * (int)sizeof(T));
    static constexpr int SMEM = kNS2 * BYTES + 2 * L1B;
    static constexpr int MINB = SMEM > 113 * 1024 ? 1 : 2;   // CTAs per SM the smem allows
};

// The two tile points of a thread at one level, side by side.  FP32 pair:
// the components of df2 (packed FP32 instructions); FP32 and FP64: a pair of
// scalar points.  Staged arrays are read at slot offsets, level-1 planes at
// level-1 indices (the FP32 pair as a high plane followed by a low plane).
template <int PREC, bool VARK>
struct Two3 {
    using T = typename Elem<PREC>::T;
    using C = typename Elem<PREC>::C;
    using L = Plane2<PREC, VARK>;
    using P = Point<PREC, 3>;
    struct V {
        T p[2];
    };
    struct W {
        C p[2];
    };

    __device__ __forceinline__ static T ld1(const unsigned char *pl, int i) {
        if constexpr (PREC == PREC_DF)
            return df32{((const float *)pl)[i], ((const float *)(pl + kL1Lo))[i]};
        else
            return ((const T *)pl)[i];
    }
    __device__ __forceinline__ static void st1(unsigned char *pl, int i, T v) {
        if constexpr (PREC == PREC_DF) {
            ((float *)pl)[i] = v.hi;
            ((float *)(pl + kL1Lo))[i] = v.lo;
        } else {
            ((T *)pl)[i] = v;
        }
    }
    __device__ __forceinline__ static T ldu(const unsigned char *s, int i) {
        if constexpr (PREC == PREC_DF)
            return df32{*(const float *)(s + L::o_hi + i * 4), *(const float *)(s + L::o_lo + i * 4)};
        else
            return *(const T *)(s + L::o_hi + i * L::ES);
    }
    __device__ __forceinline__ static C ldc(const unsigned char *s, int off, int i) {
        return *(const C *)(s + off + i * L::ES);
    }
};

template <bool VARK>
struct Two3DF {
    using L = Plane2<PREC_DF, VARK>;
    using V = df2;
    using W = float2;
    __device__ __forceinline__ static df2 ldu(const unsigned char *s, int i0, int i1) {
        const float *h = (const float *)(s + L::o_hi), *l = (const float *)(s + L::o_lo);
        return df2{make_float2(h[i0], h[i1]), make_float2(l[i0], l[i1])};
    }
    __device__ __forceinline__ static float2 ldc(const unsigned char *s, int off, int i0, int i1) {
        const float *c = (const float *)(s + off);
        return make_float2(c[i0], c[i1]);
    }
    __device__ __forceinline__ static df2 ld1(const unsigned char *pl, int i0, int i1) {
        const float *h = (const float *)pl, *l = (const float *)(pl + kL1Lo);
        return df2{make_float2(h[i0], h[i1]), make_float2(l[i0], l[i1])};
    }
};

template <int PREC, bool VARK>
__global__ void __launch_bounds__(kT2Threads, (Plane2<PREC, VARK>::MINB))
    plane3d2_kernel(PassLaunch a, int zchunk, const __grid_constant__ Plane3dMaps maps) {
    using T = typename Elem<PREC>::T;
    using C = typename Elem<PREC>::C;
    using P = Point<PREC, 3>;
    using L = Plane2<PREC, VARK>;
    using S = Two3<PREC, VARK>;
    constexpr bool DF = PREC == PREC_DF;
    using D = Two3DF<VARK>;
    // a thread's two points: packed pairs (FP32 pair) or two scalars
    using V = std::conditional_t<DF, df2, typename S::V>;
    using W = std::conditional_t<DF, float2, typename S::W>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_bar[kNS2];
    __shared__ PassPlan s_plan;
    __shared__ double s_om[2];
    __shared__ long long s_wlim;
    __shared__ int s_mine, s_err;

    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kTX * ty;
    if (tid == 0) {
        s_plan = plan_pass(a, 2);
        // this kernel runs the passes of two sweeps; the rest of a cycle (and
        // the residual) belongs to the one-sweep kernel launched beside it
        s_mine = s_plan.run && s_plan.nsw == 2 && !s_plan.resid;
        s_om[0] = s_mine ? a.w64[s_plan.woff] : 0.0;
        s_om[1] = s_mine ? a.w64[s_plan.woff + 1] : 0.0;
        s_wlim = a.st->wait_limit;
        s_err = 0;
        if (!s_plan.run && a.cfg.use_cond && blockIdx.x == 0 && blockIdx.y == 0 &&
            blockIdx.z == 0)
            cudaGraphSetConditional(a.cfg.cond, 0);
        if (s_mine) {
            for (int k = 0; k < kNS2; ++k) bar_init(&s_bar[k]);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
    }
    __syncthreads();
    if (!s_mine) return;
    const PassPlan p = s_plan;
    const double om1 = s_om[0], om2 = s_om[1];
    const float om1f = (float)om1, om2f = (float)om2;
    const long long wlim = s_wlim;

    const GridGeo &g = a.geo;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kT2Y;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    const int src = p.cur, dst = p.cur ^ 1;
    unsigned char *l1b = smem + kNS2 * L::BYTES;  // two level-1 planes

    // plane zz (>= z0 - 2) lives in slot (zz - z0 + 2) mod 4; the n-th plane
    // of a slot completes its barrier's phase n
    auto rel = [&](int zz) { return zz - (z0 - 2); };
    auto slot = [&](int zz) -> unsigned char * { return smem + (rel(zz) % kNS2) * L::BYTES; };
    auto issue = [&](int zz) {  // one thread
        unsigned char *s = slot(zz);
        uint64_t *bar = &s_bar[rel(zz) % kNS2];
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        bar_expect(bar, L::TX);
        const int xs = x0 - kHX, ys = y0 - 2;
        tma3(s + L::o_hi, &maps.u[src], xs, ys, zz, bar);
        if constexpr (L::LO) tma3(s + L::o_lo, &maps.ulo[src], xs, ys, zz, bar);
        tma3(s + L::o_f, &maps.f, xs, ys, zz, bar);
        if constexpr (VARK) {
            tma3(s + L::o_wx, &maps.wx, xs, ys, zz, bar);
            tma3(s + L::o_wy, &maps.wy, xs, ys, zz, bar);
            tma3(s + L::o_wz, &maps.wz, xs, ys, zz, bar);
            tma3(s + L::o_id, &maps.invd, xs, ys, zz, bar);
        }
    };
    auto wait = [&](int zz, long long limit) -> bool {
        return bar_wait(&s_bar[rel(zz) % kNS2], (unsigned)((rel(zz) / kNS2) & 1), limit);
    };
    // staged arrays: index of column lx (-4 .. 35), row ly (-2 .. 17) of the tile;
    // level-1 planes: column lx (-1 .. 32), row ly (-1 .. 16)
    auto sidx = [](int lx, int ly) { return (lx + kHX) + kBW * (ly + 2); };
    auto lidx = [](int lx, int ly) { return (lx + 1) + kL1W * (ly + 1); };
    auto l1 = [&](int zz) -> unsigned char * { return l1b + (zz & 1) * L::L1B; };

    C cconst[3];
    const C invd_c = C(g.invdiag);
    cconst[0] = C(g.acx);
    cconst[1] = C(g.acy);
    cconst[2] = C(g.acz);

    // the thread's tile points (tx, ty + 8 q), q = 0, 1
    int si[2], li[2];
    bool in[2];
    long long col[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int ly = ty + 8 * q;
        si[q] = sidx(tx, ly);
        li[q] = lidx(tx, ly);
        in[q] = (x0 + tx) < g.nx && (y0 + ly) < g.ny;
        col[q] = (long long)(x0 + tx) + g.pitch * (y0 + ly);
    }
    // the halo ring (100 points: rows -1 and 16 over columns -1 .. 32, then
    // columns -1 and 32 over rows 0 .. 15): threads 0 .. 49 own ring points
    // tid and tid + 50, side by side like the tile points
    constexpr int kRing = 2 * kL1W + 2 * kT2Y;
    const bool hasH = tid < kRing / 2;
    int siH[2], liH[2];
    bool inH[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int h = tid + q * (kRing / 2);
        int hx, hy;
        if (h < kL1W) hx = h - 1, hy = -1;
        else if (h < 2 * kL1W) hx = h - kL1W - 1, hy = kT2Y;
        else if (h < 2 * kL1W + kT2Y) hx = -1, hy = h - 2 * kL1W;
        else hx = kTX, hy = h - 2 * kL1W - kT2Y;
        siH[q] = sidx(hx, hy);
        liH[q] = lidx(hx, hy);
        inH[q] = hasH && x0 + hx >= 0 && x0 + hx < g.nx && y0 + hy >= 0 && y0 + hy < g.ny;
    }

    if (tid == 0)
        for (int zz = z0 - 2; zz <= min(z0 + 1, z1 + 1); ++zz) issue(zz);
    int last_issued = min(z0 + 1, z1 + 1);
    int next_wait = z0 - 2;  // first plane this thread has not seen land
    bool ok = true;

    // loads of two points (the tile pair or the ring pair) side by side
    auto ld_u2 = [&](const unsigned char *s, const int *ix, int d) -> V {
        if constexpr (DF) return D::ldu(s, ix[0] + d, ix[1] + d);
        else return V{{S::ldu(s, ix[0] + d), S::ldu(s, ix[1] + d)}};
    };
    auto ld_c2 = [&](const unsigned char *s, int off, const int *ix, int d) -> W {
        if constexpr (DF) return D::ldc(s, off, ix[0] + d, ix[1] + d);
        else return W{{S::ldc(s, off, ix[0] + d), S::ldc(s, off, ix[1] + d)}};
    };
    auto ld_l1 = [&](const unsigned char *pl, int d) -> V {
        if constexpr (DF) return D::ld1(pl, li[0] + d, li[1] + d);
        else return V{{S::ld1(pl, li[0] + d), S::ld1(pl, li[1] + d)}};
    };
    auto zero2 = [&]() -> V {
        if constexpr (DF) return df2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        else return V{{zero_u<PREC>(), zero_u<PREC>()}};
    };
    auto wzero2 = [&]() -> W {
        if constexpr (DF) return make_float2(0.f, 0.f);
        else return W{{C(0), C(0)}};
    };
    auto get = [&](const V &v, int q) -> T {
        if constexpr (DF) return q ? df32{v.hi.y, v.lo.y} : df32{v.hi.x, v.lo.x};
        else return v.p[q];
    };
    // point q keeps its value where k[q], else zero (ghost)
    auto keep = [&](V v, bool k0, bool k1) -> V {
        if constexpr (DF) {
            if (!k0) v.hi.x = v.lo.x = 0.f;
            if (!k1) v.hi.y = v.lo.y = 0.f;
            return v;
        } else {
            if (!k0) v.p[0] = zero_u<PREC>();
            if (!k1) v.p[1] = zero_u<PREC>();
            return v;
        }
    };
    // one relaxed sweep of the two points
    auto sweep2 = [&](const V *nb, const W *wgt, W invd, W f, const V &uc, double om,
                      float omf) -> V {
        if constexpr (DF) {
            df2 q;
            if constexpr (VARK) q = df2_q_vark<6>(nb, wgt, invd, f);
            else q = df2_q_axes<3>(nb, cconst, f);
            return df2_relax_to(uc, q, omf, 1.f - omf);
        } else {
            V r;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                T n1[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) n1[j] = nb[j].p[k];
                if constexpr (VARK) {
                    C w1[6];
#pragma unroll
                    for (int j = 0; j < 6; ++j) w1[j] = wgt[j].p[k];
                    r.p[k] = P::sweep_of(n1, w1, invd.p[k], f.p[k], uc.p[k], om);
                } else {
                    r.p[k] = P::sweep_const(n1, cconst, invd_c, f.p[k], uc.p[k], om);
                }
            }
            return r;
        }
    };

    // carried values.  Level 1: the iterate at z - 1 and z, the -z face.
    // Level 2: level-1 values at z - 2 and z - 1, and the coefficients level 1
    // read for plane z - 1 (f, faces -x +x -y +y -z +z, 1/D).
    V um1 = zero2(), uc1 = zero2(), vm2 = zero2(), vc2 = zero2();
    W wzm1 = wzero2();
    W cw[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) cw[j] = wzero2();
    V um1H = zero2(), uc1H = zero2();
    W wzm1H = wzero2();

    for (int z = z0 - 1; z <= z1; ++z) {
        // planes z and z + 1 (and, at the first step, z - 1) must have landed
        while (ok && next_wait <= z + 1) {
            if (wait(next_wait, wlim)) ++next_wait;
            else ok = false;
        }
        // one decision for the block; the barrier also means every thread is
        // done with the previous step, so the slot of plane z - 1 is free
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        {
            // plane z + 3 goes into the slot plane z - 1 held (at the first
            // step that slot's plane z0 - 2 is still read: one plane less)
            const int lim = min(z == z0 - 1 ? z + 2 : z + 3, z1 + 1);
            if (tid == 0)
                for (int pl = last_issued + 1; pl <= lim; ++pl) issue(pl);
            if (lim > last_issued) last_issued = lim;
        }
        const unsigned char *s0 = slot(z), *sp = slot(z + 1);
        const bool zin = z >= 0 && z < g.nz;
        unsigned char *l1z = l1(z);
        // level 1 on a pair of points of plane z (ix: staged indices, jx:
        // level-1 indices, k: inside the grid); um, uc, wzm: the carried
        // iterate at z - 1 and z and -z face; nc returns the coefficients read
        auto level1 = [&](const int *ix, const int *jx, const bool *k, V &um, V &uc, W &wzm,
                          W *nc) -> V {
            if (z == z0 - 1) {  // the first step reads what later steps carry
                const unsigned char *sm = slot(z - 1);
                um = ld_u2(sm, ix, 0);
                uc = ld_u2(s0, ix, 0);
                if constexpr (VARK) wzm = ld_c2(sm, L::o_wz, ix, 0);
            }
            const V up = ld_u2(sp, ix, 0);
#pragma unroll
            for (int j = 1; j < 8; ++j) nc[j] = wzero2();
            nc[0] = ld_c2(s0, L::o_f, ix, 0);
            if constexpr (VARK) {
                nc[1] = ld_c2(s0, L::o_wx, ix, -1);
                nc[2] = ld_c2(s0, L::o_wx, ix, 0);
                nc[3] = ld_c2(s0, L::o_wy, ix, -kBW);
                nc[4] = ld_c2(s0, L::o_wy, ix, 0);
                nc[5] = wzm;
                nc[6] = ld_c2(s0, L::o_wz, ix, 0);
                nc[7] = ld_c2(s0, L::o_id, ix, 0);
            }
            V val = zero2();
            if (zin && (k[0] || k[1])) {
                const V nb[6] = {ld_u2(s0, ix, -1), ld_u2(s0, ix, 1), ld_u2(s0, ix, -kBW),
                                 ld_u2(s0, ix, kBW), um, up};
                val = keep(sweep2(nb, nc + 1, nc[7], nc[0], uc, om1, om1f), k[0], k[1]);
            }
            S::st1(l1z, jx[0], get(val, 0));
            S::st1(l1z, jx[1], get(val, 1));
            um = uc;
            uc = up;
            if constexpr (VARK) wzm = nc[6];
            return val;
        };
        // the thread's tile points; level 2 takes the coefficients read here
        // one step later
        W nc[8];  // f, faces -x +x -y +y -z +z, 1/D of plane z
        const V val = level1(si, li, in, um1, uc1, wzm1, nc);
        // level 2: plane z - 1 of the thread's two points, from level-1 planes
        // z - 2 (carried), z - 1 (ring: neighbours, carried: centre) and z
        // (this step's level-1 value), with the coefficients level 1 read for
        // plane z - 1.  Plane z - 1 of the level-1 ring was complete at the
        // barrier that opened this step, and nothing writes it during the
        // step (level 1 writes plane z, the other half of the ring), so no
        // barrier separates the levels.
        if (z - 1 >= z0 && (in[0] || in[1])) {
            const unsigned char *l1m = l1(z - 1);
            const V nb[6] = {ld_l1(l1m, -1), ld_l1(l1m, 1), ld_l1(l1m, -kL1W), ld_l1(l1m, kL1W),
                             vm2, val};
            const V un = sweep2(nb, cw + 1, cw[7], cw[0], vc2, om2, om2f);
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (in[q]) store_u<PREC>(a.bufs, dst, col[q] + (long long)g.plane * (z - 1), get(un, q));
        }
        vm2 = vc2;
        vc2 = val;
#pragma unroll
        for (int j = 0; j < 8; ++j) cw[j] = nc[j];
        // level 1 on the ring pair (threads 0 .. 49); level 2 reads it from
        // the next step on
        if (hasH) {
            W ncH[8];
            level1(siH, liH, inH, um1H, uc1H, wzm1H, ncH);
        }
    }
    // every copy in flight lands before the shared memory goes away (the
    // drain uses the default limit); a wait that ran out marks the solve
    for (; next_wait <= last_issued; ++next_wait) ok = wait(next_wait, kDefaultWaitLimit) && ok;
    if (!ok) atomicOr(&s_err, 1);
    __syncthreads();
    if (s_err && tid == 0) atomicExch(&a.st->status, (int)DST_TIMEOUT);
    finish_pass(a, p, 0.0);
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

template <int PREC, bool VARK>
void *plane2_entry() {
    return (void *)&plane3d2_kernel<PREC, VARK>;
}

Plane3dPlan plane3d2_plan(int prec, const GridGeo &g, bool vark, int num_sms) {
    Plane3dPlan p{};
    p.block = dim3(kTX, kTY, 1);
    int minb = 2;
#define P2_(PR, VK)                                  \
    do {                                             \
        p.kernel = plane2_entry<PR, VK>();           \
        p.smem = Plane2<PR, VK>::SMEM;               \
        minb = Plane2<PR, VK>::MINB;                 \
    } while (0)
    if (prec == PREC_F64) {
        if (vark) P2_(PREC_F64, true); else P2_(PREC_F64, false);
    } else if (prec == PREC_F32) {
        if (vark) P2_(PREC_F32, true); else P2_(PREC_F32, false);
    } else {
        if (vark) P2_(PREC_DF, true); else P2_(PREC_DF, false);
    }
#undef P2_
    // z chunks: at least four waves of CTAs over the SMs, 16 .. 64 planes each
    // (each chunk computes two extra level-1 planes and stages three extra)
    long long cxy = (long long)((g.nx + kTX - 1) / kTX) * ((g.ny + kT2Y - 1) / kT2Y);
    if (cxy < 1) cxy = 1;
    const long long want = (4LL * num_sms * minb + cxy - 1) / cxy;
    long long zc = (g.nz + want - 1) / (want > 0 ? want : 1);
    if (zc < 16) zc = 16;
    if (zc > 64) zc = 64;
    if (zc > g.nz) zc = g.nz;
    p.zchunk = (int)zc;
    p.grid = dim3((g.nx + kTX - 1) / kTX, (g.ny + kT2Y - 1) / kT2Y,
                  (unsigned)((g.nz + zc - 1) / zc));
    return p;
}

cudaError_t plane3d2_prepare(int prec, bool vark) {
    const Plane3dPlan q = plane3d2_plan(prec, GridGeo{}, vark, 1);
    return cudaFuncSetAttribute(q.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, q.smem);
}

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
                           Plane3dMaps *m, bool two_sweep) {
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
    if (two_sweep) {  // every array in the one box of the two-sweep pass
        for (int k = 0; k < 2; ++k) {
            ck(enc(&m->u[k], b.u[k], kBW, kBH));
            if (prec == PREC_DF) ck(enc(&m->ulo[k], b.ulo[k], kBW, kBH));
        }
        ck(enc(&m->f, b.f, kBW, kBH));
        if (vark) {
            ck(enc(&m->wx, b.wx, kBW, kBH));
            ck(enc(&m->wy, b.wy, kBW, kBH));
            ck(enc(&m->wz, b.wz, kBW, kBH));
            ck(enc(&m->invd, b.invd, kBW, kBH));
        }
        return e;
    }
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
