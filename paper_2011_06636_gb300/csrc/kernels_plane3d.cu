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
// 18 points, a fixed set of two or three per thread) into a two-plane ring of
// level-1 values; after a block barrier, level 2 (the second sweep) computes
// plane z - 1 of the tile (two points per thread) from the level-1 ring and
// stores it.  Each thread carries the z neighbours of its points and the
// -z face weights in registers from plane to plane, and level 2 reads the
// coefficients of its next plane one step ahead, so no slot is needed after
// the step that last reads it.  Level-1 values outside the grid are zero (the
// Dirichlet ghosts).  Only passes of two sweeps run here; the last pass of a
// cycle (fewer sweeps, the residual) runs in plane3d_kernel.
constexpr int kT2Y = 16;              // output rows per tile (two per thread)
constexpr int kBW = 40, kBH = 20;     // staged box: columns x0-4 .., rows y0-2 ..
constexpr int kL1W = 34, kL1H = 18;   // level-1 region: columns x0-1 .., rows y0-1 ..
constexpr int kL1N = kL1W * kL1H;     // 612 points
constexpr int kNS2 = 4;               // input ring slots
constexpr int kT2Threads = kTX * kTY;  // 256

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
    static constexpr int L1B = al128(kL1N * (int)sizeof(T));  // one level-1 plane
    static constexpr int SMEM = kNS2 * BYTES + 2 * L1B;
    static constexpr int MINB = SMEM > 113 * 1024 ? 1 : 2;   // CTAs per SM the smem allows
};

template <int PREC, bool VARK>
__global__ void __launch_bounds__(kT2Threads, (Plane2<PREC, VARK>::MINB))
    plane3d2_kernel(PassLaunch a, int zchunk, const __grid_constant__ Plane3dMaps maps) {
    using T = typename Elem<PREC>::T;
    using C = typename Elem<PREC>::C;
    using P = Point<PREC, 3>;
    using L = Plane2<PREC, VARK>;
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
    // staged arrays: index of column lx (-4 .. 35), row ly (-2 .. 17) of the tile
    auto sidx = [](int lx, int ly) { return (lx + kHX) + kBW * (ly + 2); };
    auto ldc = [&](const unsigned char *s, int off, int i) -> C {
        return *(const C *)(s + off + i * L::ES);
    };
    auto ldu = [&](const unsigned char *s, int i) -> T {
        if constexpr (L::LO)
            return df32{*(const float *)(s + L::o_hi + i * 4), *(const float *)(s + L::o_lo + i * 4)};
        else
            return *(const T *)(s + L::o_hi + i * L::ES);
    };
    auto l1 = [&](int zz) -> T * { return (T *)(l1b + (zz & 1) * L::L1B); };

    C cconst[3];
    const C invd_c = C(g.invdiag);
    cconst[0] = C(g.acx);
    cconst[1] = C(g.acy);
    cconst[2] = C(g.acz);

    // level-1 points of this thread: q = tid + 256 k, column q % 34 - 1,
    // row q / 34 - 1 of the tile; and level-2 points: column tx, rows ty, ty + 8
    constexpr int K1 = (kL1N + kT2Threads - 1) / kT2Threads;  // 3
    int si1[K1];
    bool has1[K1], in1[K1];
#pragma unroll
    for (int k = 0; k < K1; ++k) {
        const int q = tid + kT2Threads * k;
        has1[k] = q < kL1N;
        const int lx = q % kL1W - 1, ly = q / kL1W - 1;
        si1[k] = sidx(lx, ly);
        const int gx = x0 + lx, gy = y0 + ly;
        in1[k] = has1[k] && gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny;
    }
    int si2[2], li2[2];
    bool in2[2];
    long long col2[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int ly = ty + 8 * q;
        si2[q] = sidx(tx, ly);
        li2[q] = (tx + 1) + kL1W * (ly + 1);
        in2[q] = (x0 + tx) < g.nx && (y0 + ly) < g.ny;
        col2[q] = (long long)(x0 + tx) + g.pitch * (y0 + ly);
    }

    if (tid == 0)
        for (int zz = z0 - 2; zz <= min(z0 + 1, z1 + 1); ++zz) issue(zz);
    int last_issued = min(z0 + 1, z1 + 1);
    int next_wait = z0 - 2;  // first plane this thread has not seen land
    bool ok = true;

    // carried values: level 1 -- the iterate at z - 1 and z and the -z face;
    // level 2 -- level-1 values at z - 2 and z - 1 and the coefficients of the
    // plane it computes next
    T um1[K1], uc1[K1];
    C wzm1[K1];
#pragma unroll
    for (int k = 0; k < K1; ++k) {
        um1[k] = zero_u<PREC>();
        uc1[k] = zero_u<PREC>();
        wzm1[k] = C(0);
    }
    T vm2[2], vc2[2];
    C cf[2], cwxm[2], cwxp[2], cwym[2], cwyp[2], cwzm[2], cwzp[2], cid[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        vm2[q] = zero_u<PREC>();
        vc2[q] = zero_u<PREC>();
        cf[q] = cwxm[q] = cwxp[q] = cwym[q] = cwyp[q] = cwzm[q] = cwzp[q] = C(0);
        cid[q] = invd_c;
    }

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
        T *l1z = l1(z);
        // level 1: plane z of the tile plus halo
#pragma unroll
        for (int k = 0; k < K1; ++k) {
            if (!has1[k]) continue;
            const int i = si1[k];
            if (z == z0 - 1) {  // the first step reads what later steps carry
                const unsigned char *sm = slot(z - 1);
                um1[k] = ldu(sm, i);
                uc1[k] = ldu(s0, i);
                if constexpr (VARK) wzm1[k] = ldc(sm, L::o_wz, i);
            }
            const T up = ldu(sp, i);
            T val = zero_u<PREC>();
            C wzp = C(0);
            if constexpr (VARK) wzp = ldc(s0, L::o_wz, i);
            if (in1[k] && zin) {
                T nb[6];
                nb[0] = ldu(s0, i - 1);
                nb[1] = ldu(s0, i + 1);
                nb[2] = ldu(s0, i - kBW);
                nb[3] = ldu(s0, i + kBW);
                nb[4] = um1[k];
                nb[5] = up;
                const C fi = ldc(s0, L::o_f, i);
                if constexpr (VARK) {
                    C wgt[6];
                    wgt[0] = ldc(s0, L::o_wx, i - 1);
                    wgt[1] = ldc(s0, L::o_wx, i);
                    wgt[2] = ldc(s0, L::o_wy, i - kBW);
                    wgt[3] = ldc(s0, L::o_wy, i);
                    wgt[4] = wzm1[k];
                    wgt[5] = wzp;
                    val = P::sweep_of(nb, wgt, ldc(s0, L::o_id, i), fi, uc1[k], om1);
                } else {
                    val = P::sweep_const(nb, cconst, invd_c, fi, uc1[k], om1);
                }
            }
            l1z[tid + kT2Threads * k] = val;
            um1[k] = uc1[k];
            uc1[k] = up;
            if constexpr (VARK) wzm1[k] = wzp;
        }
        __syncthreads();
        // level 2: plane z - 1 of the tile, from level-1 planes z - 2 (carried),
        // z - 1 (ring: neighbours, carried: centre) and z (ring)
        const T *l1m = l1(z - 1);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const T vp = l1z[li2[q]];
            if (z - 1 >= z0 && in2[q]) {
                T nb[6];
                nb[0] = l1m[li2[q] - 1];
                nb[1] = l1m[li2[q] + 1];
                nb[2] = l1m[li2[q] - kL1W];
                nb[3] = l1m[li2[q] + kL1W];
                nb[4] = vm2[q];
                nb[5] = vp;
                T un;
                if constexpr (VARK) {
                    C wgt[6] = {cwxm[q], cwxp[q], cwym[q], cwyp[q], cwzm[q], cwzp[q]};
                    un = P::sweep_of(nb, wgt, cid[q], cf[q], vc2[q], om2);
                } else {
                    un = P::sweep_const(nb, cconst, invd_c, cf[q], vc2[q], om2);
                }
                store_u<PREC>(a.bufs, dst, col2[q] + (long long)g.plane * (z - 1), un);
            }
            vm2[q] = vc2[q];
            vc2[q] = vp;
            // the coefficients of plane z, for the next step
            const int i = si2[q];
            cf[q] = ldc(s0, L::o_f, i);
            if constexpr (VARK) {
                cwxm[q] = ldc(s0, L::o_wx, i - 1);
                cwxp[q] = ldc(s0, L::o_wx, i);
                cwym[q] = ldc(s0, L::o_wy, i - kBW);
                cwyp[q] = ldc(s0, L::o_wy, i);
                cwzm[q] = cwzp[q];
                cwzp[q] = ldc(s0, L::o_wz, i);
                cid[q] = ldc(s0, L::o_id, i);
            }
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
