// kernels_plane3d.cu -- the 3D SRJ pass (one relaxed sweep or one residual per
// pass, Sec. 2 Eq. relaxed-jacobi and Sec. 3 Eq. relative-residual) as a
// plane-streaming kernel: a CTA owns a 32 x 8 column tile and walks a chunk of
// z planes; every plane it needs (the iterate with a one-cell halo, the
// right-hand side and, for variable coefficients, the face weights and 1/D)
// is staged into a shared-memory ring by cp.async several planes ahead, so the
// loads of plane z + 3 are in flight while plane z is computed.  Points outside
// the grid are zero-filled by the copies (zero Dirichlet values, zero faces).
// Same pass protocol as the generic kernel: plan_pass / finish_pass.
#include <cuda_runtime.h>
#include <math.h>

#include "df32.cuh"
#include "pass_common.cuh"
#include "stencil_point.cuh"
#include "srj_internal.h"

namespace srj {
namespace {

constexpr int kTX = 32, kTY = 8;  // column tile
constexpr int kHX = 4;            // columns staged left of the tile (16-byte aligned rows)
constexpr int kSX = kTX + 2 * kHX;  // staged row width: x0 - 4 .. x0 + 35
constexpr int kPD = 3;            // planes issued ahead of the one computed
constexpr int kNS = kPD + 2;      // ring slots: planes z-1 .. z+PD

// Shared-memory layout of one ring slot.  Every staged row starts on a
// 16-byte boundary in global and shared memory so that it moves in 16-byte
// cp.async chunks: the iterate rows y0-1 .. y0+8 and x faces rows y0 .. y0+7
// cover columns x0-4 .. x0+35 (the halo columns x0-1 and x0+32 inside);
// the right-hand side, z faces and 1/D cover the tile; y faces rows
// y0-1 .. y0+7.  ES is the element size (4 or 8 bytes).
template <int PREC, bool VARK>
struct Plane {
    static constexpr bool LO = PREC == PREC_DF;
    static constexpr int ES = PREC == PREC_F64 ? 8 : 4;
    static constexpr int U = kSX * (kTY + 2);       // iterate (hi), rows y0-1 .. y0+8
    static constexpr int F = kTX * kTY;
    static constexpr int WX = VARK ? kSX * kTY : 0;
    static constexpr int WY = VARK ? kTX * (kTY + 1) : 0;
    static constexpr int WZ = VARK ? kTX * kTY : 0;
    static constexpr int ID = VARK ? kTX * kTY : 0;
    static constexpr int o_lo = U, o_f = U * (LO ? 2 : 1), o_wx = o_f + F, o_wy = o_wx + WX,
                         o_wz = o_wy + WY, o_id = o_wz + WZ;
    static constexpr int ELEMS = o_id + ID;
    static constexpr int BYTES = ((ELEMS * ES + 15) / 16) * 16;
    static constexpr int SMEM = kNS * BYTES;
    static constexpr int EPC = 16 / ES;  // elements per 16-byte chunk
};

__device__ __forceinline__ void cp16(void *smem, const void *g, bool ok, const void *safe) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const void *src = ok ? g : safe;
    const int n = ok ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(n));
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <int PREC, bool VARK>
__global__ void __launch_bounds__(kTX * kTY) plane3d_kernel(PassLaunch a, int zchunk) {
    using T = typename Elem<PREC>::T;
    using C = typename Elem<PREC>::C;
    using P = Point<PREC, 3>;
    using L = Plane<PREC, VARK>;
    constexpr int ES = L::ES;
    extern __shared__ __align__(16) unsigned char smem[];

    __shared__ PassPlan s_plan;
    __shared__ double s_omega;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + kTX * ty;
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
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    const int src = p.cur, dst = p.cur ^ 1;
    const unsigned char *uhi = (const unsigned char *)a.bufs.u[src];
    const unsigned char *ulo = (const unsigned char *)a.bufs.ulo[src];
    const unsigned char *fb = (const unsigned char *)a.bufs.f;
    const unsigned char *wxb = (const unsigned char *)a.bufs.wx;
    const unsigned char *wyb = (const unsigned char *)a.bufs.wy;
    const unsigned char *wzb = (const unsigned char *)a.bufs.wz;
    const unsigned char *idb = (const unsigned char *)a.bufs.invd;
    const bool dinf = a.dinf && p.nsw;

    // Copy plane zz into ring slot zz mod NS in 16-byte chunks.  A chunk is
    // copied when it lies inside the grid's rows and planes and inside the
    // padded row [0, pitch) (pitch is a multiple of 32, so a chunk is either
    // wholly inside or wholly outside); otherwise it is zero-filled: the
    // zero Dirichlet values of the ghost rows, columns and planes, and zero
    // faces there.  Columns in [nx, pitch) are zero in memory.
    auto issue = [&](int zz) {
        unsigned char *slot = smem + ((zz + kNS) % kNS) * L::BYTES;
        const bool zok = zz >= 0 && zz < g.nz;
        const long long pz = (long long)g.plane * (zok ? zz : 0);
        // one array segment: rows [r0, r0 + nr) of the tile, columns
        // [c0, c0 + cw), into smem at element offset so (row stride cw)
        auto seg = [&](const unsigned char *base, int so, int r0, int nr, int c0, int cw) {
            const int cpr = cw / L::EPC;
            for (int q = tid; q < nr * cpr; q += kTX * kTY) {
                const int rr = q / cpr, cc = q - rr * cpr;
                const int gy = y0 + r0 + rr, gx = x0 + c0 + cc * L::EPC;
                const bool ok = zok && gy >= 0 && gy < g.ny && gx >= 0 && gx < g.pitch;
                const long long off = (pz + (long long)g.pitch * (ok ? gy : 0) + (ok ? gx : 0)) * ES;
                cp16(slot + (so + rr * cw + cc * L::EPC) * ES, base + off, ok, base);
            }
        };
        seg(uhi, 0, -1, kTY + 2, -kHX, kSX);
        if constexpr (L::LO) seg(ulo, L::o_lo, -1, kTY + 2, -kHX, kSX);
        seg(fb, L::o_f, 0, kTY, 0, kTX);
        if constexpr (VARK) {
            seg(wxb, L::o_wx, 0, kTY, -kHX, kSX);
            seg(wyb, L::o_wy, -1, kTY + 1, 0, kTX);
            seg(wzb, L::o_wz, 0, kTY, 0, kTX);
            seg(idb, L::o_id, 0, kTY, 0, kTX);
        }
        cpa_commit();
    };
    auto sl = [&](int zz) -> const unsigned char * {
        return smem + ((zz + kNS) % kNS) * L::BYTES;
    };
    auto ld = [&](const unsigned char *slot, int idx) -> C {
        return *(const C *)(slot + idx * ES);
    };
    // iterate at tile column cx (-1 .. 32) and row cy (-1 .. 8)
    auto ldu = [&](const unsigned char *slot, int cx, int cy) -> T {
        const int c = (cx + kHX) + kSX * (cy + 1);
        if constexpr (L::LO)
            return df32{*(const float *)(slot + c * ES), *(const float *)(slot + (L::o_lo + c) * ES)};
        else
            return *(const T *)(slot + c * ES);
    };

    C cconst[3], invd_c = C(1.0 / g.diag), diag_c = C(g.diag);
    cconst[0] = C(g.cx / g.diag);
    cconst[1] = C(g.cy / g.diag);
    cconst[2] = C(g.cz / g.diag);

    // prologue: planes z0 - 1 .. z0 + PD - 1
    for (int zz = z0 - 1; zz < z0 + kPD; ++zz) issue(zz);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = gx < g.nx && gy < g.ny;
    const long long col = (long long)gx + g.pitch * gy;
    double part = 0.0;
    for (int z = z0; z < z1; ++z) {
        // issued so far: planes up to z + PD - 1, one group each; all but the
        // newest PD - 2 are complete, so planes z - 1, z, z + 1 have landed
        cpa_wait<kPD - 2>();
        __syncthreads();      // everyone's did; everyone finished plane z - 1
        issue(z + kPD);       // into the slot of plane z - 2
        const unsigned char *sm = sl(z - 1), *s0 = sl(z), *sp = sl(z + 1);
        if (active) {
            T nb[6];
            nb[0] = ldu(s0, tx - 1, ty);
            nb[1] = ldu(s0, tx + 1, ty);
            nb[2] = ldu(s0, tx, ty - 1);
            nb[3] = ldu(s0, tx, ty + 1);
            nb[4] = ldu(sm, tx, ty);
            nb[5] = ldu(sp, tx, ty);
            const T u_c = ldu(s0, tx, ty);
            const C fi = ld(s0, L::o_f + tid);
            T t;
            C diag_i = diag_c;
            if constexpr (VARK) {
                C wgt[6];
                wgt[0] = ld(s0, L::o_wx + ty * kSX + kHX + tx - 1);
                wgt[1] = ld(s0, L::o_wx + ty * kSX + kHX + tx);
                wgt[2] = ld(s0, L::o_wy + ty * kTX + tx);
                wgt[3] = ld(s0, L::o_wy + (ty + 1) * kTX + tx);
                wgt[4] = ld(sm, L::o_wz + tid);
                wgt[5] = ld(s0, L::o_wz + tid);
                const C invd_i = ld(s0, L::o_id + tid);
                t = P::t_of(nb, wgt, invd_i, fi, u_c);
                diag_i = C(1) / invd_i;
            } else {
                t = P::t_const(nb, cconst, invd_c, fi, u_c);
            }
            const long long i = col + (long long)g.plane * z;
            if (p.nsw) {
                const T un = P::relax(u_c, t, omega);
                store_u<PREC>(a.bufs, dst, i, un);
                if constexpr (PREC != PREC_DF)
                    if (dinf) part = nan_max(part, fabs((double)un - (double)u_c));
            } else {
                part += P::resid2(t, diag_i);
            }
        }
    }
    cpa_wait<0>();
    double tot = 0.0;
    if (p.resid) tot = block_sum(part);
    else if (dinf) tot = block_max(part);
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

}  // namespace srj
