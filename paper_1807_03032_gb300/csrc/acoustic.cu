// acoustic.cu -- K1: one leapfrog step of the damped isotropic acoustic wave
// equation (Eq. WE; Listing fd-3) with the compact central Laplacian of
// radius R = so/2 (Listing fd-1/fd-2), over every grid point (Dirichlet: zero
// ghosts outside the grid).
//
//   u+ = u + (1 - zeta)(u - u-) + b * lap(u),   b = dt^2 / (m + damp dt/2),
//   zeta = damp * b / dt,
// which is the centred discretisation m (u+ - 2u + u-)/dt^2 +
// damp (u+ - u-)/(2 dt) = lap(u) rearranged for u+; with damp = 0 it is
// u+ = 2u - u- + dt^2 lap(u) / m.
//
// GB300 design.  One CTA owns a BX x BY column of the grid and marches it
// through z.  Every plane p of u^n (tile plus an R-wide halo, zero-filled
// outside the grid by the TMA unit) is brought into a small ring of shared-
// memory stages by cp.async.bulk.tensor, D planes ahead of use; the same stage
// also receives the interior tiles of u^n, u^{n-1} and b for the output plane
// p - R.  Each stage has a "full" mbarrier (TMA transaction count) and an
// "empty" mbarrier (one arrival per warp), so warps run decoupled and thread 0
// refills a stage as soon as every warp has released it.
//
// The z-direction uses an accumulator pipeline: when plane p arrives, each
// thread adds w_|p-z| u(p) to the 2R pending outputs z in [p-R, p+R) it holds
// in registers, adds the x/y part of the Laplacian of plane p (read from the
// staged plane) to output p, and completes output p-R.  Per point this keeps
// 2R floats of state (instead of a 2R+1-plane queue plus R staged planes), so
// the shared-memory ring is only D+1 planes deep.  Every thread owns a 4 (x,
// one float4) by VY (y) micro-tile.  Algorithmic HBM traffic: 16 bytes per
// point (read u^n, u^{n-1}, b; write u^{n+1}); halo and centre re-reads are
// served by L2.
#include <stdio.h>
#include <string.h>

#include "f32x2.cuh"
#include "kernels.cuh"
#include "runtime.cuh"

namespace fdsweep {
namespace {
using namespace f32x2;

// DF: the damping is a 3-D field; the stage then also carries the interior
// tile of the per-point coefficient zeta = damp b / dt (stored after b as a
// second field of the coefficient tensor) instead of forming zeta from the
// per-axis profiles: 20 instead of 16 bytes per point.
template <int R, int TX, int TY, int VY, int D, bool DF = false>
struct AcCfg {
    static constexpr int BX = 4 * TX;
    static constexpr int BY = VY * TY;
    static constexpr int RA = (R + 3) / 4 * 4;  // x halo rounded to 16 bytes (TMA rule)
    static constexpr int PW = BX + 2 * RA;
    static constexpr int PH = BY + 2 * R;
    static constexpr int NSL = D + 1;           // ring slots
    static constexpr int HALO = (PW * PH + 31) / 32 * 32;
    static constexpr int INT = BX * BY;         // interior tile (multiple of 32)
    static constexpr int NINT = DF ? 4 : 3;     // interior tiles per stage
    static constexpr int STAGE = HALO + NINT * INT;  // [halo u^n][u^n][u^{n-1}][b][zeta]
    static constexpr uint32_t HALO_BYTES = PW * PH * 4;
    static constexpr uint32_t INT_BYTES = INT * 4;
    static constexpr int THREADS = TX * TY;
    static constexpr int WARPS = THREADS / 32;
    // stages, full/empty mbarriers, abort flag; + damp_z of the z chunk
    // (added at launch) and 128 bytes to align the base
    static constexpr size_t SMEM = (size_t)NSL * STAGE * 4 + NSL * 16 + 16 + 128;
    static_assert(PW <= 256 && PH <= 256 && BX <= 256 && BY <= 256, "TMA box dimension limit");
    static_assert(INT % 32 == 0 && THREADS % 32 == 0, "tile shape");
};

// Source injection by the CTA that wrote a source's corners, after its
// column is complete: thread 0 adds w_c b q to each corner node inside the
// column and z chunk, sources in order, with the sparse kernel's operations
// (w_c = wx wy wz, times b, times q, added to the stored value).  The block
// barrier before it makes the column's stores visible to thread 0; no other
// CTA touches these nodes in this launch.  Out of line, with the column
// recomputed from the block index, so that nothing stays live across the
// plane loop for it.
template <int BX, int BY>
__device__ __noinline__ void inject_column(const AcousticStepArgs *a, const AcousticInject *inj,
                                           int zchunk, int nzc) {
    const int n = inj->step + (inj->step_base ? *inj->step_base : 0);
    if (n < 0 || n >= inj->nt) return;
    const int shot = blockIdx.z / nzc;
    const int za = (blockIdx.z - shot * nzc) * zchunk;
    const int zb = min(a->L.nz, za + zchunk);
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int x1 = min(x0 + BX, a->L.nx), y1 = min(y0 + BY, a->L.ny);
    float *u = a->wave + (int64_t)(shot * a->lps + a->lev_out) * a->L.vol;
    for (int s = 0; s < inj->nsrc; ++s) {
        const SparsePoint p = inj->src_tab[shot * inj->nsrc + s];
        const int i = (int)(p.base % (uint32_t)a->L.nxp);
        const int j = (int)((p.base / (uint32_t)a->L.nxp) % (uint32_t)a->L.ny);
        const int k = (int)(p.base / (uint32_t)a->L.plane);
        if (i + 1 < x0 || i >= x1 || j + 1 < y0 || j >= y1 || k + 1 < za || k >= zb) continue;
        const float q = inj->src_wav[((int64_t)shot * inj->nt + n) * inj->nsrc + s];
        for (int c = 0; c < 8; ++c) {
            const int ci = i + (c & 1), cj = j + ((c >> 1) & 1), ck = k + ((c >> 2) & 1);
            if (ci < x0 || ci >= x1 || cj < y0 || cj >= y1 || ck < za || ck >= zb) continue;
            const float wx = (c & 1) ? p.fx : __fsub_rn(1.f, p.fx);
            const float wy = (c & 2) ? p.fy : __fsub_rn(1.f, p.fy);
            const float wz = (c & 4) ? p.fz : __fsub_rn(1.f, p.fz);
            const int64_t off = (int64_t)ck * a->L.plane + (int64_t)cj * a->L.nxp + ci;
            const float val =
                __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(wx, wy), wz), a->bcoef[off]), q);
            u[off] = __fadd_rn(u[off], val);
        }
    }
}

// U: unroll factor of the plane loop.  The pending-output registers shift by
// one plane per iteration; unrolling by U turns U - 1 of every U shifts into
// register renaming instead of moves (U = 2R removes them all).
// WL: the pipeline waits take their limit from the arguments (the
// failure-injection setting of fd_set_wait_limit_ns); otherwise it is the
// constant 2 s, which keeps the limit out of the plane loop's registers (a
// limit read at run time cost 13 % at so 8).
template <int R, int TX, int TY, int VY, int D, int U, bool DF, int MINB = 0, bool WL = false>
__global__ void __launch_bounds__(TX *TY, MINB)
    acoustic_step_kernel(const __grid_constant__ CUtensorMap map_halo,
                         const __grid_constant__ CUtensorMap map_int,
                         const __grid_constant__ CUtensorMap map_b,
                         const __grid_constant__ AcousticStepArgs a,
                         const __grid_constant__ AcousticInject inj, int zchunk, int nzc) {
    using C = AcCfg<R, TX, TY, VY, D, DF>;
    // the divergence watchdog stopped the run: nothing more to compute
    if (__ldcg(a.err) & DEV_ERR_NONFINITE) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *smem = reinterpret_cast<float *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::NSL * C::STAGE);
    uint64_t *empty = full + C::NSL;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + C::NSL);
    float *sdz = reinterpret_cast<float *>(empty + C::NSL + 2);  // damp_z / dt of this chunk

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int tx = tid % TX, ty = tid / TX;
    const int shot_i = blockIdx.z / nzc;
    const int chunk = blockIdx.z - shot_i * nzc;
    const int shot = a.slot_map ? a.slot_map[shot_i] : shot_i;
    const int x0 = blockIdx.x * C::BX, y0 = blockIdx.y * C::BY;
    const int za = chunk * zchunk;
    const int zb = min(a.L.nz, za + zchunk);
    const int nplanes = zb - za + 2 * R;  // arriving planes za-R .. zb+R-1
    const int wcur = shot * a.lps + a.lev_cur, wprev = shot * a.lps + a.lev_prev;
    const int wout = shot * a.lps + a.lev_out;
    const int gx = x0 + 4 * tx;
    const uint64_t wait_ns = WL ? (a.wait_ns ? a.wait_ns : 2000000000ull) : 2000000000ull;

    if (tid == 0) {
        prefetch_tensormap(&map_halo);
        prefetch_tensormap(&map_int);
        prefetch_tensormap(&map_b);
        for (int s = 0; s < C::NSL; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], C::WARPS);
        }
        fence_mbar_init();
        *abort_flag = 0;
    }
    for (int z = za + tid; z < zb; z += C::THREADS) sdz[z - za] = a.dpz[z];
    __syncthreads();

    // Producer (thread 0): stage for iteration jj = halo plane za-R+jj, plus
    // the interior tiles of output plane za-2R+jj once jj >= 2R.
    int issued = 0;
    auto issue = [&](int jj) -> bool {
        const int slot = jj % C::NSL;
        if (jj >= C::NSL &&
            !mbar_wait_bounded(&empty[slot], (uint32_t)(((jj - C::NSL) / C::NSL) & 1), wait_ns))
            return false;
        const bool with_out = jj >= 2 * R;
        mbar_arrive_expect_tx(&full[slot],
                              C::HALO_BYTES + (with_out ? C::NINT * C::INT_BYTES : 0));
        float *st = smem + slot * C::STAGE;
        tma_load_4d(st, &map_halo, &full[slot], x0 - C::RA, y0 - R, za - R + jj, wcur);
        if (with_out) {
            const int zo = za - 2 * R + jj;
            tma_load_4d(st + C::HALO, &map_int, &full[slot], x0, y0, zo, wcur);
            tma_load_4d(st + C::HALO + C::INT, &map_int, &full[slot], x0, y0, zo, wprev);
            tma_load_4d(st + C::HALO + 2 * C::INT, &map_b, &full[slot], x0, y0, zo, 0);
            if (DF) tma_load_4d(st + C::HALO + 3 * C::INT, &map_b, &full[slot], x0, y0, zo, 1);
        }
        issued = jj + 1;
        return true;
    };
    if (tid == 0)
        for (int jj = 0; jj < D && jj < nplanes; ++jj) issue(jj);

    const bool xok = gx < a.L.nxp;
    float dpx4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) dpx4[i] = (gx + i < a.L.nx) ? a.dpx[gx + i] : 0.f;
    const f2 dpx_lo = f2_pack(dpx4[0], dpx4[1]), dpx_hi = f2_pack(dpx4[2], dpx4[3]);
    int gy[VY];
    bool yok[VY];
    float dpyv[VY];
#pragma unroll
    for (int v = 0; v < VY; ++v) {
        gy[v] = y0 + ty * VY + v;
        yok[v] = gy[v] < a.L.ny;
        dpyv[v] = yok[v] ? a.dpy[gy[v]] : 0.f;
    }
    float *__restrict__ unew = a.wave + (int64_t)wout * a.L.vol;
    const f2 one2 = f2_splat(1.f);

    // acc[i][v]: pending output plane p - R + i (p = arriving plane)
    Q4 acc[2 * R][VY];
#pragma unroll
    for (int i = 0; i < 2 * R; ++i)
#pragma unroll
        for (int v = 0; v < VY; ++v) acc[i][v] = Q4{0ull, 0ull};

    bool failed = false;
#pragma unroll U
    for (int j = 0; j < nplanes; ++j) {
        if (tid == 0 && j + D < nplanes && !failed) {
            if (!issue(j + D)) {
                failed = true;
                *abort_flag = 1;
                atomicOr(a.err, DEV_ERR_TIMEOUT);
            }
        }
        const int slot = j % C::NSL;
        if (*abort_flag || !mbar_wait_bounded(&full[slot], (uint32_t)((j / C::NSL) & 1), wait_ns)) {
            *abort_flag = 1;
            atomicOr(a.err, DEV_ERR_TIMEOUT);
            break;
        }
        const float *H = smem + slot * C::STAGE;
        const int rbase = R + ty * VY;

        // x/y part of the Laplacian of plane p (centre weight of all axes
        // included) and the centre values
        Q4 cen[VY], lxy[VY];
#pragma unroll
        for (int v = 0; v < VY; ++v) {
            constexpr int NP = (2 * C::RA + 4) / 2;  // packed pairs in the x span
            f2 xp[NP];
            const float *row = H + (rbase + v) * C::PW + 4 * tx;
#pragma unroll
            for (int t = 0; t < NP / 2; ++t) {
                const Q4 q = lds_q4(row + 4 * t);
                xp[2 * t] = q.lo;
                xp[2 * t + 1] = q.hi;
            }
            constexpr int c0 = C::RA / 2;  // pair index of points 0,1
            const Q4 c = Q4{xp[c0], xp[c0 + 1]};
            const f2 wc2 = f2_splat(a.wc);
            Q4 s = Q4{f2_mul(wc2, c.lo), f2_mul(wc2, c.hi)};
            // even shifts keep the pair alignment: packed arithmetic
#pragma unroll
            for (int k = 2; k <= R; k += 2) {
                const f2 w2 = f2_splat(a.wx[k]);
                s.lo = f2_fma(w2, f2_add(xp[c0 + k / 2], xp[c0 - k / 2]), s.lo);
                s.hi = f2_fma(w2, f2_add(xp[c0 + 1 + k / 2], xp[c0 + 1 - k / 2]), s.hi);
            }
            // odd shifts straddle the pairs: scalar arithmetic
            float o0 = 0.f, o1 = 0.f, o2 = 0.f, o3 = 0.f;
#pragma unroll
            for (int k = 1; k <= R; k += 2) {
                auto el = [&](int idx) -> float {
                    return (idx & 1) ? f2_hi(xp[idx >> 1]) : f2_lo(xp[idx >> 1]);
                };
                const float w = a.wx[k];
                o0 = fmaf(w, el(C::RA + 0 + k) + el(C::RA + 0 - k), o0);
                o1 = fmaf(w, el(C::RA + 1 + k) + el(C::RA + 1 - k), o1);
                o2 = fmaf(w, el(C::RA + 2 + k) + el(C::RA + 2 - k), o2);
                o3 = fmaf(w, el(C::RA + 3 + k) + el(C::RA + 3 - k), o3);
            }
            s.lo = f2_add(s.lo, f2_pack(o0, o1));
            s.hi = f2_add(s.hi, f2_pack(o2, o3));
            cen[v] = c;
            lxy[v] = s;
        }
#pragma unroll
        for (int dy = -R; dy < VY + R; ++dy) {
            bool needed = false;
#pragma unroll
            for (int v = 0; v < VY; ++v) {
                const int k = dy > v ? dy - v : v - dy;
                if (k >= 1 && k <= R) needed = true;
            }
            if (!needed) continue;
            const Q4 f = lds_q4(H + (rbase + dy) * C::PW + C::RA + 4 * tx);
#pragma unroll
            for (int v = 0; v < VY; ++v) {
                const int k = dy > v ? dy - v : v - dy;
                if (k >= 1 && k <= R) {
                    const f2 w2 = f2_splat(a.wy[k]);
                    lxy[v].lo = f2_fma(w2, f.lo, lxy[v].lo);
                    lxy[v].hi = f2_fma(w2, f.hi, lxy[v].hi);
                }
            }
        }

        // z part: plane p feeds the pending outputs p-R .. p+R-1 and starts p+R
#pragma unroll
        for (int v = 0; v < VY; ++v) {
            const Q4 c = cen[v];
#pragma unroll
            for (int i = 0; i < 2 * R; ++i) {
                if (i == R) {
                    acc[i][v].lo = f2_add(acc[i][v].lo, lxy[v].lo);
                    acc[i][v].hi = f2_add(acc[i][v].hi, lxy[v].hi);
                } else {
                    const f2 w2 = f2_splat(a.wz[i < R ? R - i : i - R]);
                    acc[i][v].lo = f2_fma(w2, c.lo, acc[i][v].lo);
                    acc[i][v].hi = f2_fma(w2, c.hi, acc[i][v].hi);
                }
            }
        }

        // output plane zo = p - R is complete:
        //   u+ = u + (1 - zeta)(u - u-) + b * acc,  zeta = (dx + dy + dz) b
        if (j >= 2 * R) {
            const int zo = za - 2 * R + j;
            const float dz = sdz[zo - za];
            const float *Ui = H + C::HALO;
            const float *Pi = Ui + C::INT;
            const float *Bi = Pi + C::INT;
#pragma unroll
            for (int v = 0; v < VY; ++v) {
                if (!(xok && yok[v])) continue;
                const int q = (ty * VY + v) * C::BX + 4 * tx;
                const Q4 c = lds_q4(Ui + q);
                const Q4 p = lds_q4(Pi + q);
                const Q4 b = lds_q4(Bi + q);
                const Q4 s = acc[0][v];
                f2 zl, zh;
                if constexpr (DF) {
                    const Q4 zt = lds_q4(Bi + C::INT + q);
                    zl = zt.lo;
                    zh = zt.hi;
                } else {
                    const f2 dyz = f2_splat(dpyv[v] + dz);
                    zl = f2_mul(f2_add(dpx_lo, dyz), b.lo);
                    zh = f2_mul(f2_add(dpx_hi, dyz), b.hi);
                }
                f2 ol = f2_fma(f2_sub(one2, zl), f2_sub(c.lo, p.lo), c.lo);
                f2 oh = f2_fma(f2_sub(one2, zh), f2_sub(c.hi, p.hi), c.hi);
                ol = f2_fma(b.lo, s.lo, ol);
                oh = f2_fma(b.hi, s.hi, oh);
                const int64_t off = (int64_t)zo * a.L.plane + (int64_t)gy[v] * a.L.nxp + gx;
                *reinterpret_cast<ulonglong2 *>(unew + off) = make_ulonglong2(ol, oh);
            }
        }
        // every thread is done with the stage: release it
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);

        // rotate the pending outputs; plane p + R starts with w_R u(p)
        const f2 wR2 = f2_splat(a.wz[R]);
#pragma unroll
        for (int v = 0; v < VY; ++v) {
#pragma unroll
            for (int i = 0; i < 2 * R - 1; ++i) acc[i][v] = acc[i + 1][v];
            acc[2 * R - 1][v] = Q4{f2_mul(wR2, cen[v].lo), f2_mul(wR2, cen[v].hi)};
        }
    }
    __syncthreads();
    if (*abort_flag && tid == 0) {
        // The last NSL issued stages may still be in flight: give them a
        // bounded chance to land before the CTA's shared memory is released.
        for (int jj = issued - C::NSL; jj < issued; ++jj)
            if (jj >= 0)
                mbar_wait_bounded(&full[jj % C::NSL], (uint32_t)((jj / C::NSL) & 1), 200000000ull);
    }
    if (inj.nsrc > 0 && tid == 0 && !*abort_flag)
        inject_column<C::BX, C::BY>(&a, &inj, zchunk, nzc);
}

struct ConfigEntry {
    int radius, tx, ty, vy, d;
    const void *fn;
    size_t smem;
    int bx, by, pw, ph, threads;
    const char *name;
};

template <int R, int TX, int TY, int VY, int D, int U, bool DF = false, int MINB = 0,
          bool WL = false>
ConfigEntry make_entry(const char *name) {
    using C = AcCfg<R, TX, TY, VY, D, DF>;
    return ConfigEntry{R,       TX,    TY,    VY,    D,
                       (const void *)&acoustic_step_kernel<R, TX, TY, VY, D, U, DF, MINB, WL>,
                       C::SMEM, C::BX, C::BY, C::PW, C::PH, C::THREADS, name};
}

#define FD_AC_ENTRY(R, TX, TY, VY, D, U)                                           \
    make_entry<R, TX, TY, VY, D, U>("acoustic_step<" #R "," #TX "," #TY "," #VY "," #D \
                                    "," #U ">")
#define FD_AC_ENTRY_DF(R, TX, TY, VY, D, U, MB)                                              \
    make_entry<R, TX, TY, VY, D, U, true, MB>("acoustic_step<" #R "," #TX "," #TY "," #VY "," #D \
                                              "," #U ",damp field>")

#define FD_AC_ENTRY_WL(R, TX, TY, VY, D, U)                                                 \
    make_entry<R, TX, TY, VY, D, U, false, 0, true>("acoustic_step<" #R "," #TX "," #TY "," #VY \
                                                    "," #D "," #U ",wait limit>")

// The default configuration of each radius with the wait limit taken from the
// arguments: launched instead of it while fd_set_wait_limit_ns is set.
const ConfigEntry *config_table_wl(int radius) {
    static const ConfigEntry r1 = FD_AC_ENTRY_WL(1, 16, 16, 1, 4, 1);
    static const ConfigEntry r2 = FD_AC_ENTRY_WL(2, 16, 16, 1, 4, 4);
    static const ConfigEntry r4 = FD_AC_ENTRY_WL(4, 16, 8, 1, 4, 4);
    static const ConfigEntry r6 = FD_AC_ENTRY_WL(6, 16, 8, 1, 3, 4);
    static const ConfigEntry r8 = FD_AC_ENTRY_WL(8, 16, 4, 1, 1, 4);
    switch (radius) {
        case 1: return &r1;
        case 2: return &r2;
        case 4: return &r4;
        case 6: return &r6;
        case 8: return &r8;
        default: return nullptr;
    }
}

// 3-D damping field: one configuration per radius, the default one's tiles,
// with the prefetch depth and register bound chosen so that a 512^3 launch
// still fits in one wave despite the fourth interior tile per stage (four
// 128-thread or eight 64-thread CTAs per SM; with three 128-thread CTAs the
// 512 columns need two waves: so 8 and 12 at 0.6 of the copy bandwidth).
const ConfigEntry *config_table_df(int radius) {
    static const ConfigEntry r1 = FD_AC_ENTRY_DF(1, 16, 16, 1, 4, 1, 0);
    static const ConfigEntry r2 = FD_AC_ENTRY_DF(2, 16, 16, 1, 4, 4, 0);
    static const ConfigEntry r4 = FD_AC_ENTRY_DF(4, 16, 8, 1, 3, 4, 0);
    static const ConfigEntry r6 = FD_AC_ENTRY_DF(6, 16, 8, 1, 2, 4, 4);
    static const ConfigEntry r8 = FD_AC_ENTRY_DF(8, 16, 4, 1, 1, 4, 8);
    switch (radius) {
        case 1: return &r1;
        case 2: return &r2;
        case 4: return &r4;
        case 6: return &r6;
        case 8: return &r8;
        default: return nullptr;
    }
}

const ConfigEntry *config_table(int radius, int *count) {
    // Index 0 is the default; the others are kept for tuning sweeps
    // (fd_set_acoustic_config).  Defaults measured on GB300 at 512^3 (template
    // arguments R, TX, TY, VY, D, U): the plane-loop unroll U = 4 helps at every
    // radius; a deeper prefetch suits R = 4 (D = 4, +10 %), a shallower one
    // R = 8 (D = 1: more CTAs per SM), where 64 x 4 tiles of 64 threads (1024
    // columns in two z chunks) beat 64 x 8 tiles by 4 % (281 against 269
    // GPts/s; 32 x 8 tiles of 64 threads measured the same as 64 x 4).
    static const ConfigEntry r1[] = {FD_AC_ENTRY(1, 16, 16, 1, 4, 1)};
    static const ConfigEntry r2[] = {
        FD_AC_ENTRY(2, 16, 16, 1, 4, 4), FD_AC_ENTRY(2, 16, 16, 1, 4, 1),
        FD_AC_ENTRY(2, 16, 8, 1, 6, 1),  FD_AC_ENTRY(2, 16, 8, 2, 4, 1),
        FD_AC_ENTRY(2, 16, 16, 1, 4, 2), FD_AC_ENTRY(2, 16, 16, 1, 3, 4),
        FD_AC_ENTRY(2, 16, 16, 1, 5, 4), FD_AC_ENTRY(2, 16, 8, 1, 6, 4)};
    static const ConfigEntry r4[] = {
        FD_AC_ENTRY(4, 16, 8, 1, 4, 4),  FD_AC_ENTRY(4, 16, 8, 1, 3, 1),
        FD_AC_ENTRY(4, 16, 16, 1, 4, 1), FD_AC_ENTRY(4, 16, 8, 2, 3, 1),
        FD_AC_ENTRY(4, 16, 8, 1, 3, 4),  FD_AC_ENTRY(4, 16, 16, 1, 3, 4),
        FD_AC_ENTRY(4, 16, 8, 1, 5, 4),  FD_AC_ENTRY(4, 16, 8, 1, 6, 4),
        FD_AC_ENTRY(4, 16, 8, 1, 4, 2),  FD_AC_ENTRY(4, 16, 8, 1, 4, 8)};
    static const ConfigEntry r6[] = {
        FD_AC_ENTRY(6, 16, 8, 1, 3, 4),  FD_AC_ENTRY(6, 16, 8, 1, 2, 4),
        FD_AC_ENTRY(6, 16, 16, 1, 3, 1), FD_AC_ENTRY(6, 8, 16, 1, 3, 1),
        FD_AC_ENTRY(6, 16, 8, 1, 2, 1),  FD_AC_ENTRY(6, 16, 8, 1, 3, 2),
        FD_AC_ENTRY(6, 16, 8, 1, 4, 4),  FD_AC_ENTRY(6, 16, 8, 1, 1, 4)};
    static const ConfigEntry r8[] = {
        FD_AC_ENTRY(8, 16, 4, 1, 1, 4),  FD_AC_ENTRY(8, 16, 8, 1, 1, 4),
        FD_AC_ENTRY(8, 16, 8, 1, 2, 1),
        FD_AC_ENTRY(8, 16, 16, 1, 3, 1), FD_AC_ENTRY(8, 8, 16, 1, 3, 1),
        FD_AC_ENTRY(8, 16, 8, 1, 2, 4),  FD_AC_ENTRY(8, 16, 8, 1, 1, 2),
        FD_AC_ENTRY(8, 8, 16, 1, 1, 4),  FD_AC_ENTRY(8, 16, 8, 1, 1, 8)};
    switch (radius) {
        case 1: *count = 1; return r1;
        case 2: *count = 8; return r2;
        case 4: *count = 10; return r4;
        case 6: *count = 8; return r6;
        case 8: *count = 9; return r8;
        default: *count = 0; return nullptr;
    }
}

}  // namespace

int acoustic_num_configs(int radius) {
    int n = 0;
    config_table(radius, &n);
    return n;
}

int acoustic_default_config(int radius) {
    (void)radius;
    return 0;
}

fd_status acoustic_plan(int radius, int config, const WaveLayout &L, int nshots, int lps,
                        float *wave, const float *bcoef, AcousticPlan *plan, int map_shots,
                        bool damp_field) {
    if (map_shots < nshots) map_shots = nshots;
    int n = 0;
    const ConfigEntry *tab = config_table(radius, &n);
    if (!tab) return set_error(FD_ERR_SO, "no acoustic kernel for radius %d", radius);
    if (config < 0 || config >= n || damp_field) config = acoustic_default_config(radius);
    const ConfigEntry &e = damp_field ? *config_table_df(radius) : tab[config];
    plan->radius = radius;
    plan->config = config;
    plan->damp_field = damp_field;
    plan->name = e.name;
    plan->smem = e.smem;
    plan->block = dim3(e.threads, 1, 1);
    FD_TRY(raise_smem_limit(e.fn, e.smem));
    int dev = 0, nsm = 0, per_sm = 0;
    FD_CUDA_TRY(cudaGetDevice(&dev));
    FD_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, e.fn, e.threads, e.smem));
    if (per_sm < 1) return set_error(FD_ERR_CUDA, "kernel %s does not fit on an SM", e.name);
    const int ntx = (L.nx + e.bx - 1) / e.bx;
    const int nty = (L.ny + e.by - 1) / e.by;
    const int64_t cols = (int64_t)ntx * nty * nshots;
    const int64_t slots = (int64_t)nsm * per_sm;
    // Split z only when the columns alone cannot fill the machine; keep every
    // chunk long enough that the 2R-plane warm-up stays a small fraction.
    // The narrow stencils (R <= 2) run at the HBM limit once three quarters
    // of the slots are busy, so there a split only adds warm-up planes
    // (512^3, so 4: 413 GPts/s unsplit, 396 in two chunks); the wider ones
    // are limited per SM and gain from the finer units (so 8: 381 in two
    // chunks, 357 unsplit).
    int nzc = 1;
    if (cols < slots && !(radius <= 2 && 4 * cols >= 3 * slots)) {
        nzc = (int)((slots + cols - 1) / cols);
        const int min_chunk = 8 * radius > 32 ? 8 * radius : 32;
        const int max_nzc = L.nz / min_chunk > 1 ? L.nz / min_chunk : 1;
        if (nzc > max_nzc) nzc = max_nzc;
    }
    const int zchunk = (L.nz + nzc - 1) / nzc;
    nzc = (L.nz + zchunk - 1) / zchunk;
    if ((int64_t)nshots * nzc > 65535 || nty > 65535)
        return set_error(FD_ERR_ARG, "grid too large for the launch configuration");
    plan->grid = dim3(ntx, nty, nshots * nzc);
    plan->zchunk = zchunk;
    plan->nzc = nzc;
    plan->smem = e.smem + (size_t)zchunk * 4;
    FD_TRY(raise_smem_limit(e.fn, plan->smem));
    if (!damp_field && config == acoustic_default_config(radius))
        FD_TRY(raise_smem_limit(config_table_wl(radius)->fn, plan->smem));
    FD_TRY(make_tensor_map_4d(&plan->map_halo, wave, L.nx, L.ny, L.nz, (uint64_t)map_shots * lps,
                              (uint64_t)L.nxp * 4, (uint64_t)L.plane * 4, (uint64_t)L.vol * 4,
                              e.pw, e.ph, 1, 1));
    FD_TRY(make_tensor_map_4d(&plan->map_int, wave, L.nx, L.ny, L.nz, (uint64_t)map_shots * lps,
                              (uint64_t)L.nxp * 4, (uint64_t)L.plane * 4, (uint64_t)L.vol * 4,
                              e.bx, e.by, 1, 1));
    return make_tensor_map_4d(&plan->map_b, bcoef, L.nx, L.ny, L.nz, damp_field ? 2 : 1,
                              (uint64_t)L.nxp * 4, (uint64_t)L.plane * 4, (uint64_t)L.vol * 4,
                              e.bx, e.by, 1, 1);
}

fd_status acoustic_launch(const AcousticPlan &plan, const AcousticStepArgs &args,
                          cudaStream_t stream, const AcousticInject *inject) {
    int n = 0;
    const ConfigEntry *tab = config_table(plan.radius, &n);
    if (!tab || plan.config >= n) return set_error(FD_ERR_SO, "bad acoustic plan");
    AcousticInject inj;
    memset(&inj, 0, sizeof(inj));
    if (inject && inject->nsrc > 0) {
        if (inject->nsrc > kInjectMaxSources || args.slot_map)
            return set_error(FD_ERR_ARG, "in-kernel injection: at most %d sources, no slot map",
                             kInjectMaxSources);
        inj = *inject;
    }
    int zchunk = plan.zchunk, nzc = plan.nzc;
    AcousticStepArgs a = args;
    if (!a.wait_ns) a.wait_ns = wait_limit_ns();
    void *params[] = {(void *)&plan.map_halo, (void *)&plan.map_int, (void *)&plan.map_b,
                      (void *)&a, (void *)&inj, (void *)&zchunk, (void *)&nzc};
    const void *fn = tab[plan.config].fn;
    if (plan.damp_field)
        fn = config_table_df(plan.radius)->fn;
    else if (a.wait_ns != 0 && plan.config == acoustic_default_config(plan.radius))
        fn = config_table_wl(plan.radius)->fn;  // same tiles, ring and shared memory
    FD_CUDA_TRY(cudaLaunchKernel(fn, plan.grid, plan.block, params, plan.smem, stream));
    note_launch(stream);
    return FD_OK;
}

}  // namespace fdsweep
