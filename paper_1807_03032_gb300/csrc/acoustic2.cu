// acoustic2.cu -- time tiling of the acoustic step: two leapfrog steps of the
// damped isotropic wave equation (Eq. WE; Listing fd-3, as in acoustic.cu) per
// launch, the loop blocking across the time dimension that the paper names as
// further work.
//
// One CTA owns a BX x BY column and marches it through z, like K1, but keeps
// the intermediate level u^{n+1} on chip:
//   step 1  computes u^{n+1} on the tile extended by RA columns and R rows on
//           every side (overlapped tiling: the extension is recomputed by the
//           neighbouring CTAs too), from u^n staged with a 2RA x 2R halo;
//   step 2  computes u^{n+2} on the tile from the u^{n+1} planes in shared
//           memory, R planes behind step 1.
// Both steps use K1's z-accumulator pipeline (2R pending outputs per point in
// registers) and the same packed-FP32 arithmetic in the same order, so the
// results are bit-identical to two K1 launches.  Outside the grid b is zero
// (TMA zero fill), which makes the extended u^{n+1} vanish there: the zero
// ghosts of the Dirichlet boundary come for free.  src[n] is injected into
// u^{n+1} in shared memory (up to kStep2MaxSources sources per shot) before
// step 2 reads it; the caller injects src[n+1] into u^{n+2} and records both
// receiver samples.
//
// HBM traffic per launch: read u^n, u^{n-1}, b; write u^{n+1}, u^{n+2} = 20
// bytes per point for two steps (10 per step, against 16 for K1).  All halo
// and extension re-reads are served by L2.
#include "f32x2.cuh"
#include "kernels.cuh"
#include "runtime.cuh"

namespace fdsweep {
namespace {
using namespace f32x2;

template <int R, int TX, int TY, int D>
struct T2Cfg {
    static constexpr int BX = 4 * TX, BY = TY;
    static constexpr int RA = (R + 3) / 4 * 4;
    static constexpr int EW = BX + 2 * RA, EH = BY + 2 * R;  // u^{n+1} extended tile
    static constexpr int PW = BX + 4 * RA, PH = BY + 4 * R;  // u^n plane with its halo
    static constexpr int NT = TX * TY, WARPS = NT / 32;
    static constexpr int EQ = EW / 4;                        // float4 cells per extended row
    static constexpr int NE = EQ * EH;
    static constexpr int KE = (NE + NT - 1) / NT;            // extended cells per thread
    static constexpr int HALO = (PW * PH + 31) / 32 * 32;
    static constexpr int EXT = (EW * EH + 31) / 32 * 32;
    static constexpr int INT = BX * BY;
    // stage: [u^n plane p + halo][u^n, u^{n-1}, b extended at p-R][u^n, b tile at p-2R]
    static constexpr int STAGE = HALO + 3 * EXT + 2 * INT;
    static constexpr int NSL = D + 1;
    static constexpr int NU1 = R + 2;  // u^{n+1} planes kept (z-stencil + one in flight)
    static constexpr int MAXINJ = 8 * kStep2MaxSources;
    static constexpr uint32_t HALO_BYTES = PW * PH * 4, EXT_BYTES = EW * EH * 4,
                              INT_BYTES = INT * 4;
    static constexpr size_t SMEM = ((size_t)NSL * STAGE + (size_t)NU1 * EXT) * 4 +
                                   (size_t)MAXINJ * 24 + NSL * 16 + 16 + 128;
    static_assert(PW <= 256 && PH <= 256, "TMA box dimension limit");
    static_assert(INT % 32 == 0 && NT % 32 == 0, "tile shape");
};

// x/y part of the compact Laplacian of one float4 cell of a staged plane plus
// the cell's centre values; `row` points RA floats left of the cell, rows are
// `pitch` floats apart.  Same operations, in the same order, as K1 (VY = 1).
template <int R, int RA>
__device__ __forceinline__ void lap_xy_cell(const float *row, int pitch, const AcousticStepArgs &a,
                                            Q4 &cen, Q4 &lxy) {
    constexpr int NP = (2 * RA + 4) / 2;
    f2 xp[NP];
#pragma unroll
    for (int t = 0; t < NP / 2; ++t) {
        const Q4 q = lds_q4(row + 4 * t);
        xp[2 * t] = q.lo;
        xp[2 * t + 1] = q.hi;
    }
    constexpr int c0 = RA / 2;
    const Q4 c = Q4{xp[c0], xp[c0 + 1]};
    const f2 wc2 = f2_splat(a.wc);
    Q4 s = Q4{f2_mul(wc2, c.lo), f2_mul(wc2, c.hi)};
#pragma unroll
    for (int k = 2; k <= R; k += 2) {
        const f2 w2 = f2_splat(a.wx[k]);
        s.lo = f2_fma(w2, f2_add(xp[c0 + k / 2], xp[c0 - k / 2]), s.lo);
        s.hi = f2_fma(w2, f2_add(xp[c0 + 1 + k / 2], xp[c0 + 1 - k / 2]), s.hi);
    }
    float o0 = 0.f, o1 = 0.f, o2 = 0.f, o3 = 0.f;
#pragma unroll
    for (int k = 1; k <= R; k += 2) {
        auto el = [&](int idx) -> float {
            return (idx & 1) ? f2_hi(xp[idx >> 1]) : f2_lo(xp[idx >> 1]);
        };
        const float w = a.wx[k];
        o0 = fmaf(w, el(RA + 0 + k) + el(RA + 0 - k), o0);
        o1 = fmaf(w, el(RA + 1 + k) + el(RA + 1 - k), o1);
        o2 = fmaf(w, el(RA + 2 + k) + el(RA + 2 - k), o2);
        o3 = fmaf(w, el(RA + 3 + k) + el(RA + 3 - k), o3);
    }
    s.lo = f2_add(s.lo, f2_pack(o0, o1));
    s.hi = f2_add(s.hi, f2_pack(o2, o3));
#pragma unroll
    for (int dy = -R; dy <= R; ++dy) {
        if (dy == 0) continue;
        const int k = dy > 0 ? dy : -dy;
        const Q4 f = lds_q4(row + dy * pitch + RA);
        const f2 w2 = f2_splat(a.wy[k]);
        s.lo = f2_fma(w2, f.lo, s.lo);
        s.hi = f2_fma(w2, f.hi, s.hi);
    }
    cen = c;
    lxy = s;
}

// Plane p (centre values c, x/y part lxy) feeds the pending outputs p-R ..
// p+R-1: acc[R] (output p) takes lxy, the others w_|p-z| c.
template <int R>
__device__ __forceinline__ void z_feed(Q4 (&acc)[2 * R], const Q4 &c, const Q4 &lxy,
                                       const AcousticStepArgs &a) {
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) {
        if (i == R) {
            acc[i].lo = f2_add(acc[i].lo, lxy.lo);
            acc[i].hi = f2_add(acc[i].hi, lxy.hi);
        } else {
            const f2 w2 = f2_splat(a.wz[i < R ? R - i : i - R]);
            acc[i].lo = f2_fma(w2, c.lo, acc[i].lo);
            acc[i].hi = f2_fma(w2, c.hi, acc[i].hi);
        }
    }
}
template <int R>
__device__ __forceinline__ void z_rotate(Q4 (&acc)[2 * R], const Q4 &c, const AcousticStepArgs &a) {
    const f2 wR2 = f2_splat(a.wz[R]);
#pragma unroll
    for (int i = 0; i < 2 * R - 1; ++i) acc[i] = acc[i + 1];
    acc[2 * R - 1] = Q4{f2_mul(wR2, c.lo), f2_mul(wR2, c.hi)};
}

// u+ = u + (1 - zeta)(u - u-) + b * lap, zeta = (dx + (dy + dz)) b
__device__ __forceinline__ Q4 leapfrog(const Q4 &c, const Q4 &p, const Q4 &b, const Q4 &s,
                                       f2 dpx_lo, f2 dpx_hi, float dyz) {
    const f2 one2 = f2_splat(1.f);
    const f2 d2 = f2_splat(dyz);
    const f2 zl = f2_mul(f2_add(dpx_lo, d2), b.lo);
    const f2 zh = f2_mul(f2_add(dpx_hi, d2), b.hi);
    f2 ol = f2_fma(f2_sub(one2, zl), f2_sub(c.lo, p.lo), c.lo);
    f2 oh = f2_fma(f2_sub(one2, zh), f2_sub(c.hi, p.hi), c.hi);
    ol = f2_fma(b.lo, s.lo, ol);
    oh = f2_fma(b.hi, s.hi, oh);
    return Q4{ol, oh};
}

__device__ __forceinline__ float dp_or_zero(const float *d, int i, int n) {
    return (i >= 0 && i < n) ? __ldg(d + i) : 0.f;
}

template <int R, int TX, int TY, int D, int U>
__global__ void __launch_bounds__(TX *TY)
    acoustic_step2_kernel(const __grid_constant__ CUtensorMap map_halo,
                          const __grid_constant__ CUtensorMap map_ext,
                          const __grid_constant__ CUtensorMap map_int,
                          const __grid_constant__ CUtensorMap map_bext,
                          const __grid_constant__ CUtensorMap map_bint,
                          const AcousticStep2Args a2, int zchunk, int nzc) {
    using C = T2Cfg<R, TX, TY, D>;
    const AcousticStepArgs &a = a2.s;
    if (__ldcg(a.err) & DEV_ERR_NONFINITE) return;  // stopped by the divergence watchdog
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *smem = reinterpret_cast<float *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    float *u1ring = smem + C::NSL * C::STAGE;                      // [NU1][EXT]
    int4 *inj_pos = reinterpret_cast<int4 *>(u1ring + C::NU1 * C::EXT);  // x, y, z, -
    float2 *inj_wq = reinterpret_cast<float2 *>(inj_pos + C::MAXINJ);   // weight, sample
    uint64_t *full = reinterpret_cast<uint64_t *>(inj_wq + C::MAXINJ);
    uint64_t *empty = full + C::NSL;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + C::NSL);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int shot = blockIdx.z / nzc;
    const int chunk = blockIdx.z - shot * nzc;
    const int x0 = blockIdx.x * C::BX, y0 = blockIdx.y * C::BY;
    const int za = chunk * zchunk;
    const int zb = min(a.L.nz, za + zchunk);
    const int nplanes = zb - za + 4 * R;  // u^n planes za-2R .. zb+2R-1
    const int wcur = shot * a.lps + a.lev_cur, wprev = shot * a.lps + a.lev_prev;

    // injection of src[n] into u^{n+1}: the 8 corners of every source of the shot
    const int n_time = 2 * (a2.step + (a2.step_base ? *a2.step_base : 0));
    const int ninj = (a2.src_tab && n_time < a2.nt) ? 8 * a2.nsrc : 0;
    if (tid < ninj) {
        const int isrc = tid >> 3, c = tid & 7;
        const SparsePoint sp = a2.src_tab[(int64_t)shot * a2.nsrc + isrc];
        const int64_t base = sp.base;
        const int z = (int)(base / a.L.plane);
        const int64_t rem = base - (int64_t)z * a.L.plane;
        const int y = (int)(rem / a.L.nxp);
        const int x = (int)(rem - (int64_t)y * a.L.nxp);
        const float wx = (c & 1) ? sp.fx : 1.f - sp.fx;
        const float wy = (c & 2) ? sp.fy : 1.f - sp.fy;
        const float wz = (c & 4) ? sp.fz : 1.f - sp.fz;
        inj_pos[tid] = make_int4(x + (c & 1), y + ((c >> 1) & 1), z + ((c >> 2) & 1), 0);
        inj_wq[tid] = make_float2(wx * wy * wz,
                                  a2.src_wav[((int64_t)shot * a2.nt + n_time) * a2.nsrc + isrc]);
    }
    if (tid == 0) {
        prefetch_tensormap(&map_halo);
        prefetch_tensormap(&map_ext);
        prefetch_tensormap(&map_int);
        prefetch_tensormap(&map_bext);
        prefetch_tensormap(&map_bint);
        for (int s = 0; s < C::NSL; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], C::WARPS);
        }
        fence_mbar_init();
        *abort_flag = 0;
    }
    __syncthreads();

    // Producer (thread 0): stage jj = u^n plane p = za-2R+jj with its halo;
    // from jj >= 2R the extended u^n, u^{n-1}, b at p-R (step-1 output); from
    // jj >= 4R the u^n and b tiles at p-2R (step-2 output).
    int issued = 0;
    auto issue = [&](int jj) -> bool {
        const int slot = jj % C::NSL;
        if (jj >= C::NSL &&
            !mbar_wait_bounded(&empty[slot], (uint32_t)(((jj - C::NSL) / C::NSL) & 1)))
            return false;
        const bool o1 = jj >= 2 * R, o2 = jj >= 4 * R;
        mbar_arrive_expect_tx(&full[slot], C::HALO_BYTES + (o1 ? 3 * C::EXT_BYTES : 0) +
                                               (o2 ? 2 * C::INT_BYTES : 0));
        float *st = smem + slot * C::STAGE;
        const int p = za - 2 * R + jj;
        tma_load_4d(st, &map_halo, &full[slot], x0 - 2 * C::RA, y0 - 2 * R, p, wcur);
        if (o1) {
            float *e = st + C::HALO;
            tma_load_4d(e, &map_ext, &full[slot], x0 - C::RA, y0 - R, p - R, wcur);
            tma_load_4d(e + C::EXT, &map_ext, &full[slot], x0 - C::RA, y0 - R, p - R, wprev);
            tma_load_4d(e + 2 * C::EXT, &map_bext, &full[slot], x0 - C::RA, y0 - R, p - R, 0);
        }
        if (o2) {
            float *t = st + C::HALO + 3 * C::EXT;
            tma_load_4d(t, &map_int, &full[slot], x0, y0, p - 2 * R, wcur);
            tma_load_4d(t + C::INT, &map_bint, &full[slot], x0, y0, p - 2 * R, 0);
        }
        issued = jj + 1;
        return true;
    };
    if (tid == 0)
        for (int jj = 0; jj < D && jj < nplanes; ++jj) issue(jj);

    // step-1 cells: extended float4 cells tid, tid + NT, ...; ecell is the
    // cell's offset in an extended tile, hcell the offset of its x span
    // (RA left of the cell) in the staged u^n plane
    int ecell[C::KE], hcell[C::KE];
    bool evalid[C::KE];
    f2 edpx_lo[C::KE], edpx_hi[C::KE];
    float edpy[C::KE];
#pragma unroll
    for (int k = 0; k < C::KE; ++k) {
        const int c = tid + k * C::NT;
        evalid[k] = c < C::NE;
        const int ey = evalid[k] ? c / C::EQ : 0, eq = evalid[k] ? c % C::EQ : 0;
        ecell[k] = ey * C::EW + 4 * eq;
        hcell[k] = (ey + R) * C::PW + 4 * eq;
        const int gx = x0 - C::RA + 4 * eq, gy = y0 - R + ey;
        edpx_lo[k] = f2_pack(dp_or_zero(a.dpx, gx, a.L.nx), dp_or_zero(a.dpx, gx + 1, a.L.nx));
        edpx_hi[k] = f2_pack(dp_or_zero(a.dpx, gx + 2, a.L.nx), dp_or_zero(a.dpx, gx + 3, a.L.nx));
        edpy[k] = dp_or_zero(a.dpy, gy, a.L.ny);
    }
    // step-2 cell: interior float4 cell (tx, ty)
    const int tx = tid % TX, ty = tid / TX;
    const int gx = x0 + 4 * tx, gy = y0 + ty;
    const bool ok2 = gx < a.L.nxp && gy < a.L.ny;
    const f2 dpx_lo = f2_pack(dp_or_zero(a.dpx, gx, a.L.nx), dp_or_zero(a.dpx, gx + 1, a.L.nx));
    const f2 dpx_hi =
        f2_pack(dp_or_zero(a.dpx, gx + 2, a.L.nx), dp_or_zero(a.dpx, gx + 3, a.L.nx));
    const float dpy2 = dp_or_zero(a.dpy, gy, a.L.ny);
    float *__restrict__ out1 = a.wave + (int64_t)(shot * a.lps + a.lev_out) * a.L.vol;
    float *__restrict__ out2 = a.wave + (int64_t)(shot * a.lps + a2.lev_out2) * a.L.vol;

    Q4 acc1[C::KE][2 * R], acc2[2 * R];
#pragma unroll
    for (int k = 0; k < C::KE; ++k)
#pragma unroll
        for (int i = 0; i < 2 * R; ++i) acc1[k][i] = Q4{0ull, 0ull};
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) acc2[i] = Q4{0ull, 0ull};

    bool failed = false;
#pragma unroll U
    for (int j = 0; j < nplanes; ++j) {
        bool bad = false;
        if (tid == 0 && j + D < nplanes && !failed && !issue(j + D)) {
            failed = true;
            bad = true;
        }
        const int slot = j % C::NSL;
        if (!mbar_wait_bounded(&full[slot], (uint32_t)((j / C::NSL) & 1))) bad = true;
        const float *st = smem + slot * C::STAGE;
        const float *H = st;
        const int p = za - 2 * R + j;
        const int z1 = p - R, z2 = p - 2 * R;
        const bool o1 = j >= 2 * R, o2 = j >= 4 * R;
        float *U1 = u1ring + ((z1 + C::NU1 * (R + 1)) % C::NU1) * C::EXT;

        // ---- step 1: u^n plane p feeds the extended pending outputs; output
        //      z1 = p - R is complete
        Q4 cen1[C::KE];
#pragma unroll
        for (int k = 0; k < C::KE; ++k) {
            cen1[k] = Q4{0ull, 0ull};
            if (!evalid[k]) continue;
            Q4 lxy;
            lap_xy_cell<R, C::RA>(H + hcell[k], C::PW, a, cen1[k], lxy);
            z_feed<R>(acc1[k], cen1[k], lxy, a);
            if (o1) {
                const float *E = st + C::HALO;
                const Q4 uc = lds_q4(E + ecell[k]);
                const Q4 um = lds_q4(E + C::EXT + ecell[k]);
                const Q4 b = lds_q4(E + 2 * C::EXT + ecell[k]);
                const float dz = dp_or_zero(a.dpz, z1, a.L.nz);
                const Q4 v = leapfrog(uc, um, b, acc1[k][0], edpx_lo[k], edpx_hi[k], edpy[k] + dz);
                *reinterpret_cast<ulonglong2 *>(U1 + ecell[k]) = make_ulonglong2(v.lo, v.hi);
            }
        }
        // every thread: plane z1 of u^{n+1} complete (or abandon uniformly)
        if (__syncthreads_or(bad || *abort_flag)) {
            if (tid == 0) {
                *abort_flag = 1;
                atomicOr(a.err, DEV_ERR_TIMEOUT);
            }
            break;
        }
        if (o1 && ninj > 0) {
            // src[n] into u^{n+1}: corners in plane z1 inside the extended tile
            for (int e = tid; e < ninj; e += C::NT) {
                const int4 q = inj_pos[e];
                const int ex = q.x - (x0 - C::RA), ey = q.y - (y0 - R);
                if (q.z == z1 && ex >= 0 && ex < C::EW && ey >= 0 && ey < C::EH) {
                    const float b = st[C::HALO + 2 * C::EXT + ey * C::EW + ex];
                    const float2 wq = inj_wq[e];
                    atomicAdd(U1 + ey * C::EW + ex, wq.x * b * wq.y);
                }
            }
            __syncthreads();
        }

        // ---- step 2: u^{n+1} plane z1 feeds the pending outputs; output
        //      z2 = z1 - R is complete
        if (o1) {
            Q4 c2, lxy2;
            lap_xy_cell<R, C::RA>(U1 + (R + ty) * C::EW + 4 * tx, C::EW, a, c2, lxy2);
            z_feed<R>(acc2, c2, lxy2, a);
            if (o2 && ok2) {
                const float *U1c = u1ring + ((z2 + C::NU1 * (R + 1)) % C::NU1) * C::EXT;
                const Q4 u1c = lds_q4(U1c + (R + ty) * C::EW + C::RA + 4 * tx);
                const float *T = st + C::HALO + 3 * C::EXT;
                const Q4 un = lds_q4(T + ty * C::BX + 4 * tx);
                const Q4 b = lds_q4(T + C::INT + ty * C::BX + 4 * tx);
                const Q4 v = leapfrog(u1c, un, b, acc2[0], dpx_lo, dpx_hi,
                                      dpy2 + __ldg(a.dpz + z2));
                const int64_t off = (int64_t)z2 * a.L.plane + (int64_t)gy * a.L.nxp + gx;
                *reinterpret_cast<ulonglong2 *>(out1 + off) = make_ulonglong2(u1c.lo, u1c.hi);
                *reinterpret_cast<ulonglong2 *>(out2 + off) = make_ulonglong2(v.lo, v.hi);
            }
            z_rotate<R>(acc2, c2, a);
        }
        // the stage is consumed: release it
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
#pragma unroll
        for (int k = 0; k < C::KE; ++k)
            if (evalid[k]) z_rotate<R>(acc1[k], cen1[k], a);
    }
    __syncthreads();
    if (*abort_flag && tid == 0) {
        for (int jj = issued - C::NSL; jj < issued; ++jj)
            if (jj >= 0)
                mbar_wait_bounded(&full[jj % C::NSL], (uint32_t)((jj / C::NSL) & 1), 200000000ull);
    }
}

struct T2Entry {
    int radius;
    const void *fn;
    size_t smem;
    int bx, by, ew, eh, pw, ph, threads;
    const char *name;
};

template <int R, int TX, int TY, int D, int U>
T2Entry make_t2(const char *name) {
    using C = T2Cfg<R, TX, TY, D>;
    return T2Entry{R,     (const void *)&acoustic_step2_kernel<R, TX, TY, D, U>,
                   C::SMEM, C::BX, C::BY, C::EW, C::EH, C::PW, C::PH, C::NT, name};
}

#define FD_T2_ENTRY(R, TX, TY, D, U) \
    make_t2<R, TX, TY, D, U>("acoustic_step2<" #R "," #TX "," #TY "," #D "," #U ">")

const T2Entry *t2_table(int radius, int *count) {
    // index 0 is the default
    static const T2Entry r2[] = {FD_T2_ENTRY(2, 16, 16, 1, 1), FD_T2_ENTRY(2, 16, 16, 1, 2),
                                 FD_T2_ENTRY(2, 16, 8, 2, 1)};
    static const T2Entry r4[] = {FD_T2_ENTRY(4, 16, 16, 1, 1), FD_T2_ENTRY(4, 16, 8, 1, 1)};
    switch (radius) {
        case 2: *count = 3; return r2;
        case 4: *count = 2; return r4;
        default: *count = 0; return nullptr;
    }
}

}  // namespace

int acoustic2_num_configs(int radius) {
    int n = 0;
    t2_table(radius, &n);
    return n;
}

fd_status acoustic2_plan(int radius, int config, const WaveLayout &L, int nshots, int lps,
                         float *wave, const float *bcoef, Acoustic2Plan *plan) {
    int n = 0;
    const T2Entry *tab = t2_table(radius, &n);
    if (!tab) return set_error(FD_ERR_SO, "no time-tiled kernel for radius %d", radius);
    if (config < 0 || config >= n) config = 0;
    const T2Entry &e = tab[config];
    plan->radius = radius;
    plan->config = config;
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
    int nzc = 1;
    if (cols < slots) {
        nzc = (int)((slots + cols - 1) / cols);
        const int min_chunk = 16 * radius > 32 ? 16 * radius : 32;
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
    const uint64_t nw = (uint64_t)nshots * lps, sy = (uint64_t)L.nxp * 4,
                   sz = (uint64_t)L.plane * 4, sw = (uint64_t)L.vol * 4;
    FD_TRY(make_tensor_map_4d(&plan->map_halo, wave, L.nx, L.ny, L.nz, nw, sy, sz, sw, e.pw, e.ph,
                              1, 1));
    FD_TRY(make_tensor_map_4d(&plan->map_ext, wave, L.nx, L.ny, L.nz, nw, sy, sz, sw, e.ew, e.eh,
                              1, 1));
    FD_TRY(make_tensor_map_4d(&plan->map_int, wave, L.nx, L.ny, L.nz, nw, sy, sz, sw, e.bx, e.by,
                              1, 1));
    FD_TRY(make_tensor_map_4d(&plan->map_bext, bcoef, L.nx, L.ny, L.nz, 1, sy, sz, sw, e.ew, e.eh,
                              1, 1));
    return make_tensor_map_4d(&plan->map_bint, bcoef, L.nx, L.ny, L.nz, 1, sy, sz, sw, e.bx, e.by,
                              1, 1);
}

fd_status acoustic2_launch(const Acoustic2Plan &plan, const AcousticStep2Args &args,
                           cudaStream_t stream) {
    int n = 0;
    const T2Entry *tab = t2_table(plan.radius, &n);
    if (!tab || plan.config >= n) return set_error(FD_ERR_SO, "bad time-tiled plan");
    if (args.nsrc > kStep2MaxSources)
        return set_error(FD_ERR_ARG, "time-tiled step: %d sources per shot (at most %d)",
                         args.nsrc, kStep2MaxSources);
    int zchunk = plan.zchunk, nzc = plan.nzc;
    void *params[] = {(void *)&plan.map_halo, (void *)&plan.map_ext, (void *)&plan.map_int,
                      (void *)&plan.map_bext, (void *)&plan.map_bint, (void *)&args,
                      (void *)&zchunk, (void *)&nzc};
    FD_CUDA_TRY(cudaLaunchKernel(tab[plan.config].fn, plan.grid, plan.block, params, plan.smem,
                                 stream));
    note_launch(stream);
    return FD_OK;
}

}  // namespace fdsweep
