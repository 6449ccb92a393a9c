// acoustic_h.cu -- the acoustic leapfrog step with reduced-precision storage:
// the wavefield levels u^n, u^{n-1} and the coefficient b = dt^2/(m + damp
// dt/2) are stored in IEEE binary16, all arithmetic is FP32.  This is the
// paper's further work on mixed-precision arithmetic and on-the-fly
// compression (section "Further work"): it halves the bytes per point of a
// memory-bound step.
//
// The kernel keeps K1's design (acoustic.cu): one CTA per BX x BY column
// marching z, planes staged by cp.async.bulk.tensor into a ring of
// shared-memory stages with full/empty mbarriers and bounded waits, and the
// z-direction as an accumulator pipeline of 2R pending outputs in registers.
// What changes is the element type of the staged tiles: halves, so 8 bytes
// per point of algorithmic HBM traffic (read u^n, u^{n-1}, b; write u^{n+1})
// instead of 16, and half the shared-memory bytes.  Each thread decodes the
// halves it reads (cvt.f32.f16, exact) and evaluates K1's FP32 update with
// the same operations in the same order; the result is rounded to the
// nearest binary16 (cvt.rn.f16x2.f32) when stored.  The decoding is the
// extra cost (one conversion per value read, about 3 + 2R per point), which
// makes the kernel bound by instruction issue rather than by HBM; a block
// that decodes each staged plane once into an FP32 copy needs a block
// barrier per plane and measured twice as slow.
//
// x halo: a TMA box must start on a 16-byte boundary, so each staged row
// carries 8 halves of halo on either side, of which R are read.
#include <cuda_fp16.h>

#include "f32x2.cuh"
#include "kernels.cuh"
#include "runtime.cuh"

namespace fdsweep {
namespace {
using namespace f32x2;

template <int R, int TX, int TY, int VY, int D>
struct AhCfg {
    static constexpr int BX = 4 * TX;
    static constexpr int BY = VY * TY;
    static constexpr int RA = (R + 3) / 4 * 4;  // x reach of the arithmetic (as in K1)
    static constexpr int RH = 8;                // staged x halo: 16 bytes of halves
    static constexpr int PW = BX + 2 * RH;      // halves per staged row
    static constexpr int PH = BY + 2 * R;
    static constexpr int NSL = D + 1;
    static constexpr int HALO = (PW * PH + 63) / 64 * 64;  // halves, whole 128-byte lines
    static constexpr int INT = BX * BY;
    static constexpr int STAGE = HALO + 3 * INT;  // [halo u^n][u^n][u^{n-1}][b]
    static constexpr uint32_t HALO_BYTES = PW * PH * 2;
    static constexpr uint32_t INT_BYTES = INT * 2;
    static constexpr int THREADS = TX * TY;
    static constexpr int WARPS = THREADS / 32;
    // stages, full/empty mbarriers, abort flag; + damp_z of the z chunk
    // (added at launch) and 128 bytes to align the base
    static constexpr size_t SMEM = (size_t)NSL * STAGE * 2 + NSL * 16 + 16 + 128;
    static_assert(RA <= RH, "x reach beyond the staged halo");
    static_assert(PW <= 256 && PH <= 256 && BX <= 256 && BY <= 256, "TMA box dimension limit");
    static_assert(INT % 64 == 0 && THREADS % 32 == 0, "tile shape");
};

// two halves (low half first) -> two floats (exact)
__device__ __forceinline__ f2 h2_to_f2(uint32_t h) {
    float lo, hi;
    asm("{\n\t.reg .f16 l, u;\n\tmov.b32 {l, u}, %2;\n\t"
        "cvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, u;\n\t}"
        : "=f"(lo), "=f"(hi)
        : "r"(h));
    return f2_pack(lo, hi);
}

// two floats -> two halves, each rounded to nearest even (low half first)
__device__ __forceinline__ uint32_t f2_to_h2(f2 v) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(f2_hi(v)), "f"(f2_lo(v)));
    return r;
}

// four consecutive halves (8-byte aligned shared memory) as two packed pairs
__device__ __forceinline__ Q4 lds_h4(const half_bits *p) {
    const uint2 t = *reinterpret_cast<const uint2 *>(p);
    return Q4{h2_to_f2(t.x), h2_to_f2(t.y)};
}

// Every thread decodes the halves it reads.  A 4 x VY micro-tile per thread
// (VY rows) shares the decoded y-neighbour rows between its rows: VY + 2R
// rows decoded for VY outputs instead of 2R + 1 for each.
template <int R, int TX, int TY, int VY, int D, int U>
__global__ void __launch_bounds__(TX *TY)
    acoustic_step_h_kernel(const __grid_constant__ CUtensorMap map_halo,
                           const __grid_constant__ CUtensorMap map_int,
                           const __grid_constant__ CUtensorMap map_b, const AcousticHArgs a,
                           int zchunk, int nzc) {
    using C = AhCfg<R, TX, TY, VY, D>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    half_bits *smem = reinterpret_cast<half_bits *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::NSL * C::STAGE);
    uint64_t *empty = full + C::NSL;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + C::NSL);
    float *sdz = reinterpret_cast<float *>(empty + C::NSL + 2);  // damp_z / dt of this chunk

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int tx = tid % TX, ty = tid / TX;
    const int shot = blockIdx.z / nzc;
    const int chunk = blockIdx.z - shot * nzc;
    const int x0 = blockIdx.x * C::BX, y0 = blockIdx.y * C::BY;
    const int za = chunk * zchunk;
    const int zb = min(a.L.nz, za + zchunk);
    const int nplanes = zb - za + 2 * R;  // arriving planes za-R .. zb+R-1
    const int wcur = shot * a.lps + a.lev_cur, wprev = shot * a.lps + a.lev_prev;
    const int wout = shot * a.lps + a.lev_out;
    const int gx = x0 + 4 * tx;

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
            !mbar_wait_bounded(&empty[slot], (uint32_t)(((jj - C::NSL) / C::NSL) & 1)))
            return false;
        const bool with_out = jj >= 2 * R;
        mbar_arrive_expect_tx(&full[slot], C::HALO_BYTES + (with_out ? 3 * C::INT_BYTES : 0));
        half_bits *st = smem + slot * C::STAGE;
        tma_load_4d(st, &map_halo, &full[slot], x0 - C::RH, y0 - R, za - R + jj, wcur);
        if (with_out) {
            const int zo = za - 2 * R + jj;
            tma_load_4d(st + C::HALO, &map_int, &full[slot], x0, y0, zo, wcur);
            tma_load_4d(st + C::HALO + C::INT, &map_int, &full[slot], x0, y0, zo, wprev);
            tma_load_4d(st + C::HALO + 2 * C::INT, &map_b, &full[slot], x0, y0, zo, 0);
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
    half_bits *__restrict__ unew = a.wave + (int64_t)wout * a.L.vol;
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
        if (*abort_flag || !mbar_wait_bounded(&full[slot], (uint32_t)((j / C::NSL) & 1))) {
            *abort_flag = 1;
            atomicOr(a.err, DEV_ERR_TIMEOUT);
            break;
        }
        const half_bits *H = smem + slot * C::STAGE;
        const int rbase = R + ty * VY;

        // x/y part of the Laplacian of plane p (centre weight of all axes
        // included) and the centre values: K1's operations in K1's order on
        // the decoded values
        Q4 cen[VY], lxy[VY];
#pragma unroll
        for (int v = 0; v < VY; ++v) {
            constexpr int NP = (2 * C::RA + 4) / 2;  // packed pairs in the x span
            f2 xp[NP];
            const half_bits *row = H + (rbase + v) * C::PW + (C::RH - C::RA) + 4 * tx;
#pragma unroll
            for (int t = 0; t < NP / 2; ++t) {
                const Q4 q = lds_h4(row + 4 * t);
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
            const Q4 f = lds_h4(H + (rbase + dy) * C::PW + C::RH + 4 * tx);
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

        // z part: plane p feeds the pending outputs p-R .. p+R-1
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
            const half_bits *Ui = H + C::HALO;
#pragma unroll
            for (int v = 0; v < VY; ++v) {
                if (!(xok && yok[v])) continue;
                const int q = (ty * VY + v) * C::BX + 4 * tx;
                const Q4 c = lds_h4(Ui + q);
                const Q4 p = lds_h4(Ui + C::INT + q);
                const Q4 b = lds_h4(Ui + 2 * C::INT + q);
                const Q4 s = acc[0][v];
                const f2 dyz = f2_splat(dpyv[v] + dz);
                const f2 zl = f2_mul(f2_add(dpx_lo, dyz), b.lo);
                const f2 zh = f2_mul(f2_add(dpx_hi, dyz), b.hi);
                f2 ol = f2_fma(f2_sub(one2, zl), f2_sub(c.lo, p.lo), c.lo);
                f2 oh = f2_fma(f2_sub(one2, zh), f2_sub(c.hi, p.hi), c.hi);
                ol = f2_fma(b.lo, s.lo, ol);
                oh = f2_fma(b.hi, s.hi, oh);
                const int64_t off = (int64_t)zo * a.L.plane + (int64_t)gy[v] * a.L.nxp + gx;
                *reinterpret_cast<uint2 *>(unew + off) = make_uint2(f2_to_h2(ol), f2_to_h2(oh));
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
}

struct HEntry {
    int radius;
    const void *fn;
    size_t smem;
    int bx, by, pw, ph, threads;
    const char *name;
};

template <int R, int TX, int TY, int VY, int D, int U>
HEntry make_h_entry(const char *name) {
    using C = AhCfg<R, TX, TY, VY, D>;
    return HEntry{R,     (const void *)&acoustic_step_h_kernel<R, TX, TY, VY, D, U>,
                  C::SMEM, C::BX, C::BY, C::PW, C::PH, C::THREADS, name};
}

#define FD_AH_ENTRY(R, TX, TY, VY, D, U)                                                  \
    make_h_entry<R, TX, TY, VY, D, U>("acoustic_step_h<" #R "," #TX "," #TY "," #VY "," #D \
                                      "," #U ">")

// Index 0 is the default (template arguments R, TX, TY, VY, D, U: tile
// 4 TX x VY TY, VY rows per thread, prefetch depth D, plane-loop unroll U),
// measured on GB300 at 512^3: two rows per thread pay at R = 2 and 4 (fewer
// decoded neighbour rows per point), one row at R = 6 and 8 (registers).
const HEntry *h_table(int radius, int *count) {
    static const HEntry r1[] = {FD_AH_ENTRY(1, 16, 16, 1, 4, 1)};
    static const HEntry r2[] = {FD_AH_ENTRY(2, 16, 8, 2, 4, 2), FD_AH_ENTRY(2, 16, 8, 1, 4, 4),
                                FD_AH_ENTRY(2, 16, 8, 2, 4, 4), FD_AH_ENTRY(2, 16, 4, 4, 4, 2),
                                FD_AH_ENTRY(2, 16, 16, 1, 4, 4)};
    static const HEntry r4[] = {FD_AH_ENTRY(4, 16, 8, 2, 3, 4), FD_AH_ENTRY(4, 16, 8, 1, 3, 4),
                                FD_AH_ENTRY(4, 16, 8, 2, 3, 2), FD_AH_ENTRY(4, 16, 4, 2, 4, 2),
                                FD_AH_ENTRY(4, 16, 8, 1, 4, 4)};
    static const HEntry r6[] = {FD_AH_ENTRY(6, 16, 8, 1, 3, 4), FD_AH_ENTRY(6, 16, 8, 2, 2, 1),
                                FD_AH_ENTRY(6, 16, 8, 2, 2, 2), FD_AH_ENTRY(6, 16, 8, 1, 2, 4)};
    static const HEntry r8[] = {FD_AH_ENTRY(8, 16, 8, 1, 1, 4), FD_AH_ENTRY(8, 16, 8, 2, 1, 1),
                                FD_AH_ENTRY(8, 16, 8, 2, 2, 1), FD_AH_ENTRY(8, 16, 8, 1, 2, 4)};
    switch (radius) {
        case 1: *count = 1; return r1;
        case 2: *count = 5; return r2;
        case 4: *count = 5; return r4;
        case 6: *count = 4; return r6;
        case 8: *count = 4; return r8;
        default: *count = 0; return nullptr;
    }
}

// ---------------------------------------------------------------- sparse

__device__ __forceinline__ float h_corner_weight(const SparsePoint &p, int c) {
    const float wx = (c & 1) ? p.fx : 1.f - p.fx;
    const float wy = (c & 2) ? p.fy : 1.f - p.fy;
    const float wz = (c & 4) ? p.fz : 1.f - p.fz;
    return wx * wy * wz;
}

__device__ __forceinline__ int64_t h_corner_offset(const SparsePoint &p, int c,
                                                   const WaveLayout &L) {
    return (int64_t)p.base + ((c & 1) ? 1 : 0) + ((c & 2) ? L.nxp : 0) + ((c & 4) ? L.plane : 0);
}

__device__ __forceinline__ float h_load(const half_bits *p) {
    return __half2float(__ushort_as_half(__ldg(p)));
}

// Threads [0, nrec_total) interpolate receivers; the following
// nshots * nsrc * 8 threads inject (one per source corner).
__global__ void sparse_h_kernel(const SparseHArgs a, int step, int do_inject,
                                int64_t nrec_total) {
    const int n = step + (a.step_base ? *a.step_base : 0);
    if (n < 0 || n >= a.nt) return;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid < nrec_total) {
        const int s = (int)(gid / a.nrec);
        const int i = (int)(gid - (int64_t)s * a.nrec);
        const SparsePoint p = a.rec_tab[gid];
        const half_bits *u = a.wave + (int64_t)(s * a.fields_per_shot + a.rec_level) * a.L.vol;
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            acc = fmaf(h_corner_weight(p, c), h_load(u + h_corner_offset(p, c, a.L)), acc);
        a.rec_out[((int64_t)s * a.nt + n) * a.nrec + i] = acc;
        return;
    }
    if (!do_inject) return;
    const int64_t k = gid - nrec_total;
    if (k >= (int64_t)a.nshots * a.nsrc * 8) return;
    const int c = (int)(k & 7);
    const int64_t ps = k >> 3;  // (shot, source)
    const int s = (int)(ps / a.nsrc);
    const int isrc = (int)(ps - (int64_t)s * a.nsrc);
    const SparsePoint p = a.src_tab[ps];
    const int64_t off = h_corner_offset(p, c, a.L);
    const float q = a.src_wav[((int64_t)s * a.nt + n) * a.nsrc + isrc];
    const float val = h_corner_weight(p, c) * h_load(a.bcoef + off) * q;
    half_bits *dst = a.wave + (int64_t)(s * a.fields_per_shot + a.inj_level) * a.L.vol + off;
    atomicAdd(reinterpret_cast<__half *>(dst), __float2half_rn(val));
}

// ---------------------------------------------------------------- conversions

__global__ void narrow_rows_kernel(const float *__restrict__ src, int64_t ss,
                                   half_bits *__restrict__ dst, int64_t ds, int nx, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / nx;
        const int x = (int)(i - r * nx);
        dst[r * ds + x] = __half_as_ushort(__float2half_rn(src[r * ss + x]));
    }
}

__global__ void widen_rows_kernel(const half_bits *__restrict__ src, int64_t ss,
                                  float *__restrict__ dst, int64_t ds, int nx, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / nx;
        const int x = (int)(i - r * nx);
        dst[r * ds + x] = __half2float(__ushort_as_half(src[r * ss + x]));
    }
}

// inf and NaN are the binary16 patterns with all exponent bits set
__global__ void finite_h_kernel(const half_bits *__restrict__ f, int64_t ss, int nx, int64_t n,
                                unsigned int *flags) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / nx;
        const int x = (int)(i - r * nx);
        bad |= (f[r * ss + x] & 0x7c00u) == 0x7c00u;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, DEV_ERR_NONFINITE);
}

int h_grid(int64_t n, int threads) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t b = (n + threads - 1) / threads;
    if (b > (int64_t)nsm * 16) b = (int64_t)nsm * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

int acoustic_h_num_configs(int radius) {
    int n = 0;
    h_table(radius, &n);
    return n;
}

fd_status acoustic_h_plan(int radius, int config, const WaveLayout &L, int nshots, int lps,
                          half_bits *wave, const half_bits *bcoef, AcousticPlan *plan) {
    int n = 0;
    const HEntry *tab = h_table(radius, &n);
    if (!tab) return set_error(FD_ERR_UNIMPL, "no binary16-storage kernel for radius %d", radius);
    if (L.nxp % 8) return set_error(FD_ERR_ARG, "binary16 layout: row length not a multiple of 8");
    if (config < 0 || config >= n) config = 0;
    const HEntry &e = tab[config];
    plan->radius = radius;
    plan->config = config;
    plan->name = e.name;
    plan->block = dim3(e.threads, 1, 1);
    int dev = 0, nsm = 0, per_sm = 0;
    FD_CUDA_TRY(cudaGetDevice(&dev));
    FD_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FD_TRY(raise_smem_limit(e.fn, e.smem));
    FD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, e.fn, e.threads, e.smem));
    if (per_sm < 1) return set_error(FD_ERR_CUDA, "kernel %s does not fit on an SM", e.name);
    const int ntx = (L.nx + e.bx - 1) / e.bx;
    const int nty = (L.ny + e.by - 1) / e.by;
    const int64_t cols = (int64_t)ntx * nty * nshots;
    const int64_t slots = (int64_t)nsm * per_sm;
    // split z only when the columns alone cannot fill the machine (as K1)
    int nzc = 1;
    if (cols < slots) {
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
    const uint64_t sy = (uint64_t)L.nxp * 2, sz = (uint64_t)L.plane * 2, sw = (uint64_t)L.vol * 2;
    FD_TRY(make_tensor_map_4d_elem(&plan->map_halo, wave, 2, L.nx, L.ny, L.nz,
                                   (uint64_t)nshots * lps, sy, sz, sw, e.pw, e.ph, 1, 1));
    FD_TRY(make_tensor_map_4d_elem(&plan->map_int, wave, 2, L.nx, L.ny, L.nz,
                                   (uint64_t)nshots * lps, sy, sz, sw, e.bx, e.by, 1, 1));
    return make_tensor_map_4d_elem(&plan->map_b, bcoef, 2, L.nx, L.ny, L.nz, 1, sy, sz, sw, e.bx,
                                   e.by, 1, 1);
}

fd_status acoustic_h_launch(const AcousticPlan &plan, const AcousticHArgs &args,
                            cudaStream_t stream) {
    int n = 0;
    const HEntry *tab = h_table(plan.radius, &n);
    if (!tab || plan.config >= n) return set_error(FD_ERR_SO, "bad binary16 acoustic plan");
    int zchunk = plan.zchunk, nzc = plan.nzc;
    void *params[] = {(void *)&plan.map_halo, (void *)&plan.map_int, (void *)&plan.map_b,
                      (void *)&args, (void *)&zchunk, (void *)&nzc};
    FD_CUDA_TRY(cudaLaunchKernel(tab[plan.config].fn, plan.grid, plan.block, params, plan.smem,
                                 stream));
    note_launch(stream);
    return FD_OK;
}

fd_status sparse_h_launch(const SparseHArgs &a, int step, bool do_inject, bool do_interp,
                          cudaStream_t stream) {
    const int64_t nrec_total = do_interp ? (int64_t)a.nshots * a.nrec : 0;
    const int64_t ninj = do_inject ? (int64_t)a.nshots * a.nsrc * 8 : 0;
    const int64_t total = nrec_total + ninj;
    if (total == 0) return FD_OK;
    const int threads = 256;
    const int64_t blocks = (total + threads - 1) / threads;
    sparse_h_kernel<<<(unsigned)blocks, threads, 0, stream>>>(a, step, do_inject ? 1 : 0,
                                                              nrec_total);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

fd_status narrow_rows(const float *src, int64_t src_stride, half_bits *dst, int64_t dst_stride,
                      int nx, int64_t rows, cudaStream_t stream) {
    const int64_t n = (int64_t)nx * rows;
    if (n == 0) return FD_OK;
    narrow_rows_kernel<<<h_grid(n, 256), 256, 0, stream>>>(src, src_stride, dst, dst_stride, nx,
                                                           n);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

fd_status widen_rows(const half_bits *src, int64_t src_stride, float *dst, int64_t dst_stride,
                     int nx, int64_t rows, cudaStream_t stream) {
    const int64_t n = (int64_t)nx * rows;
    if (n == 0) return FD_OK;
    widen_rows_kernel<<<h_grid(n, 256), 256, 0, stream>>>(src, src_stride, dst, dst_stride, nx,
                                                          n);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

fd_status check_finite_h(const half_bits *field, const WaveLayout &L, int nfields,
                         unsigned int *flags, cudaStream_t stream) {
    const int64_t n = (int64_t)L.nx * L.ny * L.nz * nfields;
    if (n == 0) return FD_OK;
    // rows of all fields are equally spaced: field f row r at (f nz ny + r) nxp
    finite_h_kernel<<<h_grid(n, 256), 256, 0, stream>>>(field, L.nxp, L.nx, n, flags);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

}  // namespace fdsweep
