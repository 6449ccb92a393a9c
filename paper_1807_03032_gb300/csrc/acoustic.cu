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
// GB300 design: one CTA owns a BX x BY column of the grid and marches it
// through z.  Each xy plane of u^n (tile plus an R-wide halo, zero-filled
// outside the grid by the TMA unit) is staged into a ring of shared-memory
// stages by cp.async.bulk.tensor, D planes ahead of use, completing on one
// mbarrier per stage.  Every thread owns a 4 (x, one float4) by VY (y)
// micro-tile; the z-neighbours live in a register queue of 2R+1 planes, the x-
// and y-neighbours are read from the staged plane.  u^{n-1} and b stream in
// with float4 loads, u^{n+1} overwrites u^{n-1} in place.  Algorithmic HBM
// traffic: 16 bytes per point (read u^n, u^{n-1}, b; write u^{n+1}).
#include <stdio.h>

#include "kernels.cuh"

namespace fdsweep {
namespace {

template <int R, int TX, int TY, int VY, int D>
struct AcCfg {
    static constexpr int BX = 4 * TX;
    static constexpr int BY = VY * TY;
    static constexpr int RA = (R + 3) / 4 * 4;  // x halo rounded to 16 bytes (TMA rule)
    static constexpr int PW = BX + 2 * RA;
    static constexpr int PH = BY + 2 * R;
    static constexpr int NS = R + D + 1;        // stages: R+1 planes in use + D in flight
    static constexpr int STAGE = (PW * PH + 31) / 32 * 32;
    static constexpr uint32_t BYTES = PW * PH * 4;
    // stages, then NS mbarriers and an abort flag; +128 bytes to align the base
    static constexpr size_t SMEM = (size_t)NS * STAGE * 4 + NS * 8 + 16 + 128;
    static constexpr int THREADS = TX * TY;
    static_assert(PW <= 256 && PH <= 256, "TMA box dimension limit");
};

template <int R, int TX, int TY, int VY, int D>
__global__ void __launch_bounds__(TX *TY)
    acoustic_step_kernel(const __grid_constant__ CUtensorMap map, const AcousticStepArgs a,
                         int zchunk, int nzc) {
    using C = AcCfg<R, TX, TY, VY, D>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations: 128-byte aligned stages of STAGE floats each
    float *smem = reinterpret_cast<float *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::NS * C::STAGE);
    volatile int &s_abort = *reinterpret_cast<volatile int *>(bars + C::NS);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int shot = blockIdx.z / nzc;
    const int chunk = blockIdx.z - shot * nzc;
    const int x0 = blockIdx.x * C::BX, y0 = blockIdx.y * C::BY;
    const int za = chunk * zchunk;
    const int zb = min(a.L.nz, za + zchunk);
    const int nplanes = zb - za + 2 * R;  // planes za-R .. zb+R-1
    const int wcur = 2 * shot + a.cur;
    const int gx = x0 + 4 * tx;

    if (tid == 0) {
        prefetch_tensormap(&map);
        for (int s = 0; s < C::NS; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    if (tid == 0) {
        for (int j = 0; j < D && j < nplanes; ++j) {
            mbar_arrive_expect_tx(&bars[j], C::BYTES);
            tma_load_4d(smem + j * C::STAGE, &map, &bars[j], x0 - C::RA, y0 - R, za - R + j,
                        wcur);
        }
    }

    const bool xok = gx < a.L.nxp;
    float dpx4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) dpx4[i] = (gx + i < a.L.nx) ? a.dpx[gx + i] : 0.f;
    int gy[VY];
    bool yok[VY];
    float dpyv[VY];
#pragma unroll
    for (int v = 0; v < VY; ++v) {
        gy[v] = y0 + ty * VY + v;
        yok[v] = gy[v] < a.L.ny;
        dpyv[v] = yok[v] ? a.dpy[gy[v]] : 0.f;
    }
    float *__restrict__ unew = a.wave + (int64_t)(2 * shot + 1 - a.cur) * a.L.vol;

    float4 q[2 * R + 1][VY];
#pragma unroll
    for (int s = 0; s < 2 * R + 1; ++s)
#pragma unroll
        for (int v = 0; v < VY; ++v) q[s][v] = make_float4(0.f, 0.f, 0.f, 0.f);

    int j = 0;
    for (; j < nplanes; ++j) {
        const int zo = za + j - 2 * R;  // output plane completed by this iteration
        const bool has_out = j >= 2 * R;
        float4 um[VY], bb[VY];
#pragma unroll
        for (int v = 0; v < VY; ++v) {
            um[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            bb[v] = um[v];
            if (has_out && xok && yok[v]) {
                const int64_t off = (int64_t)zo * a.L.plane + (int64_t)gy[v] * a.L.nxp + gx;
                um[v] = *reinterpret_cast<const float4 *>(unew + off);
                bb[v] = ld_nc_f4(a.bcoef + off);
            }
        }
        if (tid == 0 && j + D < nplanes) {
            const int jj = j + D;
            const int slot = jj % C::NS;
            mbar_arrive_expect_tx(&bars[slot], C::BYTES);
            tma_load_4d(smem + slot * C::STAGE, &map, &bars[slot], x0 - C::RA, y0 - R,
                        za - R + jj, wcur);
        }
        const int slot = j % C::NS;
        const bool ok = mbar_wait_bounded(&bars[slot], (uint32_t)((j / C::NS) & 1));
        if (!ok) {
            s_abort = 1;
            atomicOr(a.err, DEV_ERR_TIMEOUT);
        } else {
#pragma unroll
            for (int s = 0; s < 2 * R; ++s)
#pragma unroll
                for (int v = 0; v < VY; ++v) q[s][v] = q[s + 1][v];
            const float *P = smem + slot * C::STAGE;
#pragma unroll
            for (int v = 0; v < VY; ++v)
                q[2 * R][v] = *reinterpret_cast<const float4 *>(
                    P + (R + ty * VY + v) * C::PW + C::RA + 4 * tx);

            if (has_out) {
                const float *Cp = smem + ((j - R) % C::NS) * C::STAGE;
                const int rbase = R + ty * VY;
                float4 acc[VY];
#pragma unroll
                for (int v = 0; v < VY; ++v) {
                    const float4 c = q[R][v];
                    float4 s;
                    s.x = a.wc * c.x;
                    s.y = a.wc * c.y;
                    s.z = a.wc * c.z;
                    s.w = a.wc * c.w;
#pragma unroll
                    for (int k = 1; k <= R; ++k) {
                        const float4 p = q[R + k][v], m = q[R - k][v];
                        s.x = fmaf(a.wz[k], p.x + m.x, s.x);
                        s.y = fmaf(a.wz[k], p.y + m.y, s.y);
                        s.z = fmaf(a.wz[k], p.z + m.z, s.z);
                        s.w = fmaf(a.wz[k], p.w + m.w, s.w);
                    }
                    float xs[2 * C::RA + 4];
                    const float *row = Cp + (rbase + v) * C::PW + 4 * tx;
#pragma unroll
                    for (int t = 0; t < (2 * C::RA + 4) / 4; ++t) {
                        const float4 f = *reinterpret_cast<const float4 *>(row + 4 * t);
                        xs[4 * t + 0] = f.x;
                        xs[4 * t + 1] = f.y;
                        xs[4 * t + 2] = f.z;
                        xs[4 * t + 3] = f.w;
                    }
#pragma unroll
                    for (int k = 1; k <= R; ++k) {
                        s.x = fmaf(a.wx[k], xs[C::RA + 0 + k] + xs[C::RA + 0 - k], s.x);
                        s.y = fmaf(a.wx[k], xs[C::RA + 1 + k] + xs[C::RA + 1 - k], s.y);
                        s.z = fmaf(a.wx[k], xs[C::RA + 2 + k] + xs[C::RA + 2 - k], s.z);
                        s.w = fmaf(a.wx[k], xs[C::RA + 3 + k] + xs[C::RA + 3 - k], s.w);
                    }
                    acc[v] = s;
                }
                // y-neighbours: stream the rows once, each feeds every output row
                // of this thread within reach.
#pragma unroll
                for (int dy = -R; dy < VY + R; ++dy) {
                    bool needed = false;
#pragma unroll
                    for (int v = 0; v < VY; ++v) {
                        const int k = dy > v ? dy - v : v - dy;
                        if (k >= 1 && k <= R) needed = true;
                    }
                    if (!needed) continue;
                    const float4 f = *reinterpret_cast<const float4 *>(
                        Cp + (rbase + dy) * C::PW + C::RA + 4 * tx);
#pragma unroll
                    for (int v = 0; v < VY; ++v) {
                        const int k = dy > v ? dy - v : v - dy;
                        if (k >= 1 && k <= R) {
                            acc[v].x = fmaf(a.wy[k], f.x, acc[v].x);
                            acc[v].y = fmaf(a.wy[k], f.y, acc[v].y);
                            acc[v].z = fmaf(a.wy[k], f.z, acc[v].z);
                            acc[v].w = fmaf(a.wy[k], f.w, acc[v].w);
                        }
                    }
                }
                const float dz = a.dpz[zo];
#pragma unroll
                for (int v = 0; v < VY; ++v) {
                    if (!(xok && yok[v])) continue;
                    const float4 c = q[R][v];
                    const float4 b = bb[v], p = um[v], s = acc[v];
                    const float dyz = dpyv[v] + dz;
                    float4 o;
                    o.x = c.x + (1.f - (dpx4[0] + dyz) * b.x) * (c.x - p.x) + b.x * s.x;
                    o.y = c.y + (1.f - (dpx4[1] + dyz) * b.y) * (c.y - p.y) + b.y * s.y;
                    o.z = c.z + (1.f - (dpx4[2] + dyz) * b.z) * (c.z - p.z) + b.z * s.z;
                    o.w = c.w + (1.f - (dpx4[3] + dyz) * b.w) * (c.w - p.w) + b.w * s.w;
                    const int64_t off = (int64_t)zo * a.L.plane + (int64_t)gy[v] * a.L.nxp + gx;
                    *reinterpret_cast<float4 *>(unew + off) = o;
                }
            }
        }
        __syncthreads();
        if (s_abort) break;
    }
    if (s_abort && tid == 0) {
        // Planes 0 .. j+D have been issued; give the ones not yet consumed a
        // bounded chance to land before the CTA's shared memory goes away.
        const int issued = min(nplanes, j + D + 1);
        for (int jj = j; jj < issued; ++jj)
            mbar_wait_bounded(&bars[jj % C::NS], (uint32_t)((jj / C::NS) & 1), 200000000ull);
    }
}

struct ConfigEntry {
    int radius, tx, ty, vy, d;
    const void *fn;
    size_t smem;
    int bx, by, pw, ph, threads;
    const char *name;
};

template <int R, int TX, int TY, int VY, int D>
ConfigEntry make_entry(const char *name) {
    using C = AcCfg<R, TX, TY, VY, D>;
    return ConfigEntry{R,      TX,     TY,     VY,         D,    (const void *)&acoustic_step_kernel<R, TX, TY, VY, D>,
                       C::SMEM, C::BX, C::BY, C::PW, C::PH, C::THREADS, name};
}

#define FD_AC_ENTRY(R, TX, TY, VY, D) make_entry<R, TX, TY, VY, D>("acoustic_step<" #R "," #TX "," #TY "," #VY "," #D ">")

const ConfigEntry *config_table(int radius, int *count) {
    static const ConfigEntry r1[] = {FD_AC_ENTRY(1, 16, 8, 2, 3)};
    static const ConfigEntry r2[] = {FD_AC_ENTRY(2, 16, 8, 2, 3), FD_AC_ENTRY(2, 16, 8, 4, 3),
                                     FD_AC_ENTRY(2, 32, 4, 2, 3)};
    static const ConfigEntry r4[] = {FD_AC_ENTRY(4, 16, 8, 2, 2), FD_AC_ENTRY(4, 16, 8, 4, 2),
                                     FD_AC_ENTRY(4, 32, 4, 2, 2)};
    static const ConfigEntry r6[] = {FD_AC_ENTRY(6, 16, 8, 2, 2), FD_AC_ENTRY(6, 16, 4, 2, 2),
                                     FD_AC_ENTRY(6, 32, 4, 2, 2)};
    static const ConfigEntry r8[] = {FD_AC_ENTRY(8, 16, 8, 1, 2), FD_AC_ENTRY(8, 16, 4, 2, 2),
                                     FD_AC_ENTRY(8, 16, 8, 2, 2)};
    switch (radius) {
        case 1: *count = 1; return r1;
        case 2: *count = 3; return r2;
        case 4: *count = 3; return r4;
        case 6: *count = 3; return r6;
        case 8: *count = 3; return r8;
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

fd_status acoustic_plan(int radius, int config, const WaveLayout &L, int nshots, float *wave,
                        AcousticPlan *plan) {
    int n = 0;
    const ConfigEntry *tab = config_table(radius, &n);
    if (!tab) return set_error(FD_ERR_SO, "no acoustic kernel for radius %d", radius);
    if (config < 0 || config >= n) config = acoustic_default_config(radius);
    const ConfigEntry &e = tab[config];
    plan->radius = radius;
    plan->config = config;
    plan->name = e.name;
    plan->smem = e.smem;
    plan->block = dim3(e.threads, 1, 1);
    FD_CUDA_TRY(cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)e.smem));
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
    return make_tensor_map_4d(&plan->map, wave, L.nx, L.ny, L.nz, 2ull * nshots,
                              (uint64_t)L.nxp * 4, (uint64_t)L.plane * 4, (uint64_t)L.vol * 4,
                              e.pw, e.ph, 1, 1);
}

fd_status acoustic_launch(const AcousticPlan &plan, const AcousticStepArgs &args,
                          cudaStream_t stream) {
    int n = 0;
    const ConfigEntry *tab = config_table(plan.radius, &n);
    if (!tab || plan.config >= n) return set_error(FD_ERR_SO, "bad acoustic plan");
    int zchunk = plan.zchunk, nzc = plan.nzc;
    void *params[] = {(void *)&plan.map, (void *)&args, (void *)&zchunk, (void *)&nzc};
    FD_CUDA_TRY(cudaLaunchKernel(tab[plan.config].fn, plan.grid, plan.block, params, plan.smem,
                                 stream));
    note_launch(stream);
    return FD_OK;
}

}  // namespace fdsweep
