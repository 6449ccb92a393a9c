// setup.cu -- K0: per-call coefficient precompute and validation.
//
//  * b = dt^2 / (m + damp dt / 2) per point, rounded once to FP32 (two-float
//    FP32 arithmetic with a residual-corrected quotient; FP64 with a
//    Newton-Raphson reciprocal for points outside its range),
//    the factor that multiplies the Laplacian in the leapfrog update and the
//    injected source (Listing finject's dt^2 q / m, generalised to the damped
//    update); damping profiles scaled by 1/dt.
//  * TTI: a = 1 + 2 eps, s = sqrt(1 + 2 delta) and the symmetry axis
//    n = (sin theta cos phi, sin theta sin phi, cos theta), precomputed once
//    because they do not change with time.
//  * Sparse tables: the trilinear corner and fractional offsets of every
//    source and receiver, x1 = floor((x - o)/h) in FP64, clamped to n - 2.
//  * Reductions for validation: min/max of m (stability bound), max eps,
//    flags for non-finite or non-physical values.
#include "kernels.cuh"

namespace fdsweep {
namespace {

// Order-preserving float <-> uint mapping for atomicMin/atomicMax on floats.
__device__ __forceinline__ unsigned int float_key(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned int k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

struct StatsKeys {
    unsigned int m_min, m_max, eps_max, flags;
};

__global__ void init_stats_kernel(StatsKeys *s) {
    s->m_min = float_key(__int_as_float(0x7f800000));  // +inf
    s->m_max = float_key(0.f);
    s->eps_max = float_key(-__int_as_float(0x7f800000));
    s->flags = 0u;
}

__global__ void finish_stats_kernel(StatsKeys *s) {
    MediumStats *out = reinterpret_cast<MediumStats *>(s);
    const StatsKeys k = *s;
    out->m_min = key_float(k.m_min);
    out->m_max = key_float(k.m_max);
    out->eps_max = key_float(k.eps_max);
    out->flags = k.flags;
}

__device__ __forceinline__ float warp_min(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// 1/x in FP64 by Newton-Raphson on the reciprocal (y <- y + y (1 - x y),
// which squares the relative error), seeded with the FP32 reciprocal: two
// steps take the 24-bit seed past FP64 precision.  GB300's FP64 rate is low,
// and this costs a third of a full-precision division.  Falls back to the
// division when the seed is not usable (x outside the FP32 normal range).
__device__ __forceinline__ double recip_newton(double x) {
    const float xf = (float)x;
    if (!(fabsf(xf) >= 1.17549435e-38f && fabsf(xf) <= 1.0e38f)) return 1.0 / x;
    double y = (double)__frcp_rn(xf);
    y = fma(y, fma(-x, y, 1.0), y);
    y = fma(y, fma(-x, y, 1.0), y);
    return y;
}

// Two-float arithmetic (a value as an unevaluated sum hi + lo of floats),
// with the error-free transformations TwoSum (Knuth) and TwoProduct (by FMA)
// and the rounding-explicit intrinsics, so that no operation is contracted.
struct TwoFloat {
    float hi, lo;
};

__device__ __forceinline__ TwoFloat two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return TwoFloat{s, e};
}

// The nearest float to (A + a) / (X + x) for two-float numerator and
// denominator (X > 0): q = A / X is within a few units of the answer; the
// residual (A + a) - q (X + x), whose leading part A - q X is exact by FMA,
// divided by X is the remaining correction, and q plus it is rounded once
// (Markstein's final step).  The correction carries about 24 bits, so the
// result can differ from exact rounding only when the quotient lies within
// about 2^-44 of its size of a rounding midpoint.
__device__ __forceinline__ float div_two_float_rn(float A, float a, float X, float x) {
    const float q = __fdiv_rn(A, X);
    float r = fmaf(-q, X, A);
    r = __fadd_rn(r, a);
    r = fmaf(-q, x, r);
    return fmaf(r, __frcp_rn(X), q);
}

// One grid row (j, k) per block iteration: the row index is split once per
// row, not per point.  b = dt^2 / (m + (dx + dy + dz) dt / 2) is formed in
// two-float FP32 arithmetic (dt^2 = A + a, dt / 2 = H + h): the damping sum
// and its product with dt / 2 carried to about 2^-44, the quotient rounded
// once (div_two_float_rn).  FP64 -- slow on this part -- remains for the
// points that fail validation or lie outside the range where the two-float
// steps are exact (m or a damping term negative, non-finite, or extreme).
// With `zeta` non-null the damping is a 3-D field damp[nz][ny][nx] (d = damp
// at the point) and zeta = fl(fl(d / dt) b) is stored beside b, the factor
// the stencil kernel's damp-field variant reads instead of forming it from
// per-axis profiles (the same two roundings as the profile path's
// fl(fl(d_x/dt + (d_y/dt + d_z/dt)) b) when a single axis is damped).
__global__ void acoustic_coeff_kernel(const float *__restrict__ m, const float *__restrict__ damp,
                                      double dt, float dt2_hi, float dt2_lo, float hdt_hi,
                                      float hdt_lo, WaveLayout L, float *__restrict__ bcoef,
                                      float *__restrict__ zeta, StatsKeys *stats) {
    const int64_t rows = (int64_t)L.ny * L.nz;
    const double dt2 = dt * dt;
    float lmin = __int_as_float(0x7f800000), lmax = 0.f;
    unsigned int bad = 0u;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int j = (int)(r % L.ny);
        const int k = (int)(r / L.ny);
        const bool dense = zeta != nullptr;
        const float dyf = damp && !dense ? damp[L.nx + j] : 0.f;
        const float dzf = damp && !dense ? damp[L.nx + L.ny + k] : 0.f;
        const bool row_ok = dyf >= 0.f && dyf <= 1.0e30f && dzf >= 0.f && dzf <= 1.0e30f;
        const float *mrow = m + r * L.nx;
        const float *drow = dense && damp ? damp + r * L.nx : nullptr;
        float *brow = bcoef + (int64_t)k * L.plane + (int64_t)j * L.nxp;
        for (int i = threadIdx.x; i < L.nx; i += blockDim.x) {
            const float mv = mrow[i];
            const float dxf = drow ? drow[i] : (damp && !dense ? damp[i] : 0.f);
            lmin = fminf(lmin, mv);
            lmax = fmaxf(lmax, mv);
            if (row_ok && dxf >= 0.f && dxf <= 1.0e30f && mv >= 1.17549435e-38f &&
                mv <= 1.0e30f) {
                // d = dx + dy + dz, eta = d dt / 2, x = m + eta, as two-floats
                const TwoFloat s1 = two_sum(dxf, dyf);
                const TwoFloat s2 = two_sum(s1.hi, dzf);
                const float dlo = __fadd_rn(s1.lo, s2.lo);
                const float ph = __fmul_rn(s2.hi, hdt_hi);
                float pl = fmaf(s2.hi, hdt_hi, -ph);
                pl = __fadd_rn(pl, __fadd_rn(__fmul_rn(s2.hi, hdt_lo), __fmul_rn(dlo, hdt_hi)));
                const TwoFloat xs = two_sum(mv, ph);
                brow[i] = div_two_float_rn(dt2_hi, dt2_lo, xs.hi, __fadd_rn(xs.lo, pl));
            } else {
                double d = 0.0;
                if (damp) d = (double)dxf + (double)dyf + (double)dzf;
                if (!(mv > 0.f) || !isfinite(mv) || !(d >= 0.0) || !isfinite(d))
                    bad = DEV_ERR_MEDIUM;
                brow[i] = (float)(dt2 * recip_newton((double)mv + 0.5 * d * dt));
            }
            if (dense)
                zeta[(int64_t)k * L.plane + (int64_t)j * L.nxp + i] =
                    __fmul_rn((float)((double)dxf / dt), brow[i]);
        }
    }
    lmin = warp_min(lmin);
    lmax = warp_max(lmax);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&stats->m_min, float_key(lmin));
        atomicMax(&stats->m_max, float_key(lmax));
    }
    if (bad) atomicOr(&stats->flags, bad);
}

__global__ void damp_scale_kernel(const float *__restrict__ damp, int n, double dt,
                                  float *__restrict__ dps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dps[i] = damp ? (float)((double)damp[i] / dt) : 0.f;
}

__global__ void tti_coeff_kernel(const float *__restrict__ eps, const float *__restrict__ delta,
                                 const float *__restrict__ theta, const float *__restrict__ phi,
                                 WaveLayout L, float *__restrict__ acoef, float *__restrict__ scoef,
                                 float *__restrict__ nvec, StatsKeys *stats) {
    const int64_t n = (int64_t)L.nx * L.ny * L.nz;
    float lmax = -__int_as_float(0x7f800000);
    unsigned int bad = 0u;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % L.nx);
        const int64_t r = p / L.nx;
        const int j = (int)(r % L.ny);
        const int k = (int)(r / L.ny);
        const float e = eps[p], d = delta[p], th = theta[p], ph = phi[p];
        if (!isfinite(e) || !isfinite(d) || !isfinite(th) || !isfinite(ph) || !(e >= d) ||
            !(1.0f + 2.0f * d >= 0.f))
            bad = DEV_ERR_MEDIUM;
        lmax = fmaxf(lmax, e);
        const int64_t q = (int64_t)k * L.plane + (int64_t)j * L.nxp + i;
        acoef[q] = (float)(1.0 + 2.0 * (double)e);
        scoef[q] = (float)sqrt(fmax(0.0, 1.0 + 2.0 * (double)d));
        double st, ct, sp, cp;
        sincos((double)th, &st, &ct);
        sincos((double)ph, &sp, &cp);
        nvec[q] = (float)(st * cp);
        nvec[L.vol + q] = (float)(st * sp);
        nvec[2 * L.vol + q] = (float)ct;
    }
    lmax = warp_max(lmax);
    if ((threadIdx.x & 31) == 0) atomicMax(&stats->eps_max, float_key(lmax));
    if (bad) atomicOr(&stats->flags, bad);
}

__global__ void sparse_table_kernel(const float *__restrict__ xyz, int npts, fd_grid g,
                                    WaveLayout L, SparsePoint *__restrict__ tab,
                                    unsigned int *flags) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    const int n[3] = {g.nx, g.ny, g.nz};
    const double h[3] = {g.hx, g.hy, g.hz};
    const double o[3] = {g.ox, g.oy, g.oz};
    int i1[3];
    float fr[3];
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
        const double s = ((double)xyz[3 * (int64_t)p + a] - o[a]) / h[a];
        if (!(s >= 0.0 && s <= (double)(n[a] - 1))) {
            ok = false;
            i1[a] = 0;
            fr[a] = 0.f;
            continue;
        }
        int x1 = (int)floor(s);
        if (x1 > n[a] - 2) x1 = n[a] - 2;
        i1[a] = x1;
        fr[a] = (float)(s - (double)x1);
    }
    if (!ok) atomicOr(flags, DEV_ERR_COORD);
    SparsePoint sp;
    sp.base = (uint32_t)((int64_t)i1[2] * L.plane + (int64_t)i1[1] * L.nxp + i1[0]);
    sp.fx = fr[0];
    sp.fy = fr[1];
    sp.fz = fr[2];
    tab[p] = sp;
}

__global__ void finite_kernel(const float *__restrict__ f, int64_t n, unsigned int *flags) {
    bool bad = false;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(f[p])) bad = true;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, DEV_ERR_NONFINITE);
}

// One thread per element of the sampled rows (see watchdog_launch).
__global__ void watchdog_kernel(const float *__restrict__ f, WaveLayout L, int nfields, int nzs,
                                int nys, unsigned int *flags) {
    const int64_t per_field = (int64_t)nzs * nys * L.nxp;
    const int64_t n = per_field * nfields;
    bool bad = false;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t fld = p / per_field;
        const int64_t r = p - fld * per_field;
        const int64_t row = r / L.nxp;
        const int x = (int)(r - row * L.nxp);
        const int zi = (int)(row / nys), yi = (int)(row - (int64_t)zi * nys);
        const int64_t off = fld * L.vol + (int64_t)zi * kWatchStride * L.plane +
                            (int64_t)yi * kWatchStride * L.nxp + x;
        if (!isfinite(f[off])) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, DEV_ERR_NONFINITE);
}

int grid_for(int64_t n, int threads) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)nsm * 8;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

fd_status init_medium_stats(MediumStats *dev_stats, cudaStream_t stream) {
    static_assert(sizeof(StatsKeys) == sizeof(MediumStats), "stats layout");
    init_stats_kernel<<<1, 1, 0, stream>>>(reinterpret_cast<StatsKeys *>(dev_stats));
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

fd_status setup_acoustic_coeffs(const float *m, const float *damp, double dt,
                                const WaveLayout &L, float *bcoef, float *dps,
                                MediumStats *dev_stats, cudaStream_t stream, bool damp_field) {
    StatsKeys *keys = reinterpret_cast<StatsKeys *>(dev_stats);
    const double dt2 = dt * dt, hdt = 0.5 * dt;
    const float dt2_hi = (float)dt2, hdt_hi = (float)hdt;
    const float dt2_lo = (float)(dt2 - (double)dt2_hi), hdt_lo = (float)(hdt - (double)hdt_hi);
    acoustic_coeff_kernel<<<grid_for((int64_t)L.ny * L.nz * 256, 256), 256, 0, stream>>>(
        m, damp, dt, dt2_hi, dt2_lo, hdt_hi, hdt_lo, L, bcoef, damp_field ? bcoef + L.vol : nullptr,
        keys);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    const int nd = L.nx + L.ny + L.nz;
    damp_scale_kernel<<<(nd + 255) / 256, 256, 0, stream>>>(damp_field ? nullptr : damp, nd, dt,
                                                            dps);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

fd_status setup_tti_coeffs(const float *eps, const float *delta, const float *theta,
                           const float *phi, const WaveLayout &L, float *acoef, float *scoef,
                           float *nvec, MediumStats *dev_stats, cudaStream_t stream) {
    StatsKeys *keys = reinterpret_cast<StatsKeys *>(dev_stats);
    const int64_t n = (int64_t)L.nx * L.ny * L.nz;
    tti_coeff_kernel<<<grid_for(n, 256), 256, 0, stream>>>(eps, delta, theta, phi, L, acoef,
                                                           scoef, nvec, keys);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

fd_status setup_sparse_table(const float *xyz, int npts, const fd_grid &g, const WaveLayout &L,
                             SparsePoint *tab, unsigned int *flags, cudaStream_t stream) {
    if (npts <= 0) return FD_OK;
    sparse_table_kernel<<<(npts + 255) / 256, 256, 0, stream>>>(xyz, npts, g, L, tab, flags);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

fd_status check_finite(const float *field, const WaveLayout &L, int nfields, unsigned int *flags,
                       cudaStream_t stream) {
    const int64_t n = L.vol * nfields;
    finite_kernel<<<grid_for(n, 256), 256, 0, stream>>>(field, n, flags);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

fd_status watchdog_launch(const float *field, const WaveLayout &L, int nfields,
                          unsigned int *flags, cudaStream_t stream) {
    const int nzs = (L.nz + kWatchStride - 1) / kWatchStride;
    const int nys = (L.ny + kWatchStride - 1) / kWatchStride;
    const int64_t n = (int64_t)nzs * nys * L.nxp * nfields;
    watchdog_kernel<<<grid_for(n, 256), 256, 0, stream>>>(field, L, nfields, nzs, nys, flags);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

// Converts the reduction keys into MediumStats in place (device side).
fd_status finish_medium_stats(MediumStats *dev_stats, cudaStream_t stream) {
    finish_stats_kernel<<<1, 1, 0, stream>>>(reinterpret_cast<StatsKeys *>(dev_stats));
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

}  // namespace fdsweep
