// tti_stencil.cuh -- first-derivative building blocks shared by the TTI
// kernels (two-pass, fused and recompute schemes): tap tables t[d + R] for
// offsets d = -R..R (centred, forward- or backward-staggered), float4 cells
// of four consecutive x points, and the z accumulator pipeline.
#pragma once

#include "common.cuh"

namespace fdsweep {
namespace tti {

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 f4fma(float w, float4 a, float4 c) {
    return make_float4(fmaf(w, a.x, c.x), fmaf(w, a.y, c.y), fmaf(w, a.z, c.z), fmaf(w, a.w, c.w));
}
__device__ __forceinline__ float4 lds4(const float *p) {
    return *reinterpret_cast<const float4 *>(p);
}

// Stencil kinds: 0 centred (taps -R..R without the centre), +1 forward-
// staggered D+ (taps -R+1..R), -1 backward-staggered D- (taps -R..R-1).
template <int KIND>
__host__ __device__ constexpr bool tap_used(int d, int R) {
    return KIND == 0 ? d != 0 : (KIND > 0 ? d > -R : d < R);
}

// First derivative along x of 4 consecutive points from a row that starts RA
// points left of them: sum_d t[d + R] q[d].
template <int R, int RA, int KIND>
__device__ __forceinline__ float4 dx4(const float *row, const float *t) {
    float xs[2 * RA + 4];
#pragma unroll
    for (int i = 0; i < (2 * RA + 4) / 4; ++i) {
        const float4 f = lds4(row + 4 * i);
        xs[4 * i] = f.x;
        xs[4 * i + 1] = f.y;
        xs[4 * i + 2] = f.z;
        xs[4 * i + 3] = f.w;
    }
    float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = -R; k <= R; ++k) {
        if (!tap_used<KIND>(k, R)) continue;
        const float w = t[k + R];
        d.x = fmaf(w, xs[RA + 0 + k], d.x);
        d.y = fmaf(w, xs[RA + 1 + k], d.y);
        d.z = fmaf(w, xs[RA + 2 + k], d.z);
        d.w = fmaf(w, xs[RA + 3 + k], d.w);
    }
    return d;
}

// First derivative along y: `centre` points at the thread's float4 in the
// centre row, rows `pitch` floats apart.
template <int R, int KIND>
__device__ __forceinline__ float4 dy4(const float *centre, int pitch, const float *t) {
    float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = -R; k <= R; ++k) {
        if (!tap_used<KIND>(k, R)) continue;
        d = f4fma(t[k + R], lds4(centre + k * pitch), d);
    }
    return d;
}

// z first-derivative accumulator pipeline: acc[i] is output plane p-R+i when
// plane p arrives with values c (plane p is at offset R - i from it); acc[0]
// is then complete.
template <int R, int KIND>
__device__ __forceinline__ void dz_feed(float4 (&acc)[2 * R], float4 c, const float *t) {
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) {
        if (!tap_used<KIND>(R - i, R)) continue;
        acc[i] = f4fma(t[2 * R - i], c, acc[i]);
    }
}
// rotate: the new last entry is output p+R, for which plane p is offset -R
template <int R, int KIND>
__device__ __forceinline__ void dz_shift(float4 (&acc)[2 * R], float4 c, const float *t) {
#pragma unroll
    for (int i = 0; i < 2 * R - 1; ++i) acc[i] = acc[i + 1];
    const float w = tap_used<KIND>(-R, R) ? t[0] : 0.f;
    acc[2 * R - 1] = make_float4(w * c.x, w * c.y, w * c.z, w * c.w);
}

}  // namespace tti
}  // namespace fdsweep
