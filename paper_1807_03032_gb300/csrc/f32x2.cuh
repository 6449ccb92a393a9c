// f32x2.cuh -- packed FP32 pair arithmetic shared by the acoustic stencil
// kernels (single-step K1 and the two-step time-tiled kernel), so that both
// evaluate the update with the same operations in the same order.
#pragma once

#include <stdint.h>

namespace fdsweep {
namespace f32x2 {

// Packed FP32 pairs: Blackwell executes fma/add/sub/mul.rn.f32x2 on a 64-bit
// register pair as two independently rounded FP32 operations, so results are
// bit-identical to the scalar forms at half the instruction count.
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float f2_lo(f2 v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo;
}
__device__ __forceinline__ float f2_hi(f2 v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return hi;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_splat(float w) { return f2_pack(w, w); }

// Four consecutive x points as two packed pairs.
struct Q4 {
    f2 lo, hi;
};
__device__ __forceinline__ Q4 lds_q4(const float *p) {
    const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(p);
    return Q4{t.x, t.y};
}

}  // namespace f32x2
}  // namespace fdsweep
