// common.cuh -- shared host/device helpers of the fdsweep CUDA library:
// status/error plumbing, hand-written PTX wrappers for mbarrier and the
// tensor-memory-accelerator (TMA) bulk tensor copy, and small device utilities.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fdsweep.h"

namespace fdsweep {

// ------------------------------------------------------------------ host side

// Records `msg` as the calling thread's last error and returns `st`.
fd_status set_error(fd_status st, const char *fmt, ...);
void clear_error();

#define FD_CUDA_TRY(expr)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            return ::fdsweep::set_error(e_ == cudaErrorMemoryAllocation ? FD_ERR_OOM       \
                                                                        : FD_ERR_CUDA,     \
                                        "%s failed: %s (%s:%d)", #expr,                    \
                                        cudaGetErrorString(e_), __FILE__, __LINE__);       \
        }                                                                                  \
    } while (0)

#define FD_TRY(expr)                          \
    do {                                      \
        fd_status s_ = (expr);                \
        if (s_ != FD_OK) return s_;           \
    } while (0)

// Device-side error bits (written with atomicOr into a device word).
enum : unsigned int {
    DEV_ERR_TIMEOUT = 1u,     // a bounded mbarrier wait ran out
    DEV_ERR_COORD = 2u,       // a sparse point lies outside the grid
    DEV_ERR_MEDIUM = 4u,      // m <= 0 or non-finite, damp < 0, eps < delta, ...
    DEV_ERR_NONFINITE = 8u,   // a wavefield became non-finite
};

// Builds a TMA descriptor for a 4-D FP32 tensor (x, y, z, w) with x
// contiguous; strides in bytes for dims 1..3.  Out-of-range elements of a
// box read as zero.
fd_status make_tensor_map_4d(CUtensorMap *map, const float *base, uint64_t nx, uint64_t ny,
                             uint64_t nz, uint64_t nw, uint64_t stride_y_bytes,
                             uint64_t stride_z_bytes, uint64_t stride_w_bytes, uint32_t box_x,
                             uint32_t box_y, uint32_t box_z, uint32_t box_w);

// Launch accounting (fd_launch_count): call note_launch(stream) after every
// kernel launch.  Launches recorded while the stream is being captured are
// counted when the graph is replayed (take_captured / add_launches).
void note_launch(cudaStream_t s);
int64_t take_captured();
void add_launches(int64_t n);
int64_t launch_count();

// Kernel-timing statistics (see fd_stats_* in fdsweep.h).
bool stats_enabled();
void stats_add(const char *family, double ms, int64_t launches, double points_per_launch);

// ------------------------------------------------------------------ device side

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Non-blocking test of an mbarrier phase.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: gives up after `limit_ns` nanoseconds
// and returns false (the caller records DEV_ERR_TIMEOUT and unwinds).  A
// limit of 1 ns or less makes it a single non-blocking test (the
// failure-injection setting of fd_set_wait_limit_ns).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns = 2000000000ull) {
    if (limit_ns <= 1) return mbar_test_wait(bar, parity);
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    uint32_t spins = 0;
    while (!mbar_try_wait(bar, parity)) {
        if ((++spins & 255u) == 0 && global_timer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// TMA tiled load of a 4-D box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z, int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ float4 ld_nc_f4(const float *p) {
    return __ldg(reinterpret_cast<const float4 *>(p));
}

}  // namespace fdsweep
