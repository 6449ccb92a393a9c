// runtime.cuh -- host runtime pieces shared by the entry points.
#pragma once

#include "common.cuh"

namespace fdsweep {

const char *last_error();
fd_status stats_enable(int on);
fd_status stats_reset();
fd_status stats_get(const char *family, double *total_ms, int64_t *launches,
                    double *points_per_launch);

// Debug tracing, controlled by the FDSWEEP_TRACE environment variable:
// 1 prints each stage of a call to stderr, 2 also synchronises after every
// stage (and disables graph capture) so that a device error is reported at the
// stage that caused it.
int trace_level();
fd_status trace_stage(cudaStream_t s, const char *stage);
#define FD_STAGE(stream, name) FD_TRY(::fdsweep::trace_stage((stream), (name)))

// make_tensor_map_4d for 4-byte (FP32) or 2-byte (IEEE binary16) elements.
fd_status make_tensor_map_4d_elem(CUtensorMap *map, const void *base, int elem_bytes,
                                  uint64_t nx, uint64_t ny, uint64_t nz, uint64_t nw,
                                  uint64_t stride_y_bytes, uint64_t stride_z_bytes,
                                  uint64_t stride_w_bytes, uint32_t box_x, uint32_t box_y,
                                  uint32_t box_z, uint32_t box_w);

// Raises a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`, never lowering it: the limit belongs to the function and is
// shared by every thread and call, so one call must not lower the limit
// another call is about to launch with (concurrent calls from host threads).
fd_status raise_smem_limit(const void *fn, size_t bytes);

// Host-side fault injection for tests: with the environment variable
// FDSWEEP_FAIL_ALLOC=1 every device allocation of the library (per-call
// workspaces, batch engines) fails as if the device were out of memory, and
// the call returns FD_ERR_OOM without launching anything.
bool simulated_alloc_failure();
void set_wait_limit_ns(uint64_t ns);

// True for managed memory, for device memory of the current device and for
// null; false for host memory and for another device's memory (which the
// entry points that accept host buffers stage like host memory, and the
// device-only entry points reject).
bool is_device_pointer(const void *p);

// One stream-ordered device allocation per call, carved into 256-byte aligned
// pieces.  Pieces are declared first (add), then allocate() assigns every
// declared pointer; the block is released (cudaFreeAsync) when the object goes
// out of scope.
class Workspace {
  public:
    ~Workspace();
    template <class T>
    void add(T **slot, size_t count) {
        add_raw(reinterpret_cast<void **>(slot), count * sizeof(T));
    }
    void add_raw(void **slot, size_t bytes);
    fd_status allocate(cudaStream_t s);
    size_t bytes() const { return total_; }
    void release();

  private:
    struct Piece {
        void **slot;
        size_t offset;
    };
    Piece pieces_[64];
    int npieces_ = 0;
    size_t total_ = 0;
    void *base_ = nullptr;
    cudaStream_t stream_ = nullptr;
};

// The library's own non-blocking stream for one call, ordered after the work
// already queued on the caller's stream (and the caller's stream after it).
// Keeping a private stream lets the time loop be captured into a CUDA graph
// even when the caller passes the legacy default stream.
class CallStream {
  public:
    ~CallStream();
    fd_status begin(cudaStream_t caller);
    fd_status finish();
    cudaStream_t get() const { return s_; }

  private:
    cudaStream_t caller_ = nullptr, s_ = nullptr;
    cudaEvent_t done_ = nullptr;
};

// A second (thread-local, non-blocking) stream for work that may overlap the
// call stream's kernels, forked from and joined back into it with events, so
// that the dependencies are also captured when the call stream is being
// recorded into a CUDA graph.
class SideLane {
  public:
    explicit SideLane(int lane = 0) : lane_(lane) {}
    ~SideLane();
    fd_status begin();
    cudaStream_t get() const { return s_; }
    fd_status fork(cudaStream_t from);  // side waits for the work queued on `from`
    fd_status join(cudaStream_t into);  // `into` waits for the work queued on side

  private:
    int lane_ = 0;  // 0 or 1: distinct thread-local streams
    cudaStream_t s_ = nullptr;
    cudaEvent_t f_ = nullptr, j_ = nullptr;
};

}  // namespace fdsweep
