// runtime.cuh -- host runtime pieces shared by the entry points.
#pragma once

#include "common.cuh"

namespace fdsweep {

const char *last_error();
fd_status stats_enable(int on);
fd_status stats_reset();
fd_status stats_get(const char *family, double *total_ms, int64_t *launches,
                    double *points_per_launch);

// True for device or managed memory (and for null); false for host memory.
bool is_device_pointer(const void *p);

// One stream-ordered device allocation per call, carved into 256-byte aligned
// pieces; released (cudaFreeAsync) when the object goes out of scope.
class Workspace {
  public:
    ~Workspace();
    void reserve(size_t bytes);
    fd_status allocate(cudaStream_t s);
    void *take(size_t bytes);
    template <class T>
    T *take_n(size_t n) {
        return static_cast<T *>(take(n * sizeof(T)));
    }
    void release();

  private:
    size_t total_ = 0, cursor_ = 0;
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

}  // namespace fdsweep
