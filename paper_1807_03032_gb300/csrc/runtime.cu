// runtime.cu -- host runtime of the fdsweep library: per-thread error
// messages, kernel-timing statistics, TMA descriptor encoding through the
// driver entry point (no link-time dependency on libcuda), pointer
// classification and the stream-ordered workspace.
#include <cudaTypedefs.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "runtime.cuh"

namespace fdsweep {

namespace {
thread_local char g_last_error[1024] = "";

struct StatEntry {
    double total_ms = 0.0;
    int64_t launches = 0;
    double points_per_launch = 0.0;
};
std::mutex g_stats_mu;
std::map<std::string, StatEntry> g_stats;
bool g_stats_on = false;
}  // namespace

namespace {
std::atomic<int64_t> g_launches{0};
thread_local int64_t t_captured = 0;
}  // namespace

void note_launch(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive)
        ++t_captured;
    else
        g_launches.fetch_add(1, std::memory_order_relaxed);
}

int64_t take_captured() {
    const int64_t n = t_captured;
    t_captured = 0;
    return n;
}

void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

fd_status set_error(fd_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

void clear_error() { g_last_error[0] = '\0'; }

const char *last_error() { return g_last_error; }

bool stats_enabled() {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    return g_stats_on;
}

void stats_add(const char *family, double ms, int64_t launches, double points_per_launch) {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    StatEntry &e = g_stats[family];
    e.total_ms += ms;
    e.launches += launches;
    e.points_per_launch = points_per_launch;
}

fd_status stats_enable(int on) {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    g_stats_on = on != 0;
    return FD_OK;
}

fd_status stats_reset() {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    g_stats.clear();
    return FD_OK;
}

fd_status stats_get(const char *family, double *total_ms, int64_t *launches,
                    double *points_per_launch) {
    if (!family) return set_error(FD_ERR_ARG, "fd_stats_get: null family");
    std::lock_guard<std::mutex> lk(g_stats_mu);
    static const char *known[] = {"acoustic_step", "acoustic_step2", "acoustic_step_h",
                                  "tti_pass1",     "tti_pass2",      "tti_recompute",
                                  "tti_fused",     "sparse"};
    bool ok = false;
    for (const char *k : known) ok = ok || strcmp(k, family) == 0;
    if (!ok) return set_error(FD_ERR_ARG, "fd_stats_get: unknown family '%s'", family);
    auto it = g_stats.find(family);
    StatEntry e = it == g_stats.end() ? StatEntry{} : it->second;
    if (total_ms) *total_ms = e.total_ms;
    if (launches) *launches = e.launches;
    if (points_per_launch) *points_per_launch = e.points_per_launch;
    return FD_OK;
}

fd_status make_tensor_map_4d(CUtensorMap *map, const float *base, uint64_t nx, uint64_t ny,
                             uint64_t nz, uint64_t nw, uint64_t stride_y_bytes,
                             uint64_t stride_z_bytes, uint64_t stride_w_bytes, uint32_t box_x,
                             uint32_t box_y, uint32_t box_z, uint32_t box_w) {
    return make_tensor_map_4d_elem(map, base, 4, nx, ny, nz, nw, stride_y_bytes, stride_z_bytes,
                                   stride_w_bytes, box_x, box_y, box_z, box_w);
}

fd_status make_tensor_map_4d_elem(CUtensorMap *map, const void *base, int elem_bytes,
                                  uint64_t nx, uint64_t ny, uint64_t nz, uint64_t nw,
                                  uint64_t stride_y_bytes, uint64_t stride_z_bytes,
                                  uint64_t stride_w_bytes, uint32_t box_x, uint32_t box_y,
                                  uint32_t box_z, uint32_t box_w) {
    if (elem_bytes != 4 && elem_bytes != 2)
        return set_error(FD_ERR_ARG, "tensor map: element size %d not supported", elem_bytes);
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    static cudaError_t lookup_err = cudaSuccess;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        lookup_err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                      cudaEnableDefault, &q);
        if (lookup_err == cudaSuccess && q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!encode)
        return set_error(FD_ERR_CUDA, "cuTensorMapEncodeTiled not available (%s)",
                         cudaGetErrorString(lookup_err));
    cuuint64_t dims[4] = {nx, ny, nz, nw};
    cuuint64_t strides[3] = {stride_y_bytes, stride_z_bytes, stride_w_bytes};
    cuuint32_t box[4] = {box_x, box_y, box_z, box_w};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dtype =
        elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    CUresult r = encode(map, dtype, 4, const_cast<void *>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(FD_ERR_CUDA,
                         "cuTensorMapEncodeTiled failed (%d): dims %llu %llu %llu %llu box %u %u",
                         (int)r, (unsigned long long)nx, (unsigned long long)ny,
                         (unsigned long long)nz, (unsigned long long)nw, box_x, box_y);
    return FD_OK;
}

int trace_level() {
    static int level = [] {
        const char *e = getenv("FDSWEEP_TRACE");
        return e ? atoi(e) : 0;
    }();
    return level;
}

fd_status trace_stage(cudaStream_t s, const char *stage) {
    const int lvl = trace_level();
    if (lvl <= 0) return FD_OK;
    fprintf(stderr, "[fdsweep] %s\n", stage);
    fflush(stderr);
    if (lvl >= 2) {
        // host time from the previous synchronised stage to the end of this
        // one (the stage's device work included)
        thread_local std::chrono::steady_clock::time_point last;
        cudaError_t e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess)
            return set_error(FD_ERR_CUDA, "after stage '%s': %s", stage, cudaGetErrorString(e));
        const auto now = std::chrono::steady_clock::now();
        const double ms =
            last.time_since_epoch().count() == 0
                ? 0.0
                : std::chrono::duration<double, std::milli>(now - last).count();
        last = now;
        fprintf(stderr, "[fdsweep] %s: ok (+%.3f ms)\n", stage, ms);
        fflush(stderr);
    }
    return FD_OK;
}

fd_status raise_smem_limit(const void *fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> limit;
    int dev = 0;
    FD_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = limit[std::make_pair(dev, fn)];
    if (bytes > cur) {
        FD_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes));
        cur = bytes;
    }
    return FD_OK;
}

bool is_device_pointer(const void *p) {
    if (!p) return true;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (attr.type == cudaMemoryTypeManaged) return true;
    if (attr.type != cudaMemoryTypeDevice) return false;
    // device memory of another GPU is not this call's to dereference
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.device == dev;
}

// ------------------------------------------------------------------ workspace

Workspace::~Workspace() { release(); }

void Workspace::add_raw(void **slot, size_t bytes) {
    total_ = (total_ + 255) / 256 * 256;
    if (npieces_ < 64) pieces_[npieces_++] = Piece{slot, total_};
    *slot = nullptr;
    total_ += bytes > 0 ? bytes : 1;
}

// ------------------------------------------------------------------ fault injection

bool simulated_alloc_failure() {
    const char *v = getenv("FDSWEEP_FAIL_ALLOC");
    return v && v[0] == '1';
}

namespace {
std::atomic<uint64_t> g_wait_limit_ns{0};
}  // namespace

uint64_t wait_limit_ns() { return g_wait_limit_ns.load(std::memory_order_relaxed); }
void set_wait_limit_ns(uint64_t ns) { g_wait_limit_ns.store(ns, std::memory_order_relaxed); }

fd_status Workspace::allocate(cudaStream_t s) {
    stream_ = s;
    if (npieces_ >= 64) return set_error(FD_ERR_ARG, "workspace: too many pieces");
    static std::once_flag once;
    std::call_once(once, [] {
        // Keep freed workspace in the stream-ordered pool instead of returning
        // it to the driver at every synchronisation.
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    });
    if (total_ == 0) return FD_OK;
    cudaError_t e = simulated_alloc_failure() ? cudaErrorMemoryAllocation
                                              : cudaMallocAsync(&base_, total_, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        base_ = nullptr;
        return set_error(e == cudaErrorMemoryAllocation ? FD_ERR_OOM : FD_ERR_CUDA,
                         "workspace allocation of %zu bytes failed: %s", total_,
                         cudaGetErrorString(e));
    }
    for (int i = 0; i < npieces_; ++i)
        *pieces_[i].slot = static_cast<char *>(base_) + pieces_[i].offset;
    return FD_OK;
}

void Workspace::release() {
    if (base_) {
        cudaFreeAsync(base_, stream_);
        base_ = nullptr;
    }
}

// ------------------------------------------------------------------ call stream

CallStream::~CallStream() {
    if (done_) cudaEventDestroy(done_);
}

fd_status CallStream::begin(cudaStream_t caller) {
    caller_ = caller;
    thread_local cudaStream_t own = nullptr;
    thread_local int own_dev = -1;
    int dev = 0;
    FD_CUDA_TRY(cudaGetDevice(&dev));
    if (!own || own_dev != dev) {
        FD_CUDA_TRY(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
        own_dev = dev;
    }
    s_ = own;
    cudaEvent_t ready;
    FD_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    cudaError_t e1 = cudaEventRecord(ready, caller_);
    cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(s_, ready, 0) : e1;
    cudaEventDestroy(ready);
    FD_CUDA_TRY(e2);
    FD_CUDA_TRY(cudaEventCreateWithFlags(&done_, cudaEventDisableTiming));
    return FD_OK;
}

SideLane::~SideLane() {
    if (f_) cudaEventDestroy(f_);
    if (j_) cudaEventDestroy(j_);
}

fd_status SideLane::begin() {
    thread_local cudaStream_t own[2] = {nullptr, nullptr};
    thread_local int own_dev[2] = {-1, -1};
    const int l = lane_ ? 1 : 0;
    int dev = 0;
    FD_CUDA_TRY(cudaGetDevice(&dev));
    if (!own[l] || own_dev[l] != dev) {
        FD_CUDA_TRY(cudaStreamCreateWithFlags(&own[l], cudaStreamNonBlocking));
        own_dev[l] = dev;
    }
    s_ = own[l];
    FD_CUDA_TRY(cudaEventCreateWithFlags(&f_, cudaEventDisableTiming));
    FD_CUDA_TRY(cudaEventCreateWithFlags(&j_, cudaEventDisableTiming));
    return FD_OK;
}

fd_status SideLane::fork(cudaStream_t from) {
    FD_CUDA_TRY(cudaEventRecord(f_, from));
    FD_CUDA_TRY(cudaStreamWaitEvent(s_, f_, 0));
    return FD_OK;
}

fd_status SideLane::join(cudaStream_t into) {
    FD_CUDA_TRY(cudaEventRecord(j_, s_));
    FD_CUDA_TRY(cudaStreamWaitEvent(into, j_, 0));
    return FD_OK;
}

fd_status CallStream::finish() {
    FD_CUDA_TRY(cudaEventRecord(done_, s_));
    FD_CUDA_TRY(cudaStreamWaitEvent(caller_, done_, 0));
    return FD_OK;
}

}  // namespace fdsweep
