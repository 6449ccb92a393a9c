// noalloc.cu -- acoustic_forward_noalloc: the acoustic forward model for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaMallocAsync is not
// allowed or not wanted -- inside a host callback or a real-time loop whose
// memory budget is fixed up front, in a process whose device memory is owned
// by another allocator (a framework's caching pool that must not be bypassed),
// or in a service that must not fail with out-of-memory halfway through a
// request.  acoustic_forward allocates its workspace (padded wavefields, the b
// coefficient, sparse tables) on every call; this entry point instead keeps
// that workspace in one file-scope __device__ array of fixed size, so a call
// allocates nothing.
//
// Limits and rules (also stated in include/fdsweep.h):
//  * The scratch array holds FD_STATIC_SCRATCH_BYTES (64 MiB).  Every GPU that
//    loads this library holds it until the process exits.  A problem whose
//    workspace does not fit is rejected with FD_ERR_ARG before any launch.
//  * Every call reuses the same array; it keeps the previous call's contents,
//    so the call clears what must start at zero itself.  Calls whose work
//    overlaps on the GPU (different streams, or different host threads using
//    the same device) race on the array: serialise them.
//  * The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture.
//  * All pointers must be device memory (host buffers would need staging).
//    Work runs on the caller's stream with direct launches (no private
//    stream, no graph, no events); the call synchronises the stream at the
//    end, like acoustic_forward.
#include <math.h>
#include <string.h>

#include <mutex>

#include "kernels.cuh"
#include "runtime.cuh"

namespace fdsweep {

fd_status finish_medium_stats(MediumStats *dev_stats, cudaStream_t stream);

namespace {

// The fixed workspace.  Its host-side name is only a stand-in for the symbol:
// host code must use the address returned by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[FD_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

fd_status scratch_for_current_device(void **out) {
    int dev = 0;
    FD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(FD_ERR_ARG, "device index %d", dev);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return set_error(FD_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed on device %d: %s",
                             dev, cudaGetErrorString(e));
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return FD_OK;
}

// Bump layout inside the fixed array (256-byte aligned pieces).  Sizes are
// counted without overflow: a piece larger than the whole array saturates
// `used` beyond the array's size, so an oversized request is rejected rather
// than wrapped to a small number.
struct Carve {
    char *base;
    size_t used = 0;
    template <class T>
    T *take(uint64_t count) {
        const uint64_t cap = (uint64_t)FD_STATIC_SCRATCH_BYTES;
        used = (used + 255) / 256 * 256;
        T *p = reinterpret_cast<T *>(base + (used <= cap ? used : 0));
        const uint64_t bytes = count <= cap / sizeof(T) ? count * sizeof(T) : cap + 1;
        used = used <= cap ? used + (bytes > 0 ? bytes : 1) : used;
        return p;
    }
};

// Counts are non-negative ints and vol < 2^32 (checked first), so every
// product below fits in 64 bits.
size_t needed_bytes(const WaveLayout &L, int nshots, int nsrc, int nrec) {
    Carve c{nullptr};
    c.take<float>((uint64_t)2 * nshots * (uint64_t)L.vol);
    c.take<float>((uint64_t)L.vol);
    c.take<float>((uint64_t)L.nx + L.ny + L.nz);
    c.take<SparsePoint>((uint64_t)nshots * nsrc);
    c.take<SparsePoint>((uint64_t)nshots * nrec);
    c.take<MediumStats>(1);
    return c.used;
}

fd_status flags_status(unsigned int f) {
    if (f & DEV_ERR_TIMEOUT) return set_error(FD_ERR_TIMEOUT, "a device-side wait ran out");
    if (f & DEV_ERR_COORD) return set_error(FD_ERR_COORD, "a sparse point lies outside the grid");
    if (f & DEV_ERR_MEDIUM)
        return set_error(FD_ERR_ARG, "medium out of range (need finite m > 0, damp >= 0)");
    if (f & DEV_ERR_NONFINITE) return set_error(FD_ERR_DIVERGED, "the wavefield became non-finite");
    return FD_OK;
}

fd_status noalloc_impl(const fd_grid *g, int so, double dt, int nt, int nshots, const float *m,
                       const float *damp, int nsrc, const float *src_xyz, const float *src_wav,
                       int nrec, const float *rec_xyz, float *rec_out, const float *u_init,
                       float *u_final, cudaStream_t s) {
    FD_TRY(validate_common(g, so, dt, nt, nshots, m, nsrc, src_xyz, src_wav, nrec, rec_xyz,
                           rec_out));
    for (const void *p : {(const void *)m, (const void *)damp, (const void *)src_xyz,
                          (const void *)src_wav, (const void *)rec_xyz, (const void *)rec_out,
                          (const void *)u_init, (const void *)u_final})
        if (p && !is_device_pointer(p))
            return set_error(FD_ERR_ARG,
                             "acoustic_forward_noalloc takes device pointers of the current "
                             "device only");
    const int R = so / 2;
    const WaveLayout L = wave_layout(*g);
    const size_t need = needed_bytes(L, nshots, nsrc, nrec);
    if (need > (size_t)FD_STATIC_SCRATCH_BYTES)
        return set_error(FD_ERR_ARG,
                         "acoustic_forward_noalloc: the problem needs %zu bytes of scratch, the "
                         "static scratch holds %zu (FD_STATIC_SCRATCH_BYTES)",
                         need, (size_t)FD_STATIC_SCRATCH_BYTES);
    void *base = nullptr;
    FD_TRY(scratch_for_current_device(&base));
    Carve c{static_cast<char *>(base)};
    float *wave = c.take<float>((size_t)2 * nshots * L.vol);
    float *bcoef = c.take<float>(L.vol);
    float *dps = c.take<float>(L.nx + L.ny + L.nz);
    SparsePoint *src_tab = c.take<SparsePoint>((size_t)nshots * nsrc);
    SparsePoint *rec_tab = c.take<SparsePoint>((size_t)nshots * nrec);
    MediumStats *dstats = c.take<MediumStats>(1);
    const size_t dense = (size_t)L.nx * L.ny * L.nz;

    // setup: the scratch keeps the previous call's data, so zero what the
    // kernels expect to start at zero (b padding, wavefields)
    FD_CUDA_TRY(cudaMemsetAsync(bcoef, 0, (size_t)L.vol * 4, s));
    FD_TRY(init_medium_stats(dstats, s));
    FD_TRY(setup_acoustic_coeffs(m, damp, dt, L, bcoef, dps, dstats, s));
    for (int sh = 0; sh < nshots; ++sh) {
        FD_TRY(setup_sparse_table(src_xyz ? src_xyz + (size_t)sh * nsrc * 3 : nullptr, nsrc, *g, L,
                                  src_tab + (size_t)sh * nsrc, &dstats->flags, s));
        FD_TRY(setup_sparse_table(rec_xyz ? rec_xyz + (size_t)sh * nrec * 3 : nullptr, nrec, *g, L,
                                  rec_tab + (size_t)sh * nrec, &dstats->flags, s));
    }
    FD_TRY(finish_medium_stats(dstats, s));
    MediumStats hs;
    FD_CUDA_TRY(cudaMemcpyAsync(&hs, dstats, sizeof(hs), cudaMemcpyDeviceToHost, s));
    FD_CUDA_TRY(cudaStreamSynchronize(s));
    FD_TRY(flags_status(hs.flags));
    const double dt_max = acoustic_dt_bound(*g, R, (double)hs.m_min);
    if (dt > dt_max * (1.0 + 1e-12))
        return set_error(FD_ERR_CFL, "dt = %.6g ms exceeds the stability bound %.6g ms", dt, dt_max);

    FD_CUDA_TRY(cudaMemsetAsync(wave, 0, (size_t)2 * nshots * L.vol * 4, s));
    if (u_init)
        for (int sh = 0; sh < nshots; ++sh)
            for (int l = 0; l < 2; ++l)
                FD_CUDA_TRY(cudaMemcpy2DAsync(wave + (int64_t)(2 * sh + l) * L.vol,
                                              (size_t)L.nxp * 4,
                                              u_init + ((size_t)sh * 2 + l) * dense,
                                              (size_t)L.nx * 4, (size_t)L.nx * 4,
                                              (size_t)L.ny * L.nz, cudaMemcpyDeviceToDevice, s));

    AcousticPlan plan;
    FD_TRY(acoustic_plan(R, acoustic_step_config(R), L, nshots, 2, wave, bcoef, &plan));
    AcousticStepArgs a;
    memset(&a, 0, sizeof(a));
    a.wave = wave;
    a.bcoef = bcoef;
    a.dpx = dps;
    a.dpy = dps + L.nx;
    a.dpz = dps + L.nx + L.ny;
    a.L = L;
    a.nshots = nshots;
    a.err = &dstats->flags;
    laplacian_weights(*g, R, &a.wc, a.wx, a.wy, a.wz);
    SparseArgs sp;
    memset(&sp, 0, sizeof(sp));
    sp.wave = wave;
    sp.fields_per_shot = 2;
    sp.L = L;
    sp.bcoef = bcoef;
    sp.nshots = nshots;
    sp.nt = nt;
    sp.nsrc = nsrc;
    sp.src_tab = src_tab;
    sp.src_wav = src_wav;
    sp.inj_level1 = -1;
    sp.inj_t0 = 0;
    sp.inj_dt = 1;
    sp.rec_t0 = 0;
    sp.rec_dt = 1;
    sp.nrec = nrec;
    sp.rec_tab = rec_tab;
    sp.rec_out = rec_out;
    sp.step_base = nullptr;
    // the schedule of acoustic_forward: up to kInjectMaxSources sources per
    // shot are injected by the stencil kernel itself, in source order
    const bool inject_in_k1 = nsrc > 0 && nsrc <= kInjectMaxSources;
    AcousticInject inj;
    memset(&inj, 0, sizeof(inj));
    if (inject_in_k1) {
        inj.src_tab = src_tab;
        inj.src_wav = src_wav;
        inj.nsrc = nsrc;
        inj.nt = nt;
    }
    for (int n = 0; n + 1 < nt; ++n) {
        set_two_levels(a, n & 1);
        inj.step = n;
        FD_TRY(acoustic_launch(plan, a, s, &inj));
        sp.inj_level0 = 1 - (n & 1);
        sp.rec_level = n & 1;
        FD_TRY(sparse_launch(sp, n, nsrc > 0 && !inject_in_k1, nrec > 0, s));
    }
    const int last = (nt - 1) & 1;
    sp.rec_level = last;
    FD_TRY(sparse_launch(sp, nt - 1, false, nrec > 0, s));
    FD_TRY(check_finite(wave, L, 2 * nshots, &dstats->flags, s));
    if (u_final)
        for (int sh = 0; sh < nshots; ++sh)
            for (int l = 0; l < 2; ++l) {
                const int lev = l == 0 ? last : 1 - last;
                FD_CUDA_TRY(cudaMemcpy2DAsync(u_final + ((size_t)sh * 2 + l) * dense,
                                              (size_t)L.nx * 4,
                                              wave + (int64_t)(2 * sh + lev) * L.vol,
                                              (size_t)L.nxp * 4, (size_t)L.nx * 4,
                                              (size_t)L.ny * L.nz, cudaMemcpyDeviceToDevice, s));
            }
    FD_CUDA_TRY(cudaMemcpyAsync(&hs, dstats, sizeof(hs), cudaMemcpyDeviceToHost, s));
    FD_CUDA_TRY(cudaStreamSynchronize(s));
    return flags_status(hs.flags);
}

}  // namespace
}  // namespace fdsweep

extern "C" fd_status acoustic_forward_noalloc(const fd_grid *grid, int so, double dt, int nt,
                                              int nshots, const float *m, const float *damp,
                                              int nsrc, const float *src_xyz,
                                              const float *src_wav, int nrec,
                                              const float *rec_xyz, float *rec_out,
                                              const float *u_init, float *u_final, void *stream) {
    fdsweep::clear_error();
    return fdsweep::noalloc_impl(grid, so, dt, nt, nshots, m, damp, nsrc, src_xyz, src_wav, nrec,
                                 rec_xyz, rec_out, u_init, u_final,
                                 static_cast<cudaStream_t>(stream));
}
