// engine.cu -- a batch engine for serving: shots that share a velocity model
// (grid, m, damp, so, dt) are slots of one engine and advance together, one
// launch of the stencil kernel per time step over all active slots (the shot
// is the outer dimension).  Every slot carries its own start step, so a shot
// can join while others are mid-run: at the global step G a slot that started
// at t0 is at its own time index n = G - t0, and the sparse kernel injects
// its wavelet sample n and records its trace sample n.  A slot added at G
// starts from the zero state like a standalone forward run, so its traces are
// those of acoustic_forward for the same shot.
//
// Each engine owns a non-blocking stream, so the engines of different models
// run concurrently on the device.  Memory is allocated once, at creation
// (the serving layer admits engines by this footprint); adding a shot,
// stepping and releasing allocate nothing.  Chunks of steps are captured into
// a CUDA graph and replayed while the set of active slots is unchanged.
#include <math.h>
#include <string.h>

#include <vector>

#include "kernels.cuh"
#include "runtime.cuh"

namespace fdsweep {

fd_status finish_medium_stats(MediumStats *dev_stats, cudaStream_t stream);

namespace {

struct SlotDesc {
    int t0, nt, nsrc, nrec;
    const float *wav;  // [nt][nsrc]
    float *out;        // [nt][nrec]
};

struct EngineSparseArgs {
    float *wave;  // [max_slots][2][vol]
    WaveLayout L;
    const float *bcoef;
    const SlotDesc *desc;
    const int *slot_map;
    const SparsePoint *src_tab, *rec_tab;  // [max_slots][max_nsrc], [max_slots][max_nrec]
    int max_nsrc, max_nrec, nactive;
    const int *gstep;
};

__device__ __forceinline__ int64_t corner_off(const SparsePoint &p, int c, const WaveLayout &L) {
    return (int64_t)p.base + ((c & 1) ? 1 : 0) + ((c & 2) ? L.nxp : 0) + ((c & 4) ? L.plane : 0);
}
__device__ __forceinline__ float corner_w(const SparsePoint &p, int c) {
    return ((c & 1) ? p.fx : 1.f - p.fx) * ((c & 2) ? p.fy : 1.f - p.fy) *
           ((c & 4) ? p.fz : 1.f - p.fz);
}

// Threads [0, nactive*max_nrec) record traces; then nactive*max_nsrc*8 inject.
__global__ void engine_sparse_kernel(const EngineSparseArgs e, int offset, int cur) {
    const int G = *e.gstep + offset;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nrec_all = (int64_t)e.nactive * e.max_nrec;
    if (gid < nrec_all) {
        const int si = (int)(gid / e.max_nrec);
        const int r = (int)(gid - (int64_t)si * e.max_nrec);
        const int slot = e.slot_map[si];
        const SlotDesc d = e.desc[slot];
        const int n = G - d.t0;
        if (r >= d.nrec || n < 0 || n >= d.nt) return;
        const SparsePoint p = e.rec_tab[(int64_t)slot * e.max_nrec + r];
        const float *u = e.wave + (int64_t)(2 * slot + cur) * e.L.vol;
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) acc = fmaf(corner_w(p, c), __ldg(u + corner_off(p, c, e.L)), acc);
        d.out[(int64_t)n * d.nrec + r] = acc;
        return;
    }
    const int64_t k = gid - nrec_all;
    if (k >= (int64_t)e.nactive * e.max_nsrc * 8) return;
    const int c = (int)(k & 7);
    const int64_t ps = k >> 3;
    const int si = (int)(ps / e.max_nsrc);
    const int s = (int)(ps - (int64_t)si * e.max_nsrc);
    const int slot = e.slot_map[si];
    const SlotDesc d = e.desc[slot];
    const int n = G - d.t0;
    if (s >= d.nsrc || n < 0 || n > d.nt - 2) return;
    const SparsePoint p = e.src_tab[(int64_t)slot * e.max_nsrc + s];
    const int64_t off = corner_off(p, c, e.L);
    const float q = d.wav[(int64_t)n * d.nsrc + s];
    atomicAdd(e.wave + (int64_t)(2 * slot + 1 - cur) * e.L.vol + off,
              corner_w(p, c) * __ldg(e.bcoef + off) * q);
}

__global__ void engine_bump(int *g, int by) { *g += by; }

}  // namespace

struct Engine {
    fd_grid grid;
    int so, R;
    double dt;
    WaveLayout L;
    int max_slots, max_nsrc, max_nrec;
    cudaStream_t stream = nullptr;
    void *base = nullptr;
    float *wave = nullptr, *bcoef = nullptr, *dps = nullptr;
    SparsePoint *src_tab = nullptr, *rec_tab = nullptr;
    SlotDesc *desc = nullptr;
    int *slot_map = nullptr, *gstep = nullptr;
    MediumStats *stats = nullptr;
    SlotDesc *h_desc = nullptr;  // pinned staging
    int *h_map = nullptr;        // pinned staging
    std::vector<int> active;     // per slot 0/1
    std::vector<int> t0, nt;
    int64_t G = 0;
    int version = 0, planned_version = -1, graph_version = -1, graph_steps = 0;
    AcousticPlan plan;
    AcousticStepArgs args;
    int nactive = 0;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_nodes = 0;
};

static size_t engine_bytes(const WaveLayout &L, int max_slots, int max_nsrc, int max_nrec,
                           size_t *offs /* 9 entries or null */) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
        o = (o + 255) / 256 * 256;
        const size_t at = o;
        o += bytes > 0 ? bytes : 1;
        return at;
    };
    size_t v[9];
    v[0] = take((size_t)max_slots * 2 * L.vol * 4);                       // wave
    v[1] = take((size_t)L.vol * 4);                                       // b
    v[2] = take((size_t)(L.nx + L.ny + L.nz) * 4);                        // damping / dt
    v[3] = take((size_t)max_slots * max_nsrc * sizeof(SparsePoint));      // source tables
    v[4] = take((size_t)max_slots * max_nrec * sizeof(SparsePoint));      // receiver tables
    v[5] = take((size_t)max_slots * sizeof(SlotDesc));
    v[6] = take((size_t)max_slots * sizeof(int));                         // slot map
    v[7] = take(64);                                                      // global step
    v[8] = take(sizeof(MediumStats));
    if (offs) memcpy(offs, v, sizeof(v));
    return o;
}

static void destroy_engine(Engine *e) {
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->graph) cudaGraphExecDestroy(e->graph);
    if (e->base) cudaFree(e->base);
    if (e->h_desc) cudaFreeHost(e->h_desc);
    if (e->h_map) cudaFreeHost(e->h_map);
    if (e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

static fd_status engine_create(const fd_grid *g, int so, double dt, const float *m,
                               const float *damp, int max_slots, int max_nsrc, int max_nrec,
                               Engine **out) {
    if (!g || !out || !m) return set_error(FD_ERR_ARG, "fd_engine_create: null argument");
    FD_TRY(validate_common(g, so, dt, 1, 1, m, 0, nullptr, nullptr, 0, nullptr, nullptr));
    if (max_slots < 1 || max_nsrc < 0 || max_nrec < 0)
        return set_error(FD_ERR_ARG, "fd_engine_create: bad slot or sparse-point counts");
    if (!is_device_pointer(m) || (damp && !is_device_pointer(damp)))
        return set_error(FD_ERR_ARG, "fd_engine_create: m and damp must be device memory");
    Engine *e = new Engine();
    e->grid = *g;
    e->so = so;
    e->R = so / 2;
    e->dt = dt;
    e->L = wave_layout(*g);
    e->max_slots = max_slots;
    e->max_nsrc = max_nsrc;
    e->max_nrec = max_nrec;
    e->active.assign(max_slots, 0);
    e->t0.assign(max_slots, 0);
    e->nt.assign(max_slots, 0);
    auto fail = [&](fd_status st) {
        destroy_engine(e);
        return st;
    };
    cudaError_t ce = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return fail(set_error(FD_ERR_CUDA, "stream: %s", cudaGetErrorString(ce)));
    size_t off[9];
    const size_t bytes = engine_bytes(e->L, max_slots, max_nsrc, max_nrec, off);
    ce = simulated_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&e->base, bytes);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        e->base = nullptr;
        return fail(set_error(ce == cudaErrorMemoryAllocation ? FD_ERR_OOM : FD_ERR_CUDA,
                              "fd_engine_create: %zu bytes: %s", bytes, cudaGetErrorString(ce)));
    }
    char *b = static_cast<char *>(e->base);
    e->wave = reinterpret_cast<float *>(b + off[0]);
    e->bcoef = reinterpret_cast<float *>(b + off[1]);
    e->dps = reinterpret_cast<float *>(b + off[2]);
    e->src_tab = reinterpret_cast<SparsePoint *>(b + off[3]);
    e->rec_tab = reinterpret_cast<SparsePoint *>(b + off[4]);
    e->desc = reinterpret_cast<SlotDesc *>(b + off[5]);
    e->slot_map = reinterpret_cast<int *>(b + off[6]);
    e->gstep = reinterpret_cast<int *>(b + off[7]);
    e->stats = reinterpret_cast<MediumStats *>(b + off[8]);
    if (cudaMallocHost(&e->h_desc, sizeof(SlotDesc)) != cudaSuccess ||
        cudaMallocHost(&e->h_map, sizeof(int) * max_slots) != cudaSuccess) {
        cudaGetLastError();
        return fail(set_error(FD_ERR_OOM, "fd_engine_create: pinned staging"));
    }
    cudaStream_t s = e->stream;
    fd_status st;
#define ENGINE_TRY(x)                   \
    do {                                \
        st = (x);                       \
        if (st != FD_OK) return fail(st); \
    } while (0)
#define ENGINE_CUDA(x)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (x);                                                               \
        if (e_ != cudaSuccess)                                                              \
            return fail(set_error(FD_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)));     \
    } while (0)
    ENGINE_CUDA(cudaMemsetAsync(e->base, 0, bytes, s));
    ENGINE_TRY(init_medium_stats(e->stats, s));
    ENGINE_TRY(setup_acoustic_coeffs(m, damp, dt, e->L, e->bcoef, e->dps, e->stats, s));
    ENGINE_TRY(finish_medium_stats(e->stats, s));
    MediumStats hs;
    ENGINE_CUDA(cudaMemcpyAsync(&hs, e->stats, sizeof(hs), cudaMemcpyDeviceToHost, s));
    ENGINE_CUDA(cudaStreamSynchronize(s));
    if (hs.flags & DEV_ERR_MEDIUM)
        return fail(set_error(FD_ERR_ARG, "fd_engine_create: need finite m > 0 and damp >= 0"));
    const double dt_max = acoustic_dt_bound(*g, e->R, (double)hs.m_min);
    if (dt > dt_max * (1.0 + 1e-12))
        return fail(set_error(FD_ERR_CFL, "dt = %.6g ms exceeds the stability bound %.6g ms", dt,
                              dt_max));
    memset(&e->args, 0, sizeof(e->args));
    e->args.wave = e->wave;
    e->args.bcoef = e->bcoef;
    e->args.dpx = e->dps;
    e->args.dpy = e->dps + e->L.nx;
    e->args.dpz = e->dps + e->L.nx + e->L.ny;
    e->args.L = e->L;
    e->args.err = &e->stats->flags;
    e->args.slot_map = e->slot_map;
    laplacian_weights(*g, e->R, &e->args.wc, e->args.wx, e->args.wy, e->args.wz);
#undef ENGINE_TRY
#undef ENGINE_CUDA
    *out = e;
    return FD_OK;
}

static fd_status engine_add(Engine *e, int nt, int nsrc, const float *src_xyz,
                            const float *src_wav, int nrec, const float *rec_xyz, float *rec_out,
                            int *slot_out) {
    if (!e || !slot_out) return set_error(FD_ERR_ARG, "fd_engine_add_shot: null argument");
    if (nt < 1 || nsrc < 0 || nrec < 0 || nsrc > e->max_nsrc || nrec > e->max_nrec)
        return set_error(FD_ERR_ARG, "fd_engine_add_shot: nt, nsrc or nrec out of range");
    if ((nsrc > 0 && (!src_xyz || !src_wav)) || (nrec > 0 && (!rec_xyz || !rec_out)))
        return set_error(FD_ERR_ARG, "fd_engine_add_shot: null source or receiver array");
    for (const void *p : {(const void *)src_xyz, (const void *)src_wav, (const void *)rec_xyz,
                          (const void *)rec_out})
        if (p && !is_device_pointer(p))
            return set_error(FD_ERR_ARG, "fd_engine_add_shot: device pointers only");
    int slot = -1;
    for (int i = 0; i < e->max_slots; ++i)
        if (!e->active[i]) {
            slot = i;
            break;
        }
    if (slot < 0) return set_error(FD_ERR_ARG, "fd_engine_add_shot: no free slot");
    cudaStream_t s = e->stream;
    FD_CUDA_TRY(cudaMemsetAsync(e->wave + (int64_t)2 * slot * e->L.vol, 0,
                                (size_t)2 * e->L.vol * 4, s));
    FD_TRY(setup_sparse_table(src_xyz, nsrc, e->grid, e->L, e->src_tab + (int64_t)slot * e->max_nsrc,
                              &e->stats->flags, s));
    FD_TRY(setup_sparse_table(rec_xyz, nrec, e->grid, e->L, e->rec_tab + (int64_t)slot * e->max_nrec,
                              &e->stats->flags, s));
    // the staging buffer is reused: wait for its previous copy to be consumed
    FD_CUDA_TRY(cudaStreamSynchronize(s));
    *e->h_desc = SlotDesc{(int)e->G, nt, nsrc, nrec, src_wav, rec_out};
    FD_CUDA_TRY(cudaMemcpyAsync(e->desc + slot, e->h_desc, sizeof(SlotDesc),
                                cudaMemcpyHostToDevice, s));
    e->active[slot] = 1;
    e->t0[slot] = (int)e->G;
    e->nt[slot] = nt;
    ++e->version;
    *slot_out = slot;
    return FD_OK;
}

static fd_status engine_refresh(Engine *e) {
    if (e->planned_version == e->version) return FD_OK;
    int n = 0;
    for (int i = 0; i < e->max_slots; ++i)
        if (e->active[i]) e->h_map[n++] = i;
    e->nactive = n;
    if (n > 0) {
        FD_CUDA_TRY(cudaStreamSynchronize(e->stream));  // h_map reuse
        FD_CUDA_TRY(cudaMemcpyAsync(e->slot_map, e->h_map, sizeof(int) * n,
                                    cudaMemcpyHostToDevice, e->stream));
        // grid over the n active slots, tensor maps over all slots' buffers
        FD_TRY(acoustic_plan(e->R, -1, e->L, n, 2, e->wave, e->bcoef, &e->plan, e->max_slots));
    }
    e->planned_version = e->version;
    return FD_OK;
}

static fd_status engine_one_step(Engine *e, int offset, int cur) {
    AcousticStepArgs a = e->args;
    a.nshots = e->nactive;
    set_two_levels(a, cur);
    FD_TRY(acoustic_launch(e->plan, a, e->stream));
    EngineSparseArgs sp;
    sp.wave = e->wave;
    sp.L = e->L;
    sp.bcoef = e->bcoef;
    sp.desc = e->desc;
    sp.slot_map = e->slot_map;
    sp.src_tab = e->src_tab;
    sp.rec_tab = e->rec_tab;
    sp.max_nsrc = e->max_nsrc;
    sp.max_nrec = e->max_nrec;
    sp.nactive = e->nactive;
    sp.gstep = e->gstep;
    const int64_t total = (int64_t)e->nactive * (e->max_nrec + 8 * e->max_nsrc);
    if (total > 0) {
        engine_sparse_kernel<<<(unsigned)((total + 255) / 256), 256, 0, e->stream>>>(sp, offset, cur);
        FD_CUDA_TRY(cudaGetLastError());
        note_launch(e->stream);
    }
    return FD_OK;
}

static fd_status engine_step(Engine *e, int nsteps) {
    if (!e) return set_error(FD_ERR_ARG, "fd_engine_step: null engine");
    if (nsteps < 0 || (nsteps & 1))
        return set_error(FD_ERR_ARG, "fd_engine_step: nsteps must be even and >= 0");
    FD_TRY(engine_refresh(e));
    if (e->nactive == 0 || nsteps == 0) {
        e->G += nsteps;
        if (nsteps) {
            engine_bump<<<1, 1, 0, e->stream>>>(e->gstep, nsteps);
            FD_CUDA_TRY(cudaGetLastError());
            note_launch(e->stream);
        }
        return FD_OK;
    }
    const bool use_graph = nsteps >= 8 && trace_level() < 2;
    if (use_graph && !(e->graph && e->graph_version == e->version && e->graph_steps == nsteps)) {
        if (e->graph) {
            FD_CUDA_TRY(cudaStreamSynchronize(e->stream));
            cudaGraphExecDestroy(e->graph);
            e->graph = nullptr;
        }
        take_captured();
        cudaGraph_t gr = nullptr;
        FD_CUDA_TRY(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
        fd_status st = FD_OK;
        for (int i = 0; i < nsteps && st == FD_OK; ++i) st = engine_one_step(e, i, i & 1);
        if (st == FD_OK) {
            engine_bump<<<1, 1, 0, e->stream>>>(e->gstep, nsteps);
            note_launch(e->stream);
        }
        cudaError_t ce = cudaStreamEndCapture(e->stream, &gr);
        e->graph_nodes = take_captured();
        if (st != FD_OK) {
            if (gr) cudaGraphDestroy(gr);
            return st;
        }
        FD_CUDA_TRY(ce);
        ce = cudaGraphInstantiate(&e->graph, gr, 0);
        cudaGraphDestroy(gr);
        FD_CUDA_TRY(ce);
        e->graph_version = e->version;
        e->graph_steps = nsteps;
    }
    if (use_graph) {
        FD_CUDA_TRY(cudaGraphLaunch(e->graph, e->stream));
        add_launches(e->graph_nodes);
    } else {
        for (int i = 0; i < nsteps; ++i) FD_TRY(engine_one_step(e, i, i & 1));
        engine_bump<<<1, 1, 0, e->stream>>>(e->gstep, nsteps);
        FD_CUDA_TRY(cudaGetLastError());
        note_launch(e->stream);
    }
    e->G += nsteps;
    return FD_OK;
}

}  // namespace fdsweep

using fdsweep::Engine;

extern "C" {

struct fd_engine {
    Engine *impl;
};

fd_status fd_engine_footprint(const fd_grid *grid, int max_slots, int max_nsrc, int max_nrec,
                              int64_t *bytes) {
    fdsweep::clear_error();
    if (!grid || !bytes || max_slots < 1 || max_nsrc < 0 || max_nrec < 0)
        return fdsweep::set_error(FD_ERR_ARG, "fd_engine_footprint: bad argument");
    FD_TRY(fdsweep::validate_grid(grid));
    *bytes = (int64_t)fdsweep::engine_bytes(fdsweep::wave_layout(*grid), max_slots, max_nsrc,
                                            max_nrec, nullptr);
    return FD_OK;
}

fd_status fd_engine_create(const fd_grid *grid, int so, double dt, const float *m,
                           const float *damp, int max_slots, int max_nsrc, int max_nrec,
                           fd_engine **out) {
    fdsweep::clear_error();
    if (!out) return fdsweep::set_error(FD_ERR_ARG, "fd_engine_create: null out");
    Engine *e = nullptr;
    fd_status st = fdsweep::engine_create(grid, so, dt, m, damp, max_slots, max_nsrc, max_nrec, &e);
    if (st != FD_OK) return st;
    *out = new fd_engine{e};
    return FD_OK;
}

fd_status fd_engine_add_shot(fd_engine *h, int nt, int nsrc, const float *src_xyz,
                             const float *src_wav, int nrec, const float *rec_xyz, float *rec_out,
                             int *slot) {
    fdsweep::clear_error();
    return fdsweep::engine_add(h ? h->impl : nullptr, nt, nsrc, src_xyz, src_wav, nrec, rec_xyz,
                               rec_out, slot);
}

fd_status fd_engine_step(fd_engine *h, int nsteps) {
    fdsweep::clear_error();
    return fdsweep::engine_step(h ? h->impl : nullptr, nsteps);
}

fd_status fd_engine_shot_status(fd_engine *h, int slot, int *active, int64_t *steps_left) {
    fdsweep::clear_error();
    if (!h || slot < 0 || slot >= h->impl->max_slots)
        return fdsweep::set_error(FD_ERR_ARG, "fd_engine_shot_status: bad slot");
    Engine *e = h->impl;
    if (active) *active = e->active[slot];
    if (steps_left) {
        const int64_t left = (int64_t)e->t0[slot] + e->nt[slot] - e->G;
        *steps_left = e->active[slot] ? (left > 0 ? left : 0) : 0;
    }
    return FD_OK;
}

fd_status fd_engine_release(fd_engine *h, int slot) {
    fdsweep::clear_error();
    if (!h || slot < 0 || slot >= h->impl->max_slots || !h->impl->active[slot])
        return fdsweep::set_error(FD_ERR_ARG, "fd_engine_release: slot not active");
    h->impl->active[slot] = 0;
    ++h->impl->version;
    return FD_OK;
}

fd_status fd_engine_stream(fd_engine *h, void **stream) {
    fdsweep::clear_error();
    if (!h || !stream) return fdsweep::set_error(FD_ERR_ARG, "fd_engine_stream: null argument");
    *stream = h->impl->stream;
    return FD_OK;
}

fd_status fd_engine_sync(fd_engine *h) {
    fdsweep::clear_error();
    if (!h) return fdsweep::set_error(FD_ERR_ARG, "fd_engine_sync: null engine");
    Engine *e = h->impl;
    FD_CUDA_TRY(cudaStreamSynchronize(e->stream));
    fdsweep::MediumStats hs;
    FD_CUDA_TRY(cudaMemcpy(&hs, e->stats, sizeof(hs), cudaMemcpyDeviceToHost));
    if (hs.flags & fdsweep::DEV_ERR_COORD)
        return fdsweep::set_error(FD_ERR_COORD, "a shot's source or receiver lies outside the grid");
    if (hs.flags & fdsweep::DEV_ERR_TIMEOUT)
        return fdsweep::set_error(FD_ERR_TIMEOUT, "a device-side wait ran out");
    return FD_OK;
}

fd_status fd_engine_destroy(fd_engine *h) {
    fdsweep::clear_error();
    if (!h) return FD_OK;
    fdsweep::destroy_engine(h->impl);
    delete h;
    return FD_OK;
}

}  // extern "C"
