// api.cu -- the C-ABI entry points (include/fdsweep.h): argument validation,
// stability check, workspace, coefficient setup and the time loop.
//
// Per time step n (the paper's schedule of one time iteration: stencil
// update, then sparse injection into the t+1 field; receivers sample t):
//   acoustic:  K1 acoustic_step  ->  K3/K4 sparse (inject src[n] into u^{n+1},
//              interpolate rec[n] from u^n)
//   TTI:       K2a tti_pass1 -> K2b tti_pass2 -> K3/K4 sparse
// Steps are captured into a CUDA graph of kGraphChunk steps that is replayed;
// the sparse kernel reads its time index from a device counter that the
// graph's last node advances.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "kernels.cuh"
#include "runtime.cuh"

namespace fdsweep {

fd_status finish_medium_stats(MediumStats *dev_stats, cudaStream_t stream);

// ------------------------------------------------ numerics shared by every entry point

// Central FD weights for radius r, closed form:
//   second derivative w_k = 2 (-1)^{k+1} (r!)^2 / (k^2 (r-k)! (r+k)!), w_0 = -2 sum w_k
//   first derivative  c_k = (-1)^{k+1} (r!)^2 / (k (r-k)! (r+k)!)
void fd_weights(int r, double *w, double *c) {
    double ratio = 1.0, sum = 0.0;
    w[0] = 0.0;
    c[0] = 0.0;
    for (int k = 1; k <= r; ++k) {
        ratio = ratio * (double)(r - k + 1) / (double)(r + k);
        const double sign = (k & 1) ? 1.0 : -1.0;
        w[k] = 2.0 * sign * ratio / ((double)k * k);
        c[k] = sign * ratio / (double)k;
        sum += w[k];
    }
    w[0] = -2.0 * sum;
}

// max over theta of the second-derivative symbol -(w0 + 2 sum w_k cos k theta)
double second_symbol_max(int r, const double *w) {
    double best = 0.0;
    for (int t = 0; t <= 4096; ++t) {
        const double th = M_PI * t / 4096.0;
        double s = w[0];
        for (int k = 1; k <= r; ++k) s += 2.0 * w[k] * cos(k * th);
        if (-s > best) best = -s;
    }
    return best;
}

double acoustic_dt_bound(const fd_grid &g, int r, double m_min) {
    double w[kMaxRadius + 1] = {0.0}, c[kMaxRadius + 1] = {0.0};
    fd_weights(r, w, c);
    const double vmax = 1.0 / sqrt(m_min);
    const double lam = second_symbol_max(r, w) *
                       (1.0 / (g.hx * g.hx) + 1.0 / (g.hy * g.hy) + 1.0 / (g.hz * g.hz));
    return 2.0 / (vmax * sqrt(lam));
}

// The FP32 weights sum to zero exactly, as the FP64 weights do (w_0 = -2 sum
// w_k): the Laplacian of a constant is then zero in the device's weights too.
// Rounding each weight to FP32 on its own leaves a residual of up to ~1e-7 of
// the centre weight, which acts as a spurious mass term (the scheme solves
// m u_tt = lap u + eps u) and shifts the phase of every wave coherently, by
// about eps / (2 k^2) relative, so that the error grows linearly in time: on
// the 1000 ms acoustic workload at so = 12 the FP32 run ended 1.1e-4 (relative
// L2) from the FP64 scheme with independently rounded weights.  So the centre
// weight is the FP32 rounding of -2 sum_k (wx_k + wy_k + wz_k) and what that
// rounding leaves is moved into the neighbour weights, in the order of their
// effect on the operator's second moment (tap k of axis d changes the k^2
// coefficient by 2 k^2 h_d^2 per unit of weight: nearest taps of the finest
// axes first), each by less than one ulp of the centre weight; the second
// moment of every axis stays within 1e-6 of its exact value (a phase
// velocity error below 5e-7).  The FP64 sums are exact while
// the spacings differ by less than a factor of about 4 (48 FP32 terms whose
// exponents then span under 24 bits); beyond that the residual left is at the
// level of FP64 rounding.
void laplacian_weights(const fd_grid &g, int r, float *wc, float *wx, float *wy, float *wz) {
    double w[kMaxRadius + 1] = {0.0}, c[kMaxRadius + 1] = {0.0};
    fd_weights(r, w, c);
    const double ih2[3] = {1.0 / (g.hx * g.hx), 1.0 / (g.hy * g.hy), 1.0 / (g.hz * g.hz)};
    float *wa[3] = {wx, wy, wz};
    double sum = 0.0;  // 2 sum_k of the FP32 neighbour weights of all axes
    for (int a = 0; a < 3; ++a) {
        wa[a][0] = 0.f;  // the centre weights of all axes are in wc
        for (int k = 1; k <= kMaxRadius; ++k) {
            wa[a][k] = (float)(w[k] * ih2[a]);
            sum += 2.0 * (double)wa[a][k];
        }
    }
    *wc = (float)(-sum);
    double residual = (double)*wc + sum;
    // taps (axis, k) by increasing k^2 h_d^2
    int order[3 * kMaxRadius];
    int ntaps = 0;
    for (int k = 1; k <= r; ++k)
        for (int a = 0; a < 3; ++a) order[ntaps++] = a * (kMaxRadius + 1) + k;
    auto impact = [&](int t) {
        const int a = t / (kMaxRadius + 1), k = t % (kMaxRadius + 1);
        return (double)k * k / ih2[a];
    };
    for (int i = 1; i < ntaps; ++i)  // insertion sort, stable
        for (int j = i; j > 0 && impact(order[j]) < impact(order[j - 1]); --j) {
            const int t = order[j];
            order[j] = order[j - 1];
            order[j - 1] = t;
        }
    for (int i = 0; i < ntaps && residual != 0.0; ++i) {
        float &wt = wa[order[i] / (kMaxRadius + 1)][order[i] % (kMaxRadius + 1)];
        const float old = wt;
        wt = (float)((double)old - 0.5 * residual);
        residual -= 2.0 * ((double)old - (double)wt);
    }
}

WaveLayout wave_layout(const fd_grid &g) {
    WaveLayout L;
    L.nx = g.nx;
    L.ny = g.ny;
    L.nz = g.nz;
    L.nxp = (g.nx + 3) / 4 * 4;
    L.plane = (int64_t)L.nxp * g.ny;
    L.vol = L.plane * g.nz;
    return L;
}

namespace {

constexpr int kGraphChunk = 16;  // steps per captured graph (even: parity repeats)

// max over theta of the squared first-derivative symbol (2 sum c_k sin k theta)^2
double first_symbol_sq_max(int r, const double *c) {
    double best = 0.0;
    for (int t = 0; t <= 4096; ++t) {
        const double th = M_PI * t / 4096.0;
        double s = 0.0;
        for (int k = 1; k <= r; ++k) s += 2.0 * c[k] * sin(k * th);
        if (s * s > best) best = s * s;
    }
    return best;
}

// Staggered first-derivative weights a_k (k = 1..r) for the derivative midway
// between nodes from the node pairs at +-(k - 1/2) h:
//   a_k = (-1)^(k+1) ((2r-1)!!)^2 / (4^(r-1) (2k-1)^2 (r+k-1)! (r-k)!),
// built as a running product from a_1 (a_{k+1}/a_k = -(2k-1)^2 (r-k) /
// ((2k+1)^2 (r+k))).
void staggered_weights(int r, double *a) {
    double a1 = 1.0;  // ((2r-1)!!)^2 / (4^(r-1) r! (r-1)!)
    for (int j = 1; j < r; ++j) a1 *= (double)((2 * j + 1) * (2 * j + 1)) / (4.0 * j * (j + 1));
    a[0] = 0.0;
    a[1] = a1;
    for (int k = 1; k < r; ++k)
        a[k + 1] = -a[k] * (double)((2 * k - 1) * (2 * k - 1)) * (r - k) /
                   ((double)((2 * k + 1) * (2 * k + 1)) * (r + k));
}

// max over theta of the squared staggered symbol (2 sum a_k sin((k - 1/2) theta))^2
double staggered_symbol_sq_max(int r, const double *a) {
    double best = 0.0;
    for (int t = 0; t <= 4096; ++t) {
        const double th = M_PI * t / 4096.0;
        double s = 0.0;
        for (int k = 1; k <= r; ++k) s += 2.0 * a[k] * sin((k - 0.5) * th);
        if (s * s > best) best = s * s;
    }
    return best;
}

bool valid_so(int so) { return so == 2 || so == 4 || so == 8 || so == 12 || so == 16; }

int g_acoustic_config[kMaxRadius + 1] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
// TTI pass configuration per radius (-1: default).
int g_tti_config[kMaxRadius + 1] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
// Time tiling per radius: -1 automatic, 0 off, 1 + k forced with configuration k.
int g_time_tiling[kMaxRadius + 1] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};

// Radii for which the two-step kernel is the automatic choice: none.  On
// GB300 the single-step kernel runs at 95 % of the HBM copy bandwidth for
// so = 4, and the two-step kernel, which recomputes the extended tile's halo
// and stages three more tiles per plane, is bound by instruction issue and
// shared memory instead: 0.83 ms per two steps at 512^3 (so = 4) against
// 2 x 0.335 ms for two single steps; 2.5x slower at so = 8.
bool time_tiling_auto(int R) {
    (void)R;
    return false;
}

// Whether acoustic_forward runs its time loop two steps per launch, and with
// which configuration of the time-tiled kernel.
bool use_time_tiling(int R, int nsrc, int nsteps, int *config) {
    const int mode = g_time_tiling[R];
    *config = mode > 0 ? mode - 1 : 0;
    if (mode == 0 || nsteps < 2 || nsrc > kStep2MaxSources || acoustic2_num_configs(R) == 0)
        return false;
    return mode > 0 || time_tiling_auto(R);
}

}  // namespace

fd_status validate_grid(const fd_grid *g) {
    if (!g) return set_error(FD_ERR_ARG, "grid is null");
    if (g->nx < 2 || g->ny < 2 || g->nz < 2)
        return set_error(FD_ERR_ARG, "grid shape %d x %d x %d: every axis needs >= 2 points",
                         g->nx, g->ny, g->nz);
    const double hs[3] = {g->hx, g->hy, g->hz}, os[3] = {g->ox, g->oy, g->oz};
    for (int a = 0; a < 3; ++a) {
        if (!(hs[a] > 0.0) || !isfinite(hs[a]))
            return set_error(FD_ERR_ARG, "grid spacing must be finite and > 0");
        if (!isfinite(os[a])) return set_error(FD_ERR_ARG, "grid origin must be finite");
    }
    // nxp * ny < 2^62 cannot overflow; the volume is formed only once the
    // plane is known to be below 2^32 (so that it stays below 2^63)
    const int64_t nxp = ((int64_t)g->nx + 3) / 4 * 4;
    const int64_t plane = nxp * g->ny;
    if (plane >= (int64_t)1 << 32 || plane * g->nz >= (int64_t)1 << 32)
        return set_error(FD_ERR_ARG, "grid of %lld x %d x %d padded points reaches 2^32",
                         (long long)nxp, g->ny, g->nz);
    return FD_OK;
}

fd_status validate_common(const fd_grid *g, int so, double dt, int nt, int nshots, const float *m,
                          int nsrc, const float *src_xyz, const float *src_wav, int nrec,
                          const float *rec_xyz, const float *rec_out) {
    if (!g) return set_error(FD_ERR_ARG, "grid is null");
    if (!valid_so(so)) return set_error(FD_ERR_SO, "space order %d not in {2,4,8,12,16}", so);
    FD_TRY(validate_grid(g));
    if (!(dt > 0.0) || !isfinite(dt)) return set_error(FD_ERR_ARG, "dt must be finite and > 0");
    if (nt < 1) return set_error(FD_ERR_ARG, "nt must be >= 1");
    if (nshots < 1) return set_error(FD_ERR_ARG, "nshots must be >= 1");
    if (!m) return set_error(FD_ERR_ARG, "m is null");
    if (nsrc < 0 || nrec < 0) return set_error(FD_ERR_ARG, "nsrc and nrec must be >= 0");
    if (nsrc > 0 && (!src_xyz || !src_wav))
        return set_error(FD_ERR_ARG, "sources given but src_xyz or src_wav is null");
    if (nrec > 0 && (!rec_xyz || !rec_out))
        return set_error(FD_ERR_ARG, "receivers given but rec_xyz or rec_out is null");
    return FD_OK;
}

int acoustic_step_config(int radius) {
    return radius >= 0 && radius <= kMaxRadius ? g_acoustic_config[radius] : -1;
}

namespace {

// An input array that may live on the host: device copy in the workspace.
struct Staged {
    const float *user = nullptr;
    size_t count = 0;
    bool host = false;
    float *dev = nullptr;
    void plan(Workspace &ws, const float *p, size_t n) {
        user = p;
        count = n;
        host = p && n && !is_device_pointer(p);
        if (host) ws.add(&dev, n);
        else dev = const_cast<float *>(p);
    }
    fd_status place(cudaStream_t s) {
        if (host)
            FD_CUDA_TRY(cudaMemcpyAsync(dev, user, count * sizeof(float), cudaMemcpyDefault, s));
        return FD_OK;
    }
};

// An output array that may live on the host: written in the workspace, copied
// back at the end.
struct StagedOut {
    float *user = nullptr;
    size_t count = 0;
    bool host = false;
    float *dev = nullptr;
    void plan(Workspace &ws, float *p, size_t n) {
        user = p;
        count = n;
        host = p && n && !is_device_pointer(p);
        if (host) ws.add(&dev, n);
        else dev = p;
    }
    fd_status copy_back(cudaStream_t s) {
        if (host)
            FD_CUDA_TRY(cudaMemcpyAsync(user, dev, count * sizeof(float), cudaMemcpyDefault, s));
        return FD_OK;
    }
};

// Copies the finished time rows [done, upto) of traces [nshots][nt][nrec]
// staged on the device back to host memory on a copy stream while the time
// loop continues (the copy waits for the rows' producer on the call stream).
struct TraceStreamer {
    StagedOut *out = nullptr;
    int nshots = 0, nt = 0, nrec = 0;
    int done = 0;
    SideLane lane{1};
    bool active() const { return out && out->host && nrec > 0; }
    fd_status begin(StagedOut *o, int ns, int t, int nr) {
        out = o;
        nshots = ns;
        nt = t;
        nrec = nr;
        done = 0;
        return active() ? lane.begin() : FD_OK;
    }
    fd_status upto(int rows, cudaStream_t s) {
        if (!active() || rows <= done) return FD_OK;
        FD_TRY(lane.fork(s));
        const size_t pitch = (size_t)nt * nrec * sizeof(float);
        FD_CUDA_TRY(cudaMemcpy2DAsync(out->user + (size_t)done * nrec, pitch,
                                      out->dev + (size_t)done * nrec, pitch,
                                      (size_t)(rows - done) * nrec * sizeof(float), nshots,
                                      cudaMemcpyDefault, lane.get()));
        done = rows;
        return FD_OK;
    }
    // the remaining rows, then the call stream waits for every copy
    fd_status finish(cudaStream_t s) {
        if (!active()) return FD_OK;
        FD_TRY(upto(nt, s));
        return lane.join(s);
    }
};

// Host copy of the device MediumStats after a synchronisation.
fd_status read_stats(const MediumStats *dev, MediumStats *host, cudaStream_t s) {
    FD_CUDA_TRY(cudaMemcpyAsync(host, dev, sizeof(MediumStats), cudaMemcpyDeviceToHost, s));
    FD_CUDA_TRY(cudaStreamSynchronize(s));
    return FD_OK;
}

fd_status flags_to_status(unsigned int flags, const char *what) {
    if (flags & DEV_ERR_TIMEOUT)
        return set_error(FD_ERR_TIMEOUT, "%s: a device-side wait ran out (kernel aborted)", what);
    if (flags & DEV_ERR_COORD)
        return set_error(FD_ERR_COORD, "%s: a source or receiver lies outside the grid", what);
    if (flags & DEV_ERR_MEDIUM)
        return set_error(FD_ERR_ARG,
                         "%s: medium out of range (need finite m > 0, damp >= 0; TTI: "
                         "eps >= delta, 1 + 2 delta >= 0, finite angles)",
                         what);
    if (flags & DEV_ERR_NONFINITE)
        return set_error(FD_ERR_DIVERGED, "%s: the wavefield became non-finite", what);
    return FD_OK;
}

// Copies nfields dense [nz][ny][nx] arrays into (or out of) padded buffers.
fd_status copy_fields_in(float *dst_base, const WaveLayout &L, const float *src, int shot,
                         int nlev, int fields_per_shot, int first_level, cudaStream_t s) {
    const size_t dense = (size_t)L.nx * L.ny * L.nz;
    for (int l = 0; l < nlev; ++l) {
        float *dst = dst_base + (int64_t)(shot * fields_per_shot + first_level + l) * L.vol;
        const float *sp = src + ((size_t)shot * nlev + l) * dense;
        FD_CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)L.nxp * 4, sp, (size_t)L.nx * 4,
                                      (size_t)L.nx * 4, (size_t)L.ny * L.nz, cudaMemcpyDefault,
                                      s));
    }
    return FD_OK;
}

fd_status copy_field_out(float *dst_dense, const float *src_buf, const WaveLayout &L,
                         cudaStream_t s) {
    FD_CUDA_TRY(cudaMemcpy2DAsync(dst_dense, (size_t)L.nx * 4, src_buf, (size_t)L.nxp * 4,
                                  (size_t)L.nx * 4, (size_t)L.ny * L.nz, cudaMemcpyDefault, s));
    return FD_OK;
}

// Runs `nsteps` steps.  step(i, parity, use_counter) enqueues one step; with
// use_counter the sparse kernel's time index is *counter + i, otherwise i.
struct NoProgress {
    fd_status operator()(int) const { return FD_OK; }
};

// `progress(n)` is called (on the host, after enqueueing) whenever the first n
// units are enqueued: after every graph replay and every kGraphChunk direct
// units, and at the end.
template <class StepFn, class ProgressFn = NoProgress>
fd_status run_time_loop(int nsteps, cudaStream_t s, int *counter, bool allow_graph,
                        StepFn step, ProgressFn progress = ProgressFn()) {
    int n = 0;
    if (allow_graph && nsteps >= 2 * kGraphChunk) {
        FD_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), s));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        take_captured();
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            fd_status st = FD_OK;
            for (int i = 0; i < kGraphChunk && st == FD_OK; ++i) st = step(i, i & 1, true);
            if (st == FD_OK) st = bump_counter(counter, kGraphChunk, s);
            cudaError_t e = cudaStreamEndCapture(s, &graph);
            const int64_t per_graph = take_captured();
            if (st != FD_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            FD_CUDA_TRY(e);
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            FD_CUDA_TRY(e);
            const int reps = nsteps / kGraphChunk;
            fd_status pst = FD_OK;
            for (int r = 0; r < reps && pst == FD_OK; ++r) {
                e = cudaGraphLaunch(exec, s);
                if (e != cudaSuccess) break;
                pst = progress((r + 1) * kGraphChunk);
            }
            cudaGraphExecDestroy(exec);  // released once the queued launches complete
            add_launches(per_graph * reps);
            FD_CUDA_TRY(e);
            FD_TRY(pst);
            n = reps * kGraphChunk;
        } else {
            cudaGetLastError();
        }
    }
    for (; n < nsteps; ++n) {
        FD_TRY(step(n, n & 1, false));
        if ((n + 1) % kGraphChunk == 0 && n + 1 < nsteps) FD_TRY(progress(n + 1));
    }
    return progress(nsteps);
}

// Events bracketing the kernels of every step when statistics are on.
struct StepEvents {
    std::vector<cudaEvent_t> ev;
    int per_step = 0;
    ~StepEvents() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    fd_status create(int nsteps, int per) {
        per_step = per;
        ev.assign((size_t)nsteps * per, nullptr);
        for (auto &e : ev) FD_CUDA_TRY(cudaEventCreate(&e));
        return FD_OK;
    }
    cudaEvent_t at(int step, int k) { return ev[(size_t)step * per_step + k]; }
    double elapsed(int step, int k0, int k1) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, at(step, k0), at(step, k1));
        return ms;
    }
};

struct GridDerived {
    WaveLayout L;
    int R;
    double w[kMaxRadius + 1], c[kMaxRadius + 1];
};

GridDerived derive(const fd_grid *g, int so) {
    GridDerived d;
    d.L = wave_layout(*g);
    d.R = so / 2;
    for (int k = 0; k <= kMaxRadius; ++k) d.w[k] = d.c[k] = 0.0;
    fd_weights(so / 2, d.w, d.c);
    return d;
}

}  // namespace

// ====================================================================== acoustic

// damp_field: damp is a 3-D field [nz][ny][nx] instead of per-axis profiles;
// the stencil kernel then reads zeta = damp b / dt per point.
static fd_status acoustic_forward_impl(const fd_grid *grid, int so, double dt, int nt, int nshots,
                                       const float *m, const float *damp, int nsrc,
                                       const float *src_xyz, const float *src_wav, int nrec,
                                       const float *rec_xyz, float *rec_out, const float *u_init,
                                       float *u_final, cudaStream_t caller,
                                       bool damp_field = false) {
    FD_TRY(validate_common(grid, so, dt, nt, nshots, m, nsrc, src_xyz, src_wav, nrec, rec_xyz,
                           rec_out));
    const int R = so / 2;
    GridDerived gd = derive(grid, so);
    const WaveLayout &L = gd.L;
    const size_t dense = (size_t)L.nx * L.ny * L.nz;
    const int ndamp = L.nx + L.ny + L.nz;
    // two steps per launch needs four distinct levels per shot
    int t2_config = 0;
    const bool tiled = !damp_field && use_time_tiling(R, nsrc, nt - 1, &t2_config);
    const int lps = tiled ? 4 : 2;

    CallStream cs;
    FD_TRY(cs.begin(caller));
    cudaStream_t s = cs.get();

    Workspace ws;
    float *wave, *bcoef, *dps;
    SparsePoint *src_tab, *rec_tab;
    MediumStats *dstats;
    int *counter;
    ws.add(&wave, (size_t)lps * nshots * L.vol);  // u levels per shot
    ws.add(&bcoef, (damp_field ? 2 : 1) * (size_t)L.vol);  // b = dt^2 / (m + damp dt/2) [, zeta]
    ws.add(&dps, ndamp);                        // damping / dt
    ws.add(&src_tab, (size_t)nshots * nsrc);
    ws.add(&rec_tab, (size_t)nshots * nrec);
    ws.add(&dstats, 1);
    ws.add(&counter, 1);
    Staged sm, sdamp, ssxyz, swav, srxyz;
    StagedOut srec;
    sm.plan(ws, m, dense);
    sdamp.plan(ws, damp, damp ? (damp_field ? dense : (size_t)ndamp) : 0);
    ssxyz.plan(ws, src_xyz, (size_t)nshots * nsrc * 3);
    swav.plan(ws, src_wav, (size_t)nshots * nt * nsrc);
    srxyz.plan(ws, rec_xyz, (size_t)nshots * nrec * 3);
    srec.plan(ws, rec_out, (size_t)nshots * nt * nrec);
    FD_TRY(ws.allocate(s));
    FD_STAGE(s, "acoustic: workspace allocated");
    TraceStreamer traces;  // host traces: copied back while the loop runs
    FD_TRY(traces.begin(&srec, nshots, nt, nrec));
    for (Staged *st : {&sm, &sdamp, &ssxyz, &swav, &srxyz}) FD_TRY(st->place(s));
    FD_STAGE(s, "acoustic: inputs staged");

    // ---- K0: coefficients, tables, validation
    FD_CUDA_TRY(cudaMemsetAsync(bcoef, 0, (damp_field ? 2 : 1) * (size_t)L.vol * 4, s));
    FD_TRY(init_medium_stats(dstats, s));
    FD_TRY(setup_acoustic_coeffs(sm.dev, sdamp.dev, dt, L, bcoef, dps, dstats, s, damp_field));
    FD_STAGE(s, "acoustic: coefficients");
    for (int sh = 0; sh < nshots; ++sh) {
        FD_TRY(setup_sparse_table(ssxyz.dev ? ssxyz.dev + (size_t)sh * nsrc * 3 : nullptr, nsrc,
                                  *grid, L, src_tab + (size_t)sh * nsrc, &dstats->flags, s));
        FD_TRY(setup_sparse_table(srxyz.dev ? srxyz.dev + (size_t)sh * nrec * 3 : nullptr, nrec,
                                  *grid, L, rec_tab + (size_t)sh * nrec, &dstats->flags, s));
    }
    FD_TRY(finish_medium_stats(dstats, s));
    FD_STAGE(s, "acoustic: setup kernels");
    MediumStats hs;
    FD_TRY(read_stats(dstats, &hs, s));
    FD_TRY(flags_to_status(hs.flags, "acoustic_forward"));
    {
        const double vmax = 1.0 / sqrt((double)hs.m_min);
        const double dt_max = acoustic_dt_bound(*grid, R, (double)hs.m_min);
        if (dt > dt_max * (1.0 + 1e-12))
            return set_error(FD_ERR_CFL,
                             "dt = %.6g ms exceeds the leapfrog stability bound %.6g ms "
                             "(v_max = %.6g km/s, so = %d)",
                             dt, dt_max, vmax, so);
    }

    // ---- initial state
    FD_CUDA_TRY(cudaMemsetAsync(wave, 0, (size_t)lps * nshots * L.vol * 4, s));
    if (u_init)
        for (int sh = 0; sh < nshots; ++sh)
            FD_TRY(copy_fields_in(wave, L, u_init, sh, 2, lps, 0, s));

    // ---- K1 plan and arguments
    AcousticPlan plan;
    FD_STAGE(s, "acoustic: initial state");
    FD_TRY(acoustic_plan(R, g_acoustic_config[R], L, nshots, lps, wave, bcoef, &plan, 0,
                         damp_field));
    FD_STAGE(s, plan.name);
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
    laplacian_weights(*grid, R, &a.wc, a.wx, a.wy, a.wz);
    SparseArgs sp;
    memset(&sp, 0, sizeof(sp));
    sp.wave = wave;
    sp.fields_per_shot = lps;
    sp.L = L;
    sp.bcoef = bcoef;
    sp.nshots = nshots;
    sp.nt = nt;
    sp.nsrc = nsrc;
    sp.src_tab = src_tab;
    sp.src_wav = swav.dev;
    sp.inj_level1 = -1;
    sp.inj_t0 = 0;
    sp.inj_dt = 1;
    sp.rec_t0 = 0;
    sp.rec_dt = 1;
    sp.nrec = nrec;
    sp.rec_tab = rec_tab;
    sp.rec_out = srec.dev;

    // ---- time loop
    const int nsteps = nt - 1;
    const bool timing = stats_enabled();
    const bool graphs = !timing && trace_level() < 2;
    int last = nsteps & 1, prev_of_last = 1 - last;  // levels of u^{nt-1}, u^{nt-2}
    // per-launch events (stats mode): one row per step, or per pair plus one
    // row for a final single step; read after the call's closing sync
    const int nunits = tiled ? nsteps / 2 : nsteps;
    StepEvents evs;
    if (timing) FD_TRY(evs.create(nunits + 1, 3));
    bool odd_tail = false;
    if (!tiled) {
        // The receivers of step n read only u^n, which the stencil kernel of
        // step n reads too and the kernel of step n+1 overwrites: they run on
        // a side stream concurrently with the stencil, and only the source
        // injection into u^{n+1} stays between two stencil launches.
        SideLane side;
        const bool overlap = nrec > 0;
        if (overlap) FD_TRY(side.begin());
        // Up to kInjectMaxSources sources per shot are injected by the
        // stencil kernel itself (the CTA that wrote the corners), which
        // removes a dependent launch from every step; more go through the
        // sparse kernel.
        const bool inject_in_k1 = nsrc > 0 && nsrc <= kInjectMaxSources;
        auto step = [&](int i, int par, bool via_counter) -> fd_status {
            AcousticStepArgs ai = a;
            set_two_levels(ai, par);
            SparseArgs si = sp;
            si.inj_level0 = 1 - par;
            si.rec_level = par;
            si.step_base = via_counter ? counter : nullptr;
            AcousticInject inj;
            memset(&inj, 0, sizeof(inj));
            if (inject_in_k1) {
                inj.src_tab = src_tab;
                inj.src_wav = swav.dev;
                inj.nsrc = nsrc;
                inj.nt = nt;
                inj.step_base = si.step_base;
                inj.step = i;
            }
            if (overlap) {
                FD_TRY(side.fork(s));
                FD_TRY(sparse_launch(si, i, false, true, side.get()));
            }
            if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(i, 0), s));
            FD_TRY(acoustic_launch(plan, ai, s, &inj));
            if (!via_counter && trace_level() >= 2) FD_STAGE(s, "acoustic_step kernel");
            if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(i, 1), s));
            FD_TRY(sparse_launch(si, i, nsrc > 0 && !inject_in_k1, !overlap && nrec > 0, s));
            if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(i, 2), s));
            if (overlap) FD_TRY(side.join(s));
            if (i % kWatchEvery == kWatchEvery - 1)
                FD_TRY(watchdog_launch(wave, L, lps * nshots, &dstats->flags, s));
            return FD_OK;
        };
        FD_TRY(run_time_loop(nsteps, s, counter, graphs, step,
                             [&](int n) { return traces.upto(n, s); }));
    } else {
        // Two steps per launch over four levels per shot: pair i (parity par)
        // reads u^n, u^{n-1} from levels (0, 1) or (3, 2) and writes u^{n+1},
        // u^{n+2} to (2, 3) or (1, 0), so every pair starts where the one
        // before the previous did.  The sparse kernel records rec[n] and
        // rec[n+1] and injects src[n+1] into u^{n+2}; src[n] is injected into
        // u^{n+1} by the two-step kernel itself.
        Acoustic2Plan plan2;
        FD_TRY(acoustic2_plan(R, t2_config, L, nshots, lps, wave, bcoef, &plan2));
        FD_STAGE(s, plan2.name);
        AcousticStep2Args a2;
        memset(&a2, 0, sizeof(a2));
        a2.s = a;
        a2.s.lps = lps;
        a2.src_tab = nsrc > 0 ? src_tab : nullptr;
        a2.src_wav = swav.dev;
        a2.nsrc = nsrc;
        a2.nt = nt;
        const int npairs = nunits;
        auto pair = [&](int i, int par, bool via_counter) -> fd_status {
            AcousticStep2Args ai = a2;
            ai.s.lev_cur = par ? 3 : 0;
            ai.s.lev_prev = par ? 2 : 1;
            ai.s.lev_out = par ? 1 : 2;
            ai.lev_out2 = par ? 0 : 3;
            ai.step = i;
            ai.step_base = via_counter ? counter : nullptr;
            if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(i, 0), s));
            FD_TRY(acoustic2_launch(plan2, ai, s));
            if (!via_counter && trace_level() >= 2) FD_STAGE(s, "acoustic_step2 kernel");
            if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(i, 1), s));
            SparseArgs si = sp;
            si.inj_level0 = ai.lev_out2;
            si.inj_t0 = 1;
            si.inj_dt = 2;
            si.rec_level = ai.s.lev_cur;
            si.rec_t0 = 0;
            si.rec_dt = 2;
            si.step_base = ai.step_base;
            FD_TRY(sparse_launch(si, i, nsrc > 0, nrec > 0, s));
            SparseArgs sj = sp;
            sj.rec_level = ai.s.lev_out;
            sj.rec_t0 = 1;
            sj.rec_dt = 2;
            sj.step_base = ai.step_base;
            FD_TRY(sparse_launch(sj, i, false, nrec > 0, s));
            if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(i, 2), s));
            if (i % (kWatchEvery / 2) == kWatchEvery / 2 - 1)
                FD_TRY(watchdog_launch(wave, L, lps * nshots, &dstats->flags, s));
            return FD_OK;
        };
        FD_TRY(run_time_loop(npairs, s, counter, graphs, pair,
                             [&](int np) { return traces.upto(2 * np, s); }));
        last = (npairs & 1) ? 3 : 0;
        prev_of_last = (npairs & 1) ? 2 : 1;
        if (nsteps & 1) {  // one single step to finish, in place
            AcousticStepArgs ai = a;
            ai.lps = lps;
            ai.lev_cur = last;
            ai.lev_prev = prev_of_last;
            ai.lev_out = prev_of_last;
            if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(nunits, 0), s));
            FD_TRY(acoustic_launch(plan, ai, s));
            if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(nunits, 1), s));
            SparseArgs si = sp;
            si.inj_level0 = prev_of_last;
            si.rec_level = last;
            FD_TRY(sparse_launch(si, nsteps - 1, nsrc > 0, nrec > 0, s));
            if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(nunits, 2), s));
            odd_tail = true;
            const int t = last;
            last = prev_of_last;
            prev_of_last = t;
        }
    }
    FD_STAGE(s, "acoustic: time loop");
    {
        SparseArgs si = sp;
        si.rec_level = last;
        si.step_base = nullptr;
        FD_TRY(sparse_launch(si, nt - 1, false, nrec > 0, s));
    }
    FD_TRY(check_finite(wave, L, lps * nshots, &dstats->flags, s));
    FD_STAGE(s, "acoustic: final interpolation and check");

    // ---- outputs
    if (u_final) {
        for (int sh = 0; sh < nshots; ++sh) {
            float *dst = u_final + (size_t)sh * 2 * dense;
            FD_TRY(copy_field_out(dst, wave + (int64_t)(lps * sh + last) * L.vol, L, s));
            FD_TRY(copy_field_out(dst + dense, wave + (int64_t)(lps * sh + prev_of_last) * L.vol,
                                  L, s));
        }
    }
    if (traces.active())
        FD_TRY(traces.finish(s));
    else
        FD_TRY(srec.copy_back(s));
    FD_TRY(read_stats(dstats, &hs, s));
    if (timing && nsteps > 0) {
        double kms = 0.0, sms = 0.0;
        for (int i = 0; i < nunits; ++i) {
            kms += evs.elapsed(i, 0, 1);
            sms += evs.elapsed(i, 1, 2);
        }
        const double pts = (double)dense * nshots;
        if (tiled) {
            if (nunits) stats_add("acoustic_step2", kms, nunits, pts);
            if (odd_tail) {
                stats_add("acoustic_step", evs.elapsed(nunits, 0, 1), 1, pts);
                sms += evs.elapsed(nunits, 1, 2);
            }
        } else {
            stats_add("acoustic_step", kms, nunits, pts);
        }
        stats_add("sparse", sms, nsteps, (double)(nrec + 8 * nsrc) * nshots);
    }
    ws.release();
    FD_TRY(cs.finish());
    return flags_to_status(hs.flags, "acoustic_forward");
}

// ====================================================================== binary16 storage

namespace {
int g_acoustic_h_config[kMaxRadius + 1] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
}  // namespace

// acoustic_forward with the wavefield levels and b stored in IEEE binary16
// (FP32 arithmetic).  Same schedule as the FP32 path without time tiling:
// per step the stencil kernel, the injection of src[n] into u^{n+1}, and the
// receivers of u^n on a side stream.
static fd_status acoustic_forward_h_impl(const fd_grid *grid, int so, double dt, int nt,
                                         int nshots, const float *m, const float *damp,
                                         int nsrc, const float *src_xyz, const float *src_wav,
                                         int nrec, const float *rec_xyz, float *rec_out,
                                         const float *u_init, float *u_final,
                                         cudaStream_t caller) {
    FD_TRY(validate_common(grid, so, dt, nt, nshots, m, nsrc, src_xyz, src_wav, nrec, rec_xyz,
                           rec_out));
    const int R = so / 2;
    if (acoustic_h_num_configs(R) == 0)
        return set_error(FD_ERR_UNIMPL, "binary16 storage: no kernel for so = %d", so);
    GridDerived gd = derive(grid, so);
    const WaveLayout &L = gd.L;  // FP32 layout of the setup
    WaveLayout LH = L;           // binary16 layout: 16-byte rows
    LH.nxp = (L.nx + 7) / 8 * 8;
    LH.plane = (int64_t)LH.nxp * L.ny;
    LH.vol = LH.plane * L.nz;
    const size_t dense = (size_t)L.nx * L.ny * L.nz;
    const int64_t rows = (int64_t)L.ny * L.nz;
    const int ndamp = L.nx + L.ny + L.nz;

    CallStream cs;
    FD_TRY(cs.begin(caller));
    cudaStream_t s = cs.get();

    Workspace ws;
    half_bits *wave, *bh;
    float *b32, *dps;
    SparsePoint *src_tab, *rec_tab;
    MediumStats *dstats;
    int *counter;
    ws.add(&wave, (size_t)2 * nshots * LH.vol);
    ws.add(&bh, LH.vol);
    ws.add(&b32, L.vol);
    ws.add(&dps, ndamp);
    ws.add(&src_tab, (size_t)nshots * nsrc);
    ws.add(&rec_tab, (size_t)nshots * nrec);
    ws.add(&dstats, 1);
    ws.add(&counter, 1);
    Staged sm, sdamp, ssxyz, swav, srxyz, sinit;
    StagedOut srec, sfinal;
    sm.plan(ws, m, dense);
    sdamp.plan(ws, damp, damp ? ndamp : 0);
    ssxyz.plan(ws, src_xyz, (size_t)nshots * nsrc * 3);
    swav.plan(ws, src_wav, (size_t)nshots * nt * nsrc);
    srxyz.plan(ws, rec_xyz, (size_t)nshots * nrec * 3);
    sinit.plan(ws, u_init, u_init ? (size_t)nshots * 2 * dense : 0);
    srec.plan(ws, rec_out, (size_t)nshots * nt * nrec);
    sfinal.plan(ws, u_final, u_final ? (size_t)nshots * 2 * dense : 0);
    FD_TRY(ws.allocate(s));
    TraceStreamer traces;
    FD_TRY(traces.begin(&srec, nshots, nt, nrec));
    for (Staged *st : {&sm, &sdamp, &ssxyz, &swav, &srxyz, &sinit}) FD_TRY(st->place(s));
    FD_STAGE(s, "acoustic f16: inputs staged");

    // ---- K0: coefficients (FP64 -> FP32 as in the FP32 path, then binary16)
    FD_CUDA_TRY(cudaMemsetAsync(b32, 0, (size_t)L.vol * 4, s));
    FD_CUDA_TRY(cudaMemsetAsync(bh, 0, (size_t)LH.vol * 2, s));
    FD_TRY(init_medium_stats(dstats, s));
    FD_TRY(setup_acoustic_coeffs(sm.dev, sdamp.dev, dt, L, b32, dps, dstats, s));
    FD_TRY(narrow_rows(b32, L.nxp, bh, LH.nxp, L.nx, rows, s));
    for (int sh = 0; sh < nshots; ++sh) {
        FD_TRY(setup_sparse_table(ssxyz.dev ? ssxyz.dev + (size_t)sh * nsrc * 3 : nullptr, nsrc,
                                  *grid, LH, src_tab + (size_t)sh * nsrc, &dstats->flags, s));
        FD_TRY(setup_sparse_table(srxyz.dev ? srxyz.dev + (size_t)sh * nrec * 3 : nullptr, nrec,
                                  *grid, LH, rec_tab + (size_t)sh * nrec, &dstats->flags, s));
    }
    FD_TRY(finish_medium_stats(dstats, s));
    MediumStats hs;
    FD_TRY(read_stats(dstats, &hs, s));
    FD_TRY(flags_to_status(hs.flags, "acoustic_forward_opts"));
    {
        const double vmax = 1.0 / sqrt((double)hs.m_min);
        const double dt_max = acoustic_dt_bound(*grid, R, (double)hs.m_min);
        if (dt > dt_max * (1.0 + 1e-12))
            return set_error(FD_ERR_CFL,
                             "dt = %.6g ms exceeds the leapfrog stability bound %.6g ms "
                             "(v_max = %.6g km/s, so = %d)",
                             dt, dt_max, vmax, so);
    }

    // ---- initial state, rounded to binary16
    FD_CUDA_TRY(cudaMemsetAsync(wave, 0, (size_t)2 * nshots * LH.vol * 2, s));
    if (u_init)
        for (int f = 0; f < 2 * nshots; ++f)
            FD_TRY(narrow_rows(sinit.dev + (size_t)f * dense, L.nx, wave + (int64_t)f * LH.vol,
                               LH.nxp, L.nx, rows, s));

    AcousticPlan plan;
    FD_TRY(acoustic_h_plan(R, g_acoustic_h_config[R], LH, nshots, 2, wave, bh, &plan));
    FD_STAGE(s, plan.name);
    AcousticHArgs a;
    memset(&a, 0, sizeof(a));
    a.wave = wave;
    a.bcoef = bh;
    a.dpx = dps;
    a.dpy = dps + L.nx;
    a.dpz = dps + L.nx + L.ny;
    a.L = LH;
    a.nshots = nshots;
    a.lps = 2;
    a.err = &dstats->flags;
    laplacian_weights(*grid, R, &a.wc, a.wx, a.wy, a.wz);
    SparseHArgs sp;
    memset(&sp, 0, sizeof(sp));
    sp.wave = wave;
    sp.fields_per_shot = 2;
    sp.L = LH;
    sp.bcoef = bh;
    sp.nshots = nshots;
    sp.nt = nt;
    sp.nsrc = nsrc;
    sp.src_tab = src_tab;
    sp.src_wav = swav.dev;
    sp.nrec = nrec;
    sp.rec_tab = rec_tab;
    sp.rec_out = srec.dev;

    // ---- time loop
    const int nsteps = nt - 1;
    const bool timing = stats_enabled();
    const bool graphs = !timing && trace_level() < 2;
    StepEvents evs;
    if (timing) FD_TRY(evs.create(nsteps + 1, 3));
    SideLane side;
    const bool overlap = nrec > 0;
    if (overlap) FD_TRY(side.begin());
    auto step = [&](int i, int par, bool via_counter) -> fd_status {
        AcousticHArgs ai = a;
        ai.lev_cur = par;
        ai.lev_prev = 1 - par;
        ai.lev_out = 1 - par;
        SparseHArgs si = sp;
        si.inj_level = 1 - par;
        si.rec_level = par;
        si.step_base = via_counter ? counter : nullptr;
        if (overlap) {
            FD_TRY(side.fork(s));
            FD_TRY(sparse_h_launch(si, i, false, true, side.get()));
        }
        if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(i, 0), s));
        FD_TRY(acoustic_h_launch(plan, ai, s));
        if (!via_counter && trace_level() >= 2) FD_STAGE(s, "acoustic_step_h kernel");
        if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(i, 1), s));
        FD_TRY(sparse_h_launch(si, i, nsrc > 0, false, s));
        if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(i, 2), s));
        if (overlap) FD_TRY(side.join(s));
        return FD_OK;
    };
    FD_TRY(run_time_loop(nsteps, s, counter, graphs, step,
                         [&](int n) { return traces.upto(n, s); }));
    const int last = nsteps & 1, prev_of_last = 1 - last;
    {
        SparseHArgs si = sp;
        si.rec_level = last;
        FD_TRY(sparse_h_launch(si, nt - 1, false, nrec > 0, s));
    }
    FD_TRY(check_finite_h(wave, LH, 2 * nshots, &dstats->flags, s));
    FD_STAGE(s, "acoustic f16: time loop");

    // ---- outputs: the stored values widened to FP32
    if (u_final) {
        for (int sh = 0; sh < nshots; ++sh) {
            float *dst = sfinal.dev + (size_t)sh * 2 * dense;
            FD_TRY(widen_rows(wave + (int64_t)(2 * sh + last) * LH.vol, LH.nxp, dst, L.nx, L.nx,
                              rows, s));
            FD_TRY(widen_rows(wave + (int64_t)(2 * sh + prev_of_last) * LH.vol, LH.nxp,
                              dst + dense, L.nx, L.nx, rows, s));
        }
        FD_TRY(sfinal.copy_back(s));
    }
    if (traces.active())
        FD_TRY(traces.finish(s));
    else
        FD_TRY(srec.copy_back(s));
    FD_TRY(read_stats(dstats, &hs, s));
    if (timing && nsteps > 0) {
        double kms = 0.0, sms = 0.0;
        for (int i = 0; i < nsteps; ++i) {
            kms += evs.elapsed(i, 0, 1);
            sms += evs.elapsed(i, 1, 2);
        }
        stats_add("acoustic_step_h", kms, nsteps, (double)dense * nshots);
        stats_add("sparse", sms, nsteps, (double)(nrec + 8 * nsrc) * nshots);
    }
    ws.release();
    FD_TRY(cs.finish());
    return flags_to_status(hs.flags, "acoustic_forward_opts");
}

// ====================================================================== TTI

static fd_status tti_forward_impl(const fd_grid *grid, int so, double dt, int nt, int nshots,
                                  const float *m, const float *damp, const float *eps,
                                  const float *delta, const float *theta, const float *phi,
                                  int nsrc, const float *src_xyz, const float *src_wav, int nrec,
                                  const float *rec_xyz, float *rec_out, const float *p_init,
                                  const float *r_init, float *p_final, float *r_final,
                                  const fd_tti_options *opts, cudaStream_t caller) {
    FD_TRY(validate_common(grid, so, dt, nt, nshots, m, nsrc, src_xyz, src_wav, nrec, rec_xyz,
                           rec_out));
    if (!eps || !delta || !theta || !phi)
        return set_error(FD_ERR_ARG, "tti_forward: epsilon, delta, theta and phi are required");
    fd_tti_options op = {FD_TTI_CENTRED, FD_TTI_REC_P, FD_TTI_AUTO};
    if (opts) op = *opts;
    if ((op.deriv != FD_TTI_CENTRED && op.deriv != FD_TTI_STAGGERED) ||
        (op.receiver != FD_TTI_REC_P && op.receiver != FD_TTI_REC_MEAN) ||
        (op.scheme != FD_TTI_AUTO && op.scheme != FD_TTI_TWO_PASS &&
         op.scheme != FD_TTI_RECOMPUTE && op.scheme != FD_TTI_FUSED))
        return set_error(FD_ERR_ARG, "tti_forward: options (%d, %d, %d) out of range", op.deriv,
                         op.receiver, op.scheme);
    // automatic: the fused kernel where it was measured faster (so <= 4:
    // 1.76 against 2.12 ms per 512^3 step at so 4), two passes otherwise
    if (op.scheme == FD_TTI_AUTO)
        op.scheme = (so <= 4 && tti_fused_supported(so / 2)) ? FD_TTI_FUSED : FD_TTI_TWO_PASS;
    if (op.scheme == FD_TTI_FUSED && !tti_fused_supported(so / 2))
        return set_error(FD_ERR_ARG, "tti_forward: the fused scheme covers so <= 8 (so = %d)",
                         so);
    const bool stag = op.deriv == FD_TTI_STAGGERED;
    const bool two_pass = op.scheme == FD_TTI_TWO_PASS;
    const bool fused = op.scheme == FD_TTI_FUSED;
    const int R = so / 2;
    GridDerived gd = derive(grid, so);
    const WaveLayout &L = gd.L;
    const size_t dense = (size_t)L.nx * L.ny * L.nz;
    const int ndamp = L.nx + L.ny + L.nz;

    CallStream cs;
    FD_TRY(cs.begin(caller));
    cudaStream_t s = cs.get();

    Workspace ws;
    float *wave, *tmp, *bcoef, *dps;
    SparsePoint *src_tab, *rec_tab;
    MediumStats *dstats;
    int *counter;
    ws.add(&wave, (size_t)4 * nshots * L.vol);  // p, r at two levels per shot
    ws.add(&tmp, two_pass ? (size_t)6 * nshots * L.vol : 0);  // pass-1 temporaries
    ws.add(&bcoef, (size_t)6 * L.vol);          // b, a, s, n_x, n_y, n_z
    ws.add(&dps, ndamp);
    ws.add(&src_tab, (size_t)nshots * nsrc);
    ws.add(&rec_tab, (size_t)nshots * nrec);
    ws.add(&dstats, 1);
    ws.add(&counter, 1);
    Staged sm, sdamp, seps, sdel, sth, sph, ssxyz, swav, srxyz;
    StagedOut srec;
    sm.plan(ws, m, dense);
    sdamp.plan(ws, damp, damp ? ndamp : 0);
    seps.plan(ws, eps, dense);
    sdel.plan(ws, delta, dense);
    sth.plan(ws, theta, dense);
    sph.plan(ws, phi, dense);
    ssxyz.plan(ws, src_xyz, (size_t)nshots * nsrc * 3);
    swav.plan(ws, src_wav, (size_t)nshots * nt * nsrc);
    srxyz.plan(ws, rec_xyz, (size_t)nshots * nrec * 3);
    srec.plan(ws, rec_out, (size_t)nshots * nt * nrec);
    FD_TRY(ws.allocate(s));
    float *acoef = bcoef + L.vol;
    float *scoef = bcoef + 2 * L.vol;
    float *nvec = bcoef + 3 * L.vol;
    for (Staged *st : {&sm, &sdamp, &seps, &sdel, &sth, &sph, &ssxyz, &swav, &srxyz})
        FD_TRY(st->place(s));

    FD_CUDA_TRY(cudaMemsetAsync(bcoef, 0, (size_t)6 * L.vol * 4, s));
    FD_TRY(init_medium_stats(dstats, s));
    FD_TRY(setup_acoustic_coeffs(sm.dev, sdamp.dev, dt, L, bcoef, dps, dstats, s));
    FD_TRY(setup_tti_coeffs(seps.dev, sdel.dev, sth.dev, sph.dev, L, acoef, scoef, nvec, dstats,
                            s));
    for (int sh = 0; sh < nshots; ++sh) {
        FD_TRY(setup_sparse_table(ssxyz.dev ? ssxyz.dev + (size_t)sh * nsrc * 3 : nullptr, nsrc,
                                  *grid, L, src_tab + (size_t)sh * nsrc, &dstats->flags, s));
        FD_TRY(setup_sparse_table(srxyz.dev ? srxyz.dev + (size_t)sh * nrec * 3 : nullptr, nrec,
                                  *grid, L, rec_tab + (size_t)sh * nrec, &dstats->flags, s));
    }
    FD_TRY(finish_medium_stats(dstats, s));
    MediumStats hs;
    FD_TRY(read_stats(dstats, &hs, s));
    FD_TRY(flags_to_status(hs.flags, "tti_forward"));
    {
        const double vmax = 1.0 / sqrt((double)hs.m_min);
        const double amax = 1.0 + 2.0 * (double)(hs.eps_max > 0.f ? hs.eps_max : 0.f);
        double sa[kMaxRadius + 1];
        staggered_weights(R, sa);
        const double sig = stag ? staggered_symbol_sq_max(R, sa) : first_symbol_sq_max(R, gd.c);
        const double lam = sig * (1.0 / (grid->hx * grid->hx) + 1.0 / (grid->hy * grid->hy) +
                                  1.0 / (grid->hz * grid->hz));
        const double dt_max = 2.0 / sqrt(amax * vmax * vmax * lam);
        if (dt > dt_max * (1.0 + 1e-12))
            return set_error(FD_ERR_CFL,
                             "dt = %.6g ms exceeds the TTI stability bound %.6g ms "
                             "(v_max = %.6g km/s, 1+2eps_max = %.4g, so = %d)",
                             dt, dt_max, vmax, amax, so);
    }

    FD_CUDA_TRY(cudaMemsetAsync(wave, 0, (size_t)4 * nshots * L.vol * 4, s));
    for (int sh = 0; sh < nshots; ++sh) {
        if (p_init) FD_TRY(copy_fields_in(wave, L, p_init, sh, 2, 4, 0, s));
        if (r_init) FD_TRY(copy_fields_in(wave, L, r_init, sh, 2, 4, 2, s));
    }

    TtiPlan tplan;
    if (fused)
        FD_TRY(tti_fused_plan(R, stag ? 1 : 0, L, nshots, wave, bcoef, &tplan,
                              g_tti_config[R] < 0 ? 0 : g_tti_config[R]));
    else
        FD_TRY(tti_plan(R, L, nshots, wave, tmp, bcoef, &tplan, stag ? 1 : 0,
                        two_pass ? kTtiTwoPass : kTtiRecompute, g_tti_config[R]));
    TtiArgs a;
    memset(&a, 0, sizeof(a));
    a.wave = wave;
    a.tmp = tmp;
    a.bcoef = bcoef;
    a.acoef = acoef;
    a.scoef = scoef;
    a.nvec = nvec;
    a.dpx = dps;
    a.dpy = dps + L.nx;
    a.dpz = dps + L.nx + L.ny;
    a.L = L;
    a.nshots = nshots;
    a.err = &dstats->flags;
    {
        // tap tables (offset d at index d + R): centred sign(d) c_|d|;
        // staggered inner D+ (a_d at +d, -a_d at 1-d), outer D- (a_d at d-1,
        // -a_d at -d); all divided by the spacing of the axis
        double sa[kMaxRadius + 1];
        staggered_weights(R, sa);
        const double hh[3] = {grid->hx, grid->hy, grid->hz};
        for (int ax = 0; ax < 3; ++ax) {
            for (int d = -R; d <= R; ++d) {
                double w1 = 0.0, w2 = 0.0;
                if (!stag) {
                    w1 = w2 = d > 0 ? gd.c[d] : (d < 0 ? -gd.c[-d] : 0.0);
                } else {
                    w1 = d >= 1 ? sa[d] : (d > -R ? -sa[1 - d] : 0.0);
                    w2 = d <= -1 ? -sa[-d] : (d < R ? sa[d + 1] : 0.0);
                }
                a.t1[ax][d + R] = (float)(w1 / hh[ax]);
                a.t2[ax][d + R] = (float)(w2 / hh[ax]);
            }
        }
    }
    SparseArgs sp;
    memset(&sp, 0, sizeof(sp));
    sp.wave = wave;
    sp.fields_per_shot = 4;
    sp.L = L;
    sp.bcoef = bcoef;
    sp.nshots = nshots;
    sp.nt = nt;
    sp.nsrc = nsrc;
    sp.src_tab = src_tab;
    sp.src_wav = swav.dev;
    sp.inj_t0 = 0;
    sp.inj_dt = 1;
    sp.rec_t0 = 0;
    sp.rec_dt = 1;
    sp.nrec = nrec;
    sp.rec_tab = rec_tab;
    sp.rec_out = srec.dev;
    sp.rec_mean = op.receiver == FD_TTI_REC_MEAN ? 1 : 0;

    const int nsteps = nt - 1;
    const bool timing = stats_enabled();
    StepEvents evs;
    if (timing) FD_TRY(evs.create(nsteps, 4));
    auto step = [&](int i, int par, bool via_counter) -> fd_status {
        TtiArgs ai = a;
        ai.cur = par;
        cudaEvent_t ev3[3];
        if (timing)
            for (int k = 0; k < 3; ++k) ev3[k] = evs.at(i, k);
        FD_TRY(tti_launch(tplan, ai, s, timing ? ev3 : nullptr));
        SparseArgs si = sp;
        si.inj_level0 = 1 - par;
        si.inj_level1 = 3 - par;
        si.rec_level = par;
        si.rec_level2 = 2 + par;
        si.step_base = via_counter ? counter : nullptr;
        FD_TRY(sparse_launch(si, i, nsrc > 0, nrec > 0, s));
        if (timing) FD_CUDA_TRY(cudaEventRecord(evs.at(i, 3), s));
        if (i % kWatchEvery == kWatchEvery - 1)
            FD_TRY(watchdog_launch(wave, L, 4 * nshots, &dstats->flags, s));
        return FD_OK;
    };
    FD_TRY(run_time_loop(nsteps, s, counter, !timing && trace_level() < 2, step));
    FD_STAGE(s, "tti: time loop");
    const int last = nsteps & 1;
    {
        SparseArgs si = sp;
        si.rec_level = last;
        si.rec_level2 = 2 + last;
        si.step_base = nullptr;
        FD_TRY(sparse_launch(si, nt - 1, false, nrec > 0, s));
    }
    FD_TRY(check_finite(wave, L, 4 * nshots, &dstats->flags, s));
    for (int sh = 0; sh < nshots; ++sh) {
        if (p_final) {
            float *dst = p_final + (size_t)sh * 2 * dense;
            FD_TRY(copy_field_out(dst, wave + (int64_t)(4 * sh + last) * L.vol, L, s));
            FD_TRY(copy_field_out(dst + dense, wave + (int64_t)(4 * sh + 1 - last) * L.vol, L, s));
        }
        if (r_final) {
            float *dst = r_final + (size_t)sh * 2 * dense;
            FD_TRY(copy_field_out(dst, wave + (int64_t)(4 * sh + 2 + last) * L.vol, L, s));
            FD_TRY(copy_field_out(dst + dense, wave + (int64_t)(4 * sh + 3 - last) * L.vol, L, s));
        }
    }
    FD_TRY(srec.copy_back(s));
    FD_TRY(read_stats(dstats, &hs, s));
    if (timing && nsteps > 0) {
        double t1 = 0.0, t2 = 0.0, ts = 0.0;
        for (int i = 0; i < nsteps; ++i) {
            t1 += evs.elapsed(i, 0, 1);
            t2 += evs.elapsed(i, 1, 2);
            ts += evs.elapsed(i, 2, 3);
        }
        if (two_pass) {
            stats_add("tti_pass1", t1, nsteps, (double)dense * nshots);
            stats_add("tti_pass2", t2, nsteps, (double)dense * nshots);
        } else {
            stats_add(fused ? "tti_fused" : "tti_recompute", t1, nsteps, (double)dense * nshots);
        }
        stats_add("sparse", ts, nsteps, (double)(nrec + 16 * nsrc) * nshots);
    }
    ws.release();
    FD_TRY(cs.finish());
    return flags_to_status(hs.flags, "tti_forward");
}

// ====================================================================== adjoint

// Shared setup of the acoustic adjoint and gradient: b, damping, sparse
// tables, validation and the stability check (the same bound as forward).
static fd_status acoustic_common_setup(const fd_grid *grid, int so, double dt, const GridDerived &gd,
                                       int nshots, const float *m, const float *damp, int nsrc,
                                       const float *src_xyz, int nrec, const float *rec_xyz,
                                       float *bcoef, float *dps, SparsePoint *src_tab,
                                       SparsePoint *rec_tab, MediumStats *dstats,
                                       const char *what, cudaStream_t s) {
    const WaveLayout &L = gd.L;
    FD_CUDA_TRY(cudaMemsetAsync(bcoef, 0, (size_t)L.vol * 4, s));
    FD_TRY(init_medium_stats(dstats, s));
    FD_TRY(setup_acoustic_coeffs(m, damp, dt, L, bcoef, dps, dstats, s));
    for (int sh = 0; sh < nshots; ++sh) {
        FD_TRY(setup_sparse_table(src_xyz ? src_xyz + (size_t)sh * nsrc * 3 : nullptr, nsrc,
                                  *grid, L, src_tab + (size_t)sh * nsrc, &dstats->flags, s));
        FD_TRY(setup_sparse_table(rec_xyz ? rec_xyz + (size_t)sh * nrec * 3 : nullptr, nrec,
                                  *grid, L, rec_tab + (size_t)sh * nrec, &dstats->flags, s));
    }
    FD_TRY(finish_medium_stats(dstats, s));
    MediumStats hs;
    FD_TRY(read_stats(dstats, &hs, s));
    FD_TRY(flags_to_status(hs.flags, what));
    const double dt_max = acoustic_dt_bound(*grid, so / 2, (double)hs.m_min);
    if (dt > dt_max * (1.0 + 1e-12))
        return set_error(FD_ERR_CFL, "%s: dt = %.6g ms exceeds the stability bound %.6g ms", what,
                         dt, dt_max);
    return FD_OK;
}

static void fill_step_args(AcousticStepArgs &a, const fd_grid *grid, const GridDerived &gd,
                           float *wave, const float *bcoef, const float *dps, int nshots,
                           unsigned int *err) {
    const WaveLayout &L = gd.L;
    memset(&a, 0, sizeof(a));
    a.wave = wave;
    a.bcoef = bcoef;
    a.dpx = dps;
    a.dpy = dps + L.nx;
    a.dpz = dps + L.nx + L.ny;
    a.L = L;
    a.nshots = nshots;
    a.err = err;
    laplacian_weights(*grid, gd.R, &a.wc, a.wx, a.wy, a.wz);
}

/*
 * Adjoint of the source-to-receiver map (zero initial state).  With the
 * scaled adjoint variable w = b * lambda, the exact discrete adjoint
 *   lambda^n = R^T dd^n + M1^T lambda^{n+1} - M2^T lambda^{n+2}
 * becomes w^n = M1 w^{n+1} - M2 w^{n+2} + B R^T dd^n -- the forward update --
 * so the adjoint runs the forward machinery backwards in time: residuals are
 * injected at the receivers (scaled by b, like a source) and the gradient for
 * source sample n is the interpolation of w^{n+1} at the sources.
 */
static fd_status acoustic_adjoint_impl(const fd_grid *grid, int so, double dt, int nt, int nshots,
                                       const float *m, const float *damp, int nsrc,
                                       const float *src_xyz, float *src_grad, int nrec,
                                       const float *rec_xyz, const float *rec_resid,
                                       cudaStream_t caller) {
    FD_TRY(validate_common(grid, so, dt, nt, nshots, m, nsrc, src_xyz, src_grad, nrec, rec_xyz,
                           rec_resid));
    const int R = so / 2;
    GridDerived gd = derive(grid, so);
    const WaveLayout &L = gd.L;
    const size_t dense = (size_t)L.nx * L.ny * L.nz;
    const int ndamp = L.nx + L.ny + L.nz;
    CallStream cs;
    FD_TRY(cs.begin(caller));
    cudaStream_t s = cs.get();
    Workspace ws;
    float *wave, *bcoef, *dps;
    SparsePoint *src_tab, *rec_tab;
    MediumStats *dstats;
    int *counter;
    ws.add(&wave, (size_t)2 * nshots * L.vol);
    ws.add(&bcoef, L.vol);
    ws.add(&dps, ndamp);
    ws.add(&src_tab, (size_t)nshots * nsrc);
    ws.add(&rec_tab, (size_t)nshots * nrec);
    ws.add(&dstats, 1);
    ws.add(&counter, 1);
    Staged sm, sdamp, ssxyz, srxyz, sres;
    StagedOut sgrad;
    sm.plan(ws, m, dense);
    sdamp.plan(ws, damp, damp ? ndamp : 0);
    ssxyz.plan(ws, src_xyz, (size_t)nshots * nsrc * 3);
    srxyz.plan(ws, rec_xyz, (size_t)nshots * nrec * 3);
    sres.plan(ws, rec_resid, (size_t)nshots * nt * nrec);
    sgrad.plan(ws, src_grad, (size_t)nshots * nt * nsrc);
    FD_TRY(ws.allocate(s));
    for (Staged *st : {&sm, &sdamp, &ssxyz, &srxyz, &sres}) FD_TRY(st->place(s));
    FD_TRY(acoustic_common_setup(grid, so, dt, gd, nshots, sm.dev, sdamp.dev, nsrc, ssxyz.dev,
                                 nrec, srxyz.dev, bcoef, dps, src_tab, rec_tab, dstats,
                                 "acoustic_adjoint", s));
    FD_CUDA_TRY(cudaMemsetAsync(wave, 0, (size_t)2 * nshots * L.vol * 4, s));
    if (sgrad.dev && nsrc > 0)
        FD_CUDA_TRY(cudaMemsetAsync(sgrad.dev, 0, (size_t)nshots * nt * nsrc * 4, s));
    AcousticPlan plan;
    FD_TRY(acoustic_plan(R, g_acoustic_config[R], L, nshots, 2, wave, bcoef, &plan));
    AcousticStepArgs a;
    fill_step_args(a, grid, gd, wave, bcoef, dps, nshots, &dstats->flags);
    // sparse roles swapped: inject residuals at the receivers, sample at the sources
    SparseArgs sp;
    memset(&sp, 0, sizeof(sp));
    sp.wave = wave;
    sp.fields_per_shot = 2;
    sp.L = L;
    sp.bcoef = bcoef;
    sp.nshots = nshots;
    sp.nt = nt;
    sp.nsrc = nrec;
    sp.src_tab = rec_tab;
    sp.src_wav = sres.dev;
    sp.inj_level1 = -1;
    sp.nrec = nsrc;
    sp.rec_tab = src_tab;
    sp.rec_out = sgrad.dev;
    // w^{nt-1} = B R^T dd^{nt-1}
    {
        SparseArgs si = sp;
        si.inj_level0 = 0;
        si.inj_t0 = nt - 1;
        si.inj_dt = 0;
        FD_TRY(sparse_launch(si, 0, nrec > 0, false, s));
    }
    // reversed step i: w~^{i+1} = K1(w~^i, w~^{i-1}) + B R^T dd^{nt-2-i};
    // dq^{nt-2-i} = S w~^i
    const int nsteps = nt - 1;
    auto step = [&](int i, int par, bool via_counter) -> fd_status {
        AcousticStepArgs ai = a;
        set_two_levels(ai, par);
        FD_TRY(acoustic_launch(plan, ai, s));
        SparseArgs si = sp;
        si.inj_level0 = 1 - par;
        si.rec_level = par;
        si.inj_t0 = nt - 2;
        si.inj_dt = -1;
        si.rec_t0 = nt - 2;
        si.rec_dt = -1;
        si.step_base = via_counter ? counter : nullptr;
        FD_TRY(sparse_launch(si, i, nrec > 0, nsrc > 0, s));
        return FD_OK;
    };
    FD_TRY(run_time_loop(nsteps, s, counter, trace_level() < 2, step));
    FD_STAGE(s, "adjoint: time loop");
    FD_TRY(check_finite(wave, L, 2 * nshots, &dstats->flags, s));
    FD_TRY(sgrad.copy_back(s));
    MediumStats hs;
    FD_TRY(read_stats(dstats, &hs, s));
    ws.release();
    FD_TRY(cs.finish());
    return flags_to_status(hs.flags, "acoustic_adjoint");
}

// ====================================================================== gradient

/*
 * FWI gradient: grad m = d<dd, d(m)>/dm, summed over shots (in batches of
 * shots stepped together, as many as the device memory holds).  Forward with a
 * checkpoint (u^t, u^{t-1}) every K steps; then, segment by segment from the
 * last, the forward states of the segment are recomputed from its checkpoint
 * and the adjoint w (see acoustic_adjoint) is stepped back through it while
 *   grad += w^k (u^k - 2 u^{k-1} + u^{k-2}),   k = nt-1 .. 1,
 * and finally grad *= -1/dt^2 (du^k/dm = -(u^k - 2u^{k-1} + u^{k-2})/(m+eta)
 * and w = dt^2/(m+eta) lambda).
 */
static fd_status acoustic_gradient_impl(const fd_grid *grid, int so, double dt, int nt,
                                        int nshots, const float *m, const float *damp, int nsrc,
                                        const float *src_xyz, const float *src_wav, int nrec,
                                        const float *rec_xyz, const float *rec_resid,
                                        int checkpoint_every, float *grad_m,
                                        cudaStream_t caller) {
    FD_TRY(validate_common(grid, so, dt, nt, nshots, m, nsrc, src_xyz, src_wav, nrec, rec_xyz,
                           rec_resid));
    if (!grad_m) return set_error(FD_ERR_ARG, "acoustic_gradient: grad_m is null");
    if (checkpoint_every < 0) return set_error(FD_ERR_ARG, "checkpoint_every must be >= 0");
    const int R = so / 2;
    GridDerived gd = derive(grid, so);
    const WaveLayout &L = gd.L;
    const size_t dense = (size_t)L.nx * L.ny * L.nz;
    const int ndamp = L.nx + L.ny + L.nz;
    const int nsteps = nt - 1;
    int K = checkpoint_every > 0 ? checkpoint_every : (int)lround(sqrt((double)(nsteps > 1 ? nsteps : 1)));
    if (K < 1) K = 1;
    if (nsteps > 0 && K > nsteps) K = nsteps;
    const int nseg = nsteps > 0 ? (nsteps + K - 1) / K : 0;
    CallStream cs;
    FD_TRY(cs.begin(caller));
    cudaStream_t s = cs.get();
    // Shots are processed in batches of B (one stencil launch per step for the
    // whole batch); B is bounded by the device memory the per-shot buffers
    // (forward and adjoint pairs, the segment, the checkpoints) need.
    const int64_t vol = L.vol;
    const int64_t per_shot = (int64_t)(4 + (K + 2) + 2 * (nseg > 0 ? nseg : 1)) * vol * 4;
    int B = 1;
    {
        size_t free_b = 0, total_b = 0;
        FD_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        const int64_t fixed = (int64_t)(4 + 2) * vol * 4 +
                              (int64_t)nshots * (int64_t)nt * (nrec + nsrc) * 4;
        const int64_t budget = (int64_t)(0.8 * (double)free_b) - fixed;
        const int64_t fit = per_shot > 0 ? budget / per_shot : 1;
        B = (int)(fit < 1 ? 1 : (fit > nshots ? nshots : fit));
        // FDSWEEP_GRAD_BATCH=n caps the batch (to exercise several batches)
        const char *cap = getenv("FDSWEEP_GRAD_BATCH");
        if (cap && atoi(cap) > 0 && atoi(cap) < B) B = atoi(cap);
    }
    Workspace ws;
    float *fwd, *adj, *seg, *ckpt, *grad, *bcoef, *dps;
    SparsePoint *src_tab, *rec_tab;
    MediumStats *dstats;
    ws.add(&fwd, (size_t)2 * B * vol);
    ws.add(&adj, (size_t)2 * B * vol);
    ws.add(&seg, (size_t)(K + 2) * B * vol);
    ws.add(&ckpt, (size_t)2 * (nseg > 0 ? nseg : 1) * B * vol);
    ws.add(&grad, vol);
    ws.add(&bcoef, vol);
    ws.add(&dps, ndamp);
    ws.add(&src_tab, (size_t)nshots * nsrc);
    ws.add(&rec_tab, (size_t)nshots * nrec);
    ws.add(&dstats, 1);
    Staged sm, sdamp, ssxyz, swav, srxyz, sres;
    StagedOut sg;
    sm.plan(ws, m, dense);
    sdamp.plan(ws, damp, damp ? ndamp : 0);
    ssxyz.plan(ws, src_xyz, (size_t)nshots * nsrc * 3);
    swav.plan(ws, src_wav, (size_t)nshots * nt * nsrc);
    srxyz.plan(ws, rec_xyz, (size_t)nshots * nrec * 3);
    sres.plan(ws, rec_resid, (size_t)nshots * nt * nrec);
    sg.plan(ws, grad_m, dense);
    FD_TRY(ws.allocate(s));
    for (Staged *st : {&sm, &sdamp, &ssxyz, &swav, &srxyz, &sres}) FD_TRY(st->place(s));
    FD_TRY(acoustic_common_setup(grid, so, dt, gd, nshots, sm.dev, sdamp.dev, nsrc, ssxyz.dev,
                                 nrec, srxyz.dev, bcoef, dps, src_tab, rec_tab, dstats,
                                 "acoustic_gradient", s));
    FD_CUDA_TRY(cudaMemsetAsync(grad, 0, (size_t)vol * 4, s));
    const size_t vb = (size_t)vol * 4;
    for (int s0 = 0; s0 < nshots && nsteps > 0; s0 += B) {
        const int nb = nshots - s0 < B ? nshots - s0 : B;
        AcousticPlan pf, pa, ps;
        FD_TRY(acoustic_plan(R, g_acoustic_config[R], L, nb, 2, fwd, bcoef, &pf));
        FD_TRY(acoustic_plan(R, g_acoustic_config[R], L, nb, 2, adj, bcoef, &pa));
        FD_TRY(acoustic_plan(R, g_acoustic_config[R], L, nb, K + 2, seg, bcoef, &ps));
        AcousticStepArgs af, aa, as;
        fill_step_args(af, grid, gd, fwd, bcoef, dps, nb, &dstats->flags);
        fill_step_args(aa, grid, gd, adj, bcoef, dps, nb, &dstats->flags);
        fill_step_args(as, grid, gd, seg, bcoef, dps, nb, &dstats->flags);
        // sources of the batch's shots, and residuals injected at their receivers
        SparseArgs src;
        memset(&src, 0, sizeof(src));
        src.L = L;
        src.bcoef = bcoef;
        src.nshots = nb;
        src.nt = nt;
        src.nsrc = nsrc;
        src.src_tab = src_tab + (size_t)s0 * nsrc;
        src.src_wav = swav.dev ? swav.dev + (size_t)s0 * nt * nsrc : nullptr;
        src.inj_level1 = -1;
        src.inj_dt = 1;
        src.rec_dt = 1;
        SparseArgs res = src;
        res.nsrc = nrec;
        res.src_tab = rec_tab + (size_t)s0 * nrec;
        res.src_wav = sres.dev + (size_t)s0 * nt * nrec;
        // 1. forward with checkpoints: ckpt[c] holds (u^{cK-1}, u^{cK}) of every
        //    shot of the batch ([nseg][nb][2][vol])
        FD_CUDA_TRY(cudaMemsetAsync(fwd, 0, 2 * nb * vb, s));
        for (int t = 0; t < nsteps; ++t) {
            const int cur = t & 1;
            if (t % K == 0) {
                float *dst = ckpt + (size_t)(t / K) * 2 * nb * vol;
                FD_CUDA_TRY(cudaMemcpy2DAsync(dst, 2 * vb, fwd + (size_t)(1 - cur) * vol, 2 * vb,
                                              vb, nb, cudaMemcpyDeviceToDevice, s));
                FD_CUDA_TRY(cudaMemcpy2DAsync(dst + vol, 2 * vb, fwd + (size_t)cur * vol, 2 * vb,
                                              vb, nb, cudaMemcpyDeviceToDevice, s));
            }
            AcousticStepArgs ai = af;
            set_two_levels(ai, cur);
            FD_TRY(acoustic_launch(pf, ai, s));
            SparseArgs si = src;
            si.wave = fwd;
            si.fields_per_shot = 2;
            si.inj_level0 = 1 - cur;
            FD_TRY(sparse_launch(si, t, nsrc > 0, false, s));
        }
        // 2. adjoint state: w^{nt-1} = B R^T dd^{nt-1} in level acur, w^{nt} = 0
        FD_CUDA_TRY(cudaMemsetAsync(adj, 0, 2 * nb * vb, s));
        int acur = 0;
        {
            SparseArgs si = res;
            si.wave = adj;
            si.fields_per_shot = 2;
            si.inj_level0 = acur;
            si.inj_t0 = nt - 1;
            si.inj_dt = 0;
            FD_TRY(sparse_launch(si, 0, nrec > 0, false, s));
        }
        // 3. segments from the last
        for (int c = nseg - 1; c >= 0; --c) {
            const int t0 = c * K;
            const int kmax = (c + 1) * K < nsteps ? (c + 1) * K : nsteps;
            // seg level l of every shot holds u^{t0 - 1 + l}
            FD_CUDA_TRY(cudaMemcpy2DAsync(seg, (size_t)(K + 2) * vb,
                                          ckpt + (size_t)c * 2 * nb * vol, 2 * vb, 2 * vb, nb,
                                          cudaMemcpyDeviceToDevice, s));
            for (int t = t0 + 1; t <= kmax; ++t) {
                AcousticStepArgs ai = as;
                ai.lps = K + 2;
                ai.lev_cur = t - t0;
                ai.lev_prev = t - t0 - 1;
                ai.lev_out = t - t0 + 1;
                FD_TRY(acoustic_launch(ps, ai, s));
                SparseArgs si = src;
                si.wave = seg;
                si.fields_per_shot = K + 2;
                si.inj_level0 = t - t0 + 1;
                FD_TRY(sparse_launch(si, t - 1, nsrc > 0, false, s));
            }
            for (int k = kmax; k >= t0 + 1; --k) {
                FD_TRY(grad_accumulate_batch(grad, adj + (size_t)acur * vol, 2 * vol,
                                             seg + (size_t)(k - t0 + 1) * vol,
                                             (int64_t)(K + 2) * vol, nb, vol, s));
                if (k >= 2) {
                    // w^{k-1} = M1 w^k - M2 w^{k+1} + B R^T dd^{k-1}
                    AcousticStepArgs ai = aa;
                    set_two_levels(ai, acur);
                    FD_TRY(acoustic_launch(pa, ai, s));
                    SparseArgs si = res;
                    si.wave = adj;
                    si.fields_per_shot = 2;
                    si.inj_level0 = 1 - acur;
                    si.inj_t0 = k - 1;
                    si.inj_dt = 0;
                    FD_TRY(sparse_launch(si, 0, nrec > 0, false, s));
                    acur = 1 - acur;
                }
            }
        }
        FD_STAGE(s, "gradient: shot batch done");
    }
    FD_TRY(scale_field(grad, (float)(-1.0 / (dt * dt)), L.vol, s));
    FD_TRY(check_finite(grad, L, 1, &dstats->flags, s));
    FD_TRY(copy_field_out(sg.dev, grad, L, s));
    FD_TRY(sg.copy_back(s));
    MediumStats hs;
    FD_TRY(read_stats(dstats, &hs, s));
    ws.release();
    FD_TRY(cs.finish());
    return flags_to_status(hs.flags, "acoustic_gradient");
}

}  // namespace fdsweep

// ====================================================================== C ABI

extern "C" {

fd_status acoustic_forward(const fd_grid *grid, int so, double dt, int nt, int nshots,
                           const float *m, const float *damp, int nsrc, const float *src_xyz,
                           const float *src_wav, int nrec, const float *rec_xyz, float *rec_out,
                           const float *u_init, float *u_final, void *stream) {
    fdsweep::clear_error();
    return fdsweep::acoustic_forward_impl(grid, so, dt, nt, nshots, m, damp, nsrc, src_xyz,
                                          src_wav, nrec, rec_xyz, rec_out, u_init, u_final,
                                          static_cast<cudaStream_t>(stream));
}

fd_status acoustic_forward_opts(const fd_grid *grid, int so, double dt, int nt, int nshots,
                                const float *m, const float *damp, int nsrc,
                                const float *src_xyz, const float *src_wav, int nrec,
                                const float *rec_xyz, float *rec_out, const float *u_init,
                                float *u_final, const fd_acoustic_options *opts, void *stream) {
    fdsweep::clear_error();
    int storage = opts ? opts->storage : FD_STORAGE_F32;
    const int layout = opts ? opts->damp_layout : FD_DAMP_AXES;
    if (layout != FD_DAMP_AXES && layout != FD_DAMP_FIELD)
        return fdsweep::set_error(FD_ERR_ARG, "acoustic_forward_opts: damp_layout %d not in {0, 1}",
                                  layout);
    // FD_STORAGE_AUTO: binary16 storage where its kernel measured faster than
    // the FP32 one on GB300 at 512^3 (so <= 8: 1.26x and 1.10x), FP32 storage
    // where it did not (so 12: 0.94x, so 16: 0.89x; the binary16 kernel is
    // bound by shared memory and conversions there), and FP32 with a 3-D
    // damping field.
    if (storage == FD_STORAGE_AUTO)
        storage = (so <= 8 && layout == FD_DAMP_AXES) ? FD_STORAGE_F16 : FD_STORAGE_F32;
    if (storage == FD_STORAGE_F32)
        return fdsweep::acoustic_forward_impl(grid, so, dt, nt, nshots, m, damp, nsrc, src_xyz,
                                              src_wav, nrec, rec_xyz, rec_out, u_init, u_final,
                                              (cudaStream_t)stream, layout == FD_DAMP_FIELD);
    if (layout == FD_DAMP_FIELD)
        return fdsweep::set_error(FD_ERR_ARG,
                                  "acoustic_forward_opts: a 3-D damping field needs FP32 storage");
    if (storage == FD_STORAGE_F16)
        return fdsweep::acoustic_forward_h_impl(grid, so, dt, nt, nshots, m, damp, nsrc, src_xyz,
                                                src_wav, nrec, rec_xyz, rec_out, u_init, u_final,
                                                (cudaStream_t)stream);
    return fdsweep::set_error(FD_ERR_ARG, "acoustic_forward_opts: storage %d not in {0, 1, 2}",
                              storage);
}

fd_status tti_forward(const fd_grid *grid, int so, double dt, int nt, int nshots, const float *m,
                      const float *damp, const float *epsilon, const float *delta,
                      const float *theta, const float *phi, int nsrc, const float *src_xyz,
                      const float *src_wav, int nrec, const float *rec_xyz, float *rec_out,
                      const float *p_init, const float *r_init, float *p_final, float *r_final,
                      void *stream) {
    fdsweep::clear_error();
    return fdsweep::tti_forward_impl(grid, so, dt, nt, nshots, m, damp, epsilon, delta, theta,
                                     phi, nsrc, src_xyz, src_wav, nrec, rec_xyz, rec_out, p_init,
                                     r_init, p_final, r_final, nullptr,
                                     static_cast<cudaStream_t>(stream));
}

fd_status tti_forward_opts(const fd_grid *grid, int so, double dt, int nt, int nshots,
                           const float *m, const float *damp, const float *epsilon,
                           const float *delta, const float *theta, const float *phi, int nsrc,
                           const float *src_xyz, const float *src_wav, int nrec,
                           const float *rec_xyz, float *rec_out, const float *p_init,
                           const float *r_init, float *p_final, float *r_final,
                           const fd_tti_options *opts, void *stream) {
    fdsweep::clear_error();
    return fdsweep::tti_forward_impl(grid, so, dt, nt, nshots, m, damp, epsilon, delta, theta,
                                     phi, nsrc, src_xyz, src_wav, nrec, rec_xyz, rec_out, p_init,
                                     r_init, p_final, r_final, opts,
                                     static_cast<cudaStream_t>(stream));
}

fd_status acoustic_adjoint(const fd_grid *grid, int so, double dt, int nt, int nshots,
                           const float *m, const float *damp, int nsrc, const float *src_xyz,
                           float *src_grad, int nrec, const float *rec_xyz,
                           const float *rec_resid, void *stream) {
    fdsweep::clear_error();
    return fdsweep::acoustic_adjoint_impl(grid, so, dt, nt, nshots, m, damp, nsrc, src_xyz,
                                          src_grad, nrec, rec_xyz, rec_resid,
                                          static_cast<cudaStream_t>(stream));
}

fd_status acoustic_gradient(const fd_grid *grid, int so, double dt, int nt, int nshots,
                            const float *m, const float *damp, int nsrc, const float *src_xyz,
                            const float *src_wav, int nrec, const float *rec_xyz,
                            const float *rec_resid, int checkpoint_every, float *grad_m,
                            void *stream) {
    fdsweep::clear_error();
    return fdsweep::acoustic_gradient_impl(grid, so, dt, nt, nshots, m, damp, nsrc, src_xyz,
                                           src_wav, nrec, rec_xyz, rec_resid, checkpoint_every,
                                           grad_m, static_cast<cudaStream_t>(stream));
}

const char *fd_last_error(void) { return fdsweep::last_error(); }

int64_t fd_launch_count(void) { return fdsweep::launch_count(); }

fd_status fd_set_wait_limit_ns(int64_t ns) {
    fdsweep::clear_error();
    fdsweep::set_wait_limit_ns(ns > 0 ? (uint64_t)ns : 0);
    return FD_OK;
}

fd_status fd_stencil_weights(const fd_grid *grid, int so, float *centre, float *w) {
    fdsweep::clear_error();
    if (!centre || !w) return fdsweep::set_error(FD_ERR_ARG, "fd_stencil_weights: null output");
    if (!fdsweep::valid_so(so))
        return fdsweep::set_error(FD_ERR_SO, "space order %d not in {2,4,8,12,16}", so);
    FD_TRY(fdsweep::validate_grid(grid));
    const int K = fdsweep::kMaxRadius + 1;
    fdsweep::laplacian_weights(*grid, so / 2, centre, w, w + K, w + 2 * K);
    return FD_OK;
}

const char *fd_version(void) { return "fdsweep 0.1 (sm_103a)"; }

fd_status fd_stats_enable(int on) { return fdsweep::stats_enable(on); }
fd_status fd_stats_reset(void) { return fdsweep::stats_reset(); }
fd_status fd_stats_get(const char *family, double *total_ms, int64_t *launches,
                       double *points_per_launch) {
    return fdsweep::stats_get(family, total_ms, launches, points_per_launch);
}

fd_status fd_set_tti_config(int so, int config) {
    fdsweep::clear_error();
    if (!fdsweep::valid_so(so)) return fdsweep::set_error(FD_ERR_SO, "space order %d", so);
    const int R = so / 2;
    if (config < -1 || config >= fdsweep::tti_num_configs(R))
        return fdsweep::set_error(FD_ERR_ARG, "TTI configuration %d out of range for so = %d",
                                  config, so);
    fdsweep::g_tti_config[R] = config;
    return FD_OK;
}

int fd_num_tti_configs(int so) {
    return fdsweep::valid_so(so) ? fdsweep::tti_num_configs(so / 2) : 0;
}

fd_status fd_set_time_tiling(int so, int mode) {
    fdsweep::clear_error();
    if (!fdsweep::valid_so(so)) return fdsweep::set_error(FD_ERR_SO, "space order %d", so);
    const int R = so / 2;
    if (mode < -1 || mode > fdsweep::acoustic2_num_configs(R))
        return fdsweep::set_error(FD_ERR_ARG, "time tiling mode %d out of range for so = %d",
                                  mode, so);
    fdsweep::g_time_tiling[R] = mode;
    return FD_OK;
}

int fd_num_time_tiling_configs(int so) {
    return fdsweep::valid_so(so) ? fdsweep::acoustic2_num_configs(so / 2) : 0;
}

fd_status fd_set_acoustic_f16_config(int so, int config) {
    if (!fdsweep::valid_so(so)) return fdsweep::set_error(FD_ERR_SO, "bad so %d", so);
    const int r = so / 2;
    if (config < -1 || config >= fdsweep::acoustic_h_num_configs(r))
        return fdsweep::set_error(FD_ERR_ARG, "binary16 config %d out of range for so %d",
                                  config, so);
    fdsweep::g_acoustic_h_config[r] = config;
    return FD_OK;
}

int fd_num_acoustic_f16_configs(int so) {
    return fdsweep::valid_so(so) ? fdsweep::acoustic_h_num_configs(so / 2) : 0;
}

fd_status fd_set_acoustic_config(int so, int config) {
    if (!fdsweep::valid_so(so)) return fdsweep::set_error(FD_ERR_SO, "bad space order %d", so);
    const int R = so / 2;
    if (config < -1 || config >= fdsweep::acoustic_num_configs(R))
        return fdsweep::set_error(FD_ERR_ARG, "config %d out of range for so %d", config, so);
    fdsweep::g_acoustic_config[R] = config;
    return FD_OK;
}

int fd_num_acoustic_configs(int so) {
    return fdsweep::valid_so(so) ? fdsweep::acoustic_num_configs(so / 2) : 0;
}

}  // extern "C"
