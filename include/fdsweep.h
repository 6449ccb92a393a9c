/*
 * fdsweep.h -- C ABI of the GB300 (sm_103a) finite-difference wave-propagation
 * sweep: the time-stepped 3-D stencil operators of arXiv:1807.03032 (Devito),
 * isotropic acoustic and TTI, with sparse source injection and receiver
 * interpolation.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Arrays are C order [z][y][x] (x fastest).  Grid index (i, j, k) sits at
 *    coordinate (ox + i hx, oy + j hy, oz + k hz).  The grid shape includes
 *    the absorbing border ("Domain" region of the paper's section "Domain,
 *    halo, and padding regions"); points outside it are zero ghosts.
 *  - Units: m, ms, km/s (= m/ms); m = 1/v^2 in ms^2/m^2.
 *  - so (space order) is one of 2, 4, 8, 12, 16; the stencil radius is so/2.
 *  - Every pointer may be device memory or host memory (pinned or pageable);
 *    the library detects which with cudaPointerGetAttributes and copies host
 *    data through its own device workspace.  Pointers are owned by the
 *    caller; the library never frees or retains them.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default
 *    stream).  The library allocates its workspace with cudaMallocAsync on
 *    that stream and frees it before returning.  Each call synchronises the
 *    stream once, at its end, to report device-side errors; when it returns
 *    FD_OK all outputs are complete.
 *  - Errors: a negative fd_status; fd_last_error() returns a message for the
 *    calling thread.  Outputs are unspecified after an error.  Arguments are
 *    validated before any launch: bad sizes or null required pointers give
 *    FD_ERR_ARG, an unsupported space order FD_ERR_SO, a time step above the
 *    stability bound FD_ERR_CFL, a sparse point outside the grid
 *    FD_ERR_COORD, a failed allocation FD_ERR_OOM, a non-finite final field
 *    FD_ERR_DIVERGED, any CUDA failure FD_ERR_CUDA, a device-side wait that
 *    ran out FD_ERR_TIMEOUT.
 *  - Shots are the outermost dimension of per-shot arrays; all shots share
 *    the medium (m, damp and the TTI fields).
 */
#ifndef FDSWEEP_H
#define FDSWEEP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Grid descriptor (the paper's Grid(shape, extent, origin), section
 * "Symbolic types"). */
typedef struct {
    int32_t nx, ny, nz; /* points per axis, including the absorbing border */
    double hx, hy, hz;  /* spacing [m] */
    double ox, oy, oz;  /* origin [m] */
} fd_grid;

typedef enum {
    FD_OK = 0,
    FD_ERR_ARG = -1,
    FD_ERR_CFL = -2,
    FD_ERR_SO = -3,
    FD_ERR_COORD = -4,
    FD_ERR_OOM = -5,
    FD_ERR_CUDA = -6,
    FD_ERR_DIVERGED = -7,
    FD_ERR_UNIMPL = -8,
    FD_ERR_TIMEOUT = -9
} fd_status;

/*
 * acoustic_forward -- isotropic acoustic forward model.
 *
 * Solves m u_tt + damp u_t - lap(u) = src (Eq. WE with an absorbing term)
 * with the explicit leapfrog of Listing fd-3, central compact Laplacian of
 * order `so` (Listing fd-1/fd-2), damping discretised centrally:
 *   u^{n+1} = (dt^2 lap u^n + m (2u^n - u^{n-1}) + eta u^{n-1}) / (m + eta),
 *   eta = damp dt / 2.
 * Per step n = 0..nt-2: stencil update; then source samples src_wav[n] are
 * injected into u^{n+1} with trilinear weights w_c and scale
 * dt^2 / (m + eta) at each node (Eq. interp, Listing finject); receivers
 * record rec[n] = sum_c w_c u^n(node_c).  Finally rec[nt-1] samples u^{nt-1}.
 * Interpolation index x1 = floor((x - o)/h) (FP64), clamped to n-2.
 *
 *   grid      shape/spacing/origin; nx, ny, nz > so.
 *   so        space order (2, 4, 8, 12, 16).
 *   dt        time step [ms]; must satisfy the leapfrog stability bound
 *             dt <= 2 / (v_max sqrt(sum_d sigma/h_d^2)), v_max = 1/sqrt(min m),
 *             sigma = max of the stencil's symbol (else FD_ERR_CFL).
 *   nt        number of time samples (>= 1); nt-1 steps are taken.
 *   nshots    independent shots sharing the medium (>= 1).
 *   m         [nz][ny][nx] squared slowness, finite and > 0.
 *   damp      NULL (no damping) or [nx + ny + nz]: per-axis profiles
 *             (x block, then y, then z); damp(i,j,k) = dx[i] + dy[j] + dz[k],
 *             finite and >= 0.
 *   nsrc, src_xyz [nshots][nsrc][3], src_wav [nshots][nt][nsrc]: sources.
 *   nrec, rec_xyz [nshots][nrec][3]: receivers; rec_out [nshots][nt][nrec]
 *             (may be NULL when nrec = 0).
 *   u_init    NULL (zero initial state, Eq. WE) or [nshots][2][nz][ny][nx]
 *             holding (u^0, u^{-1}).
 *   u_final   NULL or [nshots][2][nz][ny][nx] receiving (u^{nt-1}, u^{nt-2}).
 *   stream    cudaStream_t to run on.
 */
fd_status acoustic_forward(const fd_grid *grid, int so, double dt, int nt, int nshots,
                           const float *m, const float *damp, int nsrc, const float *src_xyz,
                           const float *src_wav, int nrec, const float *rec_xyz, float *rec_out,
                           const float *u_init, float *u_final, void *stream);

/*
 * acoustic_forward_opts -- acoustic_forward with a choice of storage
 * precision and of the damping input's layout.  The paper names mixed-precision arithmetic and on-the-fly data
 * compression as further performance work (section "Further work"); the step
 * is memory bound, so halving the stored bytes per point is the lever.
 *
 *   opts->storage  FD_STORAGE_F32: FP32 storage, identical to acoustic_forward.
 *                  FD_STORAGE_F16: the wavefield levels and the coefficient
 *                  b = dt^2/(m + damp dt/2) are held in IEEE binary16 on the
 *                  device (8 instead of 16 bytes per point and step); every
 *                  value is decoded exactly to FP32, the update and the
 *                  sparse operations compute in FP32, and each stored result
 *                  is rounded to the nearest binary16 (ties to even; a source
 *                  contribution is rounded to binary16 and added with one
 *                  more rounding).  u_init is rounded on entry; u_final and
 *                  the traces are the FP32 values of the stored binary16
 *                  fields.  The stored values carry a relative rounding error
 *                  of up to 2^-11 per step, which accumulates: expect traces
 *                  within about 1e-3 and late wavefields within about 1e-2 of
 *                  the FP32 result after a few hundred steps, and no value
 *                  above 65504 in magnitude (beyond it the run reports
 *                  FD_ERR_DIVERGED).  Radii with a binary16 kernel: so = 2..16
 *                  (FD_ERR_UNIMPL otherwise); time tiling is not combined
 *                  with it.
 *                  FD_STORAGE_AUTO: the faster of the two on GB300 for the
 *                  space order, measured at 512^3: binary16 for so <= 8 (its
 *                  kernel 1.26x / 1.10x the FP32 one at so 4 / 8), FP32 for
 *                  so 12 and 16 (where the binary16 kernel, bound by shared
 *                  memory and conversions, ran 0.94x / 0.89x), and FP32 with
 *                  FD_DAMP_FIELD.  The results are those of the storage
 *                  chosen.
 *   opts->damp_layout
 *                  FD_DAMP_AXES: damp holds the per-axis profiles
 *                  [nx + ny + nz] of acoustic_forward (damp(i,j,k) = d_x[i] +
 *                  d_y[j] + d_z[k]; the stencil forms the damping from them,
 *                  16 bytes per point and step).
 *                  FD_DAMP_FIELD: damp is a 3-D field [nz][ny][nx] (any
 *                  finite non-negative absorbing mask, separable or not; the
 *                  paper's section "Test case setup" names only "absorbing
 *                  boundaries with a 10 point mask").  The stencil kernel
 *                  then reads one more coefficient per point, zeta = damp b
 *                  / dt (20 bytes per point and step).  FP32 storage only
 *                  (FD_ERR_ARG with FD_STORAGE_F16); time tiling is not
 *                  combined with it.  NULL damp: no damping, either layout.
 *   opts           NULL selects FD_STORAGE_F32 and FD_DAMP_AXES.
 *                  Out-of-range values return FD_ERR_ARG.
 * Other arguments, ownership and errors as for acoustic_forward.
 */
enum { FD_STORAGE_F32 = 0, FD_STORAGE_F16 = 1, FD_STORAGE_AUTO = 2 };
enum { FD_DAMP_AXES = 0, FD_DAMP_FIELD = 1 };
typedef struct {
    int32_t storage;
    int32_t damp_layout;
} fd_acoustic_options;

fd_status acoustic_forward_opts(const fd_grid *grid, int so, double dt, int nt, int nshots,
                                const float *m, const float *damp, int nsrc,
                                const float *src_xyz, const float *src_wav, int nrec,
                                const float *rec_xyz, float *rec_out, const float *u_init,
                                float *u_final, const fd_acoustic_options *opts, void *stream);

/*
 * tti_forward -- tilted transverse isotropy (TTI) forward model.
 *
 * Two coupled acoustic equations whose Laplacians are built from rotated
 * first-derivative operators (section "Test case setup"):
 *   Hz q  = sum_i D_i( n_i sum_j n_j D_j q ),  L q = sum_i D_i D_i q,
 *   Hxy q = L q - Hz q,  n = (sin(theta) cos(phi), sin(theta) sin(phi), cos(theta)),
 *   m p_tt + damp p_t = (1 + 2 eps) Hxy p + sqrt(1 + 2 delta) Hz r,
 *   m r_tt + damp r_t = sqrt(1 + 2 delta) Hxy p + Hz r,
 * D_i the central first derivative of order so along axis i (zero ghosts
 * outside the grid, also for the intermediate D_j q terms).  Each equation is
 * advanced with the same centred leapfrog as acoustic_forward; the source is
 * injected into p and r with the same scale; receivers record p.
 *
 *   epsilon, delta, theta, phi  [nz][ny][nx]; eps >= delta >= -1/2 pointwise
 *             (otherwise the system is not hyperbolic: FD_ERR_ARG).
 *   dt        must satisfy dt <= 2 / sqrt(max(1+2eps) v_max^2 sum_d s/h_d^2),
 *             s = max of the squared first-derivative symbol (else FD_ERR_CFL).
 *   p_init, r_init  NULL or [nshots][2][nz][ny][nx] (levels n, n-1).
 *   p_final, r_final NULL or [nshots][2][nz][ny][nx].
 *   rec_out   [nshots][nt][nrec] samples of p.
 *   Other arguments as for acoustic_forward.
 * The kernels: one fused kernel per step with the first-derivative
 * temporaries in shared memory for so <= 4, two passes with the temporaries
 * in device memory above (see tti_forward_opts).
 */
fd_status tti_forward(const fd_grid *grid, int so, double dt, int nt, int nshots, const float *m,
                      const float *damp, const float *epsilon, const float *delta,
                      const float *theta, const float *phi, int nsrc, const float *src_xyz,
                      const float *src_wav, int nrec, const float *rec_xyz, float *rec_out,
                      const float *p_init, const float *r_init, float *p_final, float *r_final,
                      void *stream);

/*
 * tti_forward_opts -- tti_forward with the alternative readings and schemes
 * of the TTI ablation.  The paper builds the TTI Laplacians from "rotated
 * first derivative operators" (section "Test case setup") without saying
 * which first derivative, nor which field the receivers record; its
 * performance section compares operators generated with and without
 * shift-invariant temporaries (`advanced` vs `aggressive`, Table tti:ops).
 *
 *   opts->deriv     FD_TTI_CENTRED: D_i central of order so (tti_forward);
 *                   FD_TTI_STAGGERED: inner derivatives D+_j (half a node
 *                   ahead) and outer D-_i (half a node behind), weights
 *                   a_k = (-1)^(k+1) ((2r-1)!!)^2 / (4^(r-1) (2k-1)^2
 *                   (r+k-1)! (r-k)!), so that D- = -(D+)^T and
 *                   L q = sum_i D-_i D+_i q; n stays at the nodes.  The
 *                   stability bound uses the staggered symbol.
 *   opts->receiver  FD_TTI_REC_P: receivers record p; FD_TTI_REC_MEAN: they
 *                   record (p + r)/2.
 *   opts->scheme    FD_TTI_AUTO (what tti_forward uses): FD_TTI_FUSED for
 *                   so <= 4, FD_TTI_TWO_PASS otherwise (the faster on GB300);
 *                   FD_TTI_TWO_PASS: six first-derivative temporaries per
 *                   point are written to device memory once and
 *                   differentiated again by a second kernel (the default,
 *                   linear work in so); FD_TTI_FUSED: one kernel, the
 *                   temporaries of each plane kept in shared memory
 *                   (so <= 8, else FD_ERR_ARG); FD_TTI_RECOMPUTE: no
 *                   temporaries, the inner derivatives are recomputed at
 *                   every outer stencil point (work quadratic in so).  The
 *                   last two use 6 fewer fields of device memory.
 *   opts            NULL selects the tti_forward defaults (centred, p,
 *                   automatic scheme).  Out-of-range values return FD_ERR_ARG.
 * Other arguments, ownership and errors as for tti_forward.
 */
enum { FD_TTI_CENTRED = 0, FD_TTI_STAGGERED = 1 };
enum { FD_TTI_REC_P = 0, FD_TTI_REC_MEAN = 1 };
enum { FD_TTI_AUTO = -1, FD_TTI_TWO_PASS = 0, FD_TTI_RECOMPUTE = 1, FD_TTI_FUSED = 2 };
typedef struct {
    int32_t deriv;
    int32_t receiver;
    int32_t scheme;
} fd_tti_options;

fd_status tti_forward_opts(const fd_grid *grid, int so, double dt, int nt, int nshots,
                           const float *m, const float *damp, const float *epsilon,
                           const float *delta, const float *theta, const float *phi, int nsrc,
                           const float *src_xyz, const float *src_wav, int nrec,
                           const float *rec_xyz, float *rec_out, const float *p_init,
                           const float *r_init, float *p_final, float *r_final,
                           const fd_tti_options *opts, void *stream);

/*
 * acoustic_adjoint -- adjoint of acoustic_forward's source-to-receiver map.
 *
 * The paper motivates saving the forward wavefield with "data inversion using
 * adjoint-state methods" (section "Control flow") but prints no adjoint; this
 * is the exact transpose of the discrete forward map of acoustic_forward
 * (zero initial state), so that <F q, d> = <q, F^T d> holds to rounding:
 *   lambda^n = R^T d^n + M1^T lambda^{n+1} - M2^T lambda^{n+2},
 *   q_adj^n = S B lambda^{n+1} (n <= nt-2),  q_adj^{nt-1} = 0,
 * with M1 = 2 - zeta + B L, M2 = 1 - zeta, B = dt^2/(m + damp dt/2), R the
 * receiver and S the source interpolation.  It runs the forward kernels
 * backwards in time on w = B lambda.
 *
 *   rec_resid [nshots][nt][nrec]  input traces (residuals) at the receivers.
 *   src_grad  [nshots][nt][nsrc]  output: adjoint source wavelets.
 *   Other arguments, validation and errors as for acoustic_forward.
 */
fd_status acoustic_adjoint(const fd_grid *grid, int so, double dt, int nt, int nshots,
                           const float *m, const float *damp, int nsrc, const float *src_xyz,
                           float *src_grad, int nrec, const float *rec_xyz,
                           const float *rec_resid, void *stream);

/*
 * acoustic_gradient -- gradient with respect to m of <rec_resid, d(m)>, where
 * d(m) are acoustic_forward's traces (zero initial state), summed over shots.
 * With rec_resid = d(m) - d_obs this is the FWI gradient of
 * J(m) = 1/2 sum ||d(m) - d_obs||^2 (adjoint-state method):
 *   grad m = -(1/dt^2) sum_{k=1}^{nt-1} w^k (u^k - 2u^{k-1} + u^{k-2}),
 * w the adjoint of acoustic_adjoint.  The forward wavefield is checkpointed
 * (both time levels) every `checkpoint_every` steps (0: round(sqrt(nt-1)))
 * and recomputed segment by segment during the reverse sweep (the paper's
 * time-subsampled save, Listing fd-4, used for inversion).
 *
 *   src_wav   [nshots][nt][nsrc]  source wavelets of the forward model.
 *   rec_resid [nshots][nt][nrec]  residual traces.
 *   grad_m    [nz][ny][nx]        output.
 *   Device memory: 4 + K + 2 + 2 ceil((nt-1)/K) wavefield volumes per shot
 *   of a batch, K the checkpoint interval; shots are stepped together in
 *   batches of as many as fit in 80 % of the free device memory (at least
 *   one; the environment variable FDSWEEP_GRAD_BATCH=n caps the batch).
 *   Other arguments as for acoustic_forward.
 */
fd_status acoustic_gradient(const fd_grid *grid, int so, double dt, int nt, int nshots,
                            const float *m, const float *damp, int nsrc, const float *src_xyz,
                            const float *src_wav, int nrec, const float *rec_xyz,
                            const float *rec_resid, int checkpoint_every, float *grad_m,
                            void *stream);

/*
 * acoustic_forward_noalloc -- acoustic_forward for callers that cannot
 * allocate device memory.  The paper has no counterpart; this is a library
 * convenience.
 *
 * acoustic_forward allocates its workspace (padded wavefields, the b
 * coefficient, sparse tables) with cudaMallocAsync on every call.  Some callers
 * cannot allow that: code running under a fixed device-memory budget decided
 * up front, a process whose device memory belongs to another allocator (a
 * framework's caching pool), or a service that must not hit out-of-memory in
 * the middle of a request.  This entry point runs acoustic_forward's
 * schedule with the same kernels and launch configuration but keeps the
 * workspace in one fixed, file-scope device array of FD_STATIC_SCRATCH_BYTES,
 * so a call allocates nothing (no cudaMalloc, cudaFree, stream, event or
 * graph creation).  With at most 16 sources per shot (injected by the stencil
 * kernel in source order, as acoustic_forward does) the results are
 * bit-identical to acoustic_forward's; with more, sources whose trilinear
 * stencils share a node are added atomically in an unspecified order, and the
 * two agree to FP32 rounding.
 *
 *  - Arguments, layouts and results are those of acoustic_forward, except
 *    that every pointer must be device memory of the current device or
 *    managed memory (FD_ERR_ARG otherwise) and the work runs directly on
 *    `stream` (synchronised once at the end).  The grid checks are
 *    acoustic_forward's (padded volume below 2^32 points, finite spacing and
 *    origin), made before the scratch is sized.
 *  - A problem whose workspace, 4 * (2 nshots + 1) * nz * ny * nxp bytes
 *    (nxp = nx rounded up to a multiple of 4) plus its sparse tables, exceeds
 *    FD_STATIC_SCRATCH_BYTES is rejected with FD_ERR_ARG before any launch.
 *  - Every GPU that loads the library holds the array until the process
 *    exits.  All calls share it and it keeps the last call's contents; each
 *    call clears what must start at zero.  Calls that overlap on the GPU
 *    (other streams or host threads on the same device) race on the array and
 *    must be serialised by the caller.
 *  - The first call on a device looks up the array's address with
 *    cudaGetSymbolAddress (that device current) and caches it; make that first
 *    call before any CUDA stream capture.
 */
#define FD_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
fd_status acoustic_forward_noalloc(const fd_grid *grid, int so, double dt, int nt, int nshots,
                                   const float *m, const float *damp, int nsrc,
                                   const float *src_xyz, const float *src_wav, int nrec,
                                   const float *rec_xyz, float *rec_out, const float *u_init,
                                   float *u_final, void *stream);

/*
 * Batch engine for serving (no counterpart in the paper).
 *
 * Shots that share a velocity model (grid, so, dt, m, damp) are slots of one
 * engine.  fd_engine_step advances every active slot by the same number of
 * time steps with one stencil launch per step over all active slots (the
 * shot is the outer dimension); chunks are captured into CUDA graphs and
 * replayed while the set of active slots is unchanged.  A slot added at the
 * engine's global step G starts from the zero state at its own time index
 * n = 0 and runs the scheme of acoustic_forward (injection of src[n] into
 * u^{n+1}, trace rec[n] = interp(u^n)), so its traces equal acoustic_forward's
 * for the same shot; other slots may be at any time index.  Each engine owns
 * a non-blocking CUDA stream (fd_engine_stream), so engines run concurrently.
 * All memory is allocated by fd_engine_create (fd_engine_footprint gives the
 * bytes); adding, stepping and releasing allocate nothing.  Pointers are
 * device memory and must stay valid until the shot is released.
 */
typedef struct fd_engine fd_engine;
fd_status fd_engine_footprint(const fd_grid *grid, int max_slots, int max_nsrc, int max_nrec,
                              int64_t *bytes);
fd_status fd_engine_create(const fd_grid *grid, int so, double dt, const float *m,
                           const float *damp, int max_slots, int max_nsrc, int max_nrec,
                           fd_engine **engine);
/* src_wav [nt][nsrc], rec_out [nt][nrec]; *slot receives the slot index.
 * FD_ERR_ARG if no slot is free or sizes exceed the engine's maxima. */
fd_status fd_engine_add_shot(fd_engine *engine, int nt, int nsrc, const float *src_xyz,
                             const float *src_wav, int nrec, const float *rec_xyz, float *rec_out,
                             int *slot);
/* Advance all active slots by nsteps (even, >= 0) time steps (asynchronous). */
fd_status fd_engine_step(fd_engine *engine, int nsteps);
/* Host-side view: whether the slot is active and how many of its time steps
 * have not been enqueued yet (0: its last trace sample is enqueued; it is
 * complete once the engine's stream has reached that point). */
fd_status fd_engine_shot_status(fd_engine *engine, int slot, int *active, int64_t *steps_left);
fd_status fd_engine_release(fd_engine *engine, int slot);
fd_status fd_engine_stream(fd_engine *engine, void **stream);
/* Wait for the engine's queued work and report device-side errors. */
fd_status fd_engine_sync(fd_engine *engine);
fd_status fd_engine_destroy(fd_engine *engine);

/* Message describing the last error on the calling thread ("" if none). */
const char *fd_last_error(void);

/* Library version string. */
const char *fd_version(void);

/*
 * Kernel timing statistics.  When enabled (fd_stats_enable(1)), the forward
 * entry points launch their time loop without CUDA graphs and bracket every
 * stencil-kernel launch with CUDA events on the call's stream; the elapsed
 * times are accumulated per kernel family when the call completes.
 * Families: "acoustic_step", "acoustic_step2" (two time steps per launch, see
 * fd_set_time_tiling; points_per_launch counts the points of one step),
 * "acoustic_step_h" (binary16 storage, acoustic_forward_opts),
 * "tti_pass1", "tti_pass2", "tti_recompute", "tti_fused" (the one-kernel TTI
 * schemes of tti_forward_opts), "sparse".
 * fd_stats_get returns FD_ERR_ARG for an unknown family.
 */
fd_status fd_stats_enable(int on);
fd_status fd_stats_reset(void);
fd_status fd_stats_get(const char *family, double *total_ms, int64_t *launches,
                       double *points_per_launch);

/* Number of kernel launches this library has enqueued since it was loaded
 * (a replayed CUDA graph counts each of its kernel nodes). */
int64_t fd_launch_count(void);

/*
 * Limit of the acoustic stencil kernel's bounded pipeline waits, in
 * nanoseconds (a stage of the shared-memory ring that is not filled, or not
 * released, within the limit makes the kernel stop its column, let the copies
 * it already issued land, and report FD_ERR_TIMEOUT).  ns <= 0 restores the
 * built-in 2 s.  A failure-injection knob for tests: with ns = 1 every such
 * wait is a single non-blocking test, so the waits give up on copies that are
 * merely in flight, the call returns FD_ERR_TIMEOUT and the device stays
 * usable (the copies already issued are still waited for, with their own
 * limit, before a stopped kernel exits).  Process-wide; it applies to the
 * stencil kernel's default launch configuration with per-axis damping (a
 * variant of it that reads the limit is launched while the setting is
 * non-zero, so the production kernel keeps a constant limit), and to launches
 * enqueued after the call (a CUDA graph keeps the variant it was captured
 * with).
 */
fd_status fd_set_wait_limit_ns(int64_t ns);

/*
 * The FP32 Laplacian weights the acoustic kernels use for a grid and space
 * order (Listing fd-1's compact second derivative of radius so/2 per axis,
 * divided by h_d^2): *centre receives the sum over the axes of the centre
 * weights, w[9 d + k] the weight of the offset +-k along axis d (x, y, z;
 * k = 1 .. so/2; entries k = 0 and beyond so/2 are zero).  The weights are
 * the FP32 roundings of the closed-form FP64 weights, except that the centre
 * is the rounding of -2 times the sum of the neighbour weights and the
 * residual of that rounding is moved into the neighbour weights (nearest taps
 * first): in the device's weights, as in the exact ones, the Laplacian of a
 * constant field is zero.  Host-only (no CUDA call); FD_ERR_SO / FD_ERR_ARG
 * for a bad space order or grid.
 */
fd_status fd_stencil_weights(const fd_grid *grid, int so, float *centre, float *w /* [3][9] */);

/*
 * Time tiling of acoustic_forward (loop blocking across the time dimension,
 * named in the paper's section "Further work"): two leapfrog
 * steps per kernel launch, the intermediate level kept in shared memory and
 * its halo recomputed by neighbouring tiles; results are bit-identical to
 * single steps.  Applies to space orders with a two-step kernel
 * (fd_num_time_tiling_configs(so) > 0), at most 16 sources per shot and
 * nt >= 3; it uses four wavefield levels per shot instead of two.
 *   mode -1  automatic (the default; off for every space order, since two
 *            single steps measured faster on GB300: the single-step kernel
 *            is near the HBM bound, the two-step one issue-bound),
 *         0  off,
 *     1 + k  on, with configuration k of the two-step kernel.
 * Process-wide setting, not synchronised with calls in flight.  Returns
 * FD_ERR_SO / FD_ERR_ARG for an unknown space order or mode.
 */
fd_status fd_set_time_tiling(int so, int mode);
int fd_num_time_tiling_configs(int so);

/*
 * Launch configuration override of the two TTI passes (prefetch depths and
 * loop unroll; for tuning sweeps): index into the compiled table for the
 * given space order (0 .. fd_num_tti_configs(so) - 1), or -1 for the
 * built-in choice.  Applies to centred derivatives of the two-pass scheme
 * (the staggered reading always uses the built-in choice); for the fused
 * scheme configuration 1 selects 64 x 16 tiles instead of 64 x 8 (other
 * values: the built-in choice).  Process-wide; FD_ERR_ARG if out of range.
 */
fd_status fd_set_tti_config(int so, int config);
int fd_num_tti_configs(int so);

/*
 * Tile configuration override for the acoustic stencil kernel (for tuning
 * sweeps): index into the compiled configuration table for the given space
 * order, or -1 for the built-in choice.  Returns FD_ERR_ARG if out of range.
 */
fd_status fd_set_acoustic_config(int so, int config);
int fd_num_acoustic_configs(int so);

/* The same for the binary16-storage kernel (acoustic_forward_opts with
 * FD_STORAGE_F16); 0 configurations for a space order without one. */
fd_status fd_set_acoustic_f16_config(int so, int config);
int fd_num_acoustic_f16_configs(int so);

#ifdef __cplusplus
}
#endif

#endif /* FDSWEEP_H */
