// kernels.cuh -- argument blocks and host launchers of the fdsweep kernels.
//
// Device data layout (all FP32):
//   wavefields  [nbuf][nz][ny][nxp], nxp = nx rounded up to a multiple of 4
//               (16-byte rows for TMA and float4 access); buffer index
//               (shot * fields_per_shot + level).  Columns nx..nxp-1 are
//               padding that no kernel reads.
//   coefficient fields (b = dt^2/(m + damp dt/2), TTI a, s, n) share the
//               [nz][ny][nxp] layout.
//   sparse tables one SparsePoint (16 bytes) per source/receiver.
#pragma once

#include "common.cuh"

namespace fdsweep {

struct WaveLayout {
    int nx, ny, nz, nxp;
    int64_t plane;  // ny * nxp
    int64_t vol;    // nz * plane
};

// Padded device layout of a grid (nxp = nx rounded up to a multiple of 4).
WaveLayout wave_layout(const fd_grid &g);

// Trilinear stencil of one sparse point: index of the (x1, y1, z1) corner in
// the padded layout and the fractional offsets along each axis (computed in
// FP64, stored rounded to FP32).
struct SparsePoint {
    uint32_t base;
    float fx, fy, fz;
};

constexpr int kMaxRadius = 8;

// ---------------------------------------------------------------- host numerics
//
// One definition, in api.cu, for every entry point (forward, adjoint,
// gradient, the batch engine, the allocation-free call), so that their FD
// weights, stability bounds and argument checks cannot drift apart.

// Central FD weights for radius r, closed form (second derivative w[0..r],
// first derivative c[0..r]).
void fd_weights(int r, double *w, double *c);
// max over theta of the second-derivative symbol -(w_0 + 2 sum w_k cos k theta)
double second_symbol_max(int r, const double *w);
// Exact constant-coefficient stability bound of the acoustic leapfrog with the
// compact Laplacian of radius r: 2 / (v_max sqrt(sigma_max sum_d h_d^-2)),
// v_max = 1/sqrt(m_min).
double acoustic_dt_bound(const fd_grid &g, int r, double m_min);
// Laplacian weights of radius r as the stencil kernels take them: the sum of
// the centre weights over the axes (wc) and w_k / h_d^2 for k = 1..kMaxRadius
// (zero beyond r and at k = 0).
void laplacian_weights(const fd_grid &g, int r, float *wc, float *wx, float *wy, float *wz);
// The grid alone: >= 2 points per axis, finite spacing > 0 and origin, padded
// volume below 2^32 points (the sparse tables index it in 32 bits).
fd_status validate_grid(const fd_grid *g);
// Checks shared by the entry points: the grid (>= 2 points per axis, finite
// spacing > 0 and origin, padded volume below 2^32 points, which the sparse
// tables index in 32 bits), so, dt, nt >= 1, nshots >= 1, m and the sparse
// arrays present when their counts are non-zero.
fd_status validate_common(const fd_grid *g, int so, double dt, int nt, int nshots, const float *m,
                          int nsrc, const float *src_xyz, const float *src_wav, int nrec,
                          const float *rec_xyz, const float *rec_out);
// K1 launch configuration acoustic_forward uses for a radius (-1: default).
int acoustic_step_config(int radius);

// ---------------------------------------------------------------- acoustic K1

struct AcousticStepArgs {
    float *wave;          // 2 buffers per shot: index 2 s + level
    const float *bcoef;   // b = dt^2 / (m + damp dt / 2)
    const float *dpx;     // damp_x / dt, [nx]
    const float *dpy;     // damp_y / dt, [ny]
    const float *dpz;     // damp_z / dt, [nz]
    WaveLayout L;
    int nshots;
    // Buffer index of a level: shot * lps + level.  u^n is read from lev_cur,
    // u^{n-1} from lev_prev, u^{n+1} written to lev_out (== lev_prev for the
    // in-place two-level scheme; distinct when a history is being kept).
    int lps, lev_cur, lev_prev, lev_out;
    // Optional map from blockIdx.z's shot index to the shot (slot) actually
    // stepped, so that a batch engine can step only its active slots.
    const int *slot_map;
    float wc;             // sum over axes of w_0 / h_d^2
    float wx[kMaxRadius + 1], wy[kMaxRadius + 1], wz[kMaxRadius + 1];  // w_k / h_d^2
    unsigned int *err;    // device error bits; a launch that finds DEV_ERR_NONFINITE
                          // set (by the watchdog) returns at once
    uint64_t wait_ns;     // limit of the pipeline's bounded waits (0: 2 s); filled
                          // in by acoustic_launch from fd_set_wait_limit_ns
};

struct AcousticPlan {
    int radius = 0;
    int config = 0;
    CUtensorMap map_halo;  // wavefield buffers, tile + halo box
    CUtensorMap map_int;   // wavefield buffers, interior tile box
    CUtensorMap map_b;     // b coefficient, interior tile box
    dim3 grid, block;
    size_t smem = 0;
    int zchunk = 0, nzc = 1;
    bool damp_field = false;  // the kernel variant that reads zeta per point
    const char *name = "";
};

// Two-level in-place scheme: u^n in level `cur`, u^{n-1} and u^{n+1} in 1 - cur.
inline void set_two_levels(AcousticStepArgs &a, int cur) {
    a.lps = 2;
    a.lev_cur = cur;
    a.lev_prev = 1 - cur;
    a.lev_out = 1 - cur;
}

// Source injection done by K1 itself (acoustic forward): src[n] is added
// to u^{n+1} by the threads that write the source's trilinear corners, in
// source order, with the operations of the sparse kernel (w_c b q added to
// the stored value).  n = step + *step_base (step_base may be null).  At most
// kInjectMaxSources sources per shot; nsrc = 0 disables it.
constexpr int kInjectMaxSources = 16;

struct AcousticInject {
    const SparsePoint *src_tab;  // [nshots][nsrc]
    const float *src_wav;        // [nshots][nt][nsrc]
    int nsrc, nt;
    const int *step_base;
    int step;
};

int acoustic_num_configs(int radius);
int acoustic_default_config(int radius);
// `lps` levels per shot are addressable (buffers nshots * lps).  The launch
// covers `nshots` shots; the tensor maps cover `map_shots` shots (default:
// nshots) for callers that map launch shots to slots (slot_map).
// damp_field: the damping is a 3-D field; bcoef then holds two fields, b and
// zeta = damp b / dt ([2][vol]), and the default configuration is used.
fd_status acoustic_plan(int radius, int config, const WaveLayout &L, int nshots, int lps,
                        float *wave, const float *bcoef, AcousticPlan *plan, int map_shots = 0,
                        bool damp_field = false);
fd_status acoustic_launch(const AcousticPlan &plan, const AcousticStepArgs &args,
                          cudaStream_t stream, const AcousticInject *inject = nullptr);

// ---------------------------------------------------------------- time-tiled K1

// Two leapfrog steps per launch (acoustic2.cu): u^n (lev_cur), u^{n-1}
// (lev_prev) -> u^{n+1} (lev_out) and u^{n+2} (lev_out2), all distinct levels;
// src[n] (n = 2 (step + *step_base)) is injected into u^{n+1} in the kernel.
constexpr int kStep2MaxSources = 16;

struct AcousticStep2Args {
    AcousticStepArgs s;          // slot_map must be null
    int lev_out2;
    const SparsePoint *src_tab;  // [nshots][nsrc] or null
    const float *src_wav;        // [nshots][nt][nsrc]
    int nsrc, nt;
    const int *step_base;        // device pair counter (may be null)
    int step;                    // pair index added to *step_base
};

struct Acoustic2Plan {
    int radius = 0;
    int config = 0;
    CUtensorMap map_halo, map_ext, map_int, map_bext, map_bint;
    dim3 grid, block;
    size_t smem = 0;
    int zchunk = 0, nzc = 1;
    const char *name = "";
};

int acoustic2_num_configs(int radius);  // 0: no time-tiled kernel for this radius
fd_status acoustic2_plan(int radius, int config, const WaveLayout &L, int nshots, int lps,
                         float *wave, const float *bcoef, Acoustic2Plan *plan);
fd_status acoustic2_launch(const Acoustic2Plan &plan, const AcousticStep2Args &args,
                           cudaStream_t stream);

// ---------------------------------------------------------------- sparse K3/K4

struct SparseArgs {
    float *wave;                 // wavefield buffers
    int fields_per_shot;         // 2 (acoustic) or 4 (TTI: p levels 0,1; r levels 2,3)
    WaveLayout L;
    const float *bcoef;          // injection scale per node
    int nshots, nt;
    // injection into level `inj_level[0]` (and `inj_level[1]` if >= 0)
    int nsrc;
    const SparsePoint *src_tab;  // [nshots][nsrc]
    const float *src_wav;        // [nshots][nt][nsrc]
    int inj_level0, inj_level1;
    // wavelet sample injected at step n: inj_t0 + inj_dt * n; trace sample
    // written at step n: rec_t0 + rec_dt * n (forward: 0 + n; adjoint runs
    // reversed time: nt - 2 - n)
    int inj_t0, inj_dt, rec_t0, rec_dt;
    // interpolation of level `rec_level`
    int nrec;
    const SparsePoint *rec_tab;  // [nshots][nrec]
    float *rec_out;              // [nshots][nt][nrec]
    int rec_level;
    // rec_mean != 0: record the mean of levels rec_level and rec_level2
    // (the (p + r)/2 receiver reading of the TTI system)
    int rec_mean, rec_level2;
    const int *step_base;        // device counter added to `step` (may be null)
};

// One launch performs the injection of src[n] (if do_inject) and the
// interpolation rec[n] (if do_interp), n = step + (*step_base if given).
fd_status sparse_launch(const SparseArgs &a, int step, bool do_inject, bool do_interp,
                        cudaStream_t stream);
fd_status bump_counter(int *counter, int by, cudaStream_t stream);
// grad += sum_b w_b (u_b - 2 u_b' + u_b'') over `n` floats, the FWI imaging
// condition of one time step for nb shots (scaled by -1/dt^2 once at the end):
// w_b = w + b w_stride, u_b = u + b u_stride is the level of u^k and u_b',
// u_b'' (u^{k-1}, u^{k-2}) are the n and 2n floats below it; shots are
// accumulated in order.
fd_status grad_accumulate_batch(float *grad, const float *w, int64_t w_stride, const float *u,
                                int64_t u_stride, int nb, int64_t n, cudaStream_t stream);
fd_status scale_field(float *f, float s, int64_t n, cudaStream_t stream);

// ---------------------------------------------------------------- setup K0

struct MediumStats {
    float m_min, m_max;
    float eps_max;
    unsigned int flags;  // DEV_ERR_* bits
};

// b = dt^2 / (m + damp dt/2) in the padded layout; damp per-axis profiles
// scaled by 1/dt into dps[nx + ny + nz].  m and damp are dense device arrays.
// damp_field: damp is a 3-D field [nz][ny][nx]; bcoef then has two fields,
// b and zeta = damp b / dt, and dps is zero.
fd_status setup_acoustic_coeffs(const float *m, const float *damp, double dt,
                                const WaveLayout &L, float *bcoef, float *dps,
                                MediumStats *dev_stats, cudaStream_t stream,
                                bool damp_field = false);
// TTI extra fields: a = 1 + 2 eps, s = sqrt(1 + 2 delta), n = (nx, ny, nz).
fd_status setup_tti_coeffs(const float *eps, const float *delta, const float *theta,
                           const float *phi, const WaveLayout &L, float *acoef, float *scoef,
                           float *nvec /* 3 fields */, MediumStats *dev_stats,
                           cudaStream_t stream);
fd_status setup_sparse_table(const float *xyz, int npts, const fd_grid &g, const WaveLayout &L,
                             SparsePoint *tab, unsigned int *flags, cudaStream_t stream);
fd_status init_medium_stats(MediumStats *dev_stats, cudaStream_t stream);
// Sets DEV_ERR_NONFINITE in *flags if any element of the field is not finite.
fd_status check_finite(const float *field, const WaveLayout &L, int nfields,
                       unsigned int *flags, cudaStream_t stream);
// Divergence watchdog of the time loops: checks every x row of every
// kWatchStride-th y row of every kWatchStride-th z plane of `nfields`
// consecutive fields (1/64 of the points) and sets DEV_ERR_NONFINITE in
// *flags if one is not finite.  The stencil kernels launched after that
// return at once, so a diverging run stops within one watchdog period
// instead of running its whole time budget.
constexpr int kWatchStride = 8;
constexpr int kWatchEvery = 16;  // time steps between two watchdog launches
fd_status watchdog_launch(const float *field, const WaveLayout &L, int nfields,
                          unsigned int *flags, cudaStream_t stream);
// Process-wide limit of the acoustic stencil kernel's bounded pipeline waits
// (fd_set_wait_limit_ns); 0 = the built-in 2 s.
uint64_t wait_limit_ns();

// ---------------------------------------------------------------- TTI K2a/K2b

// First-derivative stencils of the TTI operators as tap tables: entry d + R
// (d = -R..R) of t[axis] weights the value at offset d along the axis,
// already divided by h.  Centred: t[d] = sign(d) c_|d|.  Staggered: the inner
// derivative (pass 1) is D+ (taps -R+1..R), the outer one (pass 2) D- (taps
// -R..R-1).
constexpr int kTaps = 2 * kMaxRadius + 1;

struct TtiArgs {
    float *wave;           // 4 buffers per shot: p levels (0,1), r levels (2,3)
    float *tmp;            // 6 temporaries per shot [6][vol]
    const float *bcoef, *acoef, *scoef, *nvec;
    const float *dpx, *dpy, *dpz;
    WaveLayout L;
    int nshots;
    int cur;
    float t1[3][kTaps];    // inner first derivative (of p, r)
    float t2[3][kTaps];    // outer first derivative (of the temporaries)
    unsigned int *err;
};

enum TtiScheme { kTtiTwoPass = 0, kTtiRecompute = 1, kTtiFused = 2 };

struct TtiPlan {
    int radius = 0;
    int stag = 0;    // 0: centred first derivatives, 1: staggered (D+ inner, D- outer)
    int scheme = kTtiTwoPass;
    int config = 0;  // launch configuration of the two passes (tti_num_configs)
    CUtensorMap map_wint, map_whalo;          // p/r buffers: interior, x+y halo boxes
    CUtensorMap map_tint, map_tx, map_ty;     // temporaries: interior, x-halo, y-halo
    CUtensorMap map_cint;                     // b, a, s, n_x, n_y, n_z: interior box
    CUtensorMap map_fbox, map_fnbox;          // fused scheme: p/r plane box, n box
    dim3 grid, block;
    size_t smem1 = 0, smem2 = 0;
    int zchunk = 0, nzc = 1;
};

// z chunks per column of the TTI kernels (machine filling and SM balance)
int tti_z_chunks(int64_t cols, int64_t slots, int nz, int min_chunk);

// coef: 6 consecutive fields b, a, s, n_x, n_y, n_z ([6][vol]).  scheme
// kTtiTwoPass: K2a writes the six first-derivative temporaries and K2b
// differentiates them again; kTtiRecompute: one kernel recomputes the inner
// derivatives at every outer stencil point (no temporaries; tmp unused).
fd_status tti_plan(int radius, const WaveLayout &L, int nshots, float *wave, float *tmp,
                   const float *coef, TtiPlan *plan, int stag = 0, int scheme = kTtiTwoPass,
                   int config = 0);
int tti_num_configs(int radius);
// Fused scheme (tti_fused.cu): one kernel per step, temporaries in shared
// memory; radii 1, 2 and 4.
bool tti_fused_supported(int radius);
fd_status tti_fused_plan(int radius, int stag, const WaveLayout &L, int nshots, float *wave,
                         const float *coef, TtiPlan *plan, int config = 0);
fd_status tti_fused_launch(const TtiPlan &plan, const TtiArgs &a, cudaStream_t stream);
fd_status tti_launch(const TtiPlan &plan, const TtiArgs &a, cudaStream_t stream,
                     cudaEvent_t *ev /* 3 events or null */);

// ---------------------------------------------------------------- binary16 storage

// Reduced-precision storage (acoustic_h.cu): the wavefield levels and the
// coefficient b are stored in IEEE binary16, the arithmetic is FP32.  Layout
// [nbuf][nz][ny][nxp] halves with nxp = nx rounded up to a multiple of 8
// (16-byte rows for TMA); raw binary16 bit patterns are held as half_bits.
typedef unsigned short half_bits;

struct AcousticHArgs {
    half_bits *wave;          // lps buffers per shot: index shot * lps + level
    const half_bits *bcoef;   // b = dt^2 / (m + damp dt / 2), binary16
    const float *dpx, *dpy, *dpz;  // damp_d / dt per axis (FP32)
    WaveLayout L;             // binary16 layout
    int nshots;
    int lps, lev_cur, lev_prev, lev_out;
    float wc;
    float wx[kMaxRadius + 1], wy[kMaxRadius + 1], wz[kMaxRadius + 1];
    unsigned int *err;
};

int acoustic_h_num_configs(int radius);  // 0: no binary16 kernel for this radius
fd_status acoustic_h_plan(int radius, int config, const WaveLayout &L, int nshots, int lps,
                          half_bits *wave, const half_bits *bcoef, AcousticPlan *plan);
fd_status acoustic_h_launch(const AcousticPlan &plan, const AcousticHArgs &args,
                            cudaStream_t stream);

// Sparse injection / interpolation on binary16 levels (forward schedule:
// src[n] into level inj_level, rec[n] from level rec_level at step n).  The
// injected value w_c b q is rounded to binary16 and added atomically (one
// binary16 rounding of the sum).
struct SparseHArgs {
    half_bits *wave;
    int fields_per_shot;
    WaveLayout L;
    const half_bits *bcoef;
    int nshots, nt;
    int nsrc;
    const SparsePoint *src_tab;
    const float *src_wav;
    int inj_level;
    int nrec;
    const SparsePoint *rec_tab;
    float *rec_out;
    int rec_level;
    const int *step_base;
};
fd_status sparse_h_launch(const SparseHArgs &a, int step, bool do_inject, bool do_interp,
                          cudaStream_t stream);

// dst row r (stride dst_stride halves) = nearest binary16 values of src row r
// (stride src_stride floats), nx values per row, `rows` rows; and back.
fd_status narrow_rows(const float *src, int64_t src_stride, half_bits *dst, int64_t dst_stride,
                      int nx, int64_t rows, cudaStream_t stream);
fd_status widen_rows(const half_bits *src, int64_t src_stride, float *dst, int64_t dst_stride,
                     int nx, int64_t rows, cudaStream_t stream);
// Sets DEV_ERR_NONFINITE in *flags if any value of the fields is inf or NaN.
fd_status check_finite_h(const half_bits *field, const WaveLayout &L, int nfields,
                         unsigned int *flags, cudaStream_t stream);

}  // namespace fdsweep
