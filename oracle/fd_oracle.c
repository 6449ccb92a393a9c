/*
 * fd_oracle.c -- FP64 CPU oracle for the time-stepped 3-D finite-difference
 * wave-propagation sweep of arXiv:1807.03032 (Devito).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke check
 * and the benchmark's CPU-baseline leg may load this library.  It shares no
 * code, header or constant generator with the CUDA path.
 *
 * It is written to be read against the paper, not to be fast: plain loops,
 * FP64 arithmetic, one grid point at a time, no blocking and no fusion.  The
 * only parallelism is an OpenMP loop over independent grid points, which does
 * not change any result.  Inputs arrive as FP32 (the exact bits the GPU
 * receives) and are widened to FP64 on entry.
 *
 * Paper passages followed (section / equation / listing labels of the paper):
 *   - Eq. (WE), section "Symbolic types": m u_tt - lap(u) = q_s, zero initial
 *     conditions; m = 1/c^2.
 *   - Listing fd-1 / fd-2 / fd-3, section "Discretization": central FD
 *     derivatives and the explicit leapfrog update obtained with `solve`.
 *   - Eq. (interp) and Listing finject: linear (trilinear in 3-D)
 *     interpolation and injection as its adjoint, scaled dt^2 q / m, added to
 *     the field at t+1.
 *   - Section "Test case setup": zero initial conditions, Dirichlet boundary,
 *     absorbing border, space orders 4..16, second order in time; TTI is two
 *     coupled acoustic equations whose Laplacians are built from rotated
 *     first-derivative operators.
 *   - Section "Domain, halo, and padding regions": the computational domain
 *     includes the absorbing layers; halo points are ghosts (zero here).
 *
 * Readings where the paper is silent (the same readings bind the CUDA path):
 *   - space order so -> stencil radius r = so/2 for both the compact second
 *     derivative and the central first derivative;
 *   - Dirichlet: every grid point is updated, values outside the grid are 0;
 *   - damping enters as damp * u_t, discretised centrally:
 *       m (u+ - 2u + u-)/dt^2 + damp (u+ - u-)/(2 dt) = lap(u);
 *     damp(i,j,k) = dx[i] + dy[j] + dz[k] (sum of per-axis 1-D profiles);
 *   - injection at step n adds w_c dt^2 q[n] / (m + damp dt/2) to u^{n+1}
 *     (reduces to the paper's dt^2 q / m where damp = 0);
 *   - receivers sample u^n for n = 0..nt-1;
 *   - interpolation index x1 = floor((x-o)/h) clamped to n-2, computed in FP64;
 *   - TTI (pseudo-acoustic, rotated first derivatives):
 *       Hz q  = sum_i D_i( n_i * sum_j n_j D_j q ),  L q = sum_i D_i D_i q,
 *       Hxy q = L q - Hz q,  n = (sin t cos f, sin t sin f, cos t),
 *       m p_tt + damp p_t = (1+2 eps) Hxy p + sqrt(1+2 delta) Hz r,
 *       m r_tt + damp r_t = sqrt(1+2 delta) Hxy p + Hz r;
 *     the source is injected into p and r, receivers record p.
 *     Alternative readings (selectable, defaults as above): staggered first
 *     derivatives (inner D+, outer D-, each the other's negative transpose)
 *     and receivers recording (p + r)/2.
 *
 * Layout: C order [z][y][x] (x fastest), index (k*ny + j)*nx + i.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny, nz;
    double hx, hy, hz;
    double ox, oy, oz;
} ora_grid;

enum { ORA_OK = 0, ORA_ERR_ARG = -1, ORA_ERR_COORD = -4, ORA_ERR_OOM = -5 };

static size_t npts(const ora_grid *g) { return (size_t)g->nx * g->ny * g->nz; }

static size_t lin(const ora_grid *g, int i, int j, int k) {
    return ((size_t)k * g->ny + j) * g->nx + i;
}

static int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

/* Value of a grid function at (i,j,k).  Outside the grid it is the zero ghost
 * of the Dirichlet boundary, or the periodic image (a test-only mode used by
 * the plane-wave pins). */
static double at(const ora_grid *g, int periodic, const double *f, int i, int j, int k) {
    if (periodic) {
        i = wrap(i, g->nx);
        j = wrap(j, g->ny);
        k = wrap(k, g->nz);
    } else if (i < 0 || j < 0 || k < 0 || i >= g->nx || j >= g->ny || k >= g->nz) {
        return 0.0;
    }
    return f[lin(g, i, j, k)];
}

/* Central FD weights for stencil radius r (space order 2r), closed form.
 * Second derivative:  w[k] = 2(-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!),
 *                     w[0] = -2 sum_k w[k].
 * First derivative:   c[k] = (-1)^(k+1) (r!)^2 / (k (r-k)! (r+k)!), c[0] = 0.
 * For r = 1 these are Listing fd-1's [1, -2, 1]/h^2 and +-1/(2h). */
void ora_fd_weights(int r, double *w, double *c) {
    double ratio = 1.0; /* (r!)^2 / ((r-k)! (r+k)!) */
    double sum = 0.0;
    c[0] = 0.0;
    for (int k = 1; k <= r; ++k) {
        ratio *= (double)(r - k + 1) / (double)(r + k);
        double sgn = (k % 2 == 1) ? 1.0 : -1.0;
        w[k] = 2.0 * sgn * ratio / ((double)k * (double)k);
        c[k] = sgn * ratio / (double)k;
        sum += w[k];
    }
    w[0] = -2.0 * sum;
}

/* Staggered first-derivative weights for radius r (order 2r): the derivative
 * at a point midway between nodes, from the r node pairs at distances
 * (k - 1/2) h on either side,
 *   f'(x) ~ sum_k a[k] (f(x + (k - 1/2) h) - f(x - (k - 1/2) h)) / h,
 * closed form a[k] = (-1)^(k+1) ((2r-1)!!)^2 / (4^(r-1) (2k-1)^2 (r+k-1)! (r-k)!).
 * For r = 1 this is a[1] = 1 (the two-point difference), r = 2 gives 9/8, -1/24.
 * Used by the staggered reading of the rotated TTI operators. */
void ora_staggered_weights(int r, double *a) {
    double dfact = 1.0; /* (2r-1)!! */
    for (int j = 1; j <= 2 * r - 1; j += 2) dfact *= (double)j;
    double p4 = 1.0; /* 4^(r-1) */
    for (int j = 1; j < r; ++j) p4 *= 4.0;
    a[0] = 0.0;
    for (int k = 1; k <= r; ++k) {
        double f1 = 1.0, f2 = 1.0; /* (r+k-1)!, (r-k)! */
        for (int j = 2; j <= r + k - 1; ++j) f1 *= (double)j;
        for (int j = 2; j <= r - k; ++j) f2 *= (double)j;
        double sgn = (k % 2 == 1) ? 1.0 : -1.0;
        double odd = (double)(2 * k - 1);
        a[k] = sgn * dfact * dfact / (p4 * odd * odd * f1 * f2);
    }
}

static int radius_of(int so) {
    if (so < 2 || so > 32 || (so % 2) != 0) return -1;
    return so / 2;
}

/* Compact Laplacian: sum over axes of the 1-D central second derivative. */
int ora_laplacian(const ora_grid *g, int so, int periodic, const double *u, double *out) {
    int r = radius_of(so);
    if (r < 0) return ORA_ERR_ARG;
    double w[33], c[33];
    ora_fd_weights(r, w, c);
    const double ih2[3] = {1.0 / (g->hx * g->hx), 1.0 / (g->hy * g->hy), 1.0 / (g->hz * g->hz)};
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double center = u[lin(g, i, j, k)];
                double dxx = w[0] * center, dyy = w[0] * center, dzz = w[0] * center;
                for (int s = 1; s <= r; ++s) {
                    dxx += w[s] * (at(g, periodic, u, i + s, j, k) + at(g, periodic, u, i - s, j, k));
                    dyy += w[s] * (at(g, periodic, u, i, j + s, k) + at(g, periodic, u, i, j - s, k));
                    dzz += w[s] * (at(g, periodic, u, i, j, k + s) + at(g, periodic, u, i, j, k - s));
                }
                out[lin(g, i, j, k)] = dxx * ih2[0] + dyy * ih2[1] + dzz * ih2[2];
            }
    return ORA_OK;
}

/* First derivative along one axis (0 = x, 1 = y, 2 = z) of one of three kinds:
 *   kind  0: central, at the node:     sum_k c_k (f[i+k] - f[i-k]) / h;
 *   kind +1: forward-staggered D+, the derivative at i + 1/2:
 *                                      sum_k a_k (f[i+k] - f[i-k+1]) / h;
 *   kind -1: backward-staggered D-, the derivative at i - 1/2:
 *                                      sum_k a_k (f[i+k-1] - f[i-k]) / h.
 * With zero ghosts (or periodic images) D- = -(D+)^T exactly. */
int ora_first_derivative_kind(const ora_grid *g, int so, int periodic, int axis, int kind,
                              const double *f, double *out) {
    int r = radius_of(so);
    if (r < 0 || axis < 0 || axis > 2 || kind < -1 || kind > 1) return ORA_ERR_ARG;
    double w[33], c[33], a[33];
    ora_fd_weights(r, w, c);
    ora_staggered_weights(r, a);
    const int di = axis == 0, dj = axis == 1, dk = axis == 2;
    const double h = axis == 0 ? g->hx : (axis == 1 ? g->hy : g->hz);
    /* taps (offset of the "+" node, offset of the "-" node) for pair s */
    const int plus0 = kind == -1 ? -1 : 0, minus0 = kind == 1 ? 1 : 0;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double d = 0.0;
                for (int s = 1; s <= r; ++s) {
                    const int sp = s + plus0, sm = -s + minus0;
                    d += (kind == 0 ? c[s] : a[s]) *
                         (at(g, periodic, f, i + sp * di, j + sp * dj, k + sp * dk) -
                          at(g, periodic, f, i + sm * di, j + sm * dj, k + sm * dk));
                }
                out[lin(g, i, j, k)] = d / h;
            }
    return ORA_OK;
}

/* Central first derivative along one axis (0 = x, 1 = y, 2 = z). */
int ora_first_derivative(const ora_grid *g, int so, int periodic, int axis, const double *f,
                         double *out) {
    return ora_first_derivative_kind(g, so, periodic, axis, 0, f, out);
}

/* damp(i,j,k) from the damping field, one FP64 value per grid point (NULL =
 * no damping).  The callers build the field from the API's input: either the
 * per-axis 1-D profiles, damp(i,j,k) = d_x[i] + d_y[j] + d_z[k], or a 3-D
 * field given point by point (section "Test case setup" names only an
 * absorbing mask; both readings are served). */
static double damp_at(const ora_grid *g, const double *damp, int i, int j, int k) {
    if (!damp) return 0.0;
    return damp[lin(g, i, j, k)];
}

/* The FP64 damping field of per-axis FP64 profiles [nx | ny | nz]. */
static double *damping_from_axes(const ora_grid *g, const double *axes) {
    double *d = (double *)malloc(npts(g) * sizeof(double));
    if (!d) return NULL;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i)
                d[lin(g, i, j, k)] = axes[i] + axes[g->nx + j] + axes[g->nx + g->ny + k];
    return d;
}

/* Leapfrog update of the damped acoustic equation at every grid point, from
 * the Laplacian `lap` of u^n already evaluated:
 *   m (u+ - 2u + u-)/dt^2 + damp (u+ - u-)/(2dt) = lap
 *   => u+ = (dt^2 lap + m (2u - u-) + eta u-) / (m + eta),  eta = damp dt/2.
 * With damp = 0 this is Listing fd-3's u+ = 2u - u- + dt^2 lap / m. */
static void leapfrog(const ora_grid *g, double dt, const double *m, const double *damp,
                     const double *lap, const double *u, const double *uprev, double *unext) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                size_t p = lin(g, i, j, k);
                double eta = damp_at(g, damp, i, j, k) * dt * 0.5;
                unext[p] = (dt * dt * lap[p] + m[p] * (2.0 * u[p] - uprev[p]) + eta * uprev[p]) /
                           (m[p] + eta);
            }
}

/* One acoustic time step u^{n+1} from (u^n, u^{n-1}); damp is a damping
 * field (one value per point) or NULL. */
static int acoustic_step_field(const ora_grid *g, int so, int periodic, double dt,
                               const double *m, const double *damp, const double *u,
                               const double *uprev, double *unext) {
    double *lap = (double *)malloc(npts(g) * sizeof(double));
    if (!lap) return ORA_ERR_OOM;
    int st = ora_laplacian(g, so, periodic, u, lap);
    if (st == ORA_OK) leapfrog(g, dt, m, damp, lap, u, uprev, unext);
    free(lap);
    return st;
}

/* One acoustic time step u^{n+1} from (u^n, u^{n-1}); damp holds the per-axis
 * profiles [nx | ny | nz] or is NULL. */
int ora_acoustic_step(const ora_grid *g, int so, int periodic, double dt, const double *m,
                      const double *damp, const double *u, const double *uprev, double *unext) {
    double *field = damp ? damping_from_axes(g, damp) : NULL;
    if (damp && !field) return ORA_ERR_OOM;
    int st = acoustic_step_field(g, so, periodic, dt, m, field, u, uprev, unext);
    free(field);
    return st;
}

/* Trilinear stencil of one sparse point (Eq. interp, tensor product over the
 * three axes): the 8 node indices and FP64 weights.  x1 = floor((x-o)/h),
 * clamped to n-2 so that a point on the last node uses x1 = n-2, frac = 1. */
static int sparse_point(const ora_grid *g, const float *xyz, size_t idx[8], double wgt[8]) {
    const int n[3] = {g->nx, g->ny, g->nz};
    const double h[3] = {g->hx, g->hy, g->hz};
    const double o[3] = {g->ox, g->oy, g->oz};
    int i1[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        double s = ((double)xyz[a] - o[a]) / h[a];
        if (!(s >= 0.0 && s <= (double)(n[a] - 1))) return ORA_ERR_COORD;
        int x1 = (int)floor(s);
        if (x1 > n[a] - 2) x1 = n[a] - 2;
        i1[a] = x1;
        fr[a] = s - (double)x1;
    }
    for (int c = 0; c < 8; ++c) {
        int a = c & 1, b = (c >> 1) & 1, d = (c >> 2) & 1;
        idx[c] = lin(g, i1[0] + a, i1[1] + b, i1[2] + d);
        wgt[c] = (a ? fr[0] : 1.0 - fr[0]) * (b ? fr[1] : 1.0 - fr[1]) * (d ? fr[2] : 1.0 - fr[2]);
    }
    return ORA_OK;
}

/* Receiver interpolation (Eq. interp): out[i] = sum_c w_c u[node_c]. */
int ora_interpolate(const ora_grid *g, int npt, const float *xyz, const double *u, double *out) {
    for (int p = 0; p < npt; ++p) {
        size_t idx[8];
        double w[8];
        int st = sparse_point(g, xyz + 3 * (size_t)p, idx, w);
        if (st) return st;
        double acc = 0.0;
        for (int c = 0; c < 8; ++c) acc += w[c] * u[idx[c]];
        out[p] = acc;
    }
    return ORA_OK;
}

/* Source injection (Listing finject): u[node_c] += w_c * scale[node_c] * q[p],
 * accumulated.  `scale` is dt^2/(m + damp dt/2) per node (dt^2/m undamped). */
int ora_inject(const ora_grid *g, int npt, const float *xyz, const double *q, const double *scale,
               double *u) {
    for (int p = 0; p < npt; ++p) {
        size_t idx[8];
        double w[8];
        int st = sparse_point(g, xyz + 3 * (size_t)p, idx, w);
        if (st) return st;
        for (int c = 0; c < 8; ++c) u[idx[c]] += w[c] * scale[idx[c]] * q[p];
    }
    return ORA_OK;
}

static double *widen(const float *src, size_t n) {
    double *d = (double *)malloc(n * sizeof(double));
    if (d)
        for (size_t i = 0; i < n; ++i) d[i] = (double)src[i];
    return d;
}

/* The FP64 damping field of the API's FP32 damping input (NULL: none):
 * per-axis profiles [nx | ny | nz] (dense = 0) or one value per point
 * [nz][ny][nx] (dense = 1). */
static double *damping_field(const ora_grid *g, const float *damp32, int dense) {
    if (!damp32) return NULL;
    if (dense) return widen(damp32, npts(g));
    double *axes = widen(damp32, (size_t)g->nx + g->ny + g->nz);
    if (!axes) return NULL;
    double *d = damping_from_axes(g, axes);
    free(axes);
    return d;
}

static int check_sparse(const ora_grid *g, int npt, const float *xyz) {
    for (int p = 0; p < npt; ++p) {
        size_t idx[8];
        double w[8];
        if (sparse_point(g, xyz + 3 * (size_t)p, idx, w)) return ORA_ERR_COORD;
    }
    return ORA_OK;
}

/* Injection scale per node: dt^2 / (m + damp dt/2). */
static void injection_scale(const ora_grid *g, double dt, const double *m, const double *damp,
                            double *scale) {
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                size_t p = lin(g, i, j, k);
                scale[p] = dt * dt / (m[p] + damp_at(g, damp, i, j, k) * dt * 0.5);
            }
}

/*
 * Acoustic forward model.  For every shot (shots share m and damp):
 *   u^0, u^{-1} = u_init (or 0, Eq. WE's zero initial conditions);
 *   for n = 0 .. nt-2:  u^{n+1} = step(u^n, u^{n-1});
 *                       inject src[n] into u^{n+1};
 *                       rec[n] = interp(u^n);
 *   rec[nt-1] = interp(u^{nt-1});  u_final = (u^{nt-1}, u^{nt-2}).
 * The per-step order is the paper's schedule of a time iteration: stencil
 * update, then the sparse injection into the t+1 field.
 * Array shapes: m [nz][ny][nx]; damp [nx+ny+nz] (per-axis profiles,
 * damp_dense = 0) or [nz][ny][nx] (a 3-D field, damp_dense = 1) or NULL;
 * src_xyz [nshots][nsrc][3]; src_wav [nshots][nt][nsrc]; rec_xyz
 * [nshots][nrec][3]; rec_out [nshots][nt][nrec]; u_init/u_final
 * [nshots][2][nz][ny][nx] or NULL.
 */
static int acoustic_forward_impl(const ora_grid *g, int so, int periodic, double dt, int nt,
                                 int nshots, const float *m32, const float *damp32,
                                 int damp_dense, int nsrc, const float *src_xyz,
                                 const float *src_wav, int nrec, const float *rec_xyz,
                                 double *rec_out, const float *u_init, double *u_final) {
    if (radius_of(so) < 0 || nt < 1 || nshots < 1 || nsrc < 0 || nrec < 0) return ORA_ERR_ARG;
    const size_t N = npts(g);
    for (int s = 0; s < nshots; ++s) {
        if (check_sparse(g, nsrc, src_xyz + (size_t)s * nsrc * 3)) return ORA_ERR_COORD;
        if (check_sparse(g, nrec, rec_xyz + (size_t)s * nrec * 3)) return ORA_ERR_COORD;
    }
    double *m = widen(m32, N);
    double *damp = damping_field(g, damp32, damp_dense);
    double *scale = (double *)malloc(N * sizeof(double));
    double *u = (double *)malloc(N * sizeof(double));
    double *um = (double *)malloc(N * sizeof(double));
    double *un = (double *)malloc(N * sizeof(double));
    double *q = (double *)malloc(((size_t)nsrc + 1) * sizeof(double));
    int st = ORA_OK;
    if (!m || (damp32 && !damp) || !scale || !u || !um || !un || !q) {
        st = ORA_ERR_OOM;
        goto done;
    }
    injection_scale(g, dt, m, damp, scale);
    for (int s = 0; s < nshots; ++s) {
        const float *sxyz = src_xyz + (size_t)s * nsrc * 3;
        const float *rxyz = rec_xyz + (size_t)s * nrec * 3;
        double *rec = rec_out ? rec_out + (size_t)s * nt * nrec : NULL;
        for (size_t p = 0; p < N; ++p) {
            u[p] = u_init ? (double)u_init[((size_t)s * 2 + 0) * N + p] : 0.0;
            um[p] = u_init ? (double)u_init[((size_t)s * 2 + 1) * N + p] : 0.0;
        }
        for (int n = 0; n + 1 < nt; ++n) {
            st = acoustic_step_field(g, so, periodic, dt, m, damp, u, um, un);
            if (st) goto done;
            for (int p = 0; p < nsrc; ++p) q[p] = (double)src_wav[((size_t)s * nt + n) * nsrc + p];
            ora_inject(g, nsrc, sxyz, q, scale, un);
            if (rec) ora_interpolate(g, nrec, rxyz, u, rec + (size_t)n * nrec);
            double *t = um;
            um = u;
            u = un;
            un = t;
        }
        if (rec) ora_interpolate(g, nrec, rxyz, u, rec + (size_t)(nt - 1) * nrec);
        if (u_final) {
            memcpy(u_final + ((size_t)s * 2 + 0) * N, u, N * sizeof(double));
            memcpy(u_final + ((size_t)s * 2 + 1) * N, um, N * sizeof(double));
        }
    }
done:
    free(m);
    free(damp);
    free(scale);
    free(u);
    free(um);
    free(un);
    free(q);
    return st;
}

int ora_acoustic_forward(const ora_grid *g, int so, int periodic, double dt, int nt, int nshots,
                         const float *m32, const float *damp32, int nsrc, const float *src_xyz,
                         const float *src_wav, int nrec, const float *rec_xyz, double *rec_out,
                         const float *u_init, double *u_final) {
    return acoustic_forward_impl(g, so, periodic, dt, nt, nshots, m32, damp32, 0, nsrc, src_xyz,
                                 src_wav, nrec, rec_xyz, rec_out, u_init, u_final);
}

/* The acoustic forward model with the damping given as a 3-D field
 * damp[nz][ny][nx] (one value per point, NULL = none) instead of per-axis
 * profiles. */
int ora_acoustic_forward_field(const ora_grid *g, int so, int periodic, double dt, int nt,
                               int nshots, const float *m32, const float *damp32, int nsrc,
                               const float *src_xyz, const float *src_wav, int nrec,
                               const float *rec_xyz, double *rec_out, const float *u_init,
                               double *u_final) {
    return acoustic_forward_impl(g, so, periodic, dt, nt, nshots, m32, damp32, 1, nsrc, src_xyz,
                                 src_wav, nrec, rec_xyz, rec_out, u_init, u_final);
}

/*
 * ---- Reduced-precision storage ------------------------------------------
 *
 * The paper lists mixed-precision arithmetic and on-the-fly data compression
 * among its further performance work (section "Further work").  Reading used
 * here: the bulk fields are STORED in IEEE binary16 and all arithmetic stays
 * in FP32 on the device; the oracle models the storage exactly and keeps its
 * own arithmetic in FP64.  What is stored:
 *   - the wavefield levels u^n, u^{n-1} (every value written is rounded);
 *   - the coefficient b = dt^2 / (m + damp dt/2) that multiplies the
 *     Laplacian and the injected source.
 * A value that the device computes in FP32 and then stores is rounded to
 * FP32 first and to binary16 second (the decision taken in the device's
 * precision); the sum of two binary16 values (source injection into a stored
 * field) is rounded once.
 */

/* Nearest IEEE binary16 value of x, ties to even, as a double.  From the
 * format's definition: 11 significant bits for normal numbers (unbiased
 * exponents -14..15); below 2^-14 the spacing is fixed at 2^-24 (subnormal
 * numbers); magnitudes from 65520 (the midpoint between the largest finite
 * value 65504 and 2^16) up round to infinity.  The sign of zero and NaN are
 * kept. */
double ora_round_binary16(double x) {
    if (x != x) return x;
    const double a = fabs(x);
    if (a == 0.0) return x;
    if (a >= 65520.0) return copysign(INFINITY, x);
    int e2;
    frexp(a, &e2); /* a in [2^(e2-1), 2^e2) */
    int ex = e2 - 1;
    if (ex < -14) ex = -14;
    const double q = ldexp(1.0, ex - 10); /* spacing of binary16 values near a */
    return copysign(nearbyint(a / q) * q, x); /* a / q exact; default mode: ties to even */
}

/* A value computed on the device in FP32 and stored in binary16. */
static double store16(double x) { return ora_round_binary16((double)(float)x); }

/*
 * Acoustic forward model with the storage of `storage`:
 *   0  no rounding: the same model as ora_acoustic_forward, with the update
 *      written in the b form below (equal to it up to FP64 rounding);
 *   1  binary16 storage of u and b as described above;
 *   2  binary16 storage of b only (u kept exact): one step of it, stored,
 *      is one step of storage 1.
 * The update in b form (b = dt^2/(m + eta), eta = damp dt/2; algebraically
 * the damped leapfrog update of ora_acoustic_forward):
 *   u+ = u + (1 - b damp/dt)(u - u-) + b lap(u).
 * Per step n: u^{n+1} = S(update); then for every source p and corner c in
 * order, u^{n+1}[node] = S16(u^{n+1}[node] + S(w_c b[node] q_p[n])), where S
 * is store16 (storage 1) or the identity, and S16 the single binary16
 * rounding of the exact sum; rec[n] = interp(u^n).  Shapes as in
 * ora_acoustic_forward; u_init is rounded on entry; u_final holds the stored
 * values.
 */
int ora_acoustic_forward_storage(const ora_grid *g, int so, int periodic, double dt, int nt,
                                 int nshots, const float *m32, const float *damp32, int nsrc,
                                 const float *src_xyz, const float *src_wav, int nrec,
                                 const float *rec_xyz, double *rec_out, const float *u_init,
                                 double *u_final, int storage) {
    if (radius_of(so) < 0 || nt < 1 || nshots < 1 || nsrc < 0 || nrec < 0 || storage < 0 ||
        storage > 2)
        return ORA_ERR_ARG;
    const size_t N = npts(g);
    for (int s = 0; s < nshots; ++s) {
        if (check_sparse(g, nsrc, src_xyz + (size_t)s * nsrc * 3)) return ORA_ERR_COORD;
        if (check_sparse(g, nrec, rec_xyz + (size_t)s * nrec * 3)) return ORA_ERR_COORD;
    }
    double *m = widen(m32, N);
    double *damp = damping_field(g, damp32, 0);
    double *b = (double *)malloc(N * sizeof(double));
    double *lap = (double *)malloc(N * sizeof(double));
    double *u = (double *)malloc(N * sizeof(double));
    double *um = (double *)malloc(N * sizeof(double));
    double *un = (double *)malloc(N * sizeof(double));
    int st = ORA_OK;
    if (!m || (damp32 && !damp) || !b || !lap || !u || !um || !un) {
        st = ORA_ERR_OOM;
        goto done;
    }
    injection_scale(g, dt, m, damp, b); /* b = dt^2 / (m + damp dt/2) */
    if (storage >= 1)
        for (size_t p = 0; p < N; ++p) b[p] = store16(b[p]);
    for (int s = 0; s < nshots; ++s) {
        const float *sxyz = src_xyz + (size_t)s * nsrc * 3;
        const float *rxyz = rec_xyz + (size_t)s * nrec * 3;
        double *rec = rec_out ? rec_out + (size_t)s * nt * nrec : NULL;
        for (size_t p = 0; p < N; ++p) {
            u[p] = u_init ? (double)u_init[((size_t)s * 2 + 0) * N + p] : 0.0;
            um[p] = u_init ? (double)u_init[((size_t)s * 2 + 1) * N + p] : 0.0;
            if (storage == 1) {
                u[p] = store16(u[p]);
                um[p] = store16(um[p]);
            }
        }
        for (int n = 0; n + 1 < nt; ++n) {
            st = ora_laplacian(g, so, periodic, u, lap);
            if (st) goto done;
            for (int k = 0; k < g->nz; ++k)
                for (int j = 0; j < g->ny; ++j)
                    for (int i = 0; i < g->nx; ++i) {
                        const size_t p = lin(g, i, j, k);
                        const double zeta = b[p] * damp_at(g, damp, i, j, k) / dt;
                        const double v = u[p] + (1.0 - zeta) * (u[p] - um[p]) + b[p] * lap[p];
                        un[p] = storage == 1 ? store16(v) : v;
                    }
            for (int p = 0; p < nsrc; ++p) {
                size_t idx[8];
                double w[8];
                sparse_point(g, sxyz + 3 * (size_t)p, idx, w);
                const double q = (double)src_wav[((size_t)s * nt + n) * nsrc + p];
                for (int c = 0; c < 8; ++c) {
                    const double add = w[c] * b[idx[c]] * q;
                    if (storage == 1)
                        un[idx[c]] = ora_round_binary16(un[idx[c]] + store16(add));
                    else
                        un[idx[c]] += add;
                }
            }
            if (rec) ora_interpolate(g, nrec, rxyz, u, rec + (size_t)n * nrec);
            double *t = um;
            um = u;
            u = un;
            un = t;
        }
        if (rec) ora_interpolate(g, nrec, rxyz, u, rec + (size_t)(nt - 1) * nrec);
        if (u_final) {
            memcpy(u_final + ((size_t)s * 2 + 0) * N, u, N * sizeof(double));
            memcpy(u_final + ((size_t)s * 2 + 1) * N, um, N * sizeof(double));
        }
    }
done:
    free(m);
    free(damp);
    free(b);
    free(lap);
    free(u);
    free(um);
    free(un);
    return st;
}

/*
 * TTI operators for one field q: Hz q = sum_i D_i(n_i (n . grad q)) and
 * L q = sum_i D_i D_i q, with n = (sin t cos f, sin t sin f, cos t) per point.
 * deriv = 0: D is the central first derivative of order so (inner and outer);
 * deriv = 1: the staggered reading, inner derivatives D+ and outer D-
 *   Hz q = sum_i D-_i(n_i sum_j n_j D+_j q),  L q = sum_i D-_i D+_i q,
 * with n sampled at the nodes (the half-point shifts are not interpolated).
 * Temporaries outside the grid are zero ghosts (or periodic images).
 * Evaluated literally: gradient, projection on n, scaling by n_i, second
 * first-derivative pass.
 */
int ora_tti_operators_kind(const ora_grid *g, int so, int periodic, int deriv,
                           const double *theta, const double *phi, const double *q, double *hz,
                           double *lq) {
    if (deriv < 0 || deriv > 1) return ORA_ERR_ARG;
    const int inner = deriv ? 1 : 0, outer = deriv ? -1 : 0;
    const size_t N = npts(g);
    double *grad[3], *proj, *tmp, *dtmp;
    int st = ORA_OK;
    for (int a = 0; a < 3; ++a) grad[a] = (double *)malloc(N * sizeof(double));
    proj = (double *)malloc(N * sizeof(double));
    tmp = (double *)malloc(N * sizeof(double));
    dtmp = (double *)malloc(N * sizeof(double));
    if (!grad[0] || !grad[1] || !grad[2] || !proj || !tmp || !dtmp) {
        st = ORA_ERR_OOM;
        goto done;
    }
    /* gradient of q */
    for (int a = 0; a < 3; ++a) {
        st = ora_first_derivative_kind(g, so, periodic, a, inner, q, grad[a]);
        if (st) goto done;
    }
    /* projection on the symmetry axis: proj = n . grad q */
#pragma omp parallel for schedule(static)
    for (size_t p = 0; p < N; ++p) {
        double nx = sin(theta[p]) * cos(phi[p]), ny = sin(theta[p]) * sin(phi[p]),
               nz = cos(theta[p]);
        proj[p] = nx * grad[0][p] + ny * grad[1][p] + nz * grad[2][p];
    }
    if (hz) memset(hz, 0, N * sizeof(double));
    if (lq) memset(lq, 0, N * sizeof(double));
    for (int a = 0; a < 3; ++a) {
        if (hz) {
            /* hz += D_a (n_a * proj) */
#pragma omp parallel for schedule(static)
            for (size_t p = 0; p < N; ++p) {
                double na = a == 0   ? sin(theta[p]) * cos(phi[p])
                            : a == 1 ? sin(theta[p]) * sin(phi[p])
                                     : cos(theta[p]);
                tmp[p] = na * proj[p];
            }
            ora_first_derivative_kind(g, so, periodic, a, outer, tmp, dtmp);
#pragma omp parallel for schedule(static)
            for (size_t p = 0; p < N; ++p) hz[p] += dtmp[p];
        }
        if (lq) {
            /* lq += D_a (D_a q) */
            ora_first_derivative_kind(g, so, periodic, a, outer, grad[a], dtmp);
#pragma omp parallel for schedule(static)
            for (size_t p = 0; p < N; ++p) lq[p] += dtmp[p];
        }
    }
done:
    for (int a = 0; a < 3; ++a) free(grad[a]);
    free(proj);
    free(tmp);
    free(dtmp);
    return st;
}

int ora_tti_operators(const ora_grid *g, int so, int periodic, const double *theta,
                      const double *phi, const double *q, double *hz, double *lq) {
    return ora_tti_operators_kind(g, so, periodic, 0, theta, phi, q, hz, lq);
}

/* TTI coefficients a = 1 + 2 eps and s = sqrt(1 + 2 delta); with storage = 1
 * rounded to FP32, as a device that stores them in FP32 uses them. */
static double coef_a(double eps, int storage) {
    const double a = 1.0 + 2.0 * eps;
    return storage ? (double)(float)a : a;
}
static double coef_s(double delta, int storage) {
    const double sv = sqrt(1.0 + 2.0 * delta);
    return storage ? (double)(float)sv : sv;
}

/* TTI receivers: interp(p), or interp((p + r)/2) with receiver = 1 (tmp is
 * scratch of one field). */
static void record(const ora_grid *g, int receiver, int nrec, const float *rxyz,
                   const double *p, const double *r, double *tmp, double *out) {
    if (!receiver) {
        ora_interpolate(g, nrec, rxyz, p, out);
        return;
    }
    const size_t N = npts(g);
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < N; ++i) tmp[i] = 0.5 * (p[i] + r[i]);
    ora_interpolate(g, nrec, rxyz, tmp, out);
}

/*
 * TTI forward model (two coupled fields p, r).  Per shot and step n:
 *   Hxy p = L p - Hz p;
 *   m p_tt + damp p_t = (1+2 eps) Hxy p + sqrt(1+2 delta) Hz r
 *   m r_tt + damp r_t = sqrt(1+2 delta) Hxy p + Hz r
 * each advanced with the same centred leapfrog as the acoustic case; src[n]
 * is injected into p^{n+1} and r^{n+1}; rec[n] = interp(p^n), or with
 * receiver = 1 the alternative reading rec[n] = interp((p^n + r^n) / 2).
 * deriv selects the central (0) or staggered (1) first derivatives of
 * ora_tti_operators_kind.
 * Fields eps, delta, theta, phi are [nz][ny][nx].  p_init/r_init and
 * p_final/r_final are [nshots][2][nz][ny][nx] (levels n, n-1) or NULL.
 *
 * storage = 1 is a model of FP32 storage (not a reading of the paper; a
 * yardstick for the device's rounding): the coefficients a = 1 + 2 eps and
 * s = sqrt(1 + 2 delta) are rounded to FP32 once, and p^{n+1}, r^{n+1} are
 * rounded to FP32 after every step (after the injection); all arithmetic
 * stays FP64.  storage = 0 is the FP64 model.
 */
static int tti_forward_impl(const ora_grid *g, int so, int periodic, int deriv, int receiver,
                            double dt, int nt, int nshots, const float *m32, const float *damp32,
                            const float *eps32, const float *delta32, const float *theta32,
                            const float *phi32, int nsrc, const float *src_xyz,
                            const float *src_wav, int nrec, const float *rec_xyz,
                            double *rec_out, const float *p_init, const float *r_init,
                            double *p_final, double *r_final, int storage) {
    if (radius_of(so) < 0 || nt < 1 || nshots < 1 || nsrc < 0 || nrec < 0) return ORA_ERR_ARG;
    if (storage < 0 || storage > 1) return ORA_ERR_ARG;
    if (deriv < 0 || deriv > 1 || receiver < 0 || receiver > 1) return ORA_ERR_ARG;
    const size_t N = npts(g);
    for (int s = 0; s < nshots; ++s) {
        if (check_sparse(g, nsrc, src_xyz + (size_t)s * nsrc * 3)) return ORA_ERR_COORD;
        if (check_sparse(g, nrec, rec_xyz + (size_t)s * nrec * 3)) return ORA_ERR_COORD;
    }
    int st = ORA_OK;
    double *m = widen(m32, N), *eps = widen(eps32, N), *del = widen(delta32, N);
    double *th = widen(theta32, N), *ph = widen(phi32, N);
    double *damp = damping_field(g, damp32, 0);
    double *scale = (double *)malloc(N * sizeof(double));
    double *bufs[10];
    for (int b = 0; b < 10; ++b) bufs[b] = (double *)malloc(N * sizeof(double));
    double *q = (double *)malloc(((size_t)nsrc + 1) * sizeof(double));
    double *p = bufs[0], *pm = bufs[1], *pn = bufs[2], *r = bufs[3], *rm = bufs[4], *rn = bufs[5];
    double *hzp = bufs[6], *lp = bufs[7], *hzr = bufs[8], *rhs = bufs[9];
    int ok = m && eps && del && th && ph && (!damp32 || damp) && scale && q;
    for (int b = 0; b < 10; ++b) ok = ok && bufs[b];
    if (!ok) {
        st = ORA_ERR_OOM;
        goto done;
    }
    injection_scale(g, dt, m, damp, scale);
    for (int s = 0; s < nshots; ++s) {
        const float *sxyz = src_xyz + (size_t)s * nsrc * 3;
        const float *rxyz = rec_xyz + (size_t)s * nrec * 3;
        double *rec = rec_out ? rec_out + (size_t)s * nt * nrec : NULL;
        for (size_t i = 0; i < N; ++i) {
            p[i] = p_init ? (double)p_init[((size_t)s * 2 + 0) * N + i] : 0.0;
            pm[i] = p_init ? (double)p_init[((size_t)s * 2 + 1) * N + i] : 0.0;
            r[i] = r_init ? (double)r_init[((size_t)s * 2 + 0) * N + i] : 0.0;
            rm[i] = r_init ? (double)r_init[((size_t)s * 2 + 1) * N + i] : 0.0;
        }
        for (int n = 0; n + 1 < nt; ++n) {
            st = ora_tti_operators_kind(g, so, periodic, deriv, th, ph, p, hzp, lp);
            if (!st) st = ora_tti_operators_kind(g, so, periodic, deriv, th, ph, r, hzr, NULL);
            if (st) goto done;
            /* p equation: rhs = (1+2eps)(Lp - Hz p) + sqrt(1+2delta) Hz r */
#pragma omp parallel for schedule(static)
            for (size_t i = 0; i < N; ++i)
                rhs[i] = coef_a(eps[i], storage) * (lp[i] - hzp[i]) +
                         coef_s(del[i], storage) * hzr[i];
            leapfrog(g, dt, m, damp, rhs, p, pm, pn);
            /* r equation: rhs = sqrt(1+2delta)(Lp - Hz p) + Hz r */
#pragma omp parallel for schedule(static)
            for (size_t i = 0; i < N; ++i)
                rhs[i] = coef_s(del[i], storage) * (lp[i] - hzp[i]) + hzr[i];
            leapfrog(g, dt, m, damp, rhs, r, rm, rn);
            for (int k = 0; k < nsrc; ++k) q[k] = (double)src_wav[((size_t)s * nt + n) * nsrc + k];
            ora_inject(g, nsrc, sxyz, q, scale, pn);
            ora_inject(g, nsrc, sxyz, q, scale, rn);
            if (storage) {
#pragma omp parallel for schedule(static)
                for (size_t i = 0; i < N; ++i) {
                    pn[i] = (double)(float)pn[i];
                    rn[i] = (double)(float)rn[i];
                }
            }
            if (rec) record(g, receiver, nrec, rxyz, p, r, rhs, rec + (size_t)n * nrec);
            double *t = pm;
            pm = p;
            p = pn;
            pn = t;
            t = rm;
            rm = r;
            r = rn;
            rn = t;
        }
        if (rec) record(g, receiver, nrec, rxyz, p, r, rhs, rec + (size_t)(nt - 1) * nrec);
        if (p_final) {
            memcpy(p_final + ((size_t)s * 2 + 0) * N, p, N * sizeof(double));
            memcpy(p_final + ((size_t)s * 2 + 1) * N, pm, N * sizeof(double));
        }
        if (r_final) {
            memcpy(r_final + ((size_t)s * 2 + 0) * N, r, N * sizeof(double));
            memcpy(r_final + ((size_t)s * 2 + 1) * N, rm, N * sizeof(double));
        }
    }
done:
    free(m);
    free(eps);
    free(del);
    free(th);
    free(ph);
    free(damp);
    free(scale);
    free(q);
    for (int b = 0; b < 10; ++b) free(bufs[b]);
    return st;
}

int ora_tti_forward_opts(const ora_grid *g, int so, int periodic, int deriv, int receiver,
                         double dt, int nt, int nshots, const float *m32, const float *damp32,
                         const float *eps32, const float *delta32, const float *theta32,
                         const float *phi32, int nsrc, const float *src_xyz,
                         const float *src_wav, int nrec, const float *rec_xyz, double *rec_out,
                         const float *p_init, const float *r_init, double *p_final,
                         double *r_final) {
    return tti_forward_impl(g, so, periodic, deriv, receiver, dt, nt, nshots, m32, damp32, eps32,
                            delta32, theta32, phi32, nsrc, src_xyz, src_wav, nrec, rec_xyz,
                            rec_out, p_init, r_init, p_final, r_final, 0);
}

/* The TTI forward model (central derivatives, receivers on p) with the FP32
 * storage model of tti_forward_impl (storage = 1) or without it (0). */
int ora_tti_forward_storage(const ora_grid *g, int so, int periodic, double dt, int nt,
                            int nshots, const float *m32, const float *damp32, const float *eps32,
                            const float *delta32, const float *theta32, const float *phi32,
                            int nsrc, const float *src_xyz, const float *src_wav, int nrec,
                            const float *rec_xyz, double *rec_out, const float *p_init,
                            const float *r_init, double *p_final, double *r_final, int storage) {
    return tti_forward_impl(g, so, periodic, 0, 0, dt, nt, nshots, m32, damp32, eps32, delta32,
                            theta32, phi32, nsrc, src_xyz, src_wav, nrec, rec_xyz, rec_out, p_init,
                            r_init, p_final, r_final, storage);
}

int ora_tti_forward(const ora_grid *g, int so, int periodic, double dt, int nt, int nshots,
                    const float *m32, const float *damp32, const float *eps32,
                    const float *delta32, const float *theta32, const float *phi32, int nsrc,
                    const float *src_xyz, const float *src_wav, int nrec, const float *rec_xyz,
                    double *rec_out, const float *p_init, const float *r_init, double *p_final,
                    double *r_final) {
    return ora_tti_forward_opts(g, so, periodic, 0, 0, dt, nt, nshots, m32, damp32, eps32,
                                delta32, theta32, phi32, nsrc, src_xyz, src_wav, nrec, rec_xyz,
                                rec_out, p_init, r_init, p_final, r_final);
}

/* ------------------------------------------------------------------------- */
/* Adjoint and gradient (the adjoint-state method the paper names as the
 * purpose of time-subsampled saving: "data inversion using adjoint-state
 * methods").  The paper prints no adjoint; what follows is the exact transpose
 * of the discrete forward map above, derived from it:
 *
 *   forward   u^{n+1} = M1 u^n - M2 u^{n-1} + B S^T q^n,  d^n = R u^n,
 *             M1 = 2 - zeta + B L,  M2 = 1 - zeta,  B = dt^2/(m + eta),
 *             zeta = damp dt/(m + eta)   (all diagonal except L),
 *   adjoint   lambda^n = R^T dd^n + M1^T lambda^{n+1} - M2^T lambda^{n+2},
 *             M1^T x = (2 - zeta) x + L (B x),  M2^T x = (1 - zeta) x,
 *             lambda^{nt} = lambda^{nt+1} = 0,
 *             dq^n = S B lambda^{n+1}  (n <= nt-2),  dq^{nt-1} = 0,
 *   gradient  of <dd, d(m)> with respect to m:
 *             sum_{n=0}^{nt-2} lambda^{n+1} * du^{n+1}/dm,
 *             du^{n+1}/dm = -(u^{n+1} - 2u^n + u^{n-1}) / (m + eta).
 * S = source interpolation, R = receiver interpolation (trilinear, Eq. interp).
 */

/* lam_n = rtd + (2 - zeta) lam1 + L(B lam1) - (1 - zeta) lam2 */
static int adjoint_step(const ora_grid *g, int so, int periodic, double dt, const double *m,
                        const double *damp, const double *lam1, const double *lam2,
                        double *lam_n, double *tmp, double *ltmp) {
    const size_t N = npts(g);
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                size_t p = lin(g, i, j, k);
                double eta = damp_at(g, damp, i, j, k) * dt * 0.5;
                tmp[p] = dt * dt / (m[p] + eta) * lam1[p];
            }
    int st = ora_laplacian(g, so, periodic, tmp, ltmp);
    if (st) return st;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                size_t p = lin(g, i, j, k);
                double eta = damp_at(g, damp, i, j, k) * dt * 0.5;
                double zeta = 2.0 * eta / (m[p] + eta);
                lam_n[p] = (2.0 - zeta) * lam1[p] + ltmp[p] - (1.0 - zeta) * lam2[p];
            }
    (void)N;
    return ORA_OK;
}

/* Adjoint of ora_acoustic_forward's source-to-receiver map (zero initial
 * state).  rec_resid [nshots][nt][nrec] in; src_grad [nshots][nt][nsrc] out. */
int ora_acoustic_adjoint(const ora_grid *g, int so, int periodic, double dt, int nt, int nshots,
                         const float *m32, const float *damp32, int nsrc, const float *src_xyz,
                         double *src_grad, int nrec, const float *rec_xyz,
                         const double *rec_resid) {
    if (radius_of(so) < 0 || nt < 1 || nshots < 1 || nsrc < 0 || nrec < 0) return ORA_ERR_ARG;
    const size_t N = npts(g);
    for (int s = 0; s < nshots; ++s) {
        if (check_sparse(g, nsrc, src_xyz + (size_t)s * nsrc * 3)) return ORA_ERR_COORD;
        if (check_sparse(g, nrec, rec_xyz + (size_t)s * nrec * 3)) return ORA_ERR_COORD;
    }
    int st = ORA_OK;
    double *m = widen(m32, N);
    double *damp = damping_field(g, damp32, 0);
    double *l0 = (double *)calloc(N, sizeof(double)), *l1 = (double *)calloc(N, sizeof(double));
    double *l2 = (double *)calloc(N, sizeof(double)), *tmp = (double *)malloc(N * sizeof(double));
    double *ltmp = (double *)malloc(N * sizeof(double)), *ones = (double *)malloc(N * sizeof(double));
    double *bl = (double *)malloc(N * sizeof(double));
    if (!m || (damp32 && !damp) || !l0 || !l1 || !l2 || !tmp || !ltmp || !ones || !bl) {
        st = ORA_ERR_OOM;
        goto done;
    }
    for (size_t p = 0; p < N; ++p) ones[p] = 1.0;
    for (int s = 0; s < nshots; ++s) {
        const float *sxyz = src_xyz + (size_t)s * nsrc * 3;
        const float *rxyz = rec_xyz + (size_t)s * nrec * 3;
        const double *dd = rec_resid + (size_t)s * nt * nrec;
        double *dq = src_grad + (size_t)s * nt * nsrc;
        memset(l1, 0, N * sizeof(double)); /* lambda^{n+1} */
        memset(l2, 0, N * sizeof(double)); /* lambda^{n+2} */
        for (int n = nt - 1; n >= 0; --n) {
            /* dq^n = S B lambda^{n+1} */
            if (nsrc > 0) {
                if (n <= nt - 2) {
                    for (int k = 0; k < g->nz; ++k)
                        for (int j = 0; j < g->ny; ++j)
                            for (int i = 0; i < g->nx; ++i) {
                                size_t p = lin(g, i, j, k);
                                double eta = damp_at(g, damp, i, j, k) * dt * 0.5;
                                bl[p] = dt * dt / (m[p] + eta) * l1[p];
                            }
                    ora_interpolate(g, nsrc, sxyz, bl, dq + (size_t)n * nsrc);
                } else {
                    for (int k = 0; k < nsrc; ++k) dq[(size_t)n * nsrc + k] = 0.0;
                }
            }
            st = adjoint_step(g, so, periodic, dt, m, damp, l1, l2, l0, tmp, ltmp);
            if (st) goto done;
            /* + R^T dd^n */
            st = ora_inject(g, nrec, rxyz, dd + (size_t)n * nrec, ones, l0);
            if (st) goto done;
            double *t = l2;
            l2 = l1;
            l1 = l0;
            l0 = t;
        }
    }
done:
    free(m);
    free(damp);
    free(l0);
    free(l1);
    free(l2);
    free(tmp);
    free(ltmp);
    free(ones);
    free(bl);
    return st;
}

/* Gradient with respect to m of <rec_resid, d(m)> (the FWI gradient when
 * rec_resid = d(m) - d_obs), zero initial state, summed over shots; keeps the
 * whole forward history in memory (small grids only).  grad [nz][ny][nx]. */
int ora_acoustic_gradient(const ora_grid *g, int so, double dt, int nt, int nshots,
                          const float *m32, const float *damp32, int nsrc, const float *src_xyz,
                          const float *src_wav, int nrec, const float *rec_xyz,
                          const double *rec_resid, double *grad) {
    if (radius_of(so) < 0 || nt < 1 || nshots < 1 || nsrc < 0 || nrec < 0) return ORA_ERR_ARG;
    const size_t N = npts(g);
    for (int s = 0; s < nshots; ++s) {
        if (check_sparse(g, nsrc, src_xyz + (size_t)s * nsrc * 3)) return ORA_ERR_COORD;
        if (check_sparse(g, nrec, rec_xyz + (size_t)s * nrec * 3)) return ORA_ERR_COORD;
    }
    int st = ORA_OK;
    double *m = widen(m32, N);
    double *damp = damping_field(g, damp32, 0);
    double *hist = (double *)malloc((size_t)(nt + 1) * N * sizeof(double)); /* u^{-1..nt-1} */
    double *scale = (double *)malloc(N * sizeof(double));
    double *q = (double *)malloc(((size_t)nsrc + 1) * sizeof(double));
    double *l0 = (double *)calloc(N, sizeof(double)), *l1 = (double *)calloc(N, sizeof(double));
    double *l2 = (double *)calloc(N, sizeof(double)), *tmp = (double *)malloc(N * sizeof(double));
    double *ltmp = (double *)malloc(N * sizeof(double)), *ones = (double *)malloc(N * sizeof(double));
    if (!m || (damp32 && !damp) || !hist || !scale || !q || !l0 || !l1 || !l2 || !tmp || !ltmp ||
        !ones) {
        st = ORA_ERR_OOM;
        goto done;
    }
    for (size_t p = 0; p < N; ++p) {
        ones[p] = 1.0;
        grad[p] = 0.0;
    }
    injection_scale(g, dt, m, damp, scale);
    for (int s = 0; s < nshots; ++s) {
        const float *sxyz = src_xyz + (size_t)s * nsrc * 3;
        const float *rxyz = rec_xyz + (size_t)s * nrec * 3;
        const double *dd = rec_resid + (size_t)s * nt * nrec;
#define U(n) (hist + (size_t)((n) + 1) * N)
        memset(U(-1), 0, N * sizeof(double));
        memset(U(0), 0, N * sizeof(double));
        for (int n = 0; n + 1 < nt; ++n) {
            st = acoustic_step_field(g, so, 0, dt, m, damp, U(n), U(n - 1), U(n + 1));
            if (st) goto done;
            for (int k = 0; k < nsrc; ++k) q[k] = (double)src_wav[((size_t)s * nt + n) * nsrc + k];
            ora_inject(g, nsrc, sxyz, q, scale, U(n + 1));
        }
        memset(l1, 0, N * sizeof(double));
        memset(l2, 0, N * sizeof(double));
        for (int n = nt - 1; n >= 0; --n) {
            /* gradient term of step n -> n+1 uses lambda^{n+1} */
            if (n <= nt - 2)
                for (int k = 0; k < g->nz; ++k)
                    for (int j = 0; j < g->ny; ++j)
                        for (int i = 0; i < g->nx; ++i) {
                            size_t p = lin(g, i, j, k);
                            double eta = damp_at(g, damp, i, j, k) * dt * 0.5;
                            double du = -(U(n + 1)[p] - 2.0 * U(n)[p] + U(n - 1)[p]) / (m[p] + eta);
                            grad[p] += l1[p] * du;
                        }
            st = adjoint_step(g, so, 0, dt, m, damp, l1, l2, l0, tmp, ltmp);
            if (st) goto done;
            st = ora_inject(g, nrec, rxyz, dd + (size_t)n * nrec, ones, l0);
            if (st) goto done;
            double *t = l2;
            l2 = l1;
            l1 = l0;
            l0 = t;
        }
#undef U
    }
done:
    free(m);
    free(damp);
    free(hist);
    free(scale);
    free(q);
    free(l0);
    free(l1);
    free(l2);
    free(tmp);
    free(ltmp);
    free(ones);
    return st;
}
