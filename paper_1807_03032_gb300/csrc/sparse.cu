// sparse.cu -- K3/K4: sparse source injection and receiver interpolation.
//
// Trilinear interpolation (Eq. interp, the tensor product of the 1-D linear
// weights 1 - frac and frac along x, y and z) gathers
//   rec[n][i] = sum_c w_c u^n(node_c),
// and injection, its adjoint (Listing finject), scatters
//   u^{n+1}(node_c) += w_c * b(node_c) * q[n],  b = dt^2 / (m + damp dt/2),
// with atomicAdd so that sources sharing a node accumulate (injection is a
// reduction).  One launch does both: receiver threads first, then one thread
// per (source, corner).
#include "kernels.cuh"

namespace fdsweep {
namespace {

__device__ __forceinline__ float corner_weight(const SparsePoint &p, int c) {
    const float wx = (c & 1) ? p.fx : 1.f - p.fx;
    const float wy = (c & 2) ? p.fy : 1.f - p.fy;
    const float wz = (c & 4) ? p.fz : 1.f - p.fz;
    return wx * wy * wz;
}

__device__ __forceinline__ int64_t corner_offset(const SparsePoint &p, int c, const WaveLayout &L) {
    return (int64_t)p.base + ((c & 1) ? 1 : 0) + ((c & 2) ? L.nxp : 0) + ((c & 4) ? L.plane : 0);
}

// Threads [0, nrec_total) interpolate receivers (nrec_total = 0 when only
// injecting); the following nshots*nsrc*8 threads inject.
__global__ void sparse_kernel(const SparseArgs a, int step, int do_inject, int64_t nrec_total) {
    const int n = step + (a.step_base ? *a.step_base : 0);
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid < nrec_total) {
        const int ro = a.rec_t0 + a.rec_dt * n;
        if (ro < 0 || ro >= a.nt) return;
        const int s = (int)(gid / a.nrec);
        const int i = (int)(gid - (int64_t)s * a.nrec);
        const SparsePoint p = a.rec_tab[gid];
        const float *u = a.wave + (int64_t)(s * a.fields_per_shot + a.rec_level) * a.L.vol;
        float acc = 0.f;
        if (a.rec_mean) {  // interpolate (u + u2) / 2
            const float *u2 = a.wave + (int64_t)(s * a.fields_per_shot + a.rec_level2) * a.L.vol;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int64_t o = corner_offset(p, c, a.L);
                acc = fmaf(corner_weight(p, c), 0.5f * (__ldg(u + o) + __ldg(u2 + o)), acc);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c)
                acc = fmaf(corner_weight(p, c), __ldg(u + corner_offset(p, c, a.L)), acc);
        }
        a.rec_out[((int64_t)s * a.nt + ro) * a.nrec + i] = acc;
        return;
    }
    if (!do_inject) return;
    const int64_t k = gid - nrec_total;
    if (k >= (int64_t)a.nshots * a.nsrc * 8) return;
    const int c = (int)(k & 7);
    const int64_t ps = k >> 3;  // (shot, source)
    const int s = (int)(ps / a.nsrc);
    const int isrc = (int)(ps - (int64_t)s * a.nsrc);
    const int qi = a.inj_t0 + a.inj_dt * n;
    if (qi < 0 || qi >= a.nt) return;
    const SparsePoint p = a.src_tab[ps];
    const int64_t off = corner_offset(p, c, a.L);
    const float q = a.src_wav[((int64_t)s * a.nt + qi) * a.nsrc + isrc];
    const float val = corner_weight(p, c) * __ldg(a.bcoef + off) * q;
    atomicAdd(a.wave + (int64_t)(s * a.fields_per_shot + a.inj_level0) * a.L.vol + off, val);
    if (a.inj_level1 >= 0)
        atomicAdd(a.wave + (int64_t)(s * a.fields_per_shot + a.inj_level1) * a.L.vol + off, val);
}

__global__ void bump_kernel(int *counter, int by) { *counter += by; }

// g += sum_b w_b (u_b - 2 u_b' + u_b''), shots b in order; u_b' and u_b'' are
// the two levels below u_b (one field apart).  Strides and n in float4 units.
__global__ void grad_batch_kernel(float *__restrict__ g, const float *__restrict__ w,
                                  int64_t w_stride, const float *__restrict__ u,
                                  int64_t u_stride, int64_t level, int nb, int64_t n4) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 o = reinterpret_cast<float4 *>(g)[i];
        for (int b = 0; b < nb; ++b) {
            const float4 a = reinterpret_cast<const float4 *>(w)[b * w_stride + i];
            const float4 *ub = reinterpret_cast<const float4 *>(u) + b * u_stride + i;
            const float4 p = ub[0], q = ub[-level], r = ub[-2 * level];
            o.x = fmaf(a.x, p.x - 2.f * q.x + r.x, o.x);
            o.y = fmaf(a.y, p.y - 2.f * q.y + r.y, o.y);
            o.z = fmaf(a.z, p.z - 2.f * q.z + r.z, o.z);
            o.w = fmaf(a.w, p.w - 2.f * q.w + r.w, o.w);
        }
        reinterpret_cast<float4 *>(g)[i] = o;
    }
}

__global__ void scale_kernel(float *__restrict__ f, float s, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        f[i] *= s;
}

int stream_grid(int64_t n, int threads) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t b = (n + threads - 1) / threads;
    if (b > (int64_t)nsm * 16) b = (int64_t)nsm * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

fd_status sparse_launch(const SparseArgs &a, int step, bool do_inject, bool do_interp,
                        cudaStream_t stream) {
    const int64_t nrec_total = do_interp ? (int64_t)a.nshots * a.nrec : 0;
    const int64_t ninj = do_inject ? (int64_t)a.nshots * a.nsrc * 8 : 0;
    const int64_t total = nrec_total + ninj;
    if (total == 0) return FD_OK;
    const int threads = 256;
    const int64_t blocks = (total + threads - 1) / threads;
    sparse_kernel<<<(unsigned)blocks, threads, 0, stream>>>(a, step, do_inject ? 1 : 0,
                                                            nrec_total);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

fd_status bump_counter(int *counter, int by, cudaStream_t stream) {
    bump_kernel<<<1, 1, 0, stream>>>(counter, by);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

fd_status grad_accumulate_batch(float *grad, const float *w, int64_t w_stride, const float *u,
                                int64_t u_stride, int nb, int64_t n, cudaStream_t stream) {
    if (n % 4 || w_stride % 4 || u_stride % 4)
        return set_error(FD_ERR_ARG, "grad_accumulate_batch: sizes not multiples of 4");
    grad_batch_kernel<<<stream_grid(n / 4, 256), 256, 0, stream>>>(grad, w, w_stride / 4, u,
                                                                   u_stride / 4, n / 4, nb, n / 4);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

fd_status scale_field(float *f, float s, int64_t n, cudaStream_t stream) {
    scale_kernel<<<stream_grid(n, 256), 256, 0, stream>>>(f, s, n);
    FD_CUDA_TRY(cudaGetLastError());
    note_launch(stream);
    return FD_OK;
}

}  // namespace fdsweep
