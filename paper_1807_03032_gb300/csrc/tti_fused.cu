// tti_fused.cu -- the TTI step in one kernel with the first-derivative
// temporaries kept on chip (the paper's shift-invariant temporaries, here in
// shared memory instead of HBM), for stencil radii R <= 4.
//
// Same operators as the two passes of tti.cu (Hxy p = sum_i D_i f_i,
// Hz r = sum_i D_i e_i, f_i = D_i p - n_i (n . grad p), e_i = n_i (n . grad r)).
// One CTA owns a 64 x 8 column and marches it through z with two thread
// groups, one per field (p, r):
//   * every arriving plane of p and r comes with a halo of 2R rows and 2RA
//     columns (TMA, zero fill outside the grid) into a ring of R + 1 + D
//     planes; its values feed the z-derivative accumulators of the "cross"
//     cells -- the tile plus R rows above and below it and one float4
//     column left and right, the points whose temporaries the tile's outer
//     stencil reads;
//   * R planes behind, the gradient of the cross cells is complete: the
//     temporaries f (group p) or e (group r) of that plane are written to
//     shared memory (f_x, e_x on the x-extended tile, f_y, e_y on the
//     y-extended tile, f_z, e_z on the tile; zero outside the grid, as the
//     ghosts of the two-pass scheme);
//   * the outer derivatives of the temporaries feed a second accumulator
//     pipeline, whose output R planes further behind is complete; the groups
//     exchange Hxy p and Hz r through shared memory and update p and r.
// HBM traffic per point: p, r and n_x, n_y, n_z once with halos, p, p-, r,
// r-, b, a, s for the update, p+, r+ out: 48 bytes against 104 for the two
// passes; the price is the gradient of the cross cells (1.6x the tile's).
#include "kernels.cuh"
#include "runtime.cuh"
#include "tti_stencil.cuh"

namespace fdsweep {
namespace {
using namespace tti;

template <int R, int D, int TY_>
struct TfCfg {
    static constexpr int TX = 16, TY = TY_;
    static constexpr int BX = 4 * TX, BY = TY;
    static constexpr int RA = 4;  // x halo in whole float4 cells (R <= 4)
    static_assert(R >= 1 && R <= 4, "the fused TTI kernel covers radii 1..4");
    // p/r plane box (its rows carry 4 extra columns so that the x-strip
    // cells, one per row and 8 rows per phase of a 128-bit shared access,
    // fall on distinct banks) and the cross bounding box
    static constexpr int PX = BX + 4 * RA + 4, PY = BY + 4 * R;
    static constexpr int NXW = BX + 2 * RA, NYH = BY + 2 * R;
    static constexpr int GROUP = TX * TY, THREADS = 2 * GROUP, WARPS = THREADS / 32;
    static constexpr int INT = BX * BY;
    static constexpr int BOX = (PX * PY + 31) / 32 * 32;
    static constexpr int NBOX = (NXW * NYH + 31) / 32 * 32;
    static constexpr int NP = R + 1 + D;  // plane ring: plane s .. arriving plane, + prefetch
    static constexpr int NQ = D + 1;      // per-iteration ring: n at s, update tiles at o
    static constexpr int PSLOT = 2 * BOX;
    static constexpr int QSLOT = 3 * NBOX + 7 * INT;
    static constexpr int FX = (NXW * BY + 31) / 32 * 32;  // f_x / e_x, x-extended
    static constexpr int FY = (BX * NYH + 31) / 32 * 32;  // f_y / e_y, y-extended
    static constexpr int TMP = FX + FY + INT;             // + f_z / e_z on the tile
    static constexpr int NCELL = (BX / 4) * BY + 2 * BY + 2 * R * (BX / 4);
    static constexpr int KC = (NCELL + GROUP - 1) / GROUP;  // cross cells per thread
    static constexpr uint32_t PBYTES = 2 * PX * PY * 4;
    static constexpr uint32_t NBYTES = 3 * NXW * NYH * 4, UBYTES = 7 * INT * 4;
    static constexpr size_t SMEM =
        ((size_t)NP * PSLOT + (size_t)NQ * QSLOT + 2 * TMP + 4 * INT) * 4 +
        (size_t)(NP + NQ) * 2 * 8 + 16 + 128;
    static_assert(PX <= 256 && PY <= 256, "TMA box dimension limit");
};

__device__ __forceinline__ void group_sync(int group, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + group), "r"(nthreads) : "memory");
}

template <int R, int D, int K1, int K2, int TY>
__global__ void __launch_bounds__(32 * TY)
    tti_fused_kernel(const __grid_constant__ CUtensorMap map_box,
                     const __grid_constant__ CUtensorMap map_nbox,
                     const __grid_constant__ CUtensorMap map_wint,
                     const __grid_constant__ CUtensorMap map_cint, const TtiArgs a, int zchunk,
                     int nzc) {
    using C = TfCfg<R, D, TY>;
    if (__ldcg(a.err) & DEV_ERR_NONFINITE) return;  // stopped by the divergence watchdog
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *smem = reinterpret_cast<float *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    float *ringP = smem;
    float *ringQ = ringP + C::NP * C::PSLOT;
    float *tmp = ringQ + C::NQ * C::QSLOT;  // [field][fx | fy | fz]
    float *xchg = tmp + 2 * C::TMP;         // [2 buffers][A | B]
    uint64_t *fullP = reinterpret_cast<uint64_t *>(xchg + 4 * C::INT);
    uint64_t *emptyP = fullP + C::NP;
    uint64_t *fullQ = emptyP + C::NP;
    uint64_t *emptyQ = fullQ + C::NQ;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(emptyQ + C::NQ);

    const int tid = threadIdx.x, lane = tid & 31;
    const int field = tid / C::GROUP;  // 0: p (temporaries f), 1: r (temporaries e)
    const int t = tid - field * C::GROUP;
    const int shot = blockIdx.z / nzc, chunk = blockIdx.z - shot * nzc;
    const int x0 = blockIdx.x * C::BX, y0 = blockIdx.y * C::BY;
    const int za = chunk * zchunk, zb = min(a.L.nz, za + zchunk);
    const int nplanes = zb - za + 4 * R;
    const int P0 = za - 2 * R;  // first arriving plane
    const int wp = 4 * shot + a.cur, wr = 4 * shot + 2 + a.cur;

    if (tid == 0) {
        prefetch_tensormap(&map_box);
        prefetch_tensormap(&map_nbox);
        prefetch_tensormap(&map_wint);
        prefetch_tensormap(&map_cint);
        for (int i = 0; i < C::NP; ++i) {
            mbar_init(&fullP[i], 1);
            mbar_init(&emptyP[i], C::WARPS);
        }
        for (int i = 0; i < C::NQ; ++i) {
            mbar_init(&fullQ[i], 1);
            mbar_init(&emptyQ[i], C::WARPS);
        }
        fence_mbar_init();
        *abort_flag = 0;
    }
    __syncthreads();

    // Producer (thread 0).  Ring P slot jj % NP: planes of p and r (box);
    // ring Q slot jj % NQ: n boxes at s = P0 + jj - R (from jj >= 2R) and the
    // update tiles at o = P0 + jj - 2R (from jj >= 4R); zero bytes otherwise.
    int issuedP = 0;
    auto issue = [&](int jj) -> bool {
        const int sp = jj % C::NP, sq = jj % C::NQ;
        if (jj >= C::NP &&
            !mbar_wait_bounded(&emptyP[sp], (uint32_t)(((jj - C::NP) / C::NP) & 1)))
            return false;
        if (jj >= C::NQ &&
            !mbar_wait_bounded(&emptyQ[sq], (uint32_t)(((jj - C::NQ) / C::NQ) & 1)))
            return false;
        float *P = ringP + sp * C::PSLOT;
        mbar_arrive_expect_tx(&fullP[sp], C::PBYTES);
        tma_load_4d(P, &map_box, &fullP[sp], x0 - 2 * C::RA, y0 - 2 * R, P0 + jj, wp);
        tma_load_4d(P + C::BOX, &map_box, &fullP[sp], x0 - 2 * C::RA, y0 - 2 * R, P0 + jj, wr);
        const bool qs = jj >= 2 * R, qo = jj >= 4 * R;
        mbar_arrive_expect_tx(&fullQ[sq], (qs ? C::NBYTES : 0) + (qo ? C::UBYTES : 0));
        float *Q = ringQ + sq * C::QSLOT;
        if (qs)
            for (int c = 0; c < 3; ++c)
                tma_load_4d(Q + c * C::NBOX, &map_nbox, &fullQ[sq], x0 - C::RA, y0 - R,
                            P0 + jj - R, 3 + c);
        if (qo) {
            const int o = P0 + jj - 2 * R, wb = 4 * shot;
            float *U = Q + 3 * C::NBOX;
            tma_load_4d(U, &map_wint, &fullQ[sq], x0, y0, o, wb + a.cur);                  // p
            tma_load_4d(U + C::INT, &map_wint, &fullQ[sq], x0, y0, o, wb + 1 - a.cur);     // p-
            tma_load_4d(U + 2 * C::INT, &map_wint, &fullQ[sq], x0, y0, o, wb + 2 + a.cur); // r
            tma_load_4d(U + 3 * C::INT, &map_wint, &fullQ[sq], x0, y0, o, wb + 3 - a.cur); // r-
            for (int c = 0; c < 3; ++c)  // b, a, s
                tma_load_4d(U + (4 + c) * C::INT, &map_cint, &fullQ[sq], x0, y0, o, c);
        }
        issuedP = jj + 1;
        return true;
    };
    if (tid == 0)
        for (int jj = 0; jj < D && jj < nplanes; ++jj) issue(jj);

    // cross cells of this thread: float4 column qx in [-1, 16], row y in
    // [-R, BY + R); kind 0 tile, 1 x strip, 2 y strip
    int cbox[C::KC], cnb[C::KC], ckind[C::KC], cqx[C::KC], cy[C::KC];
    bool cvalid[C::KC];
    unsigned cmask[C::KC];  // in-grid x elements (bits 0..3) when the row is in the grid
#pragma unroll
    for (int k = 0; k < C::KC; ++k) {
        const int c = t + k * C::GROUP;
        cvalid[k] = c < C::NCELL;
        int qx = 0, y = 0, kind = 0;
        if (c < (C::BX / 4) * C::BY) {
            qx = c % (C::BX / 4);
            y = c / (C::BX / 4);
        } else if (c < (C::BX / 4) * C::BY + 2 * C::BY) {
            const int e = c - (C::BX / 4) * C::BY;
            qx = e < C::BY ? -1 : C::BX / 4;
            y = e % C::BY;
            kind = 1;
        } else if (cvalid[k]) {
            const int e = c - (C::BX / 4) * C::BY - 2 * C::BY;
            const int rr = e / (C::BX / 4);
            qx = e % (C::BX / 4);
            y = rr < R ? rr - R : C::BY + (rr - R);
            kind = 2;
        }
        cqx[k] = qx;
        cy[k] = y;
        ckind[k] = kind;
        cbox[k] = (y + 2 * R) * C::PX + 4 * qx + 2 * C::RA;  // the cell in the p/r box
        cnb[k] = (y + R) * C::NXW + 4 * qx + C::RA;          // the cell in the n box
        unsigned m = 0u;
        const int gy = y0 + y;
        if (gy >= 0 && gy < a.L.ny)
            for (int e = 0; e < 4; ++e) {
                const int gx = x0 + 4 * qx + e;
                if (gx >= 0 && gx < a.L.nx) m |= 1u << e;
            }
        cmask[k] = m;
    }
    // the thread's tile cell for the outer derivative and the update
    const int tx = t % C::TX, ty = t / C::TX;
    const int gx = x0 + 4 * tx, gy = y0 + ty;
    const bool ok = gx < a.L.nxp && gy < a.L.ny;
    float dpx4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) dpx4[i] = (gx + i < a.L.nx) ? a.dpx[gx + i] : 0.f;
    const float dpy = gy < a.L.ny ? a.dpy[gy] : 0.f;
    float *qn = a.wave + (int64_t)(4 * shot + 2 * field + 1 - a.cur) * a.L.vol;
    float *T = tmp + field * C::TMP;
    float *Tfx = T, *Tfy = T + C::FX, *Tfz = T + C::FX + C::FY;

    float4 acc1[C::KC][2 * R], acc2[2 * R];
#pragma unroll
    for (int k = 0; k < C::KC; ++k)
#pragma unroll
        for (int i = 0; i < 2 * R; ++i) acc1[k][i] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) acc2[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    bool failed = false;
    for (int j = 0; j < nplanes; ++j) {
        bool bad = false;
        if (tid == 0 && j + D < nplanes && !failed && !issue(j + D)) {
            failed = true;
            bad = true;
        }
        const int sp = j % C::NP, sq = j % C::NQ;
        if (!mbar_wait_bounded(&fullP[sp], (uint32_t)((j / C::NP) & 1))) bad = true;
        if (!mbar_wait_bounded(&fullQ[sq], (uint32_t)((j / C::NQ) & 1))) bad = true;
        const int s = P0 + j - R, o = P0 + j - 2 * R;
        const bool has_s = j >= 2 * R, has_o = j >= 4 * R;
        const float *Pa = ringP + sp * C::PSLOT + field * C::BOX;  // arriving plane
        const float *Ps = ringP + ((j - R + C::NP * (R + 1)) % C::NP) * C::PSLOT + field * C::BOX;
        const float *Q = ringQ + sq * C::QSLOT;
        const bool s_in = s >= 0 && s < a.L.nz;

        // ---- stage 1: z-derivative feed; gradient and temporaries of plane s
#pragma unroll
        for (int k = 0; k < C::KC; ++k) {
            if (!cvalid[k]) continue;
            const float4 cv = lds4(Pa + cbox[k]);
            dz_feed<R, K1>(acc1[k], cv, a.t1[2]);
            if (has_s) {
                const float4 g_x = dx4<R, C::RA, K1>(Ps + cbox[k] - C::RA, a.t1[0]);
                const float4 g_y = dy4<R, K1>(Ps + cbox[k], C::PX, a.t1[1]);
                const float4 g_z = acc1[k][0];
                const float4 nx = lds4(Q + cnb[k]), ny = lds4(Q + C::NBOX + cnb[k]),
                             nz = lds4(Q + 2 * C::NBOX + cnb[k]);
                float4 h;
                h.x = nx.x * g_x.x + ny.x * g_y.x + nz.x * g_z.x;
                h.y = nx.y * g_x.y + ny.y * g_y.y + nz.y * g_z.y;
                h.z = nx.z * g_x.z + ny.z * g_y.z + nz.z * g_z.z;
                h.w = nx.w * g_x.w + ny.w * g_y.w + nz.w * g_z.w;
                float4 o0, o1, o2;
                if (field == 0) {  // f_i = g_i - n_i h
                    o0 = make_float4(g_x.x - nx.x * h.x, g_x.y - nx.y * h.y, g_x.z - nx.z * h.z, g_x.w - nx.w * h.w);
                    o1 = make_float4(g_y.x - ny.x * h.x, g_y.y - ny.y * h.y, g_y.z - ny.z * h.z, g_y.w - ny.w * h.w);
                    o2 = make_float4(g_z.x - nz.x * h.x, g_z.y - nz.y * h.y, g_z.z - nz.z * h.z, g_z.w - nz.w * h.w);
                } else {  // e_i = n_i h
                    o0 = make_float4(nx.x * h.x, nx.y * h.y, nx.z * h.z, nx.w * h.w);
                    o1 = make_float4(ny.x * h.x, ny.y * h.y, ny.z * h.z, ny.w * h.w);
                    o2 = make_float4(nz.x * h.x, nz.y * h.y, nz.z * h.z, nz.w * h.w);
                }
                // zero ghosts: temporaries outside the grid vanish
                const unsigned m = s_in ? cmask[k] : 0u;
                auto masked = [m](float4 v) {
                    return make_float4((m & 1u) ? v.x : 0.f, (m & 2u) ? v.y : 0.f,
                                       (m & 4u) ? v.z : 0.f, (m & 8u) ? v.w : 0.f);
                };
                const int y = cy[k], qx = cqx[k];
                if (ckind[k] != 2)  // tile or x strip: f_x / e_x
                    *reinterpret_cast<float4 *>(Tfx + y * C::NXW + 4 * qx + C::RA) = masked(o0);
                if (ckind[k] != 1)  // tile or y strip: f_y / e_y
                    *reinterpret_cast<float4 *>(Tfy + (y + R) * C::BX + 4 * qx) = masked(o1);
                if (ckind[k] == 0)
                    *reinterpret_cast<float4 *>(Tfz + y * C::BX + 4 * qx) = masked(o2);
            }
            dz_shift<R, K1>(acc1[k], cv, a.t1[2]);
        }
        group_sync(field, C::GROUP);

        // ---- stage 2: outer derivatives of the temporaries of plane s feed
        //      the pending outputs; output o = s - R is complete
        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
        if (has_s) {
            const float4 cz = lds4(Tfz + ty * C::BX + 4 * tx);
            dz_feed<R, K2>(acc2, cz, a.t2[2]);
            const float4 dxv = dx4<R, C::RA, K2>(Tfx + ty * C::NXW + 4 * tx, a.t2[0]);
            const float4 dyv = dy4<R, K2>(Tfy + (ty + R) * C::BX + 4 * tx, C::BX, a.t2[1]);
            acc2[R] = f4add(acc2[R], f4add(dxv, dyv));
            val = acc2[0];
            dz_shift<R, K2>(acc2, cz, a.t2[2]);
        }
        float *XB = xchg + (j & 1) * 2 * C::INT;
        const int q = ty * C::BX + 4 * tx;
        if (has_o) *reinterpret_cast<float4 *>(XB + field * C::INT + q) = val;
        // every thread: temporaries consumed, A and B exchanged (or abandon)
        if (__syncthreads_or(bad || *abort_flag)) {
            if (tid == 0) {
                *abort_flag = 1;
                atomicOr(a.err, DEV_ERR_TIMEOUT);
            }
            break;
        }
        if (has_o) {
            const float *U = Q + 3 * C::NBOX;
            const float4 A = lds4(XB + q), B = lds4(XB + C::INT + q);
            const float4 qc = lds4(U + 2 * field * C::INT + q);
            const float4 qm = lds4(U + (2 * field + 1) * C::INT + q);
            const float4 b = lds4(U + 4 * C::INT + q), av = lds4(U + 5 * C::INT + q),
                         sv = lds4(U + 6 * C::INT + q);
            const float dyz = dpy + a.dpz[o];
            float4 rhs;
            if (field == 0)
                rhs = make_float4(av.x * A.x + sv.x * B.x, av.y * A.y + sv.y * B.y,
                                  av.z * A.z + sv.z * B.z, av.w * A.w + sv.w * B.w);
            else
                rhs = make_float4(sv.x * A.x + B.x, sv.y * A.y + B.y, sv.z * A.z + B.z,
                                  sv.w * A.w + B.w);
            float4 v;
            v.x = qc.x + (1.f - (dpx4[0] + dyz) * b.x) * (qc.x - qm.x) + b.x * rhs.x;
            v.y = qc.y + (1.f - (dpx4[1] + dyz) * b.y) * (qc.y - qm.y) + b.y * rhs.y;
            v.z = qc.z + (1.f - (dpx4[2] + dyz) * b.z) * (qc.z - qm.z) + b.z * rhs.z;
            v.w = qc.w + (1.f - (dpx4[3] + dyz) * b.w) * (qc.w - qm.w) + b.w * rhs.w;
            if (ok) {
                const int64_t off = (int64_t)o * a.L.plane + (int64_t)gy * a.L.nxp + gx;
                *reinterpret_cast<float4 *>(qn + off) = v;
            }
        }
        // release: plane s (no longer needed) and this iteration's Q slot
        __syncwarp();
        if (lane == 0) {
            if (j >= R) mbar_arrive(&emptyP[(j - R) % C::NP]);
            mbar_arrive(&emptyQ[sq]);
        }
    }
    __syncthreads();
    if (*abort_flag && tid == 0) {
        for (int jj = issuedP - C::NQ; jj < issuedP; ++jj)
            if (jj >= 0) {
                mbar_wait_bounded(&fullP[jj % C::NP], (uint32_t)((jj / C::NP) & 1), 200000000ull);
                mbar_wait_bounded(&fullQ[jj % C::NQ], (uint32_t)((jj / C::NQ) & 1), 200000000ull);
            }
    }
}

template <int R, int STAG, int TY>
const void *fused_fn() {
    return (const void *)&tti_fused_kernel<R, 1, STAG ? 1 : 0, STAG ? -1 : 0, TY>;
}

struct FusedInfo {
    const void *fn;
    size_t smem;
    int px, py, nxw, nyh, by, threads;
};

template <int R, int TY>
FusedInfo fused_info_t(int stag) {
    using C = TfCfg<R, 1, TY>;
    return FusedInfo{stag ? fused_fn<R, 1, TY>() : fused_fn<R, 0, TY>(), C::SMEM, C::PX, C::PY,
                     C::NXW, C::NYH, C::BY, C::THREADS};
}

// Configuration 0: 64 x 8 tiles, two CTAs per SM; configuration 1: 64 x 16
// tiles (fewer recomputed cross cells per tile point), one CTA per SM.
bool fused_info(int radius, int stag, int config, FusedInfo *out) {
    const bool tall = config == 1;
    switch (radius) {
        case 1: *out = tall ? fused_info_t<1, 16>(stag) : fused_info_t<1, 8>(stag); return true;
        case 2: *out = tall ? fused_info_t<2, 16>(stag) : fused_info_t<2, 8>(stag); return true;
        case 4: *out = fused_info_t<4, 8>(stag); return true;
        default: return false;
    }
}

}  // namespace

bool tti_fused_supported(int radius) {
    FusedInfo in;
    return fused_info(radius, 0, 0, &in);
}

fd_status tti_fused_plan(int radius, int stag, const WaveLayout &L, int nshots, float *wave,
                         const float *coef, TtiPlan *plan, int config) {
    FusedInfo in;
    if (!fused_info(radius, stag, config, &in))
        return set_error(FD_ERR_ARG, "the fused TTI scheme covers space orders up to 8");
    FD_TRY(raise_smem_limit(in.fn, in.smem));
    int dev = 0, nsm = 0, per_sm = 0;
    FD_CUDA_TRY(cudaGetDevice(&dev));
    FD_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, in.fn, in.threads, in.smem));
    if (per_sm < 1) return set_error(FD_ERR_CUDA, "fused TTI kernel does not fit on an SM");
    const int bx = 64, by = in.by;
    const int ntx = (L.nx + bx - 1) / bx, nty = (L.ny + by - 1) / by;
    const int64_t cols = (int64_t)ntx * nty * nshots, slots = (int64_t)nsm * per_sm;
    int nzc = tti_z_chunks(cols, slots, L.nz, 16 * radius > 32 ? 16 * radius : 32);
    const int zchunk = (L.nz + nzc - 1) / nzc;
    nzc = (L.nz + zchunk - 1) / zchunk;
    if ((int64_t)nshots * nzc > 65535 || nty > 65535)
        return set_error(FD_ERR_ARG, "grid too large for the fused TTI launch");
    plan->radius = radius;
    plan->stag = stag ? 1 : 0;
    plan->scheme = kTtiFused;
    plan->config = config == 1 ? 1 : 0;
    plan->grid = dim3(ntx, nty, nshots * nzc);
    plan->block = dim3(in.threads, 1, 1);
    plan->smem1 = in.smem;
    plan->zchunk = zchunk;
    plan->nzc = nzc;
    const uint64_t sy = (uint64_t)L.nxp * 4, sz = (uint64_t)L.plane * 4, sw = (uint64_t)L.vol * 4;
    FD_TRY(make_tensor_map_4d(&plan->map_fbox, wave, L.nx, L.ny, L.nz, 4ull * nshots, sy, sz, sw,
                              in.px, in.py, 1, 1));
    FD_TRY(make_tensor_map_4d(&plan->map_fnbox, coef, L.nx, L.ny, L.nz, 6, sy, sz, sw, in.nxw,
                              in.nyh, 1, 1));
    FD_TRY(make_tensor_map_4d(&plan->map_wint, wave, L.nx, L.ny, L.nz, 4ull * nshots, sy, sz, sw,
                              bx, by, 1, 1));
    return make_tensor_map_4d(&plan->map_cint, coef, L.nx, L.ny, L.nz, 6, sy, sz, sw, bx, by, 1,
                              1);
}

fd_status tti_fused_launch(const TtiPlan &plan, const TtiArgs &a, cudaStream_t stream) {
    FusedInfo in;
    if (!fused_info(plan.radius, plan.stag, plan.config, &in))
        return set_error(FD_ERR_SO, "bad fused TTI plan");
    int zchunk = plan.zchunk, nzc = plan.nzc;
    void *params[] = {(void *)&plan.map_fbox, (void *)&plan.map_fnbox, (void *)&plan.map_wint,
                      (void *)&plan.map_cint, (void *)&a, (void *)&zchunk, (void *)&nzc};
    FD_CUDA_TRY(cudaLaunchKernel(in.fn, plan.grid, plan.block, params, plan.smem1, stream));
    note_launch(stream);
    return FD_OK;
}

}  // namespace fdsweep
