// pd_resident.cuh -- the fused primal-dual iteration with the whole per-slice
// state held on chip for all iterations.
//
// Same data flow and FFT machinery as pd_cluster.cuh (one cluster per slice,
// spectrum spread over the cluster's shared memory, two FFT round trips per
// iteration with the proxes fused into the row passes), but a CTA owns few
// enough rows (R = rows in flight, one row pass per phase) that every thread
// handles the same 2*ER pixels of the same row in every phase of every
// iteration.  So:
//   * chi and p of a thread's pixels live in its registers;
//   * qx, qy, chibar, the field and the mask of the CTA's rows live in shared
//     memory planes (row pitch W + 16 floats, which puts the four row groups
//     of a warp on different banks);
//   * the neighbour rows of the stencils across a CTA boundary are read from
//     the adjacent CTA's planes through distributed shared memory.
// The iteration loop therefore touches no global memory: the field and mask
// are read once per slice, chi (and p, q for the diagnostics) written once.
#pragma once

#include "pd_cluster.cuh"

namespace pcs {

// PAD_: extra floats per plane row; 16 separates the four row groups of a
// warp onto different banks when a row group is 8 lanes wide (not needed for
// 16-lane groups).  MINB_: CTAs per SM the register budget is set for.
template <int H_, int W_, int C_, int NT_ = 256, int ER_ = 0, int EC_ = 0, int PAD_ = 16, int MINB_ = 1>
struct GeoRes : Geo<H_, W_, C_, MINB_, NT_, ER_, EC_> {
    using B = Geo<H_, W_, C_, MINB_, NT_, ER_, EC_>;
    static constexpr int WP = W_ + PAD_;  // plane row pitch (floats / bytes for the mask)
    static constexpr int PLANE = B::R * WP;
    static constexpr size_t SMEM_BYTES = B::SMEM_BYTES + sizeof(float) * 4 * PLANE + (size_t)PLANE;
    static_assert(B::R == B::RPP, "resident kernel: one row pass per phase");
    static_assert(SMEM_BYTES <= 227 * 1024, "resident kernel: shared memory");
};

template <class G>
struct ResPlanes {
    float* qx;
    float* qy;
    float* cb;  // chibar
    float* f;   // field
    unsigned char* m;
    const float* cb_next;  // next CTA's chibar plane (its row 0 follows our last row)
    const float* qy_prev;  // previous CTA's qy plane (its row R-1 precedes our row 0)
};

template <class G>
__global__ void __launch_bounds__(G::NT, G::MINB) pd_resident_kernel(PDParams prm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ctx<G> cx;
    ctx_init<G>(cx, smem_raw, prm.twid);
    constexpr int H = G::H, W = G::W, C = G::C, R = G::R, TR = G::TR, ER = G::ER, WP = G::WP;
    ResPlanes<G> pl;
    pl.qx = reinterpret_cast<float*>(cx.stw_c + G::SM_STW_C);
    pl.qy = pl.qx + G::PLANE;
    pl.cb = pl.qy + G::PLANE;
    pl.f = pl.cb + G::PLANE;
    pl.m = reinterpret_cast<unsigned char*>(pl.f + G::PLANE);
    pl.cb_next = nullptr;
    pl.qy_prev = nullptr;
    if constexpr (C > 1) {
        cg::cluster_group cluster = cg::this_cluster();
        if (cx.crank + 1 < C) pl.cb_next = cluster.map_shared_rank(pl.cb, cx.crank + 1);
        if (cx.crank > 0) pl.qy_prev = cluster.map_shared_rank(pl.qy, cx.crank - 1);
    }

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TR;
    const int grp = warp * (32 / TR) + lane / TR;  // == local row
    const unsigned gm = group_mask<TR>(lane);
    const int src_right = (g == TR - 1) ? lane - (TR - 1) : lane + 1;
    const int src_left = (g == 0) ? lane + (TR - 1) : lane - 1;
    float2* rs = cx.rows + grp * G::MP;
    const int il = grp;
    const int i = cx.crank * R + il;
    const bool has_up = (i > 0), has_down = (i + 1 < H);
    const float sigma = prm.sigma, tau = prm.tau;
    const int cid = blockIdx.x / C, ncl = gridDim.x / C;
    constexpr size_t SLICE = (size_t)H * W;

#pragma unroll 1
    for (int s = cid; s < prm.S; s += ncl) {
        const size_t base = (size_t)s * SLICE;
        const size_t rowoff = base + (size_t)i * W;
        const float inv_den = slice_inv_den(prm, s);
        // ---- zero start; field and mask of own rows into shared memory
        float2 chi[ER], pv[ER];
#pragma unroll
        for (int e = 0; e < ER; ++e) {
            chi[e] = make_float2(0.f, 0.f);
            pv[e] = make_float2(0.f, 0.f);
            const int o = il * WP + 2 * (g + TR * e);
            const size_t go = rowoff + 2 * (g + TR * e);
            *reinterpret_cast<float2*>(pl.qx + o) = make_float2(0.f, 0.f);
            *reinterpret_cast<float2*>(pl.qy + o) = make_float2(0.f, 0.f);
            *reinterpret_cast<float2*>(pl.cb + o) = make_float2(0.f, 0.f);
            *reinterpret_cast<float2*>(pl.f + o) = __ldg(reinterpret_cast<const float2*>(prm.field + go));
            *reinterpret_cast<uchar2*>(pl.m + o) = __ldg(reinterpret_cast<const uchar2*>(prm.mask + go));
        }
        for (int t = threadIdx.x; t < G::SM_TBUF; t += G::NT) cx.tbuf[t] = make_float2(0.f, 0.f);
        cluster_barrier<C>();

#pragma unroll 1
        for (int n = 0; n < prm.n_iter; ++n) {
            if (n > 0) {
                column_pass<G>(cx, prm.dtab, prm.ddtab);  // u-spectrum = D F chibar_n
                cluster_barrier<C>();
            }
            // ================= phase B: u = D chibar -> dual proxes -> F (W p)
            {
                float2 x[ER];
                row_inverse<G>(cx, rs, i, g, gm, x);
                const float* down = nullptr;  // chibar row i+1
                if (has_down) down = (il + 1 < R) ? pl.cb + (il + 1) * WP : pl.cb_next;
                // the halo row may be remote (DSMEM): fetch it all before the stores below
                float2 cdn[ER];
#pragma unroll
                for (int e = 0; e < ER; ++e)
                    cdn[e] = down ? *reinterpret_cast<const float2*>(down + 2 * (g + TR * e)) : make_float2(0.f, 0.f);
                // descending e: the last lane of the group takes pixel 2n+2 from lane 0 at e+1
                float s_next = 0.f;
#pragma unroll
                for (int e = ER - 1; e >= 0; --e) {
                    const int j0 = 2 * (g + TR * e);
                    const int o = il * WP + j0;
                    const float2 cb = *reinterpret_cast<const float2*>(pl.cb + o);
                    const float sr = __shfl_sync(gm, cb.x, src_right);
                    float right = sr;
                    if (g == TR - 1) right = (e + 1 < ER) ? s_next : cb.y;  // Neumann past the last column
                    s_next = sr;
                    const float2 cd = down ? cdn[e] : cb;
                    const float2 f = *reinterpret_cast<const float2*>(pl.f + o);
                    const uchar2 mk = *reinterpret_cast<const uchar2*>(pl.m + o);
                    const float m0 = mk.x ? 1.f : 0.f, m1 = mk.y ? 1.f : 0.f;
                    const float2 u = x[e];
                    pv[e].x = (pv[e].x + sigma * (m0 * (u.x - f.x))) * inv_den;
                    pv[e].y = (pv[e].y + sigma * (m1 * (u.y - f.y))) * inv_den;
                    float2 qx = *reinterpret_cast<const float2*>(pl.qx + o);
                    float2 qy = *reinterpret_cast<const float2*>(pl.qy + o);
                    qx.x = qx.x + sigma * m0 * (cb.y - cb.x);
                    qx.y = qx.y + sigma * m1 * (right - cb.y);
                    qy.x = qy.x + sigma * m0 * (cd.x - cb.x);
                    qy.y = qy.y + sigma * m1 * (cd.y - cb.y);
                    tv_prox(qx.x, qy.x, prm.tv_iso);
                    tv_prox(qx.y, qy.y, prm.tv_iso);
                    *reinterpret_cast<float2*>(pl.qx + o) = qx;
                    *reinterpret_cast<float2*>(pl.qy + o) = qy;
                    x[e] = pv[e];  // W p = p (p vanishes outside the mask)
                }
                row_forward<G>(cx, rs, i, g, gm, x);
            }
            cluster_barrier<C>();
            column_pass<G>(cx, prm.dtab, prm.ddtab);  // v-spectrum = D F (W p_{n+1})
            cluster_barrier<C>();
            // ================= phase A: v = D W p -> primal step -> over-relaxation -> F chibar
            {
                const bool last = (n + 1 == prm.n_iter);
                float2 x[ER];
                row_inverse<G>(cx, rs, i, g, gm, x);
                const float* up = nullptr;  // qy row i-1
                if (has_up) up = (il > 0) ? pl.qy + (il - 1) * WP : pl.qy_prev + (R - 1) * WP;
                float2 qun[ER];  // possibly remote: fetch before the stores below
#pragma unroll
                for (int e = 0; e < ER; ++e)
                    qun[e] = up ? *reinterpret_cast<const float2*>(up + 2 * (g + TR * e)) : make_float2(0.f, 0.f);
                // ascending e: lane 0 of the group takes pixel 2n-1 from the last lane at e-1
                float s_prev = 0.f;
#pragma unroll
                for (int e = 0; e < ER; ++e) {
                    const int j0 = 2 * (g + TR * e);
                    const int o = il * WP + j0;
                    const float2 qx = *reinterpret_cast<const float2*>(pl.qx + o);
                    const float sl = __shfl_sync(gm, qx.y, src_left);
                    float al = sl;
                    if (g == 0) al = (e > 0) ? s_prev : 0.f;
                    s_prev = sl;
                    const float a1r = (j0 + 2 < W) ? qx.y : 0.f;
                    const float2 qy = *reinterpret_cast<const float2*>(pl.qy + o);
                    const float2 qu = qun[e];
                    const float b0 = has_down ? qy.x : 0.f;
                    const float b1 = has_down ? qy.y : 0.f;
                    const float d0 = (al - qx.x) + (qu.x - b0);
                    const float d1 = (qx.x - a1r) + (qu.y - b1);
                    const float2 v = x[e];
                    float2 cn;
                    cn.x = chi[e].x - tau * v.x - tau * d0;
                    cn.y = chi[e].y - tau * v.y - tau * d1;
                    const float2 cb = make_float2(2.f * cn.x - chi[e].x, 2.f * cn.y - chi[e].y);
                    chi[e] = cn;
                    *reinterpret_cast<float2*>(pl.cb + o) = cb;
                    x[e] = cb;
                }
                if (!last) row_forward<G>(cx, rs, i, g, gm, x);
            }
            cluster_barrier<C>();
        }
        // ---- write chi_N (and p, q for the diagnostics) once
#pragma unroll
        for (int e = 0; e < ER; ++e) {
            const int j0 = 2 * (g + TR * e);
            const size_t go = rowoff + j0;
            __stcg(reinterpret_cast<float2*>(prm.chi + go), chi[e]);
            __stcg(reinterpret_cast<float2*>(prm.p + go), pv[e]);
            __stcg(reinterpret_cast<float2*>(prm.qx + go), *reinterpret_cast<const float2*>(pl.qx + il * WP + j0));
            __stcg(reinterpret_cast<float2*>(prm.qy + go), *reinterpret_cast<const float2*>(pl.qy + il * WP + j0));
        }
        cluster_barrier<C>();  // planes and spectrum are reused by the next slice
    }
}

}  // namespace pcs
