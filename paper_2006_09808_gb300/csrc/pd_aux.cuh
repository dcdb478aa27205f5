// pd_aux.cuh -- diagnostics and step-size kernels built on the same cluster
// FFT machinery as the iteration kernel.
//
//  * report: per slice, at (chi, p, q), the FP64 sums behind
//      objective   lambda/2 ||W(D chi - dB)||^2 + ||M G chi||_1          (Eq. (1))
//      gap         ||p - lambda W(D chi - dB)||^2 / (2 lambda) + sum(|g| - q.g), g = M G chi
//      stationarity ||D W p + G^T M q||
//    (two dipole convolutions per slice, FP32 operands, FP64 accumulation in
//    a fixed order per CTA; the host adds the C per-CTA partials in order).
//  * opnorm: L = ||K||_2 (pseudocode step 1) by power iteration on
//      K^T K x = D W^2 D x + G^T M^2 G x,
//    Rayleigh quotient <x, K^T K x> / <x, x>, the per-slice norms reduced
//    across the cluster through distributed shared memory in a fixed order.
#pragma once

#include "pd_cluster.cuh"

namespace pcs {

struct AuxParams {
    const float* field;
    const unsigned char* mask;
    const float* chi;
    const float* p;
    const float* qx;
    const float* qy;
    float* xa;  // opnorm iterate buffers [S][H][W]
    float* xb;
    const float* dtab;
    const float* ddtab;
    const float2* twid;
    double* partials;  // report: [S][C][5]
    double* Lout;      // opnorm: [S]
    int S;
    float lam;
    int iters;
    int tv_iso;
    const float* weight;  // NULL: W = mask
};

constexpr int kReportSums = 5;  // data_sq, tv_l1, fy1_sq, fy2, stat_sq

// Sum v over the CTA in a fixed order; result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) s += red[w];
    return s;
}

// Forward real row transforms of a real field (global, read through L2),
// optionally multiplied pointwise by mask^pw, and scatter to the cluster.
template <class G>
__device__ __forceinline__ void rows_forward_from(const Ctx<G>& cx, const float* src, const unsigned char* mask,
                                                  int pw, float scale, size_t base) {
    constexpr int W = G::W, TR = G::TR, ER = G::ER;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TR;
    const int grp = warp * (32 / TR) + lane / TR;
    const unsigned gm = group_mask<TR>(lane);
    float2* rs = cx.rows + grp * G::MP;
#pragma unroll 1
    for (int pass = 0; pass < G::R / G::RPP; ++pass) {
        const int i = cx.crank * G::R + pass * G::RPP + grp;
        const size_t rowoff = base + (size_t)i * W;
        float2 z[ER];
#pragma unroll
        for (int e = 0; e < ER; ++e) {
            const size_t o = rowoff + 2 * (g + TR * e);
            float2 v = __ldcg(reinterpret_cast<const float2*>(src + o));
            v.x *= scale;
            v.y *= scale;
            if (pw > 0) {
                const uchar2 mk = __ldg(reinterpret_cast<const uchar2*>(mask + o));
                v.x *= (float)mk.x;
                v.y *= (float)mk.y;
            }
            z[e] = v;
        }
        row_forward<G>(cx, rs, i, g, gm, z);
    }
}

template <class G>
__global__ void __launch_bounds__(G::NT, 1) aux_report_kernel(AuxParams prm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ctx<G> cx;
    ctx_init<G>(cx, smem_raw, prm.twid);
    double* red = reinterpret_cast<double*>(cx.stw_c + G::SM_STW_C);
    // every CTA of the cluster must have started before its shared memory is written remotely
    cluster_barrier<G::C>();
    constexpr int H = G::H, W = G::W, TR = G::TR, ER = G::ER;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TR;
    const int grp = warp * (32 / TR) + lane / TR;
    const unsigned gm = group_mask<TR>(lane);
    float2* rs = cx.rows + grp * G::MP;
    const float lam = prm.lam;
    const int cid = blockIdx.x / G::C, ncl = gridDim.x / G::C;

#pragma unroll 1
    for (int s = cid; s < prm.S; s += ncl) {
        const size_t base = (size_t)s * H * W;
        double acc[kReportSums] = {0, 0, 0, 0, 0};
        rows_forward_from<G>(cx, prm.chi, prm.mask, 0, 1.f, base);
        cluster_barrier<G::C>();
        column_pass<G>(cx, prm.dtab, prm.ddtab);
        cluster_barrier<G::C>();
        // u = D chi: data terms and TV terms; then forward rows of W p
#pragma unroll 1
        for (int pass = 0; pass < G::R / G::RPP; ++pass) {
            const int i = cx.crank * G::R + pass * G::RPP + grp;
            float2 x[ER];
            row_inverse<G>(cx, rs, i, g, gm, x);
            const size_t rowoff = base + (size_t)i * W;
#pragma unroll
            for (int e = 0; e < ER; ++e) {
                const int j0 = 2 * (g + TR * e);
                const size_t o = rowoff + j0;
                const float2 f = __ldg(reinterpret_cast<const float2*>(prm.field + o));
                const uchar2 mk = __ldg(reinterpret_cast<const uchar2*>(prm.mask + o));
                const float2 p = __ldcg(reinterpret_cast<const float2*>(prm.p + o));
                const float2 c = __ldcg(reinterpret_cast<const float2*>(prm.chi + o));
                const float cr = (j0 + 2 < W) ? __ldcg(prm.chi + o + 2) : c.y;
                const float2 cd = (i + 1 < H) ? __ldcg(reinterpret_cast<const float2*>(prm.chi + o + W)) : c;
                const float2 qx = __ldcg(reinterpret_cast<const float2*>(prm.qx + o));
                const float2 qy = __ldcg(reinterpret_cast<const float2*>(prm.qy + o));
                const float m[2] = {(float)mk.x, (float)mk.y};
                float w[2] = {m[0], m[1]};
                if (prm.weight) {
                    const float2 wv = __ldg(reinterpret_cast<const float2*>(prm.weight + o));
                    w[0] = wv.x;
                    w[1] = wv.y;
                }
                const float u[2] = {x[e].x, x[e].y}, ff[2] = {f.x, f.y}, pp[2] = {p.x, p.y};
                const float gx[2] = {m[0] * (c.y - c.x), m[1] * (cr - c.y)};
                const float gy[2] = {m[0] * (cd.x - c.x), m[1] * (cd.y - c.y)};
                const float qxs[2] = {qx.x, qx.y}, qys[2] = {qy.x, qy.y};
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const double r = (double)w[t] * ((double)u[t] - (double)ff[t]);
                    acc[0] += r * r;
                    const double gxd = gx[t], gyd = gy[t];
                    const double tvn = prm.tv_iso ? sqrt(gxd * gxd + gyd * gyd) : fabs(gxd) + fabs(gyd);
                    acc[1] += tvn;
                    const double d1 = (double)pp[t] - (double)lam * r;
                    acc[2] += d1 * d1;
                    acc[3] += tvn - ((double)qxs[t] * gxd + (double)qys[t] * gyd);
                }
                x[e] = make_float2(w[0] * p.x, w[1] * p.y);
            }
            row_forward<G>(cx, rs, i, g, gm, x);
        }
        cluster_barrier<G::C>();
        column_pass<G>(cx, prm.dtab, prm.ddtab);
        cluster_barrier<G::C>();
        // v = D W p: stationarity D W p + G^T M q
#pragma unroll 1
        for (int pass = 0; pass < G::R / G::RPP; ++pass) {
            const int i = cx.crank * G::R + pass * G::RPP + grp;
            float2 x[ER];
            row_inverse<G>(cx, rs, i, g, gm, x);
            const size_t rowoff = base + (size_t)i * W;
#pragma unroll
            for (int e = 0; e < ER; ++e) {
                const int j0 = 2 * (g + TR * e);
                const size_t o = rowoff + j0;
                const uchar2 mk = __ldg(reinterpret_cast<const uchar2*>(prm.mask + o));
                const float m0 = (float)mk.x, m1 = (float)mk.y;
                const float2 qx = __ldcg(reinterpret_cast<const float2*>(prm.qx + o));
                const float2 qy = __ldcg(reinterpret_cast<const float2*>(prm.qy + o));
                const float a0 = m0 * qx.x, a1 = m1 * qx.y;
                const float al = (j0 > 0) ? (float)__ldg(prm.mask + o - 1) * __ldcg(prm.qx + o - 1) : 0.f;
                const float a1r = (j0 + 2 < W) ? a1 : 0.f;
                float bu0 = 0.f, bu1 = 0.f;
                if (i > 0) {
                    const uchar2 mu = __ldg(reinterpret_cast<const uchar2*>(prm.mask + o - W));
                    const float2 qu = __ldcg(reinterpret_cast<const float2*>(prm.qy + o - W));
                    bu0 = (float)mu.x * qu.x;
                    bu1 = (float)mu.y * qu.y;
                }
                const float b0 = (i + 1 < H) ? m0 * qy.x : 0.f;
                const float b1 = (i + 1 < H) ? m1 * qy.y : 0.f;
                const double k0 = (double)x[e].x + ((double)(al - a0) + (double)(bu0 - b0));
                const double k1 = (double)x[e].y + ((double)(a0 - a1r) + (double)(bu1 - b1));
                acc[4] += k0 * k0 + k1 * k1;
            }
        }
#pragma unroll
        for (int t = 0; t < kReportSums; ++t) {
            const double v = block_sum<G::NT>(acc[t], red);
            if (threadIdx.x == 0) prm.partials[((size_t)s * G::C + cx.crank) * kReportSums + t] = v;
        }
        cluster_barrier<G::C>();
    }
}

// Cluster-wide sum of per-CTA values, same order in every CTA.
template <class G>
__device__ __forceinline__ double cluster_sum(double v_cta, double* slot) {
    if (threadIdx.x == 0) *slot = v_cta;
    cluster_barrier<G::C>();
    double s = 0.0;
    if constexpr (G::C == 1) {
        s = *slot;
    } else {
        cg::cluster_group cluster = cg::this_cluster();
        for (int q = 0; q < G::C; ++q) s += *cluster.map_shared_rank(slot, q);
    }
    cluster_barrier<G::C>();
    return s;
}

// splitmix-style hash to a float in [-1, 1): deterministic start vector
__device__ __forceinline__ float hash_unit(unsigned long long k) {
    k += 0x9E3779B97F4A7C15ull;
    k = (k ^ (k >> 30)) * 0xBF58476D1CE4E5B9ull;
    k = (k ^ (k >> 27)) * 0x94D049BB133111EBull;
    k ^= k >> 31;
    return (float)((double)(k >> 40) * (1.0 / 8388608.0) - 1.0);
}

template <class G>
__global__ void __launch_bounds__(G::NT, 1) aux_opnorm_kernel(AuxParams prm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ctx<G> cx;
    ctx_init<G>(cx, smem_raw, prm.twid);
    double* red = reinterpret_cast<double*>(cx.stw_c + G::SM_STW_C);
    double* slot = red + 32;
    cluster_barrier<G::C>();
    constexpr int H = G::H, W = G::W, TR = G::TR, ER = G::ER;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TR;
    const int grp = warp * (32 / TR) + lane / TR;
    const unsigned gm = group_mask<TR>(lane);
    float2* rs = cx.rows + grp * G::MP;
    const int cid = blockIdx.x / G::C, ncl = gridDim.x / G::C;
    constexpr int OWN = G::R * G::W;

#pragma unroll 1
    for (int s = cid; s < prm.S; s += ncl) {
        const size_t base = (size_t)s * H * W;
        float* x = prm.xa;
        float* y = prm.xb;
        // start vector
        double nrm = 0.0;
        for (int t = threadIdx.x; t < OWN; t += G::NT) {
            const size_t o = base + (size_t)cx.crank * OWN + t;
            const float v = hash_unit(o);
            __stcg(x + o, v);
            nrm += (double)v * v;
        }
        nrm = cluster_sum<G>(block_sum<G::NT>(nrm, red), slot);
        float scale = (float)(1.0 / sqrt(nrm));  // x_true = scale * x_raw
        double est = 0.0;
#pragma unroll 1
        for (int it = 0; it < prm.iters; ++it) {
            rows_forward_from<G>(cx, x, prm.mask, 0, scale, base);  // F x
            cluster_barrier<G::C>();
            column_pass<G>(cx, prm.dtab, prm.ddtab);
            cluster_barrier<G::C>();
            // u = D x -> W^2 u -> forward rows
#pragma unroll 1
            for (int pass = 0; pass < G::R / G::RPP; ++pass) {
                const int i = cx.crank * G::R + pass * G::RPP + grp;
                float2 z[ER];
                row_inverse<G>(cx, rs, i, g, gm, z);
                const size_t rowoff = base + (size_t)i * W;
#pragma unroll
                for (int e = 0; e < ER; ++e) {
                    const uchar2 mk = __ldg(reinterpret_cast<const uchar2*>(prm.mask + rowoff + 2 * (g + TR * e)));
                    z[e].x *= (float)mk.x * (float)mk.x;
                    z[e].y *= (float)mk.y * (float)mk.y;
                }
                row_forward<G>(cx, rs, i, g, gm, z);
            }
            cluster_barrier<G::C>();
            column_pass<G>(cx, prm.dtab, prm.ddtab);
            cluster_barrier<G::C>();
            // y = D W^2 D x + G^T M^2 G x
            double xy = 0.0, yy = 0.0;
#pragma unroll 1
            for (int pass = 0; pass < G::R / G::RPP; ++pass) {
                const int i = cx.crank * G::R + pass * G::RPP + grp;
                float2 z[ER];
                row_inverse<G>(cx, rs, i, g, gm, z);
                const size_t rowoff = base + (size_t)i * W;
#pragma unroll
                for (int e = 0; e < ER; ++e) {
                    const int j0 = 2 * (g + TR * e);
                    const size_t o = rowoff + j0;
                    auto X = [&](size_t idx) { return scale * __ldcg(x + idx); };
                    auto Mk = [&](size_t idx) { const float m = (float)__ldg(prm.mask + idx); return m * m; };
                    // a = M^2 gx, b = M^2 gy at the needed points
                    auto ax = [&](int jj) -> float {  // at column jj of row i
                        if (jj < 0 || jj >= W - 1) return 0.f;
                        return Mk(rowoff + jj) * (X(rowoff + jj + 1) - X(rowoff + jj));
                    };
                    auto by = [&](int ii, int jj) -> float {
                        if (ii < 0 || ii >= H - 1) return 0.f;
                        const size_t r0 = base + (size_t)ii * W + jj;
                        return Mk(r0) * (X(r0 + W) - X(r0));
                    };
                    float out[2];
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const int j = j0 + t;
                        const float gt = (ax(j - 1) - ax(j)) + (by(i - 1, j) - by(i, j));
                        out[t] = (t == 0 ? z[e].x : z[e].y) + gt;
                        xy += (double)X(o + t) * out[t];
                        yy += (double)out[t] * out[t];
                    }
                    __stcg(reinterpret_cast<float2*>(y + o), make_float2(out[0], out[1]));
                }
            }
            xy = cluster_sum<G>(block_sum<G::NT>(xy, red), slot);
            yy = cluster_sum<G>(block_sum<G::NT>(yy, red), slot);
            est = xy;  // x has unit norm
            scale = (yy > 0.0) ? (float)(1.0 / sqrt(yy)) : 0.f;
            float* t = x;
            x = y;
            y = t;
        }
        if (cx.crank == 0 && threadIdx.x == 0) prm.Lout[s] = sqrt(est > 0.0 ? est : 0.0);
        cluster_barrier<G::C>();
    }
}

}  // namespace pcs
