// pd_3d.cuh -- the 3-D variant: Eq. (1) with G in all three dimensions and the
// 3-D dipole convolution of the whole volume (B0 along z, the slice axis).
//
// The volume's half spectrum lives in global memory between the passes of
// one dipole convolution:
//
//   slice kernel (one cluster per slice, as pd_cluster.cuh):
//       load the slice's (ky, kx) spectrum columns, inverse column FFTs
//       -> row phase (dual or primal step of Sec. II.A with the z terms;
//          inverse and forward real row FFTs through the cluster)
//       -> forward column FFTs, store the slice's (ky, kx) spectrum
//   z kernel:  for every (kx, ky): FFT along z, x D(kz, ky, kx)/(S H W),
//              inverse FFT along z
//
// One iteration = slice kernel (dual) -> z kernel -> slice kernel (primal)
// -> z kernel; the host loops over iterations.  Spectrum layout
// [S][W/2 + 1][H] complex: column kx of slice s is contiguous along ky.  The
// slice kernels keep the packed DC/Nyquist column X[0] + i X[W/2] in shared
// memory; at the global boundary it is split into its kx = 0 and kx = W/2
// columns (each the spectrum of a real column) so that the z kernel
// multiplies every entry by a real D.
#pragma once

#include "pd_aux.cuh"
#include "pd_cluster.cuh"

namespace pcs {

// Spectrum of slice s, column kx, row ky: spec[(s (M+1) + kx) H + ky].
template <class G>
__device__ __forceinline__ size_t spec_index(int s, int kx, int ky) {
    return ((size_t)s * (G::M + 1) + kx) * G::H + ky;
}

// Inverse column FFTs of the CTA's own columns of slice s, from the global
// spectrum (CTA 0 re-packs column 0 from the kx = 0 and kx = W/2 columns).
template <class G>
__device__ __forceinline__ void columns_in_3d(const Ctx<G>& cx, const float2* __restrict__ spec, int s) {
    constexpr int H = G::H, TC = G::TC, EC = G::EC, M = G::M;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TC;
    const int grp = warp * (32 / TC) + lane / TC;
    const unsigned gm = group_mask<TC>(lane);
#pragma unroll 1
    for (int cl = grp; cl < G::MC; cl += G::CPP) {
        const int kx = cx.crank * G::MC + cl;
        float2* col = cx.tbuf + cl * G::HP;
        const int key = 4 * cl;
        float2 x[EC];
#pragma unroll
        for (int e = 0; e < EC; ++e) {
            const int ky = g + TC * e;
            const float2 a = __ldcg(spec + spec_index<G>(s, kx, ky));
            if (kx == 0) {
                const float2 b = __ldcg(spec + spec_index<G>(s, M, ky));
                x[e] = make_float2(a.x - b.y, a.y + b.x);  // Y0 + i YM
            } else {
                x[e] = a;
            }
        }
        fft<H, TC, true>(x, col, cx.stw_c, g, gm, key);
#pragma unroll
        for (int e = 0; e < EC; ++e) col[P(g + TC * e, key)] = x[e];
        __syncwarp(gm);
    }
}

// Forward column FFTs of the CTA's own columns and store of the slice's
// spectrum; the packed column 0 is split into its kx = 0 and kx = W/2 parts,
// Y0 = (C + conj C(-ky)) / 2 and YM = (C - conj C(-ky)) / (2i).
template <class G>
__device__ __forceinline__ void columns_out_3d(const Ctx<G>& cx, float2* __restrict__ spec, int s) {
    constexpr int H = G::H, TC = G::TC, EC = G::EC, M = G::M;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TC;
    const int grp = warp * (32 / TC) + lane / TC;
    const unsigned gm = group_mask<TC>(lane);
#pragma unroll 1
    for (int cl = grp; cl < G::MC; cl += G::CPP) {
        const int kx = cx.crank * G::MC + cl;
        float2* col = cx.tbuf + cl * G::HP;
        const int key = 4 * cl;
        float2 x[EC];
#pragma unroll
        for (int e = 0; e < EC; ++e) x[e] = col[P(g + TC * e, key)];
        fft<H, TC, false>(x, col, cx.stw_c, g, gm, key);
        if (kx == 0) {
#pragma unroll
            for (int e = 0; e < EC; ++e) col[P(g + TC * e, key)] = x[e];
            __syncwarp(gm);
#pragma unroll
            for (int e = 0; e < EC; ++e) {
                const int ky = g + TC * e;
                const float2 c = x[e], cm = col[P((H - ky) % H, key)];
                __stcg(spec + spec_index<G>(s, 0, ky), make_float2(0.5f * (c.x + cm.x), 0.5f * (c.y - cm.y)));
                __stcg(spec + spec_index<G>(s, M, ky), make_float2(0.5f * (c.y + cm.y), -0.5f * (c.x - cm.x)));
            }
            __syncwarp(gm);
        } else {
#pragma unroll
            for (int e = 0; e < EC; ++e) __stcg(spec + spec_index<G>(s, kx, g + TC * e), x[e]);
        }
    }
}

struct P3Params {
    PDParams pd;     // state, tables, steps (pd.S = slices of the volume; pd.qz set)
    float2* spec;    // [S][M+1][H]
    int phase;       // 0: dual step, 1: primal step
    int load;        // 1: start from the stored spectrum; 0: zero spectrum (chibar = 0)
    int store;       // 1: store the spectrum of the phase's output
    int reverse;     // 1: clusters take the slices from the last one down
};

template <class G>
__global__ void __launch_bounds__(G::NT, G::MINB) pd3_slice_kernel(P3Params a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ctx<G> cx;
    ctx_init<G>(cx, smem_raw, a.pd.twid);
    const PDParams& prm = a.pd;
    const int cid = blockIdx.x / G::C;
    const int ncl = gridDim.x / G::C;
    constexpr size_t SLICE = (size_t)G::H * G::W;
    __syncthreads();  // twiddle tables
    grid_dependency_wait();  // the previous launch's spectrum and state complete
#pragma unroll 1
    for (int k = cid; k < prm.S; k += ncl) {
        const int s = a.reverse ? prm.S - 1 - k : k;
        const size_t base = (size_t)s * SLICE;
        if (a.load) {
            columns_in_3d<G>(cx, a.spec, s);
        } else {
            for (int t = threadIdx.x; t < G::SM_TBUF; t += G::NT) cx.tbuf[t] = make_float2(0.f, 0.f);
        }
        cluster_arrive<G::C>();
        if (a.phase == 0) {
            phase_dual<G, true>(cx, prm, base, prm.inv_den, true, s);
        } else {
            phase_primal<G, true>(cx, prm, base, !a.store, s);
        }
        cluster_barrier<G::C>();  // all scatters in; all gathers done
        if (a.store) columns_out_3d<G>(cx, a.spec, s);
        // a cluster with several slices: the next slice's zero start writes these columns with
        // another thread mapping than the store just read them with
        __syncthreads();
    }
}

// ------------------------------------------------------------------ FP64 diagnostics
// At (chi, p, q) after the last iteration, per slice (sums over the slice's voxels;
// the volume's values are their sums, the norms their root sums of squares):
//   data_sq = ||W (D3 chi - dB)||^2, tv = ||M G3 chi||_1 (or the isotropic sum),
//   fy1 = ||p - lambda W (D3 chi - dB)||^2, fy2 = sum(|g| - q.g) with g = M G3 chi,
//   stat_sq = ||D3 W p + G3^T M q||^2.
// Three launches of this kernel with z passes between them:
//   mode 0: forward row and column transforms of chi -> spectrum
//   mode 1: inverse transforms -> D3 chi: data and TV terms; forward transforms of W p -> spectrum
//   mode 2: inverse transforms -> D3 W p: stationarity
struct P3Report {
    P3Params a;       // state, inputs, tables, spectrum
    double* partial;  // [S][C][kReportSums]
    double lam;
    int mode;
};

template <class G>
__global__ void __launch_bounds__(G::NT, 1) pd3_report_kernel(P3Report r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ctx<G> cx;
    ctx_init<G>(cx, smem_raw, r.a.pd.twid);
    double* red = reinterpret_cast<double*>(cx.stw_c + G::SM_STW_C);
    __syncthreads();
    const PDParams& prm = r.a.pd;
    constexpr int H = G::H, W = G::W, TR = G::TR, ER = G::ER;
    constexpr size_t SL = (size_t)H * W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TR;
    const int grp = warp * (32 / TR) + lane / TR;
    const unsigned gm = group_mask<TR>(lane);
    float2* rs = cx.rows + grp * G::MP;
    const int cid = blockIdx.x / G::C, ncl = gridDim.x / G::C;
    const double lam = r.lam;
#pragma unroll 1
    for (int s = cid; s < prm.S; s += ncl) {
        const size_t base = (size_t)s * SL;
        double acc[kReportSums] = {0, 0, 0, 0, 0};
        if (r.mode == 0) {
            cluster_barrier<G::C>();  // peers running before their shared memory is written
#pragma unroll 1
            for (int pass = 0; pass < G::R / G::RPP; ++pass) {
                const int i = cx.crank * G::R + pass * G::RPP + grp;
                float2 z[ER];
#pragma unroll
                for (int e = 0; e < ER; ++e)
                    z[e] = __ldcg(reinterpret_cast<const float2*>(prm.chi + base + (size_t)i * W + 2 * (g + TR * e)));
                row_forward<G>(cx, rs, i, g, gm, z);
            }
            cluster_barrier<G::C>();
            columns_out_3d<G>(cx, r.a.spec, s);
            continue;
        }
        columns_in_3d<G>(cx, r.a.spec, s);
        cluster_barrier<G::C>();
#pragma unroll 1
        for (int pass = 0; pass < G::R / G::RPP; ++pass) {
            const int i = cx.crank * G::R + pass * G::RPP + grp;
            const size_t rowoff = base + (size_t)i * W;
            float2 x[ER];
            row_inverse<G>(cx, rs, i, g, gm, x);
#pragma unroll
            for (int e = 0; e < ER; ++e) {
                const int j0 = 2 * (g + TR * e);
                const size_t o = rowoff + j0;
                const uchar2 mk2 = __ldg(reinterpret_cast<const uchar2*>(prm.mask + o));
                const double m[2] = {(double)mk2.x, (double)mk2.y};
                const float2 qx = __ldcg(reinterpret_cast<const float2*>(prm.qx + o));
                const float2 qy = __ldcg(reinterpret_cast<const float2*>(prm.qy + o));
                const float2 qz = __ldcg(reinterpret_cast<const float2*>(prm.qz + o));
                if (r.mode == 1) {
                    const float2 f = __ldg(reinterpret_cast<const float2*>(prm.field + o));
                    const float2 p = __ldcg(reinterpret_cast<const float2*>(prm.p + o));
                    const float2 c = __ldcg(reinterpret_cast<const float2*>(prm.chi + o));
                    const float cr = (j0 + 2 < W) ? __ldcg(prm.chi + o + 2) : c.y;
                    const float2 cd = (i + 1 < H) ? __ldcg(reinterpret_cast<const float2*>(prm.chi + o + W)) : c;
                    const float2 cz = (s + 1 < prm.S) ? __ldcg(reinterpret_cast<const float2*>(prm.chi + o + SL)) : c;
                    float2 wv = make_float2((float)m[0], (float)m[1]);
                    if (prm.weight) wv = __ldg(reinterpret_cast<const float2*>(prm.weight + o));
                    const double w[2] = {wv.x, wv.y}, u[2] = {x[e].x, x[e].y}, ff[2] = {f.x, f.y};
                    const double pp[2] = {p.x, p.y};
                    const double gx[2] = {m[0] * ((double)c.y - c.x), m[1] * ((double)cr - c.y)};
                    const double gy[2] = {m[0] * ((double)cd.x - c.x), m[1] * ((double)cd.y - c.y)};
                    const double gz[2] = {m[0] * ((double)cz.x - c.x), m[1] * ((double)cz.y - c.y)};
                    const double qxs[2] = {qx.x, qx.y}, qys[2] = {qy.x, qy.y}, qzs[2] = {qz.x, qz.y};
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const double res = w[t] * (u[t] - ff[t]);
                        acc[0] += res * res;
                        const double tvn = prm.tv_iso ? sqrt(gx[t] * gx[t] + gy[t] * gy[t] + gz[t] * gz[t])
                                                      : fabs(gx[t]) + fabs(gy[t]) + fabs(gz[t]);
                        acc[1] += tvn;
                        const double d1 = pp[t] - lam * res;
                        acc[2] += d1 * d1;
                        acc[3] += tvn - (qxs[t] * gx[t] + qys[t] * gy[t] + qzs[t] * gz[t]);
                    }
                    x[e] = make_float2((float)(w[0] * p.x), (float)(w[1] * p.y));  // W p
                } else {
                    // G3^T M q: x, y as the per-slice report; z: (M qz)[s-1] - (M qz)[s][s < S-1]
                    const double a0 = m[0] * qx.x, a1 = m[1] * qx.y;
                    const double al = (j0 > 0) ? (double)__ldg(prm.mask + o - 1) * __ldcg(prm.qx + o - 1) : 0.0;
                    const double a1r = (j0 + 2 < W) ? a1 : 0.0;
                    double bu0 = 0.0, bu1 = 0.0, zu0 = 0.0, zu1 = 0.0;
                    if (i > 0) {
                        const uchar2 mu = __ldg(reinterpret_cast<const uchar2*>(prm.mask + o - W));
                        const float2 qu = __ldcg(reinterpret_cast<const float2*>(prm.qy + o - W));
                        bu0 = (double)mu.x * qu.x;
                        bu1 = (double)mu.y * qu.y;
                    }
                    if (s > 0) {
                        const uchar2 mz = __ldg(reinterpret_cast<const uchar2*>(prm.mask + o - SL));
                        const float2 qp = __ldcg(reinterpret_cast<const float2*>(prm.qz + o - SL));
                        zu0 = (double)mz.x * qp.x;
                        zu1 = (double)mz.y * qp.y;
                    }
                    const double b0 = (i + 1 < H) ? m[0] * qy.x : 0.0, b1 = (i + 1 < H) ? m[1] * qy.y : 0.0;
                    const double z0 = (s + 1 < prm.S) ? m[0] * qz.x : 0.0, z1 = (s + 1 < prm.S) ? m[1] * qz.y : 0.0;
                    const double k0 = (double)x[e].x + (al - a0) + (bu0 - b0) + (zu0 - z0);
                    const double k1 = (double)x[e].y + (a0 - a1r) + (bu1 - b1) + (zu1 - z1);
                    acc[4] += k0 * k0 + k1 * k1;
                }
            }
            if (r.mode == 1) row_forward<G>(cx, rs, i, g, gm, x);
        }
        cluster_barrier<G::C>();  // all scatters in; all gathers done
        if (r.mode == 1) columns_out_3d<G>(cx, r.a.spec, s);
#pragma unroll
        for (int t = 0; t < kReportSums; ++t) {
            const double v = block_sum<G::NT>(acc[t], red);
            if (threadIdx.x == 0 && ((r.mode == 1 && t < 4) || (r.mode == 2 && t == 4)))
                r.partial[((size_t)s * G::C + cx.crank) * kReportSums + t] = v;
        }
    }
}

// z pass: pencils of TZ = NZ / EZ lanes, one per (kx, ky); a tile is NW * 32 / TZ
// consecutive ky of one kx, so that every load is a full 32-byte sector.  D(k) = 1/3 -
// kz^2 / |k|^2 (D(0) = 0) in FP32, k_i = f_i * iv_i: the integer frequencies in cycles per
// sample times the inverse voxel edges (iv = (1, 1, 1) for isotropic voxels).  One tile per
// CTA (grid NTILES): a persistent form that kept the next tile's loads in flight took 74
// registers instead of 57, three CTAs per SM instead of four, and measured slower.
template <int NZ, int H, int W, int NT = 256>
struct GeoZ {
    static constexpr int EZ = default_elems(NZ);
    static constexpr int TZ = NZ / EZ;
    static constexpr int PPW = 32 / TZ;           // pencils per warp
    static constexpr int TY = (NT / 32) * PPW;    // pencils (ky values) per tile
    static constexpr int M = W / 2;
    static constexpr int NTILES = (M + 1) * (H / TY);
    static constexpr int NP = NZ + (TZ % 16);  // pencil buffer stride: adjacent pencils on other banks
    static constexpr size_t SMEM_BYTES = sizeof(float2) * (TY * NP + StageTw<NZ, EZ>::SIZE);
    static_assert(H % TY == 0, "ky tiles");
    static_assert((NZ & (NZ - 1)) == 0 && (H & (H - 1)) == 0 && (W & (W - 1)) == 0,
                  "powers of two: i / n == i * (1 / n) exactly");
};

// Signed frequency of index k of a length-n transform in cycles per sample (n a power of two,
// so the product with the reciprocal equals the quotient).
template <int N>
__device__ __forceinline__ float signed_freq_pow2(int k) {
    return (float)(k < (N + 1) / 2 ? k : k - N) * (1.0f / (float)N);
}

template <class GZ, int NZ, int H, int W>
__global__ void __launch_bounds__(256) pd3_z_kernel(float2* __restrict__ spec, const float2* __restrict__ twid,
                                                    int ntw, float3 iv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TZ = GZ::TZ, EZ = GZ::EZ, M = GZ::M, TILES_Y = H / GZ::TY;
    constexpr size_t STRIDE = (size_t)(M + 1) * H;  // between slices
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + GZ::TY * GZ::NP;
    StageTw<NZ, EZ>::fill(stw, twid, ntw / NZ, threadIdx.x, 256);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TZ;
    const int pen = warp * GZ::PPW + lane / TZ;
    const unsigned gm = group_mask<TZ>(lane);
    float2* pb = buf + pen * GZ::NP;
    constexpr float scale = 1.0f / ((float)NZ * (float)H * (float)W);
    grid_dependency_wait();
    const int t = blockIdx.x;
    const int kx = t / TILES_Y, ky = (t - kx * TILES_Y) * GZ::TY + pen;
    float2* col = spec + (size_t)kx * H + ky;
    float2 x[EZ];
#pragma unroll
    for (int e = 0; e < EZ; ++e) x[e] = __ldcg(col + (size_t)(g + TZ * e) * STRIDE);
    fft<NZ, TZ, false>(x, pb, stw, g, gm);
    const float fx = (float)kx * (1.0f / (float)W) * iv.x, fy = signed_freq_pow2<H>(ky) * iv.y;
    const float pxy = fx * fx + fy * fy;
#pragma unroll
    for (int e = 0; e < EZ; ++e) {
        const float fz = signed_freq_pow2<NZ>(g + TZ * e) * iv.z;
        const float k2 = pxy + fz * fz;
        const float d = (k2 > 0.f) ? (1.0f / 3.0f - (fz * fz) / k2) * scale : 0.f;
        x[e] = make_float2(x[e].x * d, x[e].y * d);
    }
    fft<NZ, TZ, true>(x, pb, stw, g, gm);
#pragma unroll
    for (int e = 0; e < EZ; ++e) __stcg(col + (size_t)(g + TZ * e) * STRIDE, x[e]);
}

}  // namespace pcs
