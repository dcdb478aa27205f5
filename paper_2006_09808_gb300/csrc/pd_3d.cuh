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
#pragma unroll 1
    for (int s = cid; s < prm.S; s += ncl) {
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
    }
}

// z pass: pencils of TZ = NZ / EZ lanes, one per (kx, ky); a CTA takes
// NW * 32 / TZ consecutive ky of one kx.  D(k) = 1/3 - fz^2 / |f|^2 (D(0) = 0)
// from the integer frequencies, in FP32.
template <int NZ, int H, int W, int NT = 256>
struct GeoZ {
    static constexpr int EZ = default_elems(NZ);
    static constexpr int TZ = NZ / EZ;
    static constexpr int PPW = 32 / TZ;           // pencils per warp
    static constexpr int TY = (NT / 32) * PPW;    // pencils (ky values) per CTA
    static constexpr int M = W / 2;
    static constexpr int NP = NZ + (TZ % 16);  // pencil buffer stride: adjacent pencils on other banks
    static constexpr size_t SMEM_BYTES = sizeof(float2) * (TY * NP + StageTw<NZ, EZ>::SIZE);
    static_assert(H % TY == 0, "ky tiles");
};

__device__ __forceinline__ float signed_freq(int k, int n) { return (float)(k < (n + 1) / 2 ? k : k - n) / (float)n; }

template <class GZ, int NZ, int H, int W>
__global__ void __launch_bounds__(256) pd3_z_kernel(float2* __restrict__ spec, const float2* __restrict__ twid,
                                                    int ntw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TZ = GZ::TZ, EZ = GZ::EZ, M = GZ::M;
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + GZ::TY * GZ::NP;
    StageTw<NZ, EZ>::fill(stw, twid, ntw / NZ, threadIdx.x, 256);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TZ;
    const int pen = warp * GZ::PPW + lane / TZ;
    const unsigned gm = group_mask<TZ>(lane);
    const int kx = blockIdx.x;
    const int ky = blockIdx.y * GZ::TY + pen;
    const size_t stride = (size_t)(M + 1) * H;
    float2* col = spec + (size_t)kx * H + ky;
    float2* pb = buf + pen * GZ::NP;
    float2 x[EZ];
#pragma unroll
    for (int e = 0; e < EZ; ++e) x[e] = __ldcg(col + (size_t)(g + TZ * e) * stride);
    fft<NZ, TZ, false>(x, pb, stw, g, gm);
    const float fx = (float)kx / (float)W, fy = signed_freq(ky, H);
    const float pxy = fx * fx + fy * fy;
    const float scale = 1.0f / ((float)NZ * (float)H * (float)W);
#pragma unroll
    for (int e = 0; e < EZ; ++e) {
        const float fz = signed_freq(g + TZ * e, NZ);
        const float k2 = pxy + fz * fz;
        const float d = (k2 > 0.f) ? (1.0f / 3.0f - (fz * fz) / k2) * scale : 0.f;
        x[e] = make_float2(x[e].x * d, x[e].y * d);
    }
    fft<NZ, TZ, true>(x, pb, stw, g, gm);
#pragma unroll
    for (int e = 0; e < EZ; ++e) __stcg(col + (size_t)(g + TZ * e) * stride, x[e]);
}

}  // namespace pcs
