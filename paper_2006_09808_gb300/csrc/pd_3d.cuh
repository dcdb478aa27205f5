// pd_3d.cuh -- the 3-D variant: Eq. (1) with G in all three dimensions and the
// 3-D dipole convolution of the whole volume (B0 along z, the slice axis).
//
// The volume's half spectrum lives in global memory between the passes of one dipole
// convolution, in one of two forms (the host picks by shape):
//
// Pencil form (the end of this file), where a kx plane fits in shared memory: the spectrum as
// kx planes [kx][s][y]; a cluster-free row kernel (real row FFTs and the row phases) and a
// plane kernel (y and z FFTs with the D multiply).
//
// Slice form, for larger planes:
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
// multiplies every entry by a real D.  The FP64 report kernel uses the slice form's layout
// and kernels for either form.
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
    // pencil buffer stride: the 32 / TZ groups of a warp write the FFT's first stage to every bank
    // pair twice (a stride of NZ + 8 for TZ = 8 put all four groups on the same eight pairs)
    static constexpr int NP = NZ + TZ / 2;
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

// ------------------------------------------------------------------ pencil form
// The volume's half spectrum as kx planes spec[kx][s][y], kx = 0..M (the packed DC / Nyquist
// column split into planes 0 and M, the spectra of real rows), used where a plane fits in
// shared memory:
//   row kernel (no cluster): a CTA takes RPP consecutive rows of one slice; each row is read
//       from the planes (element k of row (s, y) at spec[(k S + s) H + y]: four rows of a warp
//       fill one 32-byte sector per k), inverse real row FFT, the dual or primal step of the
//       row phases above, forward real row FFT of its output, stored back in place;
//   plane kernel: one CTA per plane kx: forward y FFTs read straight from the plane, the
//       S x H plane in shared memory for forward z FFTs x D3 / (S H W) and inverse z FFTs,
//       inverse y FFTs written straight back.
// One iteration = rows (dual) -> planes -> rows (primal) -> planes.

// Row transport of the pencil form: a row's packed spectrum from and to the planes.
template <class G>
struct PlaneRows {
    using V = typename G::V;
    // epilogue elements whose loads go out together: 2 (129.8 us per 256x256x64 iteration);
    // 4 spills at two CTAs per SM (131.7), 4 or 8 at one CTA per SM 140.8 / 136.0
    static constexpr int kChunkElems = 2;
    const V* in;   // planes to read; NULL: zero spectrum (the zero start)
    V* out;        // planes to write (the same buffer: each row reads and writes only its own entries)
    size_t row0;   // s H: slice s inside a plane
    size_t plane;  // S H: stride between planes
    __device__ __forceinline__ void wait() const {}
    __device__ __forceinline__ void inverse(const Ctx<G>& cx, V* rs, int i, int g, unsigned gm, V (&x)[G::ER]) const {
        constexpr int TR = G::TR, ER = G::ER, M = G::M;
        if (in) {
#pragma unroll
            for (int e = 0; e < ER; ++e) {
                const int k = g + TR * e;
                const V v = __ldcg(in + (size_t)k * plane + row0 + i);
                // k = 0: planes 0 and M hold real rows' spectra, packed as X[0] + i X[M]
                x[e] = (k == 0) ? mk<V>(v.x, __ldcg(in + (size_t)M * plane + row0 + i).x) : v;
            }
        } else {
#pragma unroll
            for (int e = 0; e < ER; ++e) x[e] = mk<V>(0.f, 0.f);
        }
        row_unpack_inverse<G>(cx, rs, g, gm, x);
    }
    __device__ __forceinline__ void forward(const Ctx<G>& cx, V* rs, int i, int g, unsigned gm, V (&x)[G::ER]) const {
        constexpr int TR = G::TR, ER = G::ER, M = G::M;
        row_forward_pack<G>(cx, rs, g, gm, x);
#pragma unroll
        for (int e = 0; e < ER; ++e) {
            const int k = g + TR * e;
            if (k == 0) {
                __stcg(out + row0 + i, mk<V>(x[e].x, 0.f));
                __stcg(out + (size_t)M * plane + row0 + i, mk<V>(x[e].y, 0.f));
            } else {
                __stcg(out + (size_t)k * plane + row0 + i, x[e]);
            }
        }
    }
};

// Shared memory of the row kernel: row scratch and twiddle tables (no spectrum columns).
template <class G>
constexpr size_t pencil_rows_smem() {
    return sizeof(typename G::V) * (G::SM_ROWS + G::SM_TW + G::SM_STW_R);
}

// G: a geometry whose R equals RPP (one row pass per CTA); its C = H / RPP row tiles per
// slice are independent CTAs, not a cluster.
template <class G>
__global__ void __launch_bounds__(G::NT, G::MINB) pd3p_rows_kernel(P3Params a) {
    static_assert(G::R == G::RPP, "one row pass per CTA");
    using V = typename G::V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ctx<G> cx;
    cx.tbuf = nullptr;
    cx.rows = reinterpret_cast<V*>(smem_raw);
    cx.tw = cx.rows + G::SM_ROWS;
    cx.stw_r = cx.tw + G::SM_TW;
    cx.stw_c = nullptr;
    const PDParams& prm = a.pd;
    for (int t = threadIdx.x; t < G::NTW; t += G::NT) cx.tw[t] = prm.twid[t];
    StageTw<G::M, G::ER>::fill(cx.stw_r, prm.twid, G::NTW / G::M, threadIdx.x, G::NT);
    const int s = blockIdx.x / G::C;
    cx.crank = blockIdx.x - s * G::C;  // row tile within the slice
    __syncthreads();
    grid_dependency_wait();  // the previous launch's planes and state complete
    const size_t base = (size_t)s * G::H * G::W;
    const PlaneRows<G> io{a.load ? a.spec : nullptr, a.spec, (size_t)s * G::H, (size_t)prm.S * G::H};
    if (a.phase == 0) {
        phase_dual<G, true, PlaneRows<G>>(cx, prm, base, prm.inv_den, true, s, io);
    } else {
        phase_primal<G, true, PlaneRows<G>>(cx, prm, base, !a.store, s, io);
    }
}

// Plane kernel geometry: y transforms by groups of TYL lanes (EY elements each), z transforms
// by groups of TZ lanes; the plane's line s (S lines of H) at pl[s H], element y at
// P(y, 4 s); z scratch per group at stride ZP.
template <int S_, int H_, int W_, int NT_>
struct GeoPlane {
    static constexpr int S = S_, H = H_, W = W_, NT = NT_, M = W / 2;
    static constexpr int EY = default_elems(H), TYL = H / EY;
    static constexpr int EZ = default_elems(S), TZ = S / EZ;
    static constexpr int NGY = NT / TYL, NGZ = NT / TZ;
    static constexpr int ZP = S + TZ / 2;  // z scratch stride (see GeoZ::NP)
    static constexpr size_t PLANE = (size_t)S * H;
    static constexpr size_t SMEM_BYTES =
        sizeof(float2) * (PLANE + (size_t)NGZ * ZP + StageTw<H, EY>::SIZE + StageTw<S, EZ>::SIZE);
    static_assert(SMEM_BYTES <= 232448, "the plane fits in shared memory");
    static_assert(PLANE % 2 == 0 && (S & (S - 1)) == 0 && (H & (H - 1)) == 0 && (W & (W - 1)) == 0, "shape");
};

template <class GP>
__global__ void __launch_bounds__(GP::NT, 1) pd3p_plane_kernel(float2* __restrict__ spec,
                                                              const float2* __restrict__ twid, int ntw, float3 iv) {
    constexpr int S = GP::S, H = GP::H, W = GP::W, TYL = GP::TYL, EY = GP::EY, TZ = GP::TZ, EZ = GP::EZ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* pl = reinterpret_cast<float2*>(smem_raw);
    float2* zs = pl + GP::PLANE;
    float2* stw_y = zs + GP::NGZ * GP::ZP;
    float2* stw_z = stw_y + StageTw<H, EY>::SIZE;
    StageTw<H, EY>::fill(stw_y, twid, ntw / H, threadIdx.x, GP::NT);
    StageTw<S, EZ>::fill(stw_z, twid, ntw / S, threadIdx.x, GP::NT);
    const int kx = blockIdx.x;
    float2* src = spec + (size_t)kx * GP::PLANE;
    __syncthreads();  // stage twiddles
    grid_dependency_wait();  // the row kernel's planes complete
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {  // forward y transforms, straight from the plane in global memory (a group's lanes read
       // consecutive entries of one line)
        const int g = lane % TYL, grp = warp * (32 / TYL) + lane / TYL;
        const unsigned gm = group_mask<TYL>(lane);
#pragma unroll 1
        for (int sl = grp; sl < S; sl += GP::NGY) {
            float2* line = pl + sl * H;
            float2 x[EY];
#pragma unroll
            for (int e = 0; e < EY; ++e) x[e] = __ldcg(src + (size_t)sl * H + g + TYL * e);
            fft<H, TYL, false>(x, line, stw_y, g, gm, 4 * sl);
#pragma unroll
            for (int e = 0; e < EY; ++e) line[P(g + TYL * e, 4 * sl)] = x[e];
            __syncwarp(gm);
        }
    }
    __syncthreads();
    {  // z pencils: forward FFT, x D3 / (S H W), inverse FFT
        const int g = lane % TZ, grp = warp * (32 / TZ) + lane / TZ;
        const unsigned gm = group_mask<TZ>(lane);
        float2* zb = zs + grp * GP::ZP;
        const float fx = (float)kx * (1.0f / (float)W) * iv.x;
        constexpr float scale = 1.0f / ((float)S * (float)H * (float)W);
        float fz2[EZ];  // kz^2 of this lane's elements (the same for every pencil)
#pragma unroll
        for (int e = 0; e < EZ; ++e) {
            const float fz = signed_freq_pow2<S>(g + TZ * e) * iv.z;
            fz2[e] = fz * fz;
        }
#pragma unroll 1
        for (int ky = grp; ky < H; ky += GP::NGZ) {
            float2 x[EZ];
#pragma unroll
            for (int e = 0; e < EZ; ++e) {
                const int sl = g + TZ * e;
                x[e] = pl[sl * H + P(ky, 4 * sl)];
            }
            fft<S, TZ, false>(x, zb, stw_z, g, gm);
            const float fy = signed_freq_pow2<H>(ky) * iv.y;
            const float pxy = fx * fx + fy * fy;
#pragma unroll
            for (int e = 0; e < EZ; ++e) {
                const float k2 = pxy + fz2[e];
                const float d = (k2 > 0.f) ? (1.0f / 3.0f - fz2[e] / k2) * scale : 0.f;
                x[e] = make_float2(x[e].x * d, x[e].y * d);
            }
            fft<S, TZ, true>(x, zb, stw_z, g, gm);
#pragma unroll
            for (int e = 0; e < EZ; ++e) {
                const int sl = g + TZ * e;
                pl[sl * H + P(ky, 4 * sl)] = x[e];
            }
        }
    }
    __syncthreads();
    {  // inverse y transforms, straight back to the plane in global memory
        const int g = lane % TYL, grp = warp * (32 / TYL) + lane / TYL;
        const unsigned gm = group_mask<TYL>(lane);
#pragma unroll 1
        for (int sl = grp; sl < S; sl += GP::NGY) {
            float2* line = pl + sl * H;
            float2 x[EY];
#pragma unroll
            for (int e = 0; e < EY; ++e) x[e] = line[P(g + TYL * e, 4 * sl)];
            fft<H, TYL, true>(x, line, stw_y, g, gm, 4 * sl);
#pragma unroll
            for (int e = 0; e < EY; ++e) __stcg(src + (size_t)sl * H + g + TYL * e, x[e]);
        }
    }
}

}  // namespace pcs
