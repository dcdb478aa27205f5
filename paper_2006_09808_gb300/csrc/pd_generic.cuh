// pd_generic.cuh -- the Sec. II.A iteration for slice sizes outside the
// power-of-two / 3·2^k family: any even H x W whose lengths factor into
// primes <= 61 (the paper's own 256 x 258 and 128 x 132 slices: 258 = 2·3·43,
// 132 = 4·3·11).
//
// Per half step two launches, the half spectrum [S][H][W/2 + 1] (row-major,
// complex) held in global memory between them:
//   row kernel:    one warp per pair of rows; the two real rows travel as one
//                  complex row (a + i b) through a length-W DFT in shared memory
//                  -> the dual or primal row phase -> forward DFT, split back into
//                  the two half-spectrum rows
//   column kernel: length-H transform x D(k)/(H W), inverse: the register FFT of
//                  fft_core.cuh for H in {64, 128, 192, 256, 384, 512} (pencils
//                  of lanes, gen_cols_fft_kernel), else one warp per spectrum
//                  column with the shared-memory DFT (gen_cols_kernel)
// The shared-memory DFTs are mixed-radix Stockham passes: 2, 3, 4 as butterflies,
// larger odd primes as a symmetric direct DFT (terms q and r - q paired).
// Also here: the FP64 report kernel and the power iteration for ||K||, which reuse
// the row transforms and the column pass.
#pragma once

#include <cuda_runtime.h>

#include "pd_cluster.cuh"

namespace pcs {

constexpr int kGenMaxStages = 12;
constexpr int kGenRowWarps = 8;   // row pairs per CTA of the row, report and power-iteration kernels
constexpr int kGenColTile = 16;   // spectrum columns per CTA of the shared-memory column kernel

struct GenPlan {
    int n;                  // transform length
    int nst;                // number of stages
    int r[kGenMaxStages];   // radices, product n
};

struct GenParams {
    const float* field;
    const unsigned char* mask;
    const float* weight;  // NULL: W = mask
    float* chi;
    float* chibar;
    float* p;
    float* qx;
    float* qy;
    float2* spec;          // [S][H][M1]
    const float2* trow;    // exp(-2 pi i n / W), n < W
    const float2* tcol;    // exp(-2 pi i n / H), n < H
    GenPlan prow, pcol;
    int S, H, W, M1;       // M1 = W / 2 + 1
    float sigma, tau, inv_den;
    int tv_iso;
    int b0_axis;           // 0: B0 along y (rows), 1: along x
    int phase;             // 0: dual step, 1: primal step
    int store;             // 1: forward transforms of the phase's output to the spectrum
    const int* active;     // NULL, or per-slice flags: 0 = frozen (the row kernel leaves it alone)
    const float* inv_den_slice;  // NULL, or per-slice 1 / (1 + sigma / lambda_s) (batches)
};

__device__ __forceinline__ float2 gcmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// floor(j / d) for 0 <= j < 1024 and 1 <= d <= 512, from inv = 1/d rounded to float:
// (j + 1/2) inv stays within 1e-4 of (j + 1/2)/d, which is at least 1/(2d) >= 1e-3 from
// an integer (checked exhaustively over that range).  Replaces integer division by
// the runtime stage sizes.
__device__ __forceinline__ int qdiv(int j, float inv) { return (int)(((float)j + 0.5f) * inv); }

// Length pl.n DFT by one warp in shared memory (unnormalised; inv: exponent sign +).
// Input in a, b is scratch; returns the buffer holding the result (which one depends
// on the plan's radices).  Stage with
// radix r after the radices so far multiply to Ns (R = n / r):
//   X_out[(j / Ns) Ns r + k + q' Ns] = sum_q X_in[j + q R] w^(k q n/(Ns r)) w^(q q' R),
// k = j mod Ns, w = exp(-+2 pi i / n), for j < R, q' < r.
__device__ float2* warp_dft(float2* a, float2* b, const float2* T, const GenPlan& pl, bool inv, int lane) {
    const int N = pl.n;
    const float sg = inv ? -1.f : 1.f;  // sign applied to the imaginary part of the forward twiddles
    int Ns = 1;
#pragma unroll 1
    for (int st = 0; st < pl.nst; ++st) {
        const int r = pl.r[st];
        const int R = N / r;
        const int step = N / (Ns * r);
        const float invNs = __frcp_rn((float)Ns), invR = __frcp_rn((float)R);
        if (r == 2) {
#pragma unroll 1
            for (int j = lane; j < R; j += 32) {
                const int k = j - qdiv(j, invNs) * Ns;
                float2 t = T[k * step];
                t.y *= sg;
                const float2 v0 = a[j], v1 = gcmul(a[j + R], t);
                const int o = (j - k) * 2 + k;
                b[o] = make_float2(v0.x + v1.x, v0.y + v1.y);
                b[o + Ns] = make_float2(v0.x - v1.x, v0.y - v1.y);
            }
        } else if (r == 4) {
#pragma unroll 1
            for (int j = lane; j < R; j += 32) {
                const int k = j - qdiv(j, invNs) * Ns;
                float2 t1 = T[k * step], t2 = T[2 * k * step], t3 = T[3 * k * step];
                t1.y *= sg;
                t2.y *= sg;
                t3.y *= sg;
                const float2 v0 = a[j], v1 = gcmul(a[j + R], t1), v2 = gcmul(a[j + 2 * R], t2),
                             v3 = gcmul(a[j + 3 * R], t3);
                const float2 s02 = make_float2(v0.x + v2.x, v0.y + v2.y), d02 = make_float2(v0.x - v2.x, v0.y - v2.y);
                const float2 s13 = make_float2(v1.x + v3.x, v1.y + v3.y), d13 = make_float2(v1.x - v3.x, v1.y - v3.y);
                // -i d13 (forward) or +i d13 (inverse)
                const float2 rd = make_float2(sg * d13.y, -sg * d13.x);
                const int o = (j - k) * 4 + k;
                b[o] = make_float2(s02.x + s13.x, s02.y + s13.y);
                b[o + Ns] = make_float2(d02.x + rd.x, d02.y + rd.y);
                b[o + 2 * Ns] = make_float2(s02.x - s13.x, s02.y - s13.y);
                b[o + 3 * Ns] = make_float2(d02.x - rd.x, d02.y - rd.y);
            }
        } else if (r == 3) {
            const float h = 0.86602540378443865f;  // sin(2 pi / 3)
#pragma unroll 1
            for (int j = lane; j < R; j += 32) {
                const int k = j - qdiv(j, invNs) * Ns;
                float2 t1 = T[k * step], t2 = T[2 * k * step];
                t1.y *= sg;
                t2.y *= sg;
                const float2 v0 = a[j], v1 = gcmul(a[j + R], t1), v2 = gcmul(a[j + 2 * R], t2);
                const float2 s = make_float2(v1.x + v2.x, v1.y + v2.y), d = make_float2(v1.x - v2.x, v1.y - v2.y);
                const float2 m = make_float2(v0.x - 0.5f * s.x, v0.y - 0.5f * s.y);
                // -i h d (forward) or +i h d (inverse)
                const float2 rd = make_float2(sg * h * d.y, -sg * h * d.x);
                const int o = (j - k) * 3 + k;
                b[o] = make_float2(v0.x + s.x, v0.y + s.y);
                b[o + Ns] = make_float2(m.x + rd.x, m.y + rd.y);
                b[o + 2 * Ns] = make_float2(m.x - rd.x, m.y - rd.y);
            }
        } else {
            // odd prime r >= 5: (1) pre-twiddle in place; (2) sums s_q = v_q + v_(r-q) and
            // differences d_q = v_q - v_(r-q) into b; (3) outputs q' and r - q' together:
            // A = v_0 + sum s_q cos(2 pi m / r), B = sum d_q (-sin(2 pi m / r)), m = q q' mod r,
            // X_q' = A + i sg B, X_(r-q') = A - i sg B (forward sg = 1).  The result lands in a.
#pragma unroll 1
            for (int u = lane + R; u < N; u += 32) {
                const int q = qdiv(u, invR), j = u - q * R;
                float2 t = T[(j - qdiv(j, invNs) * Ns) * step * q];
                t.y *= sg;
                a[u] = gcmul(a[u], t);
            }
            __syncwarp();
            const int h = (r - 1) / 2;
#pragma unroll 1
            for (int u = lane; u < R * (h + 1); u += 32) {
                const int q = qdiv(u, invR), j = u - q * R;
                if (q == 0) {
                    b[j] = a[j];
                } else {
                    const float2 x = a[j + q * R], y = a[j + (r - q) * R];
                    b[j + q * R] = make_float2(x.x + y.x, x.y + y.y);
                    b[j + (r - q) * R] = make_float2(x.x - y.x, x.y - y.y);
                }
            }
            __syncwarp();
            // q' = 0: X_0 = v_0 + sum s_q
#pragma unroll 1
            for (int j = lane; j < R; j += 32) {
                float2 acc = b[j];
#pragma unroll 1
                for (int q = 1; q <= h; ++q) {
                    const float2 sq = b[j + q * R];
                    acc.x += sq.x;
                    acc.y += sq.y;
                }
                const int k = j - qdiv(j, invNs) * Ns;
                a[(j - k) * r + k] = acc;
            }
            // q' = 1..h: two (j, q') units per lane at a time (independent chains)
            const int NU = R * h;
#pragma unroll 1
            for (int u0 = lane; u0 < NU; u0 += 64) {
                const bool has1 = (u0 + 32 < NU);
                const int u1 = has1 ? u0 + 32 : u0;
                const int t0 = qdiv(u0, invR), t1 = qdiv(u1, invR);
                const int j0 = u0 - t0 * R, qp0 = 1 + t0;
                const int j1 = u1 - t1 * R, qp1 = 1 + t1;
                float2 A0 = b[j0], B0 = make_float2(0.f, 0.f);
                float2 A1 = b[j1], B1 = make_float2(0.f, 0.f);
                int m0 = 0, m1 = 0;
#pragma unroll 1
                for (int q = 1; q <= h; ++q) {
                    m0 += qp0;
                    if (m0 >= r) m0 -= r;
                    m1 += qp1;
                    if (m1 >= r) m1 -= r;
                    const float2 c0 = T[m0 * R], c1 = T[m1 * R];  // (cos, -sin) of 2 pi m / r
                    const float2 s0 = b[j0 + q * R], d0 = b[j0 + (r - q) * R];
                    const float2 s1 = b[j1 + q * R], d1 = b[j1 + (r - q) * R];
                    A0.x = fmaf(s0.x, c0.x, A0.x);
                    A0.y = fmaf(s0.y, c0.x, A0.y);
                    B0.x = fmaf(d0.x, c0.y, B0.x);
                    B0.y = fmaf(d0.y, c0.y, B0.y);
                    A1.x = fmaf(s1.x, c1.x, A1.x);
                    A1.y = fmaf(s1.y, c1.x, A1.y);
                    B1.x = fmaf(d1.x, c1.y, B1.x);
                    B1.y = fmaf(d1.y, c1.y, B1.y);
                }
                const int k0 = j0 - qdiv(j0, invNs) * Ns;
                const int ob0 = (j0 - k0) * r + k0;
                a[ob0 + qp0 * Ns] = make_float2(A0.x - sg * B0.y, A0.y + sg * B0.x);
                a[ob0 + (r - qp0) * Ns] = make_float2(A0.x + sg * B0.y, A0.y - sg * B0.x);
                if (has1) {
                    const int k1 = j1 - qdiv(j1, invNs) * Ns;
                    const int ob1 = (j1 - k1) * r + k1;
                    a[ob1 + qp1 * Ns] = make_float2(A1.x - sg * B1.y, A1.y + sg * B1.x);
                    a[ob1 + (r - qp1) * Ns] = make_float2(A1.x + sg * B1.y, A1.y - sg * B1.x);
                }
            }
            __syncwarp();
            Ns *= r;
            continue;  // result in a: no swap
        }
        __syncwarp();
        float2* t = a;
        a = b;
        b = t;
        Ns *= r;
    }
    return a;
}

// Row kernel: a warp takes rows i0 = 2 pr, i1 = i0 + 1 of one slice.
__global__ void __launch_bounds__(kGenRowWarps * 32) gen_rows_kernel(GenParams g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = g.H, W = g.W, M1 = g.M1;
    float2* T = reinterpret_cast<float2*>(smem_raw);
    for (int t = threadIdx.x; t < W; t += blockDim.x) T[t] = g.trow[t];
    __syncthreads();
    grid_dependency_wait();  // the previous launch's spectrum and state complete
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pair = blockIdx.x * kGenRowWarps + warp;
    if (pair >= g.S * (H / 2)) return;  // whole warps; no CTA barrier below
    float2* bufa = T + W + (size_t)warp * 2 * W;
    float2* bufb = bufa + W;
    const int s = pair / (H / 2);
    if (g.active && !g.active[s]) return;  // frozen slice (monitored solves): state kept as is
    const int i0 = 2 * (pair - s * (H / 2)), i1 = i0 + 1;
    const size_t r0 = ((size_t)s * H + i0) * W, r1 = r0 + W;
    float2* sp0 = g.spec + ((size_t)s * H + i0) * M1;
    float2* sp1 = sp0 + M1;

    // z = a + i b from the two half-spectrum rows (Hermitian extension beyond M1)
#pragma unroll 3
    for (int k = lane; k < W; k += 32) {
        float2 z;
        if (k < M1) {
            const float2 A = __ldcg(sp0 + k), B = __ldcg(sp1 + k);
            z = make_float2(A.x - B.y, A.y + B.x);
        } else {
            const float2 A = __ldcg(sp0 + (W - k)), B = __ldcg(sp1 + (W - k));
            z = make_float2(A.x + B.y, B.x - A.y);  // conj(A) + i conj(B)
        }
        bufa[k] = z;
    }
    __syncwarp();
    float2* u = warp_dft(bufa, bufb, T, g.prow, true, lane);
    float2* o = (u == bufa) ? bufb : bufa;
    const float sigma = g.sigma, tau = g.tau;
    // each element is read and written by one lane only: the state arrays do not alias
    const float* __restrict__ fld = g.field;
    const unsigned char* __restrict__ msk = g.mask;
    const float* __restrict__ wgt = g.weight;
    float* __restrict__ chi = g.chi;
    float* __restrict__ cbar = g.chibar;
    float* __restrict__ pp = g.p;
    float* __restrict__ qxp = g.qx;
    float* __restrict__ qyp = g.qy;
    // Each lane takes adjacent column pairs (n, n+1) of both rows with 8-byte accesses (W is
    // even, so every pair starts on an 8-byte boundary); the neighbouring column on the other
    // side of a pair is the adjacent lane's, passed by shuffle (lanes 0 and 31 of a chunk load
    // it).  Same arithmetic per element as one column at a time.
    const int NP = W / 2;
    if (g.phase == 0) {
        // dual step at both rows (Sec. II.A): p and q from u = D chibar and chibar's differences
        const bool down1 = (i1 + 1 < H);
        const float inv_den = g.inv_den_slice ? __ldg(g.inv_den_slice + s) : g.inv_den;
#pragma unroll 2
        for (int m0 = 0; m0 < NP; m0 += 32) {
            const int m = m0 + lane;
            const bool act = m < NP;
            const int n = 2 * (act ? m : NP - 1);  // inactive lanes shadow the last pair (no stores)
            const size_t a0 = r0 + n, a1 = r1 + n;
            const float4 uv = *reinterpret_cast<const float4*>(u + n);  // u[n], u[n+1]
            const float2 c0 = __ldcg(reinterpret_cast<const float2*>(cbar + a0));
            const float2 c1 = __ldcg(reinterpret_cast<const float2*>(cbar + a1));
            float c0r = __shfl_down_sync(0xffffffffu, c0.x, 1);  // column n+2 of row i0
            float c1r = __shfl_down_sync(0xffffffffu, c1.x, 1);
            if (n + 2 >= W) {  // past the last column the difference is zero (Neumann)
                c0r = c0.y;
                c1r = c1.y;
            } else if (lane == 31 || m + 1 >= NP) {
                c0r = __ldcg(cbar + a0 + 2);
                c1r = __ldcg(cbar + a1 + 2);
            }
            const float2 c2 = down1 ? __ldcg(reinterpret_cast<const float2*>(cbar + a1 + W)) : c1;
            const uchar2 mk0 = __ldg(reinterpret_cast<const uchar2*>(msk + a0));
            const uchar2 mk1 = __ldg(reinterpret_cast<const uchar2*>(msk + a1));
            const float m00 = (float)mk0.x, m01 = (float)mk0.y, m10 = (float)mk1.x, m11 = (float)mk1.y;
            float2 w0 = make_float2(m00, m01), w1 = make_float2(m10, m11);
            if (wgt) {
                w0 = __ldg(reinterpret_cast<const float2*>(wgt + a0));
                w1 = __ldg(reinterpret_cast<const float2*>(wgt + a1));
            }
            const float2 f0 = __ldg(reinterpret_cast<const float2*>(fld + a0));
            const float2 f1 = __ldg(reinterpret_cast<const float2*>(fld + a1));
            const float2 pa = __ldcg(reinterpret_cast<const float2*>(pp + a0));
            const float2 pb = __ldcg(reinterpret_cast<const float2*>(pp + a1));
            const float2 qxa = __ldcg(reinterpret_cast<const float2*>(qxp + a0));
            const float2 qxb = __ldcg(reinterpret_cast<const float2*>(qxp + a1));
            const float2 qya = __ldcg(reinterpret_cast<const float2*>(qyp + a0));
            const float2 qyb = __ldcg(reinterpret_cast<const float2*>(qyp + a1));
            // column n: (row i0, row i1) = (uv.x, uv.y); column n+1: (uv.z, uv.w)
            const float p00 = (pa.x + sigma * (w0.x * (uv.x - f0.x))) * inv_den;
            const float p10 = (pb.x + sigma * (w1.x * (uv.y - f1.x))) * inv_den;
            const float p01 = (pa.y + sigma * (w0.y * (uv.z - f0.y))) * inv_den;
            const float p11 = (pb.y + sigma * (w1.y * (uv.w - f1.y))) * inv_den;
            float qx00 = qxa.x + sigma * m00 * (c0.y - c0.x);
            float qy00 = qya.x + sigma * m00 * (c1.x - c0.x);
            float qx10 = qxb.x + sigma * m10 * (c1.y - c1.x);
            float qy10 = qyb.x + sigma * m10 * (c2.x - c1.x);
            float qx01 = qxa.y + sigma * m01 * (c0r - c0.y);
            float qy01 = qya.y + sigma * m01 * (c1.y - c0.y);
            float qx11 = qxb.y + sigma * m11 * (c1r - c1.y);
            float qy11 = qyb.y + sigma * m11 * (c2.y - c1.y);
            tv_prox(qx00, qy00, g.tv_iso);
            tv_prox(qx10, qy10, g.tv_iso);
            tv_prox(qx01, qy01, g.tv_iso);
            tv_prox(qx11, qy11, g.tv_iso);
            if (act) {
                __stcg(reinterpret_cast<float2*>(pp + a0), make_float2(p00, p01));
                __stcg(reinterpret_cast<float2*>(pp + a1), make_float2(p10, p11));
                __stcg(reinterpret_cast<float2*>(qxp + a0), make_float2(qx00, qx01));
                __stcg(reinterpret_cast<float2*>(qyp + a0), make_float2(qy00, qy01));
                __stcg(reinterpret_cast<float2*>(qxp + a1), make_float2(qx10, qx11));
                __stcg(reinterpret_cast<float2*>(qyp + a1), make_float2(qy10, qy11));
                // W p, transformed next
                *reinterpret_cast<float4*>(o + n) = make_float4(w0.x * p00, w1.x * p10, w0.y * p01, w1.y * p11);
            }
        }
    } else {
        // primal step: chi+ = chi - tau (v + G^T q), v = D W p; chibar = 2 chi+ - chi.
        // q is zero wherever the 0/1 mask is (zero start, masked increments), so M q = q.
        const bool up0 = (i0 > 0), down1 = (i1 + 1 < H);
#pragma unroll 2
        for (int m0 = 0; m0 < NP; m0 += 32) {
            const int m = m0 + lane;
            const bool act = m < NP;
            const int n = 2 * (act ? m : NP - 1);
            const size_t a0 = r0 + n, a1 = r1 + n;
            const float4 vv = *reinterpret_cast<const float4*>(u + n);
            const float2 qxa = __ldcg(reinterpret_cast<const float2*>(qxp + a0));
            const float2 qxb = __ldcg(reinterpret_cast<const float2*>(qxp + a1));
            const float2 qya = __ldcg(reinterpret_cast<const float2*>(qyp + a0));
            const float2 qyb = __ldcg(reinterpret_cast<const float2*>(qyp + a1));
            float qxl0 = __shfl_up_sync(0xffffffffu, qxa.y, 1);  // column n-1
            float qxl1 = __shfl_up_sync(0xffffffffu, qxb.y, 1);
            if (n == 0) {
                qxl0 = 0.f;
                qxl1 = 0.f;
            } else if (lane == 0) {
                qxl0 = __ldcg(qxp + a0 - 1);
                qxl1 = __ldcg(qxp + a1 - 1);
            }
            const float2 qyu = up0 ? __ldcg(reinterpret_cast<const float2*>(qyp + a0 - W)) : make_float2(0.f, 0.f);
            const bool last_col = (n + 2 == W);  // column n+1 is the last
            // column n (never the last: n <= W - 2)
            const float d00 = (qxl0 - qxa.x) + (qyu.x - qya.x);
            const float d10 = (qxl1 - qxb.x) + (qya.x - (down1 ? qyb.x : 0.f));
            // column n+1
            const float d01 = (qxa.x - (last_col ? 0.f : qxa.y)) + (qyu.y - qya.y);
            const float d11 = (qxb.x - (last_col ? 0.f : qxb.y)) + (qya.y - (down1 ? qyb.y : 0.f));
            const float2 ca = __ldcg(reinterpret_cast<const float2*>(chi + a0));
            const float2 cb2 = __ldcg(reinterpret_cast<const float2*>(chi + a1));
            const float n00 = ca.x - tau * vv.x - tau * d00;
            const float n10 = cb2.x - tau * vv.y - tau * d10;
            const float n01 = ca.y - tau * vv.z - tau * d01;
            const float n11 = cb2.y - tau * vv.w - tau * d11;
            const float b00 = 2.f * n00 - ca.x, b10 = 2.f * n10 - cb2.x;
            const float b01 = 2.f * n01 - ca.y, b11 = 2.f * n11 - cb2.y;
            if (act) {
                __stcg(reinterpret_cast<float2*>(chi + a0), make_float2(n00, n01));
                __stcg(reinterpret_cast<float2*>(chi + a1), make_float2(n10, n11));
                __stcg(reinterpret_cast<float2*>(cbar + a0), make_float2(b00, b01));
                __stcg(reinterpret_cast<float2*>(cbar + a1), make_float2(b10, b11));
                *reinterpret_cast<float4*>(o + n) = make_float4(b00, b10, b01, b11);
            }
        }
    }
    __syncwarp();
    if (g.phase == 0 || g.store) {
        float2* Z = warp_dft(o, u, T, g.prow, false, lane);
        // split: A = (Z(k) + conj Z(-k)) / 2, B = (Z(k) - conj Z(-k)) / (2 i)
#pragma unroll 3
        for (int k = lane; k < M1; k += 32) {
            const float2 zk = Z[k], zm = Z[k == 0 ? 0 : W - k];
            __stcg(sp0 + k, make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y)));
            __stcg(sp1 + k, make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x)));
        }
    }
}

// ------------------------------------------------------------------ FP64 diagnostics
// The terms of the per-slice report at (chi, p, q), per row pair (summed by the host):
//   [0] ||W (D chi - dB)||^2   [1] TV norm of M G chi   [2] ||p - lambda W (D chi - dB)||^2
//   [3] sum(|g| - q.g), g = M G chi   [4] ||D W p + G^T M q||^2
// Three launches with column passes between them: mode 0 forward transforms of chi;
// mode 1 D chi -> terms 0-3, forward transforms of W p; mode 2 D W p -> term 4.
constexpr int kGenReportSums = 5;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;  // lane 0
}

// Two real rows (a: row i0, b: row i1) packed as a + i b -> forward DFT -> half-spectrum rows.
__device__ __forceinline__ void gen_store_rows(float2* o, float2* scratch, const float2* T, const GenParams& g,
                                               float2* sp0, float2* sp1, int lane) {
    const int W = g.W;
    float2* Z = warp_dft(o, scratch, T, g.prow, false, lane);
#pragma unroll 3
    for (int k = lane; k < g.M1; k += 32) {
        const float2 zk = Z[k], zm = Z[k == 0 ? 0 : W - k];
        __stcg(sp0 + k, make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y)));
        __stcg(sp1 + k, make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x)));
    }
}

__global__ void __launch_bounds__(kGenRowWarps * 32) gen_report_kernel(GenParams g, double* partial, double lam,
                                                                        int mode) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = g.H, W = g.W, M1 = g.M1;
    float2* T = reinterpret_cast<float2*>(smem_raw);
    for (int t = threadIdx.x; t < W; t += blockDim.x) T[t] = g.trow[t];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pair = blockIdx.x * kGenRowWarps + warp;
    if (pair >= g.S * (H / 2)) return;  // whole warps; no CTA barrier below
    float2* bufa = T + W + (size_t)warp * 2 * W;
    float2* bufb = bufa + W;
    const int s = pair / (H / 2);
    const int i0 = 2 * (pair - s * (H / 2)), i1 = i0 + 1;
    const size_t r0 = ((size_t)s * H + i0) * W, r1 = r0 + W;
    float2* sp0 = g.spec + ((size_t)s * H + i0) * M1;
    float2* sp1 = sp0 + M1;
    if (mode == 0) {
        for (int n = lane; n < W; n += 32) bufa[n] = make_float2(__ldcg(g.chi + r0 + n), __ldcg(g.chi + r1 + n));
        __syncwarp();
        gen_store_rows(bufa, bufb, T, g, sp0, sp1, lane);
        return;
    }
    for (int k = lane; k < W; k += 32) {
        float2 z;
        if (k < M1) {
            const float2 A = __ldcg(sp0 + k), B = __ldcg(sp1 + k);
            z = make_float2(A.x - B.y, A.y + B.x);
        } else {
            const float2 A = __ldcg(sp0 + (W - k)), B = __ldcg(sp1 + (W - k));
            z = make_float2(A.x + B.y, B.x - A.y);
        }
        bufa[k] = z;
    }
    __syncwarp();
    float2* u = warp_dft(bufa, bufb, T, g.prow, true, lane);  // D chi (mode 1) or D W p (mode 2)
    float2* o = (u == bufa) ? bufb : bufa;
    double acc[kGenReportSums] = {0, 0, 0, 0, 0};
    for (int n = lane; n < W; n += 32) {
        const float2 uv = u[n];
        const float us[2] = {uv.x, uv.y};
        const int rows[2] = {i0, i1};
        float wp[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int i = rows[t];
            const size_t a = (t == 0 ? r0 : r1) + n;
            const double m = (double)__ldg(g.mask + a);
            const double w = g.weight ? (double)__ldg(g.weight + a) : m;
            const double qx = __ldcg(g.qx + a), qy = __ldcg(g.qy + a);
            if (mode == 1) {
                const double c = __ldcg(g.chi + a);
                const double gx = (n + 1 < W) ? m * ((double)__ldcg(g.chi + a + 1) - c) : 0.0;
                const double gy = (i + 1 < H) ? m * ((double)__ldcg(g.chi + a + W) - c) : 0.0;
                const double r = w * ((double)us[t] - (double)__ldg(g.field + a));
                const double p = __ldcg(g.p + a);
                const double tvn = g.tv_iso ? sqrt(gx * gx + gy * gy) : fabs(gx) + fabs(gy);
                acc[0] += r * r;
                acc[1] += tvn;
                acc[2] += (p - lam * r) * (p - lam * r);
                acc[3] += tvn - (qx * gx + qy * gy);
                wp[t] = (float)(w * p);
            } else {
                // G^T (M q): (a[j-1] - a[j] [j < W-1]) + (b[i-1] - b[i] [i < H-1]), a = M qx, b = M qy
                double k = us[t];
                if (n > 0) k += (double)__ldg(g.mask + a - 1) * (double)__ldcg(g.qx + a - 1);
                if (n + 1 < W) k -= m * qx;
                if (i > 0) k += (double)__ldg(g.mask + a - W) * (double)__ldcg(g.qy + a - W);
                if (i + 1 < H) k -= m * qy;
                acc[4] += k * k;
                wp[t] = 0.f;
            }
        }
        o[n] = make_float2(wp[0], wp[1]);
    }
    __syncwarp();
    double* out = partial + (size_t)pair * kGenReportSums;
#pragma unroll
    for (int t = 0; t < kGenReportSums; ++t) {
        const double v = warp_sum_d(acc[t]);
        if (lane == 0 && ((mode == 1 && t < 4) || (mode == 2 && t == 4))) out[t] = v;
    }
    if (mode == 1) gen_store_rows(o, u, T, g, sp0, sp1, lane);
}

// ------------------------------------------------------------------ power iteration for L = ||K||
// Per slice, x <- K^T K x / ||K^T K x|| with K^T K x = D M^2 D x + G^T M^2 G x (W = M = mask).
// The stored vector is unnormalised; scale[s] turns it into the unit vector.  Per iteration:
// mode 0 forward transforms of scale x; column pass; mode 1 D x -> M^2 D x -> forward;
// column pass; mode 2 y = D M^2 D x + G^T M^2 G x with <x, y> and ||y||^2 per row pair;
// then gen_opnorm_norm_kernel: est = <x, y>, scale = 1 / ||y||.

// Deterministic start vector in [-1, 1) from the voxel index (splitmix64 finaliser).
__device__ __forceinline__ float gen_hash_unit(unsigned long long k) {
    k += 0x9E3779B97F4A7C15ull;
    k = (k ^ (k >> 30)) * 0xBF58476D1CE4E5B9ull;
    k = (k ^ (k >> 27)) * 0x94D049BB133111EBull;
    k ^= k >> 31;
    return (float)((double)(k >> 40) * (1.0 / 8388608.0) - 1.0);
}

__global__ void __launch_bounds__(kGenRowWarps * 32) gen_opnorm_init_kernel(GenParams g, float* x, double* partial) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pair = blockIdx.x * kGenRowWarps + warp;
    if (pair >= g.S * (g.H / 2)) return;
    const size_t r0 = (size_t)pair * 2 * g.W;  // rows 2 pr, 2 pr + 1 of the slices laid end to end
    double nn = 0.0;
    for (int n = lane; n < 2 * g.W; n += 32) {
        const float v = gen_hash_unit(r0 + n);
        x[r0 + n] = v;
        nn += (double)v * v;
    }
    nn = warp_sum_d(nn);
    if (lane == 0) {
        partial[2 * (size_t)pair] = 0.0;
        partial[2 * (size_t)pair + 1] = nn;
    }
}

// est[s] = sum of the slice's <x, y> partials, scale[s] = 1 / sqrt(sum of ||y||^2), fixed order.
__global__ void gen_opnorm_norm_kernel(const double* partial, int pairs_per_slice, int S, float* scale,
                                       double* est) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    double xy = 0.0, yy = 0.0;
    for (int q = 0; q < pairs_per_slice; ++q) {
        xy += partial[2 * ((size_t)s * pairs_per_slice + q)];
        yy += partial[2 * ((size_t)s * pairs_per_slice + q) + 1];
    }
    est[s] = xy;
    scale[s] = (yy > 0.0) ? (float)(1.0 / sqrt(yy)) : 0.f;
}

__global__ void __launch_bounds__(kGenRowWarps * 32) gen_opnorm_rows_kernel(GenParams g, const float* x, float* y,
                                                                             const float* scale, double* partial,
                                                                             int mode) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = g.H, W = g.W, M1 = g.M1;
    float2* T = reinterpret_cast<float2*>(smem_raw);
    for (int t = threadIdx.x; t < W; t += blockDim.x) T[t] = g.trow[t];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pair = blockIdx.x * kGenRowWarps + warp;
    if (pair >= g.S * (H / 2)) return;  // whole warps; no CTA barrier below
    float2* bufa = T + W + (size_t)warp * 2 * W;
    float2* bufb = bufa + W;
    const int s = pair / (H / 2);
    const int i0 = 2 * (pair - s * (H / 2)), i1 = i0 + 1;
    const size_t r0 = ((size_t)s * H + i0) * W, r1 = r0 + W;
    float2* sp0 = g.spec + ((size_t)s * H + i0) * M1;
    float2* sp1 = sp0 + M1;
    const float sc = scale[s];
    if (mode == 0) {
        for (int n = lane; n < W; n += 32) bufa[n] = make_float2(sc * x[r0 + n], sc * x[r1 + n]);
        __syncwarp();
        gen_store_rows(bufa, bufb, T, g, sp0, sp1, lane);
        return;
    }
    for (int k = lane; k < W; k += 32) {
        float2 z;
        if (k < M1) {
            const float2 A = __ldcg(sp0 + k), B = __ldcg(sp1 + k);
            z = make_float2(A.x - B.y, A.y + B.x);
        } else {
            const float2 A = __ldcg(sp0 + (W - k)), B = __ldcg(sp1 + (W - k));
            z = make_float2(A.x + B.y, B.x - A.y);
        }
        bufa[k] = z;
    }
    __syncwarp();
    float2* u = warp_dft(bufa, bufb, T, g.prow, true, lane);
    float2* o = (u == bufa) ? bufb : bufa;
    if (mode == 1) {
        for (int n = lane; n < W; n += 32) {
            const float m0 = (float)__ldg(g.mask + r0 + n), m1 = (float)__ldg(g.mask + r1 + n);
            o[n] = make_float2(u[n].x * m0 * m0, u[n].y * m1 * m1);
        }
        __syncwarp();
        gen_store_rows(o, u, T, g, sp0, sp1, lane);
        return;
    }
    // mode 2: y = D M^2 D x + G^T M^2 G x at rows i0, i1
    auto X = [&](size_t idx) { return sc * x[idx]; };
    auto M2 = [&](size_t idx) {
        const float m = (float)__ldg(g.mask + idx);
        return m * m;
    };
    const size_t sbase = (size_t)s * H * W;
    auto ax = [&](int ii, int jj) -> float {  // M^2 gx at (ii, jj)
        if (jj < 0 || jj >= W - 1) return 0.f;
        const size_t q = sbase + (size_t)ii * W + jj;
        return M2(q) * (X(q + 1) - X(q));
    };
    auto by = [&](int ii, int jj) -> float {  // M^2 gy at (ii, jj)
        if (ii < 0 || ii >= H - 1) return 0.f;
        const size_t q = sbase + (size_t)ii * W + jj;
        return M2(q) * (X(q + W) - X(q));
    };
    double xy = 0.0, yy = 0.0;
    for (int n = lane; n < W; n += 32) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int i = t == 0 ? i0 : i1;
            const size_t q = (t == 0 ? r0 : r1) + n;
            const float gt = (ax(i, n - 1) - ax(i, n)) + (by(i - 1, n) - by(i, n));
            const float v = (t == 0 ? u[n].x : u[n].y) + gt;
            y[q] = v;
            xy += (double)X(q) * v;
            yy += (double)v * v;
        }
    }
    xy = warp_sum_d(xy);
    yy = warp_sum_d(yy);
    if (lane == 0) {
        partial[2 * (size_t)pair] = xy;
        partial[2 * (size_t)pair + 1] = yy;
    }
}

__device__ __forceinline__ float gen_freq(int k, int n) { return (float)(k < (n + 1) / 2 ? k : k - n) / (float)n; }

// Column kernel: CTA (tile of kGenColTile spectrum columns, slice); one warp per column.
// Column c's two buffers start at c (2H + 1): the odd stride puts the tile's
// columns on distinct banks for the row-wise load and store.
__global__ void __launch_bounds__(kGenColTile * 32) gen_cols_kernel(GenParams g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = g.H, W = g.W, M1 = g.M1;
    const int CS = 2 * H + 1;
    float2* T = reinterpret_cast<float2*>(smem_raw);
    float2* cols = T + H;  // [kGenColTile][CS]
    const int kx0 = blockIdx.x * kGenColTile, s = blockIdx.y;
    const int ncol = min(kGenColTile, M1 - kx0);
    float2* spec = g.spec + (size_t)s * H * M1;
    for (int t = threadIdx.x; t < H; t += blockDim.x) T[t] = g.tcol[t];
    grid_dependency_wait();  // the previous launch's spectrum complete
    // rows of the tile: adjacent threads take adjacent columns
    const int c = threadIdx.x % kGenColTile;
    const int ky0 = threadIdx.x / kGenColTile;
    constexpr int KY_STEP = kGenColTile * 32 / kGenColTile;  // rows per sweep of the CTA
    if (c < ncol) {
        const float2* src = spec + kx0 + c;
#pragma unroll 4
        for (int ky = ky0; ky < H; ky += KY_STEP) cols[(size_t)c * CS + ky] = __ldcg(src + (size_t)ky * M1);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < ncol) {
        const int kx = kx0 + warp;
        float2* a = cols + (size_t)warp * CS;
        float2* b = a + H;
        float2* X = warp_dft(a, b, T, g.pcol, false, lane);
        const float fx = (float)kx / (float)W;
        const float scale = 1.0f / ((float)H * (float)W);
#pragma unroll 1
        for (int ky = lane; ky < H; ky += 32) {
            const float fy = gen_freq(ky, H);
            const float k2 = fx * fx + fy * fy;
            const float fb = g.b0_axis ? fx : fy;
            const float d = (k2 > 0.f) ? (1.0f / 3.0f - (fb * fb) / k2) * scale : 0.f;
            X[ky] = make_float2(X[ky].x * d, X[ky].y * d);
        }
        __syncwarp();
        // both directions swap the buffers equally often: the result is back in a
        warp_dft(X, X == a ? b : a, T, g.pcol, true, lane);
    }
    __syncthreads();
    if (c < ncol) {
        float2* dst = spec + kx0 + c;
#pragma unroll 4
        for (int ky = ky0; ky < H; ky += KY_STEP) __stcg(dst + (size_t)ky * M1, cols[(size_t)c * CS + ky]);
    }
}

// Column pass for H with a compiled register FFT (64·2^k, 3·2^k up to 512):
// pencils of TZ = H / EZ lanes, one per spectrum column; a CTA takes TY adjacent
// columns of one slice, so lanes of adjacent pencils read adjacent addresses.
template <int H>
struct GeoCol {
    static constexpr int EZ = default_elems(H);
    static constexpr int TZ = H / EZ;
    static constexpr int PPW = 32 / TZ;         // pencils per warp
    static constexpr int NT = 128;              // 4 warps: more CTAs in flight (measured 4% faster than 8)
    static constexpr int TY = (NT / 32) * PPW;  // columns per CTA
    static constexpr int NP = H + (TZ % 16);    // pencil buffer stride
    static constexpr size_t SMEM_BYTES = sizeof(float2) * (TY * NP + StageTw<H, EZ>::SIZE);
};

template <int H>
__global__ void __launch_bounds__(GeoCol<H>::NT) gen_cols_fft_kernel(GenParams g) {
    using GC = GeoCol<H>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TZ = GC::TZ, EZ = GC::EZ;
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* stw = buf + GC::TY * GC::NP;
    StageTw<H, EZ>::fill(stw, g.tcol, 1, threadIdx.x, GC::NT);
    __syncthreads();
    grid_dependency_wait();  // the previous launch's spectrum complete
    const int W = g.W, M1 = g.M1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane % TZ;
    const int pen = warp * GC::PPW + lane / TZ;
    const unsigned gm = group_mask<TZ>(lane);
    const int kx_raw = blockIdx.x * GC::TY + pen;
    const bool live = kx_raw < M1;
    const int kx = live ? kx_raw : M1 - 1;  // idle pencils repeat the last column, store nothing
    float2* col = g.spec + (size_t)blockIdx.y * H * M1 + kx;
    float2* pb = buf + pen * GC::NP;
    float2 x[EZ];
#pragma unroll
    for (int e = 0; e < EZ; ++e) x[e] = __ldcg(col + (size_t)(gi + TZ * e) * M1);
    fft<H, TZ, false>(x, pb, stw, gi, gm);
    const float fx = (float)kx / (float)W;
    const float scale = 1.0f / ((float)H * (float)W);
#pragma unroll
    for (int e = 0; e < EZ; ++e) {
        const float fy = gen_freq(gi + TZ * e, H);
        const float k2 = fx * fx + fy * fy;
        const float fb = g.b0_axis ? fx : fy;
        const float d = (k2 > 0.f) ? (1.0f / 3.0f - (fb * fb) / k2) * scale : 0.f;
        x[e] = make_float2(x[e].x * d, x[e].y * d);
    }
    fft<H, TZ, true>(x, pb, stw, gi, gm);
    if (live) {
#pragma unroll
        for (int e = 0; e < EZ; ++e) __stcg(col + (size_t)(gi + TZ * e) * M1, x[e]);
    }
}

}  // namespace pcs
