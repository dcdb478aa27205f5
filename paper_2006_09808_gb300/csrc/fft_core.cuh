// fft_core.cuh -- warp-group complex FFT engine for the dipole convolution.
//
// One 1-D transform of length N is carried by a group of T lanes of one warp
// (T <= 32), E = N / T complex elements per lane.  Register order: lane g of
// the group holds element  g + T*e  in x[e], both on input (natural order) and
// on output (natural-order spectrum).  That shared order is what lets the
// solver fuse its pointwise steps between an inverse and a forward transform
// without moving data.
//
// The transform is a Stockham autosort radix-R factorisation (radices 16, 8,
// 4, 2): each stage reads its butterfly inputs at stride N/R, applies the
// twiddles W_{Ns R}^{r k}, a register DFT_R, and writes to the next stage's
// natural position; the group exchanges through a shared-memory buffer
// between stages.  Swizzle: element i lives at P(i, key) = i ^ ((i/16 + key)
// mod 16), a permutation inside each aligned block of 16 that puts the
// strided stores of a stage (16 j + r over lanes j) and the natural-order
// accesses (g + 16 e over lanes g) on distinct banks without padding, and
// keeps every aligned run of 4 elements inside one 32-byte sector.  key
// varies the pattern between buffers (columns use 4 x their index, so that 8
// adjacent columns read at 4 adjacent rows hit every bank exactly twice).
//
// Twiddles come from per-stage tables in shared memory laid out [r-1][k]
// (entry W_{Ns R}^{r k}), so the lanes of a group, which hold consecutive k,
// read consecutive words: no bank conflicts.  The tables are copied at kernel
// start from the master table tw[m] = exp(-2 pi i m / NTW) (host FP64, rounded
// to FP32).  Inverse transforms use conjugates and are unnormalised.
#pragma once

#include <cuda_runtime.h>

namespace pcs {

__device__ __forceinline__ int P(int i, int key = 0) { return i ^ (((i >> 4) + key) & 15); }

// Complex vector type of a real type: float -> float2, double -> double2.
template <class Real>
struct Cplx;
template <>
struct Cplx<float> {
    using T = float2;
};
template <>
struct Cplx<double> {
    using T = double2;
};
template <class V>
using RealOf = decltype(V::x);

template <class V>
__device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <class V>
__device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <class V>
__device__ __forceinline__ V cmul(V a, V b) {
    return V{fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)};
}
template <class V>
__device__ __forceinline__ V cscale(V a, RealOf<V> s) { return V{a.x * s, a.y * s}; }
template <class V>
__device__ __forceinline__ V conjf2(V a) { return V{a.x, -a.y}; }

// multiply by -i (forward) or +i (inverse)
template <bool INV, class V>
__device__ __forceinline__ V mul_mi(V a) {
    return INV ? V{-a.y, a.x} : V{a.y, -a.x};
}

// multiply by the constant (c, s) with s given for the forward sign; INV flips it
template <bool INV, class V>
__device__ __forceinline__ V mul_const(V a, RealOf<V> c, RealOf<V> s) {
    const RealOf<V> ss = INV ? -s : s;
    return V{fma(a.x, c, -a.y * ss), fma(a.x, ss, a.y * c)};
}

// cos / sin of 2*pi*k/16 (forward twiddles are (cos, -sin)), rounded once to the real type
constexpr double kC1 = 0.92387953251128675613;  // cos(pi/8)
constexpr double kS1 = 0.38268343236508977173;  // sin(pi/8)
constexpr double kR2 = 0.70710678118654752440;  // sqrt(1/2)

template <bool INV, class V>
__device__ __forceinline__ void dft2(V& a, V& b) {
    const V t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <bool INV, class V>
__device__ __forceinline__ void dft4(V& v0, V& v1, V& v2, V& v3) {
    const V t0 = cadd(v0, v2), t1 = csub(v0, v2);
    const V t2 = cadd(v1, v3), t3 = mul_mi<INV>(csub(v1, v3));
    v0 = cadd(t0, t2);
    v2 = csub(t0, t2);
    v1 = cadd(t1, t3);
    v3 = csub(t1, t3);
}

// in-place, natural order in and out
template <bool INV, class V>
__device__ __forceinline__ void dft8(V (&v)[8]) {
    using Rl = RealOf<V>;
    V e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    V o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = mul_const<INV>(o1, Rl(kR2), Rl(-kR2));
    o2 = mul_mi<INV>(o2);
    o3 = mul_const<INV>(o3, Rl(-kR2), Rl(-kR2));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

template <bool INV, class V>
__device__ __forceinline__ void dft16(V (&v)[16]) {
    using Rl = RealOf<V>;
    V e[8], o[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        e[t] = v[2 * t];
        o[t] = v[2 * t + 1];
    }
    dft8<INV>(e);
    dft8<INV>(o);
    // W16^k = (cos(2 pi k/16), -sin(2 pi k/16)) forward
    o[1] = mul_const<INV>(o[1], Rl(kC1), Rl(-kS1));
    o[2] = mul_const<INV>(o[2], Rl(kR2), Rl(-kR2));
    o[3] = mul_const<INV>(o[3], Rl(kS1), Rl(-kC1));
    o[4] = mul_mi<INV>(o[4]);
    o[5] = mul_const<INV>(o[5], Rl(-kS1), Rl(-kC1));
    o[6] = mul_const<INV>(o[6], Rl(-kR2), Rl(-kR2));
    o[7] = mul_const<INV>(o[7], Rl(-kC1), Rl(-kS1));
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        v[t] = cadd(e[t], o[t]);
        v[t + 8] = csub(e[t], o[t]);
    }
}

// DFT_3: with w = exp(-2 pi i/3) (forward), X1,2 = a - (b+c)/2 -/+ i (sqrt3/2)(b - c)
constexpr double kH3 = 0.86602540378443864676;  // sqrt(3)/2
template <bool INV, class V>
__device__ __forceinline__ void dft3(V& a, V& b, V& c) {
    using Rl = RealOf<V>;
    const V t1 = cadd(b, c);
    const V t2 = V{fma(Rl(-0.5), t1.x, a.x), fma(Rl(-0.5), t1.y, a.y)};
    const V t3 = cscale(mul_mi<INV>(csub(b, c)), Rl(kH3));
    a = cadd(a, t1);
    b = cadd(t2, t3);
    c = csub(t2, t3);
}

// cos and sin of 2 pi m / 24, m = 0..23 (multiples of 15 degrees)
__device__ __forceinline__ constexpr double cos24(int m) {
    constexpr double c[6] = {1.0, 0.96592582628906828675, 0.86602540378443864676,
                             0.70710678118654752440, 0.5, 0.25881904510252076235};
    m %= 24;
    if (m < 6) return c[m];
    if (m == 6) return 0.0;
    if (m < 12) return -c[12 - m];
    if (m < 18) return -c[m - 12];
    if (m == 18) return 0.0;
    return c[24 - m];
}
__device__ __forceinline__ constexpr double sin24(int m) { return cos24(m + 18); }  // sin x = cos(x - 90 deg)

template <int R, bool INV, class V>
__device__ __forceinline__ void dftR(V (&v)[R]);

// Composite DFT of length R = P*Q (Cooley-Tukey in registers): n = Q n1 + n2,
// k = k1 + P k2; P-point DFTs over n1, twiddles W_R^{n2 k1}, Q-point DFTs over n2.
// R divides 24 here, so every twiddle is a multiple of 15 degrees.
template <int P, int Q, bool INV, class V>
__device__ __forceinline__ void dft_composite(V (&v)[P * Q]) {
    using Rl = RealOf<V>;
    constexpr int R = P * Q;
    static_assert(24 % R == 0, "composite radix must divide 24");
    V y[Q][P];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) {
        V t[P];
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) t[n1] = v[Q * n1 + n2];
        dftR<P, INV>(t);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            const int m = (n2 * k1 * (24 / R)) % 24;  // compile-time after unrolling
            if (m == 0) {
                y[n2][k1] = t[k1];
            } else {
                y[n2][k1] = mul_const<INV>(t[k1], Rl(cos24(m)), Rl(-sin24(m)));
            }
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
        V t[Q];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) t[n2] = y[n2][k1];
        dftR<Q, INV>(t);
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = t[k2];
    }
}

template <int R, bool INV, class V>
__device__ __forceinline__ void dftR(V (&v)[R]) {
    if constexpr (R == 2) {
        dft2<INV>(v[0], v[1]);
    } else if constexpr (R == 3) {
        dft3<INV>(v[0], v[1], v[2]);
    } else if constexpr (R == 4) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 6) {
        dft_composite<2, 3, INV, V>(v);
    } else if constexpr (R == 8) {
        dft8<INV>(v);
    } else if constexpr (R == 12) {
        dft_composite<4, 3, INV, V>(v);
    } else if constexpr (R == 24) {
        dft_composite<8, 3, INV, V>(v);
    } else {
        static_assert(R == 16, "radix");
        dft16<INV>(v);
    }
}

// Radix plans: R1 first, RL last, RM middle (0 = two stages only).
template <int N, int E>
struct Plan;
template <> struct Plan<32, 8>   { static constexpr int R1 = 8,  RM = 0,  RL = 4; };
template <> struct Plan<64, 8>   { static constexpr int R1 = 8,  RM = 0,  RL = 8; };
template <> struct Plan<128, 16> { static constexpr int R1 = 16, RM = 0,  RL = 8; };
template <> struct Plan<256, 16> { static constexpr int R1 = 16, RM = 0,  RL = 16; };
template <> struct Plan<512, 16> { static constexpr int R1 = 16, RM = 16, RL = 2; };
// eight elements per lane: three radix-8 based stages
template <> struct Plan<128, 8>  { static constexpr int R1 = 8,  RM = 8,  RL = 2; };
template <> struct Plan<256, 8>  { static constexpr int R1 = 8,  RM = 8,  RL = 4; };
template <> struct Plan<512, 8>  { static constexpr int R1 = 8,  RM = 8,  RL = 8; };
// lengths 3 * 2^k (slice sizes 192 and 384)
template <> struct Plan<96, 12>  { static constexpr int R1 = 12, RM = 4,  RL = 2; };
template <> struct Plan<192, 12> { static constexpr int R1 = 12, RM = 4,  RL = 4; };
template <> struct Plan<384, 24> { static constexpr int R1 = 8,  RM = 8,  RL = 6; };

// Elements per lane for a transform of length N: 16 for powers of two >= 128,
// 8 below; 12 for 96 and 192; 24 for 384 (so that N / E lanes is a power of two).
constexpr int default_elems(int N) {
    return (N % 3 == 0) ? (N == 384 ? 24 : 12) : (N >= 128 ? 16 : 8);
}

// Per-stage twiddle tables of one transform length: the middle stage's
// (span R1, radix RM) entries first, then the last stage's (span N/RL, radix RL).
template <int N, int E>
struct StageTw {
    using PL = Plan<N, E>;
    static constexpr int MID = PL::RM ? (PL::RM - 1) * PL::R1 : 0;
    static constexpr int LAST = (PL::RL - 1) * (N / PL::RL);
    static constexpr int SIZE = MID + LAST;
    // dst[(r-1) NS + k] = W_{NS R}^{r k} = tw[r k (N / (NS R)) TWS], TWS = NTW / N
    template <class V>
    __device__ static void fill(V* dst, const V* __restrict__ tw, int TWS, int tid, int nthr) {
        if constexpr (MID > 0) {
            constexpr int NS = PL::R1, R = PL::RM, STEP = N / (NS * R);
            for (int t = tid; t < MID; t += nthr) {
                const int r = t / NS + 1, k = t % NS;
                dst[t] = tw[(r * k * STEP) * TWS];
            }
        }
        {
            constexpr int NS = N / PL::RL, R = PL::RL, STEP = N / (NS * R);
            for (int t = tid; t < LAST; t += nthr) {
                const int r = t / NS + 1, k = t % NS;
                dst[MID + t] = tw[(r * k * STEP) * TWS];
            }
        }
    }
};

// Twiddle the legs of one butterfly of a stage with span NS and radix R
// (stw: that stage's [r-1][k] table).
template <int R, int NS, bool INV, class V>
__device__ __forceinline__ void twiddle(V (&v)[R], int j, const V* __restrict__ stw) {
    if constexpr (NS > 1) {
        const int k = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) {
            V w = stw[(r - 1) * NS + k];
            if (INV) w.y = -w.y;
            v[r] = cmul(v[r], w);
        }
    }
}

// Complex FFT of length N (a multiple of 16) by a group of T lanes (lane g,
// group mask gm).  x: E = N/T elements, element g + T*e in x[e]; buf:
// group-private buffer of N entries addressed through P(., key) (contents
// destroyed); stw: StageTw<N, E> table.
template <int N, int T, bool INV, class V>
__device__ __forceinline__ void fft(V (&x)[N / T], V* __restrict__ buf, const V* __restrict__ stw, int g,
                                    unsigned gm, int key = 0) {
    static_assert(N % 16 == 0, "swizzle blocks");
    constexpr int E = N / T;
    using PL = Plan<N, E>;
    constexpr int R1 = PL::R1, RM = PL::RM, RL = PL::RL;
    static_assert(E % R1 == 0 && E % RL == 0, "plan");
    static_assert(R1 * (RM ? RM : 1) * RL == N, "plan product");

    __syncwarp(gm);
    // ---- stage 1: radix R1, span 1, inputs from registers
    {
        constexpr int B = E / R1;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            V v[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = x[b + r * B];
            dftR<R1, INV, V>(v);
            const int j = g + b * T;
#pragma unroll
            for (int r = 0; r < R1; ++r) buf[P(j * R1 + r, key)] = v[r];
        }
    }
    __syncwarp(gm);
    // ---- optional middle stage: radix RM, span R1, in place through registers
    if constexpr (RM != 0) {
        constexpr int B = E / RM;
        constexpr int NS = R1;
        V v[B][RM];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int j = g + b * T;
#pragma unroll
            for (int r = 0; r < RM; ++r) v[b][r] = buf[P(j + r * (N / RM), key)];
        }
        __syncwarp(gm);
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int j = g + b * T;
            twiddle<RM, NS, INV, V>(v[b], j, stw);
            dftR<RM, INV, V>(v[b]);
            const int k = j % NS;
            const int base = (j / NS) * NS * RM + k;
#pragma unroll
            for (int r = 0; r < RM; ++r) buf[P(base + r * NS, key)] = v[b][r];
        }
        __syncwarp(gm);
    }
    // ---- last stage: radix RL, span N/RL, outputs to registers (natural order)
    {
        constexpr int B = E / RL;
        constexpr int NS = N / RL;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int j = g + b * T;
            V v[RL];
#pragma unroll
            for (int r = 0; r < RL; ++r) v[r] = buf[P(j + r * NS, key)];
            twiddle<RL, NS, INV, V>(v, j, stw + StageTw<N, E>::MID);
            dftR<RL, INV, V>(v);
#pragma unroll
            for (int r = 0; r < RL; ++r) x[b + r * B] = v[r];
        }
    }
    __syncwarp(gm);
}

}  // namespace pcs
