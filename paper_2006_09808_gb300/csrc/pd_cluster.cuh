// pd_cluster.cuh -- the fused primal-dual iteration: one thread-block cluster
// per slice, the slice's spectrum distributed over the cluster's shared
// memory, every step of the Sec. II.A pseudocode fused around the FFT passes.
//
// Data flow of one iteration for slice s (C CTAs; CTA c owns rows
// [c R, (c+1) R) of the slice and spectrum columns [c MC, (c+1) MC)):
//
//   column pass   (own spectrum columns)  F_y, x D(k)/(HW), F_y^-1         -> u-spectrum
//   cluster barrier
//   row phase B   (own rows)   gather row from all CTAs (DSMEM), real F_x^-1 -> u = D chibar
//                              p <- (p + sigma W (u - f)) / (1 + sigma/lambda)     dual data prox
//                              q <- clamp(q + sigma M G chibar)                   dual TV prox
//                              real F_x of W p, scatter row to all CTAs (DSMEM)
//   cluster barrier
//   column pass                                                            -> v-spectrum
//   cluster barrier
//   row phase A   (own rows)   gather, real F_x^-1 -> v = D W p
//                              chi+ = chi - tau v - tau G^T M q                 primal step
//                              chibar = 2 chi+ - chi                             over-relaxation
//                              real F_x of chibar, scatter (not on the last iteration)
//   cluster barrier
//
// The real row transforms use the half-length complex FFT of
// z[n] = x[2n] + i x[2n+1]; the packed row spectrum stores X[0] + i X[W/2] in
// column 0.  Splitting that FFT into the real row's spectrum (and merging it
// back) pairs column k with column M-k of the same row; in the lane layout of
// the transforms (lane g holds k = g + TR*e) the partner sits in lane TR-g at
// element ER-1-e (lane 0: its own element ER-e), so the pairing is a warp
// shuffle.  The column pass handles that packed column by pairing ky with -ky
// (both halves are spectra of real columns):
//   Y[ky] = Dm[ky] C[ky] + Dd[ky] conj(C[-ky]),  Dm,Dd = (D(ky,0) +- D(ky,W/2))/2.
// All normalisation (1/(H W)) is folded into the D table.
//
// State (chi = the caller's chi_out, chibar, p, qx, qy) stays in global
// memory (L2/HBM) and is touched once per phase; the FFT intermediates never
// leave the chip.  The kernel is persistent: a cluster loops over slices
// s = cluster_id, cluster_id + n_clusters, ..., or, with more slices than
// clusters, over the segments of the balanced schedule (pd_cluster_kernel).
// There is no grid-wide synchronisation; apart from hardware cluster barriers
// the only wait is the schedule's bounded wait for a slice's first part.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fft_core.cuh"

namespace pcs {

namespace cg = cooperative_groups;

template <class Real>
struct PDParamsT {
    using V = typename Cplx<Real>::T;
    const Real* field;          // [S][H][W]
    const unsigned char* mask;  // [S][H][W]
    Real* chi;                  // [S][H][W]  (caller's chi_out)
    Real* chibar;               // [S][H][W]  scratch
    Real* p;                    // [S][H][W]  scratch
    Real* qx;                   // [S][H][W]  scratch
    Real* qy;                   // [S][H][W]  scratch
    const Real* dtab;           // [W/2][H]: D(ky,kx)/(HW), column kx=0 holds Dm
    const Real* ddtab;          // [H]: Dd for the packed column
    const V* twid;              // [NTW]: exp(-2 pi i m / NTW)
    int S;
    int n_iter;
    Real sigma;
    Real tau;
    Real inv_den;               // 1 / (1 + sigma / lambda)
    const Real* inv_den_slice;  // NULL, or per-slice 1 / (1 + sigma / lambda_s) [S]
    const int* active;          // NULL, or per-slice flag [S]: 0 = leave this slice untouched
    int resume;                 // 0: zero start; 1: continue from chi (chi_out), chibar, p, q
    int tv_iso;                 // 0: componentwise clamp (anisotropic TV); 1: unit-disc projection (isotropic)
    const Real* weight;         // NULL: data weighting W = mask; else W [S][H][W] (values in [0, 1])
    Real* qz;                   // 3-D variant only: z component of q [S][H][W]
    // Balanced schedule (streaming kernel, more slices than resident clusters): cluster c
    // runs the iteration segments sched[sched_off[c] .. sched_off[c+1]) = (slice, first
    // iteration, end iteration, flags); flags bit 0: wait for seg_flags[slice] (the first part
    // of the slice runs on another cluster), bit 1: set seg_flags[slice] when done.
    const int4* sched;          // NULL: persistent loop over whole slices
    const int* sched_off;       // [clusters + 1]
    int* seg_flags;             // [S], zeroed before each launch
    int* err;                   // set to 1 when a wait gives up (that launch's result is invalid)
    long long wait_limit;       // clock64 cycles a cluster waits before giving up
};

// Bounded wait for *flag != 0 (acquire, GPU scope).  Returns false once `limit`
// clock64 cycles have passed without the flag being set.
__device__ __forceinline__ bool wait_flag(const int* flag, long long limit) {
    const long long t0 = clock64();
    while (true) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v != 0) return true;
        if (clock64() - t0 > limit) return false;
        __nanosleep(200);
    }
}

// Release a flag (GPU scope) after the writes that precede it.
__device__ __forceinline__ void set_flag(int* flag) {
    __threadfence();
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(flag), "r"(1) : "memory");
}

// Dual TV prox of one pixel: v = q + sigma M G chibar; clamp each component, or
// project (vx, vy) onto the unit disc.
// Three components (3-D variant).
// Wait for the grid this launch depends on (programmatic dependent launch: the launch may
// begin before that grid has ended; this wait returns once it has, with its memory visible).
// A no-op for a launch without that attribute.  The kernels that use it issue no explicit
// early trigger: each CTA of the previous grid triggers as it exits, which measured faster
// than a trigger at kernel start (the next grid's CTAs then took SM slots while the previous
// grid still ran: 45.9 against 37.8 ms on the any-size workload, 42.6 without the attribute).
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class Real>
__device__ __forceinline__ void tv_prox3(Real& vx, Real& vy, Real& vz, int iso) {
    if (iso) {
        const Real n = fmax(Real(1), sqrt(vx * vx + vy * vy + vz * vz));
        vx = vx / n;
        vy = vy / n;
        vz = vz / n;
    } else {
        vx = fmin(Real(1), fmax(Real(-1), vx));
        vy = fmin(Real(1), fmax(Real(-1), vy));
        vz = fmin(Real(1), fmax(Real(-1), vz));
    }
}

template <class Real>
__device__ __forceinline__ void tv_prox(Real& vx, Real& vy, int iso) {
    if (iso) {
        const Real n = fmax(Real(1), sqrt(vx * vx + vy * vy));
        vx = vx / n;
        vy = vy / n;
    } else {
        vx = fmin(Real(1), fmax(Real(-1), vx));
        vy = fmin(Real(1), fmax(Real(-1), vy));
    }
}
using PDParams = PDParamsT<float>;

template <class Real>
__device__ __forceinline__ Real slice_inv_den(const PDParamsT<Real>& prm, int s) {
    return prm.inv_den_slice ? __ldg(prm.inv_den_slice + s) : prm.inv_den;
}

template <class V>
__device__ __forceinline__ V mk(RealOf<V> a, RealOf<V> b) {
    return V{a, b};
}


// ER_, EC_: elements per lane of the row / column transforms (0 = 16 for
// lengths >= 128, else 8).
template <int H_, int W_, int C_, int MINB_ = 1, int NT_ = 256, int ER_ = 0, int EC_ = 0, class Real_ = float>
struct Geo {
    using Real = Real_;                       // arithmetic type of state and transforms
    using V = typename Cplx<Real>::T;         // its complex vector type
    static constexpr int H = H_, W = W_, C = C_, NT = NT_, MINB = MINB_;
    static constexpr int M = W / 2;    // complex row length (packed half spectrum)
    static constexpr int R = H / C;    // rows per CTA
    static constexpr int MC = M / C;   // spectrum columns per CTA
    static constexpr int NTW = (H > W) ? H : W;
    // row transforms (length M)
    static constexpr int ER = ER_ ? ER_ : default_elems(M);
    static constexpr int TR = M / ER;
    // column transforms (length H)
    static constexpr int EC = EC_ ? EC_ : default_elems(H);
    static constexpr int TC = H / EC;
    static constexpr int NW = NT / 32;
    static constexpr int RPP = NW * (32 / TR);  // rows in flight per CTA
    static constexpr int CPP = NW * (32 / TC);  // columns in flight per CTA
    // shared-memory layout (complex units)
    static constexpr int HP = H;              // column stride (columns swizzled with key 4 cl)
    static constexpr int MP = M + (TR % 16);  // row-scratch stride: adjacent groups on other banks
    static constexpr int SM_TBUF = MC * HP;
    static constexpr int SM_ROWS = RPP * MP;
    static constexpr int SM_TW = NTW;
    static constexpr int SM_STW_R = StageTw<M, ER>::SIZE;  // row-transform stage twiddles
    static constexpr int SM_STW_C = StageTw<H, EC>::SIZE;  // column-transform stage twiddles
    // + 16 bytes: a cluster's decision word (balanced schedule).  No static shared memory in
    // these kernels: it would shift the dynamic buffer off the alignment the swizzle relies on.
    static constexpr size_t SMEM_BYTES = sizeof(V) * (SM_TBUF + SM_ROWS + SM_TW + SM_STW_R + SM_STW_C) + 16;

    static_assert(TR <= 32 && TC <= 32, "group fits a warp");
    static_assert(R % RPP == 0, "row passes");
    static_assert(MC % CPP == 0 || CPP % MC == 0, "column passes");
    static constexpr int CPASSES = (MC >= CPP) ? MC / CPP : 1;  // groups beyond MC idle
    // owner CTA of spectrum column k = g + TR*e is compile-time per e when MC % TR == 0,
    // else it is mapped at run time (one mapa per element)
    static constexpr bool STATIC_OWNER = (MC % TR == 0);
    static_assert(W % 4 == 0 && H % 16 == 0, "shape");
    static_assert((TR & (TR - 1)) == 0 && (TC & (TC - 1)) == 0, "lane groups tile a warp");
};

template <int T>
__device__ __forceinline__ unsigned group_mask(int lane) {
    if constexpr (T == 32) {
        return 0xffffffffu;
    } else {
        return ((1u << T) - 1u) << ((lane / T) * T);
    }
}

template <int C>
__device__ __forceinline__ void cluster_barrier() {
    if constexpr (C == 1) {
        __syncthreads();
    } else {
        cg::this_cluster().sync();
    }
}

// Split form of the cluster barrier: arrive (release) after a CTA's last write
// of a phase, wait (acquire) before its first read of the peers' data, with
// independent work in between.  C = 1: the wait is a CTA barrier.
template <int C>
__device__ __forceinline__ void cluster_arrive() {
    if constexpr (C > 1) __cluster_barrier_arrive();
}
template <int C>
__device__ __forceinline__ void cluster_wait() {
    if constexpr (C == 1) {
        __syncthreads();
    } else {
        __cluster_barrier_wait();
    }
}

template <class G>
struct Ctx {
    using V = typename G::V;
    V* tbuf;     // own spectrum columns, [MC][HP]
    V* rows;     // row scratch, [RPP][MP]
    V* tw;       // twiddles [NTW]
    V* stw_r;    // stage twiddles of the row transforms
    V* stw_c;    // stage twiddles of the column transforms
    int crank;
};

// Carve the shared-memory layout and load the twiddle tables (no barrier).
template <class G>
__device__ __forceinline__ void ctx_init(Ctx<G>& cx, unsigned char* smem_raw, const typename G::V* __restrict__ twid) {
    using V = typename G::V;
    using Real = typename G::Real;
    cx.tbuf = reinterpret_cast<V*>(smem_raw);
    cx.rows = cx.tbuf + G::SM_TBUF;
    cx.tw = cx.rows + G::SM_ROWS;
    cx.stw_r = cx.tw + G::SM_TW;
    cx.stw_c = cx.stw_r + G::SM_STW_R;
    for (int t = threadIdx.x; t < G::NTW; t += G::NT) cx.tw[t] = twid[t];
    StageTw<G::M, G::ER>::fill(cx.stw_r, twid, G::NTW / G::M, threadIdx.x, G::NT);
    StageTw<G::H, G::EC>::fill(cx.stw_c, twid, G::NTW / G::H, threadIdx.x, G::NT);
    if constexpr (G::C == 1) {
        cx.crank = 0;
    } else {
        cx.crank = (int)cg::this_cluster().block_rank();
    }
}

// Spectrum columns of cluster CTA q (mapped at each use: holding C pointers costs registers).
template <class G>
__device__ __forceinline__ typename G::V* remote_tbuf(const Ctx<G>& cx, int q) {
    if constexpr (G::C == 1) {
        return cx.tbuf;
    } else {
        return cg::this_cluster().map_shared_rank(cx.tbuf, q);
    }
}

// ------------------------------------------------------------------ column pass
// Forward column FFT, multiply by D/(HW), inverse column FFT, in place on the
// CTA's own spectrum columns.
template <class G>
__device__ __forceinline__ void column_pass(const Ctx<G>& cx, const typename G::Real* __restrict__ dtab,
                                            const typename G::Real* __restrict__ ddtab) {
    using V = typename G::V;
    using Real = typename G::Real;
    constexpr int H = G::H, TC = G::TC, EC = G::EC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TC;
    const int grp = warp * (32 / TC) + lane / TC;
    const unsigned gm = group_mask<TC>(lane);
#pragma unroll 1
    for (int pass = 0; pass < G::CPASSES; ++pass) {
        const int cl = pass * G::CPP + grp;
        if (G::CPP > G::MC && cl >= G::MC) break;  // whole group idles (uniform per group)
        const int kx = cx.crank * G::MC + cl;
        V* col = cx.tbuf + cl * G::HP;
        const int key = 4 * cl;
        V x[EC];
#pragma unroll
        for (int e = 0; e < EC; ++e) x[e] = col[P(g + TC * e, key)];
        // the column's D(k) entries (Dm, Dd for the packed column), in flight during the FFT
        Real dk[EC], ddk[EC];
        const Real* d = dtab + (size_t)kx * H;
#pragma unroll
        for (int e = 0; e < EC; ++e) {
            dk[e] = __ldg(d + g + TC * e);
            ddk[e] = (kx == 0) ? __ldg(ddtab + g + TC * e) : Real(0);
        }
        fft<H, TC, false>(x, col, cx.stw_c, g, gm, key);
        if (kx != 0) {
#pragma unroll
            for (int e = 0; e < EC; ++e) x[e] = cscale(x[e], dk[e]);
        } else {
            // packed DC / Nyquist column: pair ky with -ky
#pragma unroll
            for (int e = 0; e < EC; ++e) col[P(g + TC * e, key)] = x[e];
            __syncwarp(gm);
#pragma unroll
            for (int e = 0; e < EC; ++e) {
                const int ky = g + TC * e;
                const V ym = col[P((H - ky) % H, key)];
                const Real dm = dk[e], dd = ddk[e];
                x[e] = mk<V>(fma(dm, x[e].x, dd * ym.x), fma(dm, x[e].y, -dd * ym.y));
            }
        }
        fft<H, TC, true>(x, col, cx.stw_c, g, gm, key);
#pragma unroll
        for (int e = 0; e < EC; ++e) col[P(g + TC * e, key)] = x[e];
        __syncwarp(gm);
    }
}

// ------------------------------------------------------------------ row transforms
// Swizzled position of row i in the spectrum columns a row lane g touches:
// P(i, 4 cl) with cl = g + TR e - q MC, whose key mod 16 is 4 (g mod 4) for
// every element (TR and MC are multiples of 4).
template <class G>
__device__ __forceinline__ int row_slot(int i, int g) {
    static_assert(G::TR % 4 == 0 && G::MC % 4 == 0, "row-lane swizzle key");
    return P(i, 4 * (g & 3));
}

// Pair every element of a row with its mirror column M-k (see the file
// comment) and apply op(k, X[k], X[M-k]) in place.  Elements are taken in pairs
// (e, ER-1-e), whose mirrors in lanes g >= 1 are each other's; lane 0's
// mirrors are its own elements ER-e, read before they are overwritten (one
// carried value).
template <class G, class Op>
__device__ __forceinline__ void mirror_pairs(typename G::V (&x)[G::ER], int g, unsigned gm, Op op) {
    using V = typename G::V;
    constexpr int TR = G::TR, ER = G::ER;
    static_assert(ER % 2 == 0, "element pairs");
    const int lane = threadIdx.x & 31;
    const int src = (lane - g) + ((TR - g) & (TR - 1));  // mirror lane in the group
    V carry = x[0];
#pragma unroll
    for (int e = 0; e < ER / 2; ++e) {
        const int e2 = ER - 1 - e;
        const V a = x[e], b = x[e2];
        V va, vb;
        va.x = __shfl_sync(gm, b.x, src);
        va.y = __shfl_sync(gm, b.y, src);
        vb.x = __shfl_sync(gm, a.x, src);
        vb.y = __shfl_sync(gm, a.y, src);
        const V own_a = (e == 0) ? a : carry;           // lane 0: element ER-e
        const V own_b = (e + 1 == e2) ? b : x[e + 1];   // lane 0: element e+1
        carry = b;
        x[e] = op(g + TR * e, a, (g == 0) ? own_a : va);
        x[e2] = op(g + TR * e2, b, (g == 0) ? own_b : vb);
    }
}

// Inverse real row transform of the packed spectrum row in x (element k = g + TR*e in x[e];
// k = 0 packs X[0] + i X[M]).  Result: x[e] = W * (y[2n], y[2n+1]) for n = g + TR*e, where y
// is the real row (the D table carries 1/(HW), so x is the true D-product).
template <class G>
__device__ __forceinline__ void row_unpack_inverse(const Ctx<G>& cx, typename G::V* rs, int g, unsigned gm,
                                                   typename G::V (&x)[G::ER]) {
    using V = typename G::V;
    constexpr int M = G::M, TR = G::TR, NTW = G::NTW, W = G::W;
    const V* tw = cx.tw;
    mirror_pairs<G>(x, g, gm, [tw](int k, V X, V Xm) {
        if (k == 0) return mk<V>(X.x + X.y, X.x - X.y);  // X[0] = Re, X[M] = Im of the packed entry
        const V ec = mk<V>(X.x + Xm.x, X.y - Xm.y);     // X + conj(Xm)
        const V od0 = mk<V>(X.x - Xm.x, X.y + Xm.y);    // X - conj(Xm)
        const V w = tw[k * (NTW / W)];                    // exp(-2 pi i k / W)
        const V od = cmul(od0, conjf2(w));
        return mk<V>(ec.x - od.y, ec.y + od.x);  // ec + i od
    });
    fft<M, TR, true>(x, rs, cx.stw_r, g, gm);
}

// Forward real row transform of z[e] = (x[2n], x[2n+1]), n = g + TR*e, in place: the packed
// spectrum row, element k = g + TR*e in z[e], k = 0 packing X[0] + i X[M].
template <class G>
__device__ __forceinline__ void row_forward_pack(const Ctx<G>& cx, typename G::V* rs, int g, unsigned gm,
                                                 typename G::V (&z)[G::ER]) {
    using V = typename G::V;
    using Real = typename G::Real;
    constexpr int M = G::M, TR = G::TR, NTW = G::NTW, W = G::W;
    fft<M, TR, false>(z, rs, cx.stw_r, g, gm);
    const V* tw = cx.tw;
    mirror_pairs<G>(z, g, gm, [tw](int k, V A, V Zm) {
        if (k == 0) return mk<V>(A.x + A.y, A.x - A.y);  // X[0] + i X[M]
        // E = (A + conj(Zm))/2, O = -i (A - conj(Zm))/2, X = E + w^k O
        const V E = mk<V>(Real(0.5) * (A.x + Zm.x), Real(0.5) * (A.y - Zm.y));
        const V dlt = mk<V>(A.x - Zm.x, A.y + Zm.y);
        const V O = mk<V>(Real(0.5) * dlt.y, -Real(0.5) * dlt.x);
        const V w = tw[k * (NTW / W)];
        return cadd(E, cmul(w, O));
    });
}

// Gather packed spectrum row i from the cluster and apply the inverse real row transform.
template <class G>
__device__ __forceinline__ void row_inverse(const Ctx<G>& cx, typename G::V* rs, int i, int g, unsigned gm,
                                            typename G::V (&x)[G::ER]) {
    constexpr int TR = G::TR, ER = G::ER, MC = G::MC;
    const int pi = row_slot<G>(i, g);
#pragma unroll
    for (int e = 0; e < ER; ++e) {
        const int k = g + TR * e;
        if constexpr (G::STATIC_OWNER) {
            const int q = (TR * e) / MC;  // compile-time after unrolling
            x[e] = remote_tbuf<G>(cx, q)[(k - q * MC) * G::HP + pi];
        } else {
            const int q = k / MC;
            x[e] = remote_tbuf<G>(cx, q)[(k - q * MC) * G::HP + pi];
        }
    }
    row_unpack_inverse<G>(cx, rs, g, gm, x);
}

// Forward real row transform of z[e] = (x[2n], x[2n+1]), n = g + TR*e, and
// scatter of the packed spectrum row i to the owners of its columns.
template <class G>
__device__ __forceinline__ void row_forward(const Ctx<G>& cx, typename G::V* rs, int i, int g, unsigned gm,
                                            typename G::V (&z)[G::ER]) {
    constexpr int TR = G::TR, ER = G::ER, MC = G::MC;
    row_forward_pack<G>(cx, rs, g, gm, z);
    const int pi = row_slot<G>(i, g);
#pragma unroll
    for (int e = 0; e < ER; ++e) {
        const int k = g + TR * e;
        if constexpr (G::STATIC_OWNER) {
            const int q = (TR * e) / MC;
            remote_tbuf<G>(cx, q)[(k - q * MC) * G::HP + pi] = z[e];
        } else {
            const int q = k / MC;
            remote_tbuf<G>(cx, q)[(k - q * MC) * G::HP + pi] = z[e];
        }
    }
}

// ------------------------------------------------------------------ row phases

// Epilogue element chunk: the loads of CH elements are issued together, then
// computed and stored (restrict-qualified pointers let the next chunk's loads
// move ahead of this chunk's stores).  2 measured fastest (1: +1.7%, 4: +3%, 8: +13%).
constexpr int kChunk = 2;

// Row transport of the row phases: where the packed spectrum rows come from and go to.  The
// default is the cluster's distributed spectrum columns (gather before the inverse transform,
// scatter after the forward one, and the wait for the peers' scatters); the 3-D variant's
// plane-major rows in global memory (pd_3d.cuh) provide the same three calls.
template <class G>
struct ClusterRows {
    using V = typename G::V;
    static constexpr int kChunkElems = kChunk;  // epilogue elements whose loads go out together
    __device__ __forceinline__ void wait() const { cluster_wait<G::C>(); }
    __device__ __forceinline__ void inverse(const Ctx<G>& cx, V* rs, int i, int g, unsigned gm, V (&x)[G::ER]) const {
        row_inverse<G>(cx, rs, i, g, gm, x);
    }
    __device__ __forceinline__ void forward(const Ctx<G>& cx, V* rs, int i, int g, unsigned gm, V (&x)[G::ER]) const {
        row_forward<G>(cx, rs, i, g, gm, x);
    }
};

// Elements of one slice (the 3-D variant's offset between neighbouring slices).
template <class G>
constexpr size_t SL3 = (size_t)G::H * G::W;

// Phase B: u = D chibar -> dual proxes -> forward transform of W p.
// q stays exactly zero wherever the 0/1 mask M is zero (zero start, masked
// increments), so M q = q; p likewise wherever W is zero.  With W = mask the
// product W p equals p bit for bit.
// Entered after cluster_arrive(): the first row pass waits for the peers once
// its own-row chibar is in flight (early_cb: that row was written by this
// thread, or by an earlier launch; not so right after the zero start).
// Z3 (3-D variant): q also has a z component, updated from chibar of the next
// slice (zero difference on the last slice); s is the slice of base.
template <class G, bool Z3 = false, class IO = ClusterRows<G>>
__device__ __forceinline__ void phase_dual(const Ctx<G>& cx, const PDParamsT<typename G::Real>& prm, size_t base,
                                           typename G::Real inv_den, bool early_cb, int s = 0, const IO& io = IO()) {
    using V = typename G::V;
    using Real = typename G::Real;
    constexpr int H = G::H, W = G::W, TR = G::TR, ER = G::ER;
    constexpr int CH = (ER < IO::kChunkElems) ? ER : IO::kChunkElems;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TR;
    const int grp = warp * (32 / TR) + lane / TR;
    const unsigned gm = group_mask<TR>(lane);
    const int src_right = (g == TR - 1) ? lane - (TR - 1) : lane + 1;  // lane holding pixel 2n+2
    V* rs = cx.rows + grp * G::MP;
    const Real sigma = prm.sigma;
    const Real* __restrict__ fld = prm.field;
    const unsigned char* __restrict__ msk = prm.mask;
    const Real* __restrict__ cbar = prm.chibar;
    Real* __restrict__ pp = prm.p;
    Real* __restrict__ qxp = prm.qx;
    Real* __restrict__ qyp = prm.qy;
    Real* __restrict__ qzp = prm.qz;  // 3-D variant only
#pragma unroll 1
    for (int pass = 0; pass < G::R / G::RPP; ++pass) {
        const int i = cx.crank * G::R + pass * G::RPP + grp;
        const size_t rowoff = base + (size_t)i * W;
        const bool has_down = (i + 1 < H);
        // chibar of this row; its right neighbours come from the next lane by shuffle
        if (pass == 0 && !early_cb) io.wait();
        V cb[ER];
#pragma unroll
        for (int e = 0; e < ER; ++e) cb[e] = __ldcg(reinterpret_cast<const V*>(cbar + rowoff + 2 * (g + TR * e)));
        if (pass == 0 && early_cb) io.wait();
        V x[ER];
        io.inverse(cx, rs, i, g, gm, x);
        Real cr[ER];
#pragma unroll
        for (int e = 0; e < ER; ++e) cr[e] = __shfl_sync(gm, cb[e].x, src_right);
#pragma unroll
        for (int e0 = 0; e0 < ER; e0 += CH) {
            V f[CH], p[CH], cd[CH], qx[CH], qy[CH];
            V qz[CH], cz[CH];  // 3-D variant only
            uchar2 mk[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const size_t o = rowoff + 2 * (g + TR * (e0 + c));
                f[c] = __ldg(reinterpret_cast<const V*>(fld + o));
                mk[c] = __ldg(reinterpret_cast<const uchar2*>(msk + o));
                p[c] = __ldcg(reinterpret_cast<const V*>(pp + o));
                cd[c] = has_down ? __ldcg(reinterpret_cast<const V*>(cbar + o + W)) : cb[e0 + c];
                qx[c] = __ldcg(reinterpret_cast<const V*>(qxp + o));
                qy[c] = __ldcg(reinterpret_cast<const V*>(qyp + o));
                if constexpr (Z3) {  // with the chunk's other loads, ahead of its stores
                    qz[c] = __ldcg(reinterpret_cast<const V*>(qzp + o));
                    cz[c] = (s + 1 < prm.S) ? __ldcg(reinterpret_cast<const V*>(cbar + o + SL3<G>)) : cb[e0 + c];
                }
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int e = e0 + c;
                const size_t o = rowoff + 2 * (g + TR * e);
                // pixel 2n+2 is in the next lane at the same e, or in lane 0 at e+1; past the
                // last column the difference is zero (Neumann)
                Real right = cr[e];
                if (g == TR - 1) right = (e + 1 < ER) ? cr[e + 1] : cb[e].y;
                const Real m0 = mk[c].x ? Real(1) : Real(0), m1 = mk[c].y ? Real(1) : Real(0);
                Real w0 = m0, w1 = m1;
                if (prm.weight) {  // non-binary W (weighted solves only)
                    const V wv = __ldg(reinterpret_cast<const V*>(prm.weight + o));
                    w0 = wv.x;
                    w1 = wv.y;
                }
                const V u = x[e];
                // dual data prox (W dB formed on the fly)
                V pn;
                pn.x = (p[c].x + sigma * (w0 * (u.x - f[c].x))) * inv_den;
                pn.y = (p[c].y + sigma * (w1 * (u.y - f[c].y))) * inv_den;
                // dual TV prox (forward differences of chibar, Neumann boundary)
                V qxn, qyn;
                qxn.x = qx[c].x + sigma * m0 * (cb[e].y - cb[e].x);
                qxn.y = qx[c].y + sigma * m1 * (right - cb[e].y);
                qyn.x = qy[c].x + sigma * m0 * (cd[c].x - cb[e].x);
                qyn.y = qy[c].y + sigma * m1 * (cd[c].y - cb[e].y);
                if constexpr (Z3) {
                    V qzn = qz[c];
                    if (s + 1 < prm.S) {
                        qzn.x += sigma * m0 * (cz[c].x - cb[e].x);
                        qzn.y += sigma * m1 * (cz[c].y - cb[e].y);
                    }
                    tv_prox3(qxn.x, qyn.x, qzn.x, prm.tv_iso);
                    tv_prox3(qxn.y, qyn.y, qzn.y, prm.tv_iso);
                    __stcg(reinterpret_cast<V*>(qzp + o), qzn);
                } else {
                    tv_prox(qxn.x, qyn.x, prm.tv_iso);
                    tv_prox(qxn.y, qyn.y, prm.tv_iso);
                }
                __stcg(reinterpret_cast<V*>(pp + o), pn);
                __stcg(reinterpret_cast<V*>(qxp + o), qxn);
                __stcg(reinterpret_cast<V*>(qyp + o), qyn);
                x[e].x = w0 * pn.x;  // W p: input of the adjoint transform
                x[e].y = w1 * pn.y;
            }
        }
        io.forward(cx, rs, i, g, gm, x);
    }
}

// Phase A: v = D W p -> primal step -> over-relaxation -> forward transform of chibar.
// G^T M q = G^T q because q vanishes outside the mask (see phase_dual).
// Entered after cluster_arrive(): the own-row qx (written by this thread in
// the dual phase) is loaded before the wait.
// Z3 (3-D variant): G^T also takes the z differences, qz[s-1] - qz[s] with the
// same boundary rule as the rows.
template <class G, bool Z3 = false, class IO = ClusterRows<G>>
__device__ __forceinline__ void phase_primal(const Ctx<G>& cx, const PDParamsT<typename G::Real>& prm, size_t base,
                                             bool last, int s = 0, const IO& io = IO()) {
    using V = typename G::V;
    using Real = typename G::Real;
    constexpr int H = G::H, W = G::W, TR = G::TR, ER = G::ER;
    constexpr int CH = (ER < IO::kChunkElems) ? ER : IO::kChunkElems;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TR;
    const int grp = warp * (32 / TR) + lane / TR;
    const unsigned gm = group_mask<TR>(lane);
    const int src_left = (g == 0) ? lane + (TR - 1) : lane - 1;  // lane holding pixel 2n-1
    V* rs = cx.rows + grp * G::MP;
    const Real tau = prm.tau;
    const Real* __restrict__ qxp = prm.qx;
    const Real* __restrict__ qyp = prm.qy;
    const Real* __restrict__ qzp = prm.qz;  // 3-D variant only
    Real* __restrict__ chip = prm.chi;
    Real* __restrict__ cbar = prm.chibar;
#pragma unroll 1
    for (int pass = 0; pass < G::R / G::RPP; ++pass) {
        const int i = cx.crank * G::R + pass * G::RPP + grp;
        const size_t rowoff = base + (size_t)i * W;
        const bool has_up = (i > 0), has_down = (i + 1 < H);
        V qx[ER];
#pragma unroll
        for (int e = 0; e < ER; ++e) qx[e] = __ldcg(reinterpret_cast<const V*>(qxp + rowoff + 2 * (g + TR * e)));
        if (pass == 0) io.wait();
        V x[ER];
        io.inverse(cx, rs, i, g, gm, x);
        Real ql[ER];
#pragma unroll
        for (int e = 0; e < ER; ++e) ql[e] = __shfl_sync(gm, qx[e].y, src_left);
#pragma unroll
        for (int e0 = 0; e0 < ER; e0 += CH) {
            V qy[CH], qu[CH], chi[CH];
            V zc[CH], zp[CH];  // 3-D variant only: qz of this slice and of the slice before
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const size_t o = rowoff + 2 * (g + TR * (e0 + c));
                qy[c] = __ldcg(reinterpret_cast<const V*>(qyp + o));
                qu[c] = has_up ? __ldcg(reinterpret_cast<const V*>(qyp + o - W)) : mk<V>(Real(0), Real(0));
                chi[c] = __ldcg(reinterpret_cast<const V*>(chip + o));
                if constexpr (Z3) {  // with the chunk's other loads, ahead of its stores
                    zc[c] = (s + 1 < prm.S) ? __ldcg(reinterpret_cast<const V*>(qzp + o)) : mk<V>(Real(0), Real(0));
                    zp[c] = (s > 0) ? __ldcg(reinterpret_cast<const V*>(qzp + o - SL3<G>)) : mk<V>(Real(0), Real(0));
                }
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int e = e0 + c;
                const int j0 = 2 * (g + TR * e);
                const size_t o = rowoff + j0;
                const V v = x[e];
                // G^T(a,b)[j] = a[j-1][j>0] - a[j][j<W-1] + b[i-1][i>0] - b[i][i<H-1], a = qx, b = qy
                Real al = ql[e];
                if (g == 0) al = (e > 0) ? ql[e - 1] : Real(0);
                const Real a1r = (j0 + 2 < W) ? qx[e].y : Real(0);
                const Real b0 = has_down ? qy[c].x : Real(0);
                const Real b1 = has_down ? qy[c].y : Real(0);
                Real d0 = (al - qx[e].x) + (qu[c].x - b0);
                Real d1 = (qx[e].x - a1r) + (qu[c].y - b1);
                if constexpr (Z3) {
                    d0 += zp[c].x - zc[c].x;
                    d1 += zp[c].y - zc[c].y;
                }
                V cn;
                cn.x = chi[c].x - tau * v.x - tau * d0;
                cn.y = chi[c].y - tau * v.y - tau * d1;
                __stcg(reinterpret_cast<V*>(chip + o), cn);
                const V cb = mk<V>(Real(2) * cn.x - chi[c].x, Real(2) * cn.y - chi[c].y);
                __stcg(reinterpret_cast<V*>(cbar + o), cb);  // kept for a later resume
                x[e] = cb;
            }
        }
        if (!last) io.forward(cx, rs, i, g, gm, x);
    }
}

// Forward real row transforms of a stored field (own rows) and scatter: the
// spectrum a resumed solve starts from.
template <class G>
__device__ __forceinline__ void rows_forward_state(const Ctx<G>& cx, const typename G::Real* src, size_t base) {
    using V = typename G::V;
    constexpr int W = G::W, TR = G::TR, ER = G::ER;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane % TR;
    const int grp = warp * (32 / TR) + lane / TR;
    const unsigned gm = group_mask<TR>(lane);
    V* rs = cx.rows + grp * G::MP;
#pragma unroll 1
    for (int pass = 0; pass < G::R / G::RPP; ++pass) {
        const int i = cx.crank * G::R + pass * G::RPP + grp;
        const size_t rowoff = base + (size_t)i * W;
        V z[ER];
#pragma unroll
        for (int e = 0; e < ER; ++e) z[e] = __ldcg(reinterpret_cast<const V*>(src + rowoff + 2 * (g + TR * e)));
        row_forward<G>(cx, rs, i, g, gm, z);
    }
}

// ------------------------------------------------------------------ kernel

// Iterations [it_b, it_e) of slice s: a zero start when it_b = 0 (and no resume),
// else a continuation from the stored state.
template <class G>
__device__ __forceinline__ void run_slice(Ctx<G>& cx, const PDParamsT<typename G::Real>& prm, int s, int it_b,
                                          int it_e) {
    using V = typename G::V;
    using Real = typename G::Real;
    constexpr size_t SLICE = (size_t)G::H * G::W;
    constexpr int OWN = G::R * G::W;  // floats of own rows
    const size_t base = (size_t)s * SLICE;
    const Real inv_den = slice_inv_den(prm, s);
    const bool cont = prm.resume || it_b > 0;
    if (cont) {
        // continue: the spectrum of the stored chibar, then the loop as after iteration 0
        cluster_barrier<G::C>();  // peers running before their shared memory is written
        rows_forward_state<G>(cx, prm.chibar, base);
    } else {
        // zero start (pseudocode steps 2-3): chi, chibar, p, q of own rows, own spectrum
        const size_t o = base + (size_t)cx.crank * OWN;
        V* ptrs[5] = {reinterpret_cast<V*>(prm.chi + o), reinterpret_cast<V*>(prm.chibar + o),
                      reinterpret_cast<V*>(prm.p + o), reinterpret_cast<V*>(prm.qx + o),
                      reinterpret_cast<V*>(prm.qy + o)};
        const V z2 = mk<V>(Real(0), Real(0));
#pragma unroll
        for (int a = 0; a < 5; ++a)
            for (int t = threadIdx.x; t < OWN / 2; t += G::NT) __stcg(ptrs[a] + t, z2);
        for (int t = threadIdx.x; t < G::SM_TBUF; t += G::NT) cx.tbuf[t] = mk<V>(Real(0), Real(0));
    }
    // half-steps: even = column pass (u-spectrum = D F chibar_n; skipped at a zero
    // start, where it is zero) + dual phase, odd = column pass (v-spectrum = D F W p_{n+1})
    // + primal phase.  Each phase appears once in the code.  A row phase is
    // entered after cluster_arrive() and waits inside, after its own-row loads.
    const int nh = 2 * (it_e - it_b);
#pragma unroll 1
    for (int h = 0; h < nh; ++h) {
        if (h > 0 || cont) {
            cluster_barrier<G::C>();
            column_pass<G>(cx, prm.dtab, prm.ddtab);
        }
        cluster_arrive<G::C>();
        if ((h & 1) == 0) {
            phase_dual<G>(cx, prm, base, inv_den, h > 0 || cont);
        } else {
            phase_primal<G>(cx, prm, base, h + 1 == nh);
        }
    }
    cluster_barrier<G::C>();  // the last phase's gathers done before the next slice writes
}

// SCHED: run the balanced schedule's segments (a separate instantiation: the plain
// persistent loop keeps the registers the schedule's bookkeeping would take).
template <class G, bool SCHED = false>
__global__ void __launch_bounds__(G::NT, G::MINB) pd_cluster_kernel(PDParamsT<typename G::Real> prm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ctx<G> cx;
    ctx_init<G>(cx, smem_raw, prm.twid);
    const int cid = blockIdx.x / G::C;
    if constexpr (!SCHED) {
#pragma unroll 1
        for (int s = cid; s < prm.S; s += gridDim.x / G::C) {
            if (prm.active && __ldg(prm.active + s) == 0) continue;  // same decision in every CTA of the cluster
            run_slice<G>(cx, prm, s, 0, prm.n_iter);
        }
    } else {
#pragma unroll 1
        for (int k = __ldg(prm.sched_off + cid); k < __ldg(prm.sched_off + cid + 1); ++k) {
            const int4 sg = __ldg(prm.sched + k);
            if (sg.w & 1) {
                // the slice's first part runs on another cluster: CTA 0 waits (bounded) and the
                // cluster follows its decision (a word after the tables), so that every CTA
                // proceeds or every CTA returns
                int* go = reinterpret_cast<int*>(cx.stw_c + G::SM_STW_C);
                if (cx.crank == 0 && threadIdx.x == 0)
                    *go = wait_flag(prm.seg_flags + sg.x, prm.wait_limit) ? 1 : 0;
                cluster_barrier<G::C>();
                int ok;
                if constexpr (G::C == 1) {
                    ok = *go;
                } else {
                    ok = *cg::this_cluster().map_shared_rank(go, 0);
                }
                cluster_barrier<G::C>();  // every CTA has read CTA 0's decision
                if (!ok) {
                    if (cx.crank == 0 && threadIdx.x == 0) atomicExch(prm.err, 1);
                    return;
                }
                if (threadIdx.x == 0) (void)wait_flag(prm.seg_flags + sg.x, prm.wait_limit);  // this CTA's acquire
                __syncthreads();
            }
            run_slice<G>(cx, prm, sg.x, sg.y, sg.z);
            if (cx.crank == 0 && threadIdx.x == 0) {
                const int4 done = __ldg(prm.sched + k);
                if (done.w & 2) set_flag(prm.seg_flags + done.x);
            }
        }
    }
}

}  // namespace pcs
