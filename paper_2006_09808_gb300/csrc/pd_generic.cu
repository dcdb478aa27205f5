// pd_generic.cu -- C-ABI entry of the any-size per-slice solver
// (pcs_solve_slices_generic; kernels in pd_generic.cuh).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>

#include "../../include/pcs.h"
#include "pd_generic.cuh"
#include "pcs_trace.h"

namespace pcs {
void build_twiddles(int n, std::vector<float2>& tw);
pcs_status set_last_error(pcs_status st, const char* msg);
}  // namespace pcs

namespace {

using pcs::GenParams;
using pcs::GenPlan;

constexpr int kGenMinLen = 8;
constexpr int kGenMaxLen = 512;
constexpr int kGenMaxRadix = 61;

// Radices of n: factors 4 first, then 2, then the odd primes in increasing order.
bool gen_plan(int n, GenPlan* pl) {
    std::memset(pl, 0, sizeof(*pl));
    if (n < kGenMinLen || n > kGenMaxLen) return false;
    pl->n = n;
    int m = n;
    auto push = [&](int r) {
        if (pl->nst >= pcs::kGenMaxStages) return false;
        pl->r[pl->nst++] = r;
        m /= r;
        return true;
    };
    while (m % 4 == 0)
        if (!push(4)) return false;
    while (m % 2 == 0)
        if (!push(2)) return false;
    for (int p = 3; p <= kGenMaxRadix && m > 1; p += 2)
        while (m % p == 0)
            if (!push(p)) return false;
    return m == 1;
}

pcs_status failg(pcs_status st, const char* what, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess) {
        snprintf(buf, sizeof(buf), "pcs_solve_slices_generic: %s: %s", what, cudaGetErrorString(e));
    } else {
        snprintf(buf, sizeof(buf), "pcs_solve_slices_generic: %s", what);
    }
    return pcs::set_last_error(st, buf);
}

// Column pass: the register-FFT kernel for these H, else the shared-memory DFT kernel.
struct ColEntry {
    int H;
    size_t smem;
    void (*kern)(GenParams);
    int tile;     // columns per CTA
    int threads;  // threads per CTA
};
template <int H>
constexpr ColEntry col_entry() {
    return ColEntry{H, pcs::GeoCol<H>::SMEM_BYTES, &pcs::gen_cols_fft_kernel<H>, pcs::GeoCol<H>::TY,
                    pcs::GeoCol<H>::NT};
}
const ColEntry k_cols[] = {col_entry<64>(),  col_entry<128>(), col_entry<192>(),
                           col_entry<256>(), col_entry<384>(), col_entry<512>()};

size_t rows_smem(int W) { return sizeof(float2) * (size_t)W * (1 + 2 * pcs::kGenRowWarps); }
size_t cols_smem(int H) { return sizeof(float2) * ((size_t)H + (size_t)(2 * H + 1) * pcs::kGenColTile); }

bool gen_shape_ok(int H, int W, GenPlan* prow, GenPlan* pcol) {
    return H % 2 == 0 && W % 2 == 0 && gen_plan(W, prow) && gen_plan(H, pcol);
}

}  // namespace

namespace pcs {

// Tables, plans, kernel choice and the half-spectrum scratch of one H x W size.
struct GenSolver {
    GenParams g;  // plans, sizes, tables and spectrum set; state pointers per solve
    float2* tabs = nullptr;
    float2* spec = nullptr;
    double* partial = nullptr;  // FP64 report: [max_slices][H/2][kGenReportSums]
    int max_slices = 0;
    void (*cols_kern)(GenParams) = nullptr;
    int col_tile = 0, col_threads = 0;
    size_t srows = 0, scols = 0;
};

bool gen_supported(int H, int W) {
    GenPlan a, b;
    return gen_shape_ok(H, W, &a, &b);
}

void gen_destroy(GenSolver* gs) {
    if (!gs) return;
    cudaFree(gs->tabs);
    cudaFree(gs->spec);
    cudaFree(gs->partial);
    delete gs;
}

// Returns cudaSuccess and *out, or an error with *out = NULL.  The twiddle tables are
// uploaded synchronously.
// Launch kern(args) on st; dep: programmatic dependent launch (the kernel waits for the
// previous grid in the stream before it touches memory).
template <class... KA, class... A>
cudaError_t launch_dep(void (*kern)(KA...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool dep,
                       A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = dep ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

cudaError_t gen_create(GenSolver** out, int H, int W, int max_slices, int b0_axis, int tv) {
    *out = nullptr;
    GenSolver* gs = new GenSolver();
    std::memset(&gs->g, 0, sizeof(gs->g));
    if (!gen_shape_ok(H, W, &gs->g.prow, &gs->g.pcol)) {
        delete gs;
        return cudaErrorInvalidValue;
    }
    const int M1 = W / 2 + 1;
    const ColEntry* ce = nullptr;
    for (const auto& c : k_cols)
        if (c.H == H) ce = &c;
    gs->cols_kern = ce ? ce->kern : gen_cols_kernel;
    gs->col_tile = ce ? ce->tile : kGenColTile;
    gs->col_threads = ce ? ce->threads : kGenColTile * 32;
    gs->srows = rows_smem(W);
    gs->scols = ce ? ce->smem : cols_smem(H);
    gs->max_slices = max_slices;
    std::vector<float2> tw_r, tw_c;
    build_twiddles(W, tw_r);
    build_twiddles(H, tw_c);
    // the dynamic shared-memory limit is a per-function attribute shared by every size: set it
    // to what the largest accepted size needs, so that solvers of several sizes coexist
    const int rows_max = (int)rows_smem(kGenMaxLen), cols_max = (int)cols_smem(kGenMaxLen);
    cudaError_t e;
    if ((e = cudaMalloc(&gs->tabs, (size_t)(W + H) * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&gs->spec, (size_t)max_slices * H * M1 * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&gs->partial, (size_t)max_slices * (H / 2) * kGenReportSums * sizeof(double))) !=
            cudaSuccess ||
        (e = cudaMemcpy(gs->tabs, tw_r.data(), W * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(gs->tabs + W, tw_c.data(), H * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(gen_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, rows_max)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(gen_report_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, rows_max)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(gen_opnorm_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, rows_max)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(gs->cols_kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ce ? (int)gs->scols : cols_max)) != cudaSuccess) {  // per-H instances: own size
        gen_destroy(gs);
        return e;
    }
    GenParams& g = gs->g;
    g.spec = gs->spec;
    g.trow = gs->tabs;
    g.tcol = gs->tabs + W;
    g.H = H;
    g.W = W;
    g.M1 = M1;
    g.tv_iso = tv;
    g.b0_axis = b0_axis;
    *out = gs;
    return cudaSuccess;
}

// Enqueue a solve of S <= max_slices slices on st: zero state, chi and spectrum (or, with
// resume, continue from the stored chi, chibar, p, q: the spectrum D F chibar is rebuilt),
// then n_iter iterations of four launches; slices with active[s] = 0 stay as they are;
// inv_den_slice (optional) gives each slice its own lambda; spec (optional) replaces the
// solver's spectrum scratch ([S][H][W/2 + 1] complex).
// Asynchronous; no allocation.
cudaError_t gen_enqueue(GenSolver* gs, const float* field, const unsigned char* mask, const float* weight,
                        float* chi, float* chibar, float* p, float* qx, float* qy, int S, double lambda, double tau,
                        double sigma, int n_iter, cudaStream_t st, int resume, const int* active,
                        const float* inv_den_slice, float2* spec) {
    GenParams g = gs->g;
    if (spec) g.spec = spec;  // a caller-owned spectrum (concurrent solves of one size)
    const size_t n = (size_t)S * g.H * g.W;
    cudaError_t e;
    if (!resume &&
        ((e = cudaMemsetAsync(chibar, 0, n * sizeof(float), st)) != cudaSuccess ||
         (e = cudaMemsetAsync(p, 0, n * sizeof(float), st)) != cudaSuccess ||
         (e = cudaMemsetAsync(qx, 0, n * sizeof(float), st)) != cudaSuccess ||
         (e = cudaMemsetAsync(qy, 0, n * sizeof(float), st)) != cudaSuccess ||
         (e = cudaMemsetAsync(chi, 0, n * sizeof(float), st)) != cudaSuccess ||
         (e = cudaMemsetAsync(g.spec, 0, (size_t)S * g.H * g.M1 * sizeof(float2), st)) != cudaSuccess))
        return e;
    g.active = active;
    g.inv_den_slice = inv_den_slice;
    g.field = field;
    g.mask = mask;
    g.weight = weight;
    g.chi = chi;
    g.chibar = chibar;
    g.p = p;
    g.qx = qx;
    g.qy = qy;
    g.S = S;
    g.sigma = (float)sigma;
    g.tau = (float)tau;
    g.inv_den = (float)(1.0 / (1.0 + sigma / lambda));
    const int pairs = S * (g.H / 2);
    const dim3 grid_r((pairs + kGenRowWarps - 1) / kGenRowWarps);
    const dim3 grid_c((g.M1 + gs->col_tile - 1) / gs->col_tile, S);
    if (resume && n_iter > 0) {
        // forward transforms of the stored chibar (the report kernel's first mode), column pass
        GenParams r = g;
        r.chi = chibar;
        gen_report_kernel<<<grid_r, kGenRowWarps * 32, gs->srows, st>>>(r, gs->partial, lambda, 0);
        gs->cols_kern<<<grid_c, gs->col_threads, gs->scols, st>>>(g);
    }
    // iteration n: dual step from the spectrum D F chibar_n (zero at n = 0), column pass
    // (spectrum of W p), primal step, column pass (spectrum of chibar_{n+1}; not after the last)
    // Programmatic dependent launch for every launch that follows one of these kernels: each
    // waits for the previous grid before it touches memory, and its launch overlaps the end of
    // that grid (37.8 against 42.6 ms per 256x258x25 solve).  The first launch follows the
    // caller's own stream work and is serialised.
    const dim3 blk_r(kGenRowWarps * 32), blk_c(gs->col_threads);
    for (int it = 0; it < n_iter; ++it) {
        g.phase = 0;
        g.store = 1;
        if ((e = launch_dep(gen_rows_kernel, grid_r, blk_r, gs->srows, st, it > 0, g)) != cudaSuccess ||
            (e = launch_dep(gs->cols_kern, grid_c, blk_c, gs->scols, st, true, g)) != cudaSuccess)
            return e;
        g.phase = 1;
        g.store = it + 1 < n_iter;
        if ((e = launch_dep(gen_rows_kernel, grid_r, blk_r, gs->srows, st, true, g)) != cudaSuccess ||
            (g.store && (e = launch_dep(gs->cols_kern, grid_c, blk_c, gs->scols, st, true, g)) != cudaSuccess))
            return e;
    }
    return cudaSuccess;
}

// FP64 diagnostics of every slice at (chi, p, q) (three report launches, two column
// passes), then a synchronising read-back and fixed-order sums per slice.
cudaError_t gen_report(GenSolver* gs, const float* field, const unsigned char* mask, const float* weight,
                       const float* chi, const float* p, const float* qx, const float* qy, int S, double lambda,
                       int iters, pcs_slice_report* rep, cudaStream_t st) {
    GenParams g = gs->g;
    g.field = field;
    g.mask = mask;
    g.weight = weight;
    g.chi = const_cast<float*>(chi);
    g.p = const_cast<float*>(p);
    g.qx = const_cast<float*>(qx);
    g.qy = const_cast<float*>(qy);
    g.S = S;
    const int pairs = S * (g.H / 2);
    const dim3 grid_r((pairs + kGenRowWarps - 1) / kGenRowWarps);
    const dim3 grid_c((g.M1 + gs->col_tile - 1) / gs->col_tile, S);
    cudaError_t e;
    for (int mode = 0; mode < 3; ++mode) {
        gen_report_kernel<<<grid_r, kGenRowWarps * 32, gs->srows, st>>>(g, gs->partial, lambda, mode);
        if (mode < 2) gs->cols_kern<<<grid_c, gs->col_threads, gs->scols, st>>>(g);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    std::vector<double> h((size_t)pairs * kGenReportSums);
    if ((e = cudaMemcpyAsync(h.data(), gs->partial, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return e;
    const int PP = g.H / 2;
    for (int sl = 0; sl < S; ++sl) {
        double v[kGenReportSums] = {0, 0, 0, 0, 0};
        for (int q = 0; q < PP; ++q)
            for (int t = 0; t < kGenReportSums; ++t) v[t] += h[((size_t)sl * PP + q) * kGenReportSums + t];
        rep[sl].objective = 0.5 * lambda * v[0] + v[1];
        rep[sl].gap = v[2] / (2.0 * lambda) + v[3];
        rep[sl].stationarity = std::sqrt(v[4]);
        rep[sl].data_residual = std::sqrt(v[0]);
        rep[sl].iters = iters;
        rep[sl].pad = 0;
    }
    return cudaSuccess;
}

// L = ||K|| of every slice's operator (W = M = mask) by power_iters steps of the power
// iteration on K^T K from a fixed pseudo-random start; synchronises st.
cudaError_t gen_opnorm(GenSolver* gs, const unsigned char* mask, int S, int power_iters, double* L_out,
                       cudaStream_t st) {
    GenParams g = gs->g;
    g.mask = mask;
    g.S = S;
    const size_t n = (size_t)S * g.H * g.W;
    const int pairs = S * (g.H / 2);
    const dim3 grid_r((pairs + kGenRowWarps - 1) / kGenRowWarps);
    const dim3 grid_c((g.M1 + gs->col_tile - 1) / gs->col_tile, S);
    const dim3 grid_n((S + 127) / 128);
    float* buf = nullptr;  // x, y [n] each, scale [S]
    double* est = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&buf, (2 * n + S) * sizeof(float))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&est, (size_t)S * sizeof(double))) != cudaSuccess) {
        cudaFree(buf);
        return e;
    }
    float* x = buf;
    float* y = buf + n;
    float* scale = buf + 2 * n;
    gen_opnorm_init_kernel<<<grid_r, kGenRowWarps * 32, 0, st>>>(g, x, gs->partial);
    gen_opnorm_norm_kernel<<<grid_n, 128, 0, st>>>(gs->partial, g.H / 2, S, scale, est);
    for (int it = 0; it < power_iters; ++it) {
        gen_opnorm_rows_kernel<<<grid_r, kGenRowWarps * 32, gs->srows, st>>>(g, x, y, scale, gs->partial, 0);
        gs->cols_kern<<<grid_c, gs->col_threads, gs->scols, st>>>(g);
        gen_opnorm_rows_kernel<<<grid_r, kGenRowWarps * 32, gs->srows, st>>>(g, x, y, scale, gs->partial, 1);
        gs->cols_kern<<<grid_c, gs->col_threads, gs->scols, st>>>(g);
        gen_opnorm_rows_kernel<<<grid_r, kGenRowWarps * 32, gs->srows, st>>>(g, x, y, scale, gs->partial, 2);
        gen_opnorm_norm_kernel<<<grid_n, 128, 0, st>>>(gs->partial, g.H / 2, S, scale, est);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        float* t = x;
        x = y;
        y = t;
    }
    std::vector<double> h(S);
    if (e == cudaSuccess &&
        (e = cudaMemcpyAsync(h.data(), est, (size_t)S * sizeof(double), cudaMemcpyDeviceToHost, st)) == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        for (int sl = 0; sl < S; ++sl) L_out[sl] = std::sqrt(h[sl] > 0.0 ? h[sl] : 0.0);
    cudaStreamSynchronize(st);
    cudaFree(buf);
    cudaFree(est);
    return e;
}

}  // namespace pcs

extern "C" {

int pcs_supported_generic(int H, int W) { return pcs::gen_supported(H, W) ? 1 : 0; }

pcs_status pcs_solve_slices_generic(const float* field, const unsigned char* mask, const float* weight, int S,
                                    int H, int W, int b0_axis, double lambda, double tau, double sigma, int n_iter,
                                    int tv, float* chi_out, pcs_slice_report* rep, void* cuda_stream) {
    PCS_TRACE("pcs_solve_slices_generic");
    if (S < 0) return failg(PCS_EINVAL, "S must be >= 0");
    if (!(lambda > 0.0) || !(tau > 0.0) || !(sigma > 0.0)) return failg(PCS_EINVAL, "lambda, tau, sigma must be > 0");
    if (n_iter < 0) return failg(PCS_EINVAL, "n_iter must be >= 0");
    if (tv != 0 && tv != 1) return failg(PCS_EINVAL, "tv must be 0 or 1");
    if (b0_axis != 0 && b0_axis != 1) return failg(PCS_EINVAL, "b0_axis must be 0 or 1");
    if (!pcs::gen_supported(H, W))
        return failg(PCS_EUNSUPPORTED, "H and W must be even, in [8, 512], with prime factors <= 61");
    if (S == 0) return PCS_OK;
    if (!field || !mask || !chi_out) return failg(PCS_EINVAL, "NULL argument");
    if (field == chi_out) return failg(PCS_EINVAL, "chi_out must not alias field");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t n = (size_t)S * H * W;
    pcs::GenSolver* gs = nullptr;
    float* state = nullptr;  // chibar, p, qx, qy
    pcs_status ret = PCS_OK;
    cudaError_t e;
    if ((e = pcs::gen_create(&gs, H, W, S, b0_axis, tv)) != cudaSuccess ||
        (e = cudaMalloc(&state, 4 * n * sizeof(float))) != cudaSuccess) {
        ret = failg(PCS_ECUDA, "set-up", e);
    } else if ((e = pcs::gen_enqueue(gs, field, mask, weight, chi_out, state, state + n, state + 2 * n, state + 3 * n,
                                     S, lambda, tau, sigma, n_iter, st, 0, nullptr, nullptr, nullptr)) != cudaSuccess) {
        ret = failg(PCS_ECUDA, "launch", e);
    } else if (rep && (e = pcs::gen_report(gs, field, mask, weight, chi_out, state + n, state + 2 * n, state + 3 * n, S,
                                           lambda, n_iter, rep, st)) != cudaSuccess) {
        ret = failg(PCS_ECUDA, "report", e);
    }
    // synchronous: the call owns its scratch
    cudaError_t se = cudaStreamSynchronize(st);
    if (ret == PCS_OK && se != cudaSuccess) ret = failg(PCS_ECUDA, "stream sync", se);
    cudaFree(state);
    pcs::gen_destroy(gs);
    return ret;
}

}  // extern "C"
