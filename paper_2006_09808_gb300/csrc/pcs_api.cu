// pcs_api.cu -- the C ABI of libpcs (declared in include/pcs.h).
//
// Host side of the solver: argument validation, the FP64 dipole-kernel and
// twiddle tables, context-owned scratch, kernel variant selection and launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pcs.h"
#include "pd_launch.cuh"
#include "pcs_trace.h"

namespace {

thread_local std::string g_last_error;

pcs_status fail(pcs_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

pcs_status cuda_fail(cudaError_t e, const char* what) {
    pcs_status st = (e == cudaErrorMemoryAllocation) ? PCS_ENOMEM : PCS_ECUDA;
    return fail(st, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define PCS_CUDA(call, what)                         \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

std::vector<pcs::KernelEntry> all_entries() {
    std::vector<pcs::KernelEntry> v;
    const pcs::KernelEntry* (*fns[])(int*) = {pcs::entries_64,  pcs::entries_128, pcs::entries_192,
                                               pcs::entries_256, pcs::entries_384, pcs::entries_512};
    for (auto fn : fns) {
        int n = 0;
        const pcs::KernelEntry* e = fn(&n);
        for (int k = 0; k < n; ++k) v.push_back(e[k]);
    }
    return v;
}

const std::vector<pcs::KernelEntry>& entries() {
    static const std::vector<pcs::KernelEntry> v = all_entries();
    return v;
}

// First matching entry for (H, W) is the default; cluster_size > 0, kernel
// (1 streaming, 2 resident), threads and tile narrow the choice.
const pcs::KernelEntry* find_entry(int H, int W, int cluster_size, int kernel = 0, int threads = 0, int tile = 0) {
    for (const auto& e : entries())
        if (e.H == H && e.W == W && (cluster_size <= 0 || e.C == cluster_size) &&
            (kernel <= 0 || e.resident == (kernel == 2 ? 1 : 0)) && (threads <= 0 || e.threads == threads) &&
            (tile <= 0 || e.tile == tile))
            return &e;
    return nullptr;
}

}  // namespace

namespace pcs {
// error text for the other translation units of the library
pcs_status set_last_error(pcs_status st, const char* msg) { return fail(st, "%s", msg); }
}  // namespace pcs

// ------------------------------------------------------------------ tables (FP64 on the host)

namespace pcs {

// D(k) = 1/3 - k_par^2/|k|^2 with D(0) = 0 on the FFT grid (Eq. (1)'s dipole
// kernel), laid out for the column pass: dtab[kx][ky], kx in [0, W/2), every
// entry divided by H*W (the unnormalised transforms' scale).  Column kx = 0
// holds Dm = (D(ky,0) + D(ky,W/2))/2 and ddtab[ky] = (D(ky,0) - D(ky,W/2))/2,
// the two halves of the packed DC/Nyquist column.
template <class T>
void build_dipole_tables_t(int H, int W, int b0_axis, std::vector<T>& dtab, std::vector<T>& ddtab) {
    const int M = W / 2;
    auto freq = [](int idx, int n) {  // cycles per pixel, numpy.fft.fftfreq convention
        return (idx < (n + 1) / 2) ? (double)idx / n : (double)(idx - n) / n;
    };
    auto D = [&](int ky_idx, int kx_idx) {
        const double ky = freq(ky_idx, H), kx = freq(kx_idx, W);
        const double k2 = kx * kx + ky * ky;
        if (k2 == 0.0) return 0.0;
        const double kp = (b0_axis == 0) ? ky : kx;
        return 1.0 / 3.0 - kp * kp / k2;
    };
    const double scale = 1.0 / ((double)H * (double)W);
    dtab.assign((size_t)M * H, T(0));
    ddtab.assign((size_t)H, T(0));
    for (int kx = 0; kx < M; ++kx)
        for (int ky = 0; ky < H; ++ky) dtab[(size_t)kx * H + ky] = (T)(D(ky, kx) * scale);
    for (int ky = 0; ky < H; ++ky) {
        const double d0 = D(ky, 0), d1 = D(ky, M);
        dtab[ky] = (T)(0.5 * (d0 + d1) * scale);
        ddtab[ky] = (T)(0.5 * (d0 - d1) * scale);
    }
}
void build_dipole_tables(int H, int W, int b0_axis, std::vector<float>& dtab, std::vector<float>& ddtab) {
    build_dipole_tables_t<float>(H, W, b0_axis, dtab, ddtab);
}

// tw[m] = exp(-2 pi i m / n), m in [0, n)
template <class V>
void build_twiddles_t(int n, std::vector<V>& tw) {
    tw.resize(n);
    const double two_pi = 6.283185307179586476925286766559;
    for (int m = 0; m < n; ++m) {
        const double a = two_pi * (double)m / (double)n;
        tw[m].x = (decltype(tw[m].x))std::cos(a);
        tw[m].y = (decltype(tw[m].y))-std::sin(a);
    }
}
void build_twiddles(int n, std::vector<float2>& tw) { build_twiddles_t<float2>(n, tw); }

}  // namespace pcs

// ------------------------------------------------------------------ context

namespace pcs {
// any-size slices (pd_generic.cu)
struct GenSolver;
bool gen_supported(int H, int W);
cudaError_t gen_create(GenSolver** out, int H, int W, int max_slices, int b0_axis, int tv);
void gen_destroy(GenSolver* gs);
cudaError_t gen_enqueue(GenSolver* gs, const float* field, const unsigned char* mask, const float* weight,
                        float* chi, float* chibar, float* p, float* qx, float* qy, int S, double lambda, double tau,
                        double sigma, int n_iter, cudaStream_t st, int resume, const int* active,
                        const float* inv_den_slice, float2* spec);
cudaError_t gen_report(GenSolver* gs, const float* field, const unsigned char* mask, const float* weight,
                       const float* chi, const float* p, const float* qx, const float* qy, int S, double lambda,
                       int iters, pcs_slice_report* rep, cudaStream_t st);
cudaError_t gen_opnorm(GenSolver* gs, const unsigned char* mask, int S, int power_iters, double* L_out,
                       cudaStream_t st);
}  // namespace pcs

struct pcs_ctx {
    int H = 0, W = 0, max_slices = 0;
    pcs_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0;
    const pcs::KernelEntry* entry = nullptr;  // NULL for an any-size context
    pcs::GenSolver* gen = nullptr;            // any-size context: row/column kernels (pd_generic.cu)
    int max_clusters = 0;
    int max_clusters_aux = 0;
    int last_iters = 0;
    // device tables
    float* dtab = nullptr;
    float* ddtab = nullptr;
    float2* twid = nullptr;
    // scratch state
    float* chibar = nullptr;
    float* p = nullptr;
    float* qx = nullptr;
    float* qy = nullptr;
    // staging for the host-buffer entry point (allocated on first use)
    float* st_field = nullptr;
    unsigned char* st_mask = nullptr;
    float* st_chi = nullptr;
    // diagnostics / power iteration (allocated on first use)
    double* partials = nullptr;
    double* Ldev = nullptr;
    float* xa = nullptr;
    float* xb = nullptr;
    int* active = nullptr;  // monitored solves: per-slice flags
    // balanced schedule (more slices than resident clusters): segments, offsets, per-slice
    // flags, and the key (S, n_iter, clusters) the uploaded schedule was built for
    int4* sched = nullptr;
    int* sched_off = nullptr;
    int* seg_flags = nullptr;
    int sched_S = -1, sched_N = -1, sched_K = -1;
    int* err = nullptr;  // device error word of the schedule's bounded waits
    // CUDA-graph replay (use_graph): the last captured solve and its arguments
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    pcs::PDParams graph_prm{};
    int graph_ncl = 0;
    std::mutex mu;
};

namespace {

void free_ctx(pcs_ctx* c) {
    if (!c) return;
    void* ptrs[] = {c->dtab,     c->ddtab,  c->twid,     c->chibar, c->p,  c->qx,   c->qy,
                    c->st_field, c->st_mask, c->st_chi,  c->partials, c->Ldev, c->xa,  c->xb,
                    c->active,   c->sched,   c->sched_off, c->seg_flags, c->err};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    pcs::gen_destroy(c->gen);
    delete c;
}

size_t slice_elems(const pcs_ctx* c) { return (size_t)c->H * (size_t)c->W; }

bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

pcs_status validate_solve(pcs_ctx* ctx, const void* field, const void* mask, int S, double lambda, double tau,
                          double sigma, int n_iter, const void* chi_out) {
    if (!ctx) return fail(PCS_EINVAL, "ctx is NULL");
    if (S < 0 || S > ctx->max_slices) return fail(PCS_EINVAL, "S=%d outside [0, max_slices=%d]", S, ctx->max_slices);
    if (S == 0) return PCS_OK;
    if (!field || !mask || !chi_out) return fail(PCS_EINVAL, "NULL field/mask/chi_out");
    if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(PCS_EINVAL, "lambda must be > 0 (got %g)", lambda);
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(PCS_EINVAL, "tau must be > 0 (got %g)", tau);
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(PCS_EINVAL, "sigma must be > 0 (got %g)", sigma);
    if (n_iter < 0) return fail(PCS_EINVAL, "n_iter must be >= 0 (got %d)", n_iter);
    if (field == chi_out) return fail(PCS_EINVAL, "chi_out must not alias field");
    return PCS_OK;
}

// McNaughton's wrap-around rule over clusters with the slices' iterations laid end to end:
// cluster c covers positions [c T, (c+1) T), T = ceil(S N / K) >= N, so a slice is split at most
// once.  Each cluster runs its pieces in reverse order, so the first part of a split slice (the
// end of one cluster's range) runs at the start of that cluster's time and its second part (the
// start of the next cluster's range) at the end of the next cluster's time: with equal speeds
// the first part is done T - N iterations early, and the second waits on a flag only as a
// guard.  Segment = (slice, first iteration, end iteration, bit 0 wait / bit 1 signal).
void build_schedule(int S, int N, int K, std::vector<int4>& segs, std::vector<int>& off) {
    segs.clear();
    off.assign(K + 1, 0);
    const long long U = (long long)S * N;
    const long long T = (U + K - 1) / K;
    for (int c = 0; c < K; ++c) {
        off[c] = (int)segs.size();
        const long long lo = c * T, hi = std::min(U, lo + T);
        std::vector<int4> pieces;
        for (long long q = lo; q < hi;) {
            const int sl = (int)(q / N);
            const int b = (int)(q - (long long)sl * N);
            const int e = (int)std::min<long long>(N, b + (hi - q));
            pieces.push_back(make_int4(sl, b, e, (b > 0 ? 1 : 0) | (e < N ? 2 : 0)));
            q += e - b;
        }
        for (auto it = pieces.rbegin(); it != pieces.rend(); ++it) segs.push_back(*it);
    }
    off[K] = (int)segs.size();
}

constexpr long long kWaitLimitCycles = 4000000000LL;  // ~2 s at the maximum SM clock

pcs_status launch_solve(pcs_ctx* ctx, const float* field, const unsigned char* mask, int S, double lambda,
                        double tau, double sigma, int n_iter, float* chi_out,
                        const float* inv_den_slice = nullptr, const pcs::KernelEntry* entry = nullptr,
                        int ncl_override = 0, int resume = 0, const int* active = nullptr,
                        const float* weight = nullptr) {
    if (!aligned16(field) || !aligned16(mask) || !aligned16(chi_out) || !aligned16(weight))
        return fail(PCS_EINVAL, "device buffers must be 16-byte aligned");
    if (ctx->gen) {
        if (entry) return fail(PCS_EUNSUPPORTED, "a compiled variant was asked for an any-size context");
        PCS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
        PCS_CUDA(pcs::gen_enqueue(ctx->gen, field, mask, weight, chi_out, ctx->chibar, ctx->p, ctx->qx, ctx->qy, S,
                                  lambda, tau, sigma, n_iter, ctx->stream, resume, active, inv_den_slice,
                                  nullptr),
                 "launch of the any-size kernels");
        ctx->last_iters = n_iter;
        return PCS_OK;
    }
    pcs::PDParams prm;
    std::memset(&prm, 0, sizeof(prm));  // padding too: the graph cache compares whole structs
    prm.field = field;
    prm.mask = mask;
    prm.chi = chi_out;
    prm.chibar = ctx->chibar;
    prm.p = ctx->p;
    prm.qx = ctx->qx;
    prm.qy = ctx->qy;
    prm.dtab = ctx->dtab;
    prm.ddtab = ctx->ddtab;
    prm.twid = ctx->twid;
    prm.S = S;
    prm.n_iter = n_iter;
    prm.sigma = (float)sigma;
    prm.tau = (float)tau;
    prm.inv_den = (float)(1.0 / (1.0 + sigma / lambda));
    prm.inv_den_slice = inv_den_slice;
    prm.active = active;
    prm.resume = resume;
    prm.tv_iso = ctx->opt.tv;
    prm.weight = weight;
    int ncl = ncl_override > 0 ? ncl_override : ctx->max_clusters;
    if (ctx->opt.max_clusters > 0 && ctx->opt.max_clusters < ncl) ncl = ctx->opt.max_clusters;
    if (ncl > S) ncl = S;
    if (ncl < 1) ncl = 1;
    PCS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    // more slices than resident clusters: balance the iterations over the clusters (streaming
    // kernel, plain solves; the monitored path's active flags keep whole slices)
    const bool balanced = !active && ncl < S && n_iter > 0 && (entry ? entry : ctx->entry)->launch_sched;
    if (balanced) {
        if (!ctx->sched) {
            const size_t nseg = (size_t)ctx->max_slices * 2 + 1;
            PCS_CUDA(cudaMalloc(&ctx->sched, nseg * sizeof(int4)), "cudaMalloc schedule");
            PCS_CUDA(cudaMalloc(&ctx->sched_off, (size_t)(ctx->max_slices + 1) * sizeof(int)), "cudaMalloc schedule");
            PCS_CUDA(cudaMalloc(&ctx->seg_flags, (size_t)ctx->max_slices * sizeof(int)), "cudaMalloc flags");
        }
        if (ctx->sched_S != S || ctx->sched_N != n_iter || ctx->sched_K != ncl) {
            std::vector<int4> segs;
            std::vector<int> off;
            build_schedule(S, n_iter, ncl, segs, off);
            PCS_CUDA(cudaMemcpyAsync(ctx->sched, segs.data(), segs.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                     ctx->stream), "schedule upload");
            PCS_CUDA(cudaMemcpyAsync(ctx->sched_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice,
                                     ctx->stream), "schedule upload");
            PCS_CUDA(cudaStreamSynchronize(ctx->stream), "schedule upload");  // host vectors go out of scope
            ctx->sched_S = S;
            ctx->sched_N = n_iter;
            ctx->sched_K = ncl;
        }
        prm.sched = ctx->sched;
        prm.sched_off = ctx->sched_off;
        prm.seg_flags = ctx->seg_flags;
        prm.err = ctx->err;
        prm.wait_limit = kWaitLimitCycles;
    }
    // the flags are cleared on the stream right before every launch (inside a captured graph too)
    auto launch = [&](const pcs::KernelEntry* e) -> cudaError_t {
        if (balanced) {
            cudaError_t me = cudaMemsetAsync(ctx->seg_flags, 0, (size_t)S * sizeof(int), ctx->stream);
            if (me != cudaSuccess) return me;
        }
        return balanced ? e->launch_sched(prm, ncl, ctx->stream) : e->launch(prm, ncl, ctx->stream);
    };
    if (entry && entry != ctx->entry) {  // another variant of the same size (monitored solves)
        PCS_CUDA(launch(entry), "launch of the primal-dual kernel");
        ctx->last_iters = n_iter;
        return PCS_OK;
    }
    if (ctx->opt.use_graph) {
        // replay the captured graph when the arguments are those it was captured with
        const bool same = ctx->graph_exec && ncl == ctx->graph_ncl &&
                          std::memcmp(&prm, &ctx->graph_prm, sizeof(prm)) == 0;
        if (!same) {
            if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
            if (ctx->graph) cudaGraphDestroy(ctx->graph);
            ctx->graph_exec = nullptr;
            ctx->graph = nullptr;
            PCS_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
            cudaError_t le = launch(ctx->entry);
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
            if (le != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return cuda_fail(le, "launch during graph capture");
            }
            PCS_CUDA(ce, "graph capture end");
            ctx->graph = g;
            PCS_CUDA(cudaGraphInstantiate(&ctx->graph_exec, g, 0), "graph instantiate");
            ctx->graph_prm = prm;
            ctx->graph_ncl = ncl;
        }
        PCS_CUDA(cudaGraphLaunch(ctx->graph_exec, ctx->stream), "graph launch");
    } else {
        PCS_CUDA(launch(ctx->entry), "launch of the primal-dual kernel");
    }
    ctx->last_iters = n_iter;
    return PCS_OK;
}

// The context's error word, read after the work on its stream: set when a bounded wait of
// the balanced schedule gave up, which makes that solve's results invalid.  Clears the word.
pcs_status check_err_word(pcs_ctx* ctx) {
    int flag = 0;
    PCS_CUDA(cudaMemcpyAsync(&flag, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "D2H error word");
    PCS_CUDA(cudaStreamSynchronize(ctx->stream), "stream sync");
    if (flag) {
        PCS_CUDA(cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream), "clear error word");
        return fail(PCS_ETIMEOUT, "a solve on this context gave up waiting for another cluster (its results are invalid)");
    }
    return PCS_OK;
}

// Bounded wait of the balanced schedule on a flag nothing sets.
__global__ void wait_selftest_kernel(const int* flag, long long limit, int* out) {
    if (threadIdx.x == 0) out[0] = pcs::wait_flag(flag, limit) ? 0 : 1;
}

}  // namespace

// ------------------------------------------------------------------ diagnostics and step size

namespace {

pcs_status ensure_aux(pcs_ctx* c) {
    if (c->partials) return PCS_OK;
    const size_t n = slice_elems(c) * (size_t)c->max_slices;
    PCS_CUDA(cudaMalloc(&c->partials, (size_t)c->max_slices * c->entry->C * pcs::kReportSums * sizeof(double)),
             "cudaMalloc partials");
    PCS_CUDA(cudaMalloc(&c->Ldev, (size_t)c->max_slices * sizeof(double)), "cudaMalloc L");
    PCS_CUDA(cudaMalloc(&c->xa, n * sizeof(float)), "cudaMalloc power-iteration buffer");
    PCS_CUDA(cudaMalloc(&c->xb, n * sizeof(float)), "cudaMalloc power-iteration buffer");
    return PCS_OK;
}

pcs::AuxParams aux_params(pcs_ctx* c, int S) {
    pcs::AuxParams a{};
    a.dtab = c->dtab;
    a.ddtab = c->ddtab;
    a.twid = c->twid;
    a.partials = c->partials;
    a.Lout = c->Ldev;
    a.xa = c->xa;
    a.xb = c->xb;
    a.p = c->p;
    a.qx = c->qx;
    a.qy = c->qy;
    a.S = S;
    return a;
}

int aux_clusters(pcs_ctx* c, int S) {
    int ncl = c->max_clusters_aux;
    if (ncl > S) ncl = S;
    return ncl < 1 ? 1 : ncl;
}

}  // namespace

namespace pcs {

// Objective, Fenchel-Young gap, stationarity and residual of every slice at
// (chi, p, q) where p, q are the context's dual state of the last solve.
pcs_status ctx_report(pcs_ctx* c, const float* field, const unsigned char* mask, int S, double lambda,
                      const float* chi, pcs_slice_report* rep, const float* weight) {
    if (c->gen) {
        PCS_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
        PCS_CUDA(gen_report(c->gen, field, mask, weight, chi, c->p, c->qx, c->qy, S, lambda, c->last_iters, rep,
                            c->stream),
                 "any-size report");
        return PCS_OK;
    }
    pcs_status st = ensure_aux(c);
    if (st != PCS_OK) return st;
    AuxParams a = aux_params(c, S);
    a.field = field;
    a.mask = mask;
    a.chi = chi;
    a.lam = (float)lambda;
    a.tv_iso = c->opt.tv;
    a.weight = weight;
    PCS_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    PCS_CUDA(c->entry->launch_report(a, aux_clusters(c, S), c->stream), "launch of the report kernel");
    const int C = c->entry->C;
    std::vector<double> h((size_t)S * C * kReportSums);
    PCS_CUDA(cudaMemcpyAsync(h.data(), c->partials, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
             "D2H partials");
    PCS_CUDA(cudaStreamSynchronize(c->stream), "stream sync");
    for (int s = 0; s < S; ++s) {
        double v[kReportSums] = {0, 0, 0, 0, 0};
        for (int q = 0; q < C; ++q)
            for (int t = 0; t < kReportSums; ++t) v[t] += h[((size_t)s * C + q) * kReportSums + t];
        rep[s].objective = 0.5 * lambda * v[0] + v[1];
        rep[s].gap = v[2] / (2.0 * lambda) + v[3];
        rep[s].stationarity = std::sqrt(v[4]);
        rep[s].data_residual = std::sqrt(v[0]);
        rep[s].iters = c->last_iters;
        rep[s].pad = 0;
    }
    return PCS_OK;
}

pcs_status ctx_opnorm(pcs_ctx* c, const unsigned char* mask, int S, int power_iters, double* L_out) {
    if (c->gen) {
        PCS_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
        PCS_CUDA(gen_opnorm(c->gen, mask, S, power_iters, L_out, c->stream), "any-size power iteration");
        return PCS_OK;
    }
    pcs_status st = ensure_aux(c);
    if (st != PCS_OK) return st;
    AuxParams a = aux_params(c, S);
    a.mask = mask;
    a.iters = power_iters;
    PCS_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    PCS_CUDA(c->entry->launch_opnorm(a, aux_clusters(c, S), c->stream), "launch of the power-iteration kernel");
    PCS_CUDA(cudaMemcpyAsync(L_out, c->Ldev, (size_t)S * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
             "D2H L");
    PCS_CUDA(cudaStreamSynchronize(c->stream), "stream sync");
    return PCS_OK;
}

}  // namespace pcs

extern "C" {

pcs_status pcs_options_default(pcs_options* opt) {
    if (!opt) return fail(PCS_EINVAL, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    return PCS_OK;
}

int pcs_supported_size(int H, int W) { return find_entry(H, W, 0) != nullptr ? 1 : 0; }

pcs_status pcs_create(pcs_ctx** out, int H, int W, int max_slices, const pcs_options* opt, void* cuda_stream) {
    PCS_TRACE("pcs_create");
    if (!out) return fail(PCS_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_slices < 1) return fail(PCS_EINVAL, "max_slices must be >= 1 (got %d)", max_slices);
    pcs_options o;
    pcs_options_default(&o);
    if (opt) o = *opt;
    if (o.b0_axis != 0 && o.b0_axis != 1) return fail(PCS_EINVAL, "b0_axis must be 0 or 1");
    if (o.kernel < 0 || o.kernel > 2) return fail(PCS_EINVAL, "kernel must be 0, 1 or 2");
    if (o.tv != 0 && o.tv != 1) return fail(PCS_EINVAL, "tv must be 0 (anisotropic) or 1 (isotropic)");
    if (o.use_graph && cuda_stream == nullptr)
        return fail(PCS_EINVAL, "use_graph needs a non-NULL stream (the legacy stream cannot be captured)");
    const pcs::KernelEntry* entry = find_entry(H, W, o.cluster_size, o.kernel, o.threads, o.tile);
    const bool any_size = !entry && find_entry(H, W, 0) == nullptr && o.cluster_size == 0 && o.kernel == 0 &&
                          o.threads == 0 && o.tile == 0 && pcs::gen_supported(H, W);
    if (!entry && !any_size)
        return fail(PCS_EUNSUPPORTED, "no kernel for %d x %d slices with cluster_size %d, kernel %d, threads %d, tile %d",
                    H, W, o.cluster_size, o.kernel, o.threads, o.tile);

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1) return fail(PCS_ECUDA, "no CUDA device (%s)", cudaGetErrorString(e));

    pcs_ctx* c = new pcs_ctx();
    c->H = H;
    c->W = W;
    c->max_slices = max_slices;
    c->opt = o;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->entry = entry;
    auto bail = [&](pcs_status st) {
        free_ctx(c);
        return st;
    };
    if ((e = cudaGetDevice(&c->device)) != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
    if (any_size) {
        // the any-size row/column kernels: their own tables and spectrum; the state as below
        const size_t n = slice_elems(c) * (size_t)max_slices;
        if ((e = pcs::gen_create(&c->gen, H, W, max_slices, o.b0_axis, o.tv)) != cudaSuccess)
            return bail(cuda_fail(e, "any-size set-up"));
        float** st[] = {&c->chibar, &c->p, &c->qx, &c->qy};
        for (float** q : st)
            if ((e = cudaMalloc(q, n * sizeof(float))) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
        if ((e = cudaMalloc(&c->err, sizeof(int))) != cudaSuccess || (e = cudaMemset(c->err, 0, sizeof(int))) != cudaSuccess)
            return bail(cuda_fail(e, "cudaMalloc"));
        *out = c;
        return PCS_OK;
    }
    if ((e = entry->prepare(&c->max_clusters, &c->max_clusters_aux)) != cudaSuccess) return bail(cuda_fail(e, "kernel attributes"));
    if (c->max_clusters < 1)
        return bail(fail(PCS_ECUDA, "kernel %dx%d/C=%d cannot be made resident", H, W, entry->C));

    std::vector<float> dtab, ddtab;
    std::vector<float2> tw;
    pcs::build_dipole_tables(H, W, o.b0_axis, dtab, ddtab);
    pcs::build_twiddles(H > W ? H : W, tw);
    const size_t n = slice_elems(c) * (size_t)max_slices;
    struct {
        void** ptr;
        size_t bytes;
    } allocs[] = {
        {(void**)&c->dtab, dtab.size() * sizeof(float)},  {(void**)&c->ddtab, ddtab.size() * sizeof(float)},
        {(void**)&c->twid, tw.size() * sizeof(float2)},   {(void**)&c->chibar, n * sizeof(float)},
        {(void**)&c->p, n * sizeof(float)},               {(void**)&c->qx, n * sizeof(float)},
        {(void**)&c->qy, n * sizeof(float)},              {(void**)&c->err, sizeof(int)},
    };
    for (auto& a : allocs)
        if ((e = cudaMalloc(a.ptr, a.bytes)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    if ((e = cudaMemcpy(c->dtab, dtab.data(), dtab.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->ddtab, ddtab.data(), ddtab.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->twid, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(c->err, 0, sizeof(int))) != cudaSuccess)
        return bail(cuda_fail(e, "table upload"));
    *out = c;
    return PCS_OK;
}

pcs_status pcs_schedule_plan(int S, int n_iter, int clusters, int* segments, int* n_segments, int* offsets) {
    if (S < 1 || n_iter < 1 || clusters < 1 || clusters >= S || !n_segments)
        return fail(PCS_EINVAL, "needs 1 <= clusters < S and n_iter >= 1");
    std::vector<int4> segs;
    std::vector<int> off;
    build_schedule(S, n_iter, clusters, segs, off);
    const int cap = *n_segments;
    *n_segments = (int)segs.size();
    if (!segments || !offsets) return PCS_OK;  // size query
    if (cap < (int)segs.size()) return fail(PCS_EINVAL, "segments holds %d entries, %zu needed", cap, segs.size());
    for (size_t k = 0; k < segs.size(); ++k) {
        segments[4 * k + 0] = segs[k].x;
        segments[4 * k + 1] = segs[k].y;
        segments[4 * k + 2] = segs[k].z;
        segments[4 * k + 3] = segs[k].w;
    }
    for (int c = 0; c <= clusters; ++c) offsets[c] = off[c];
    return PCS_OK;
}

pcs_status pcs_check(pcs_ctx* ctx) {
    if (!ctx) return fail(PCS_EINVAL, "ctx is NULL");
    PCS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    return check_err_word(ctx);
}

pcs_status pcs_selftest_wait(void* cuda_stream, long long limit_cycles, int* gave_up) {
    if (!gave_up || limit_cycles < 0) return fail(PCS_EINVAL, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int* d = nullptr;
    PCS_CUDA(cudaMalloc(&d, 2 * sizeof(int)), "cudaMalloc");
    cudaError_t e;
    if ((e = cudaMemsetAsync(d, 0, 2 * sizeof(int), st)) == cudaSuccess) {
        wait_selftest_kernel<<<1, 32, 0, st>>>(d, limit_cycles, d + 1);
        if ((e = cudaGetLastError()) == cudaSuccess &&
            (e = cudaMemcpyAsync(gave_up, d + 1, sizeof(int), cudaMemcpyDeviceToHost, st)) == cudaSuccess)
            e = cudaStreamSynchronize(st);
    }
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    return PCS_OK;
}

pcs_status pcs_set_stream(pcs_ctx* ctx, void* cuda_stream) {
    if (!ctx) return fail(PCS_EINVAL, "ctx is NULL");
    if (ctx->opt.use_graph && cuda_stream == nullptr) return fail(PCS_EINVAL, "use_graph needs a non-NULL stream");
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return PCS_OK;
}

pcs_status pcs_solve_slices(pcs_ctx* ctx, const float* field, const unsigned char* mask, int S, double lambda,
                            double tau, double sigma, int n_iter, float* chi_out, pcs_slice_report* rep) {
    PCS_TRACE("pcs_solve_slices");
    pcs_status st = validate_solve(ctx, field, mask, S, lambda, tau, sigma, n_iter, chi_out);
    if (st != PCS_OK || S == 0) return st;
    std::unique_lock<std::mutex> lk(ctx->mu, std::try_to_lock);
    if (!lk.owns_lock()) return fail(PCS_EBUSY, "context in use by another thread");
    st = launch_solve(ctx, field, mask, S, lambda, tau, sigma, n_iter, chi_out);
    if (st != PCS_OK || !rep) return st;
    st = pcs::ctx_report(ctx, field, mask, S, lambda, chi_out, rep, nullptr);  // synchronises the stream
    return st != PCS_OK ? st : check_err_word(ctx);
}

pcs_status pcs_solve_slices_weighted(pcs_ctx* ctx, const float* field, const unsigned char* mask,
                                     const float* weight, int S, double lambda, double tau, double sigma,
                                     int n_iter, float* chi_out, pcs_slice_report* rep) {
    PCS_TRACE("pcs_solve_slices_weighted");
    pcs_status st = validate_solve(ctx, field, mask, S, lambda, tau, sigma, n_iter, chi_out);
    if (st != PCS_OK || S == 0) return st;
    if (!weight) return fail(PCS_EINVAL, "weight is NULL");
    if (ctx->entry && ctx->entry->resident)
        return fail(PCS_EUNSUPPORTED, "weighted solves run on the streaming kernel (create the context with kernel 1)");
    std::unique_lock<std::mutex> lk(ctx->mu, std::try_to_lock);
    if (!lk.owns_lock()) return fail(PCS_EBUSY, "context in use by another thread");
    st = launch_solve(ctx, field, mask, S, lambda, tau, sigma, n_iter, chi_out, nullptr, nullptr, 0, 0, nullptr,
                      weight);
    if (st != PCS_OK || !rep) return st;
    st = pcs::ctx_report(ctx, field, mask, S, lambda, chi_out, rep, weight);  // synchronises the stream
    return st != PCS_OK ? st : check_err_word(ctx);
}

pcs_status pcs_solve_slices_host(pcs_ctx* ctx, const float* field_host, const unsigned char* mask_host, int S,
                                 double lambda, double tau, double sigma, int n_iter, float* chi_out_host,
                                 pcs_slice_report* rep) {
    PCS_TRACE("pcs_solve_slices_host");
    pcs_status st = validate_solve(ctx, field_host, mask_host, S, lambda, tau, sigma, n_iter, chi_out_host);
    if (st != PCS_OK || S == 0) return st;
    std::unique_lock<std::mutex> lk(ctx->mu, std::try_to_lock);
    if (!lk.owns_lock()) return fail(PCS_EBUSY, "context in use by another thread");
    PCS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    const size_t n = slice_elems(ctx) * (size_t)ctx->max_slices;
    if (!ctx->st_field) {
        PCS_CUDA(cudaMalloc(&ctx->st_field, n * sizeof(float)), "cudaMalloc staging");
        PCS_CUDA(cudaMalloc(&ctx->st_mask, n), "cudaMalloc staging");
        PCS_CUDA(cudaMalloc(&ctx->st_chi, n * sizeof(float)), "cudaMalloc staging");
    }
    const size_t m = slice_elems(ctx) * (size_t)S;
    PCS_CUDA(cudaMemcpyAsync(ctx->st_field, field_host, m * sizeof(float), cudaMemcpyHostToDevice, ctx->stream),
             "H2D field");
    PCS_CUDA(cudaMemcpyAsync(ctx->st_mask, mask_host, m, cudaMemcpyHostToDevice, ctx->stream), "H2D mask");
    st = launch_solve(ctx, ctx->st_field, ctx->st_mask, S, lambda, tau, sigma, n_iter, ctx->st_chi);
    if (st != PCS_OK) return st;
    PCS_CUDA(cudaMemcpyAsync(chi_out_host, ctx->st_chi, m * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream),
             "D2H chi");
    st = check_err_word(ctx);  // synchronises the stream
    if (st != PCS_OK) return st;
    if (rep) return pcs::ctx_report(ctx, ctx->st_field, ctx->st_mask, S, lambda, ctx->st_chi, rep, nullptr);
    return PCS_OK;
}

pcs_status pcs_report(pcs_ctx* ctx, const float* field, const unsigned char* mask, int S, double lambda,
                      const float* chi, pcs_slice_report* rep) {
    PCS_TRACE("pcs_report");
    if (!ctx) return fail(PCS_EINVAL, "ctx is NULL");
    if (S < 0 || S > ctx->max_slices) return fail(PCS_EINVAL, "S=%d outside [0, max_slices]", S);
    if (S == 0) return PCS_OK;
    if (!field || !mask || !chi || !rep) return fail(PCS_EINVAL, "NULL argument");
    if (!(lambda > 0.0)) return fail(PCS_EINVAL, "lambda must be > 0");
    return pcs::ctx_report(ctx, field, mask, S, lambda, chi, rep, nullptr);
}

pcs_status pcs_opnorm(pcs_ctx* ctx, const unsigned char* mask, int S, int power_iters, double* L_out) {
    PCS_TRACE("pcs_opnorm");
    if (!ctx) return fail(PCS_EINVAL, "ctx is NULL");
    if (S < 0 || S > ctx->max_slices) return fail(PCS_EINVAL, "S=%d outside [0, max_slices]", S);
    if (S == 0) return PCS_OK;
    if (!mask || !L_out) return fail(PCS_EINVAL, "NULL argument");
    if (power_iters < 1) return fail(PCS_EINVAL, "power_iters must be >= 1");
    return pcs::ctx_opnorm(ctx, mask, S, power_iters, L_out);
}

pcs_status pcs_solve_slices_monitored(pcs_ctx* ctx, const float* field, const unsigned char* mask, int S,
                                      double lambda, double tau, double sigma, int n_iter, int check_every,
                                      double rel_gap_tol, float* chi_out, pcs_slice_report* rep) {
    PCS_TRACE("pcs_solve_slices_monitored");
    pcs_status st = validate_solve(ctx, field, mask, S, lambda, tau, sigma, n_iter, chi_out);
    if (st != PCS_OK || S == 0) return st;
    if (!rep) return fail(PCS_EINVAL, "rep is required");
    if (check_every < 1) return fail(PCS_EINVAL, "check_every must be >= 1");
    if (!(rel_gap_tol >= 0.0)) return fail(PCS_EINVAL, "rel_gap_tol must be >= 0");
    std::unique_lock<std::mutex> lk(ctx->mu, std::try_to_lock);
    if (!lk.owns_lock()) return fail(PCS_EBUSY, "context in use by another thread");
    PCS_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    // chunked solves resume from the stored state: a streaming variant of this size (any-size
    // contexts resume with their own kernels)
    const pcs::KernelEntry* e = nullptr;
    int ncl = 0;
    if (!ctx->gen) {
        e = ctx->entry->resident ? find_entry(ctx->H, ctx->W, 0, 1) : ctx->entry;
        if (!e) return fail(PCS_EUNSUPPORTED, "no streaming kernel for %d x %d", ctx->H, ctx->W);
        ncl = ctx->max_clusters;
        if (e != ctx->entry) {
            int aux = 0;
            PCS_CUDA(e->prepare(&ncl, &aux), "kernel attributes");
        }
    }
    if (!ctx->active) PCS_CUDA(cudaMalloc(&ctx->active, (size_t)ctx->max_slices * sizeof(int)), "cudaMalloc flags");
    std::vector<int> act(S, 1);
    std::vector<int> iters(S, 0);
    int done = 0;
    while (done < n_iter) {
        const int k = std::min(check_every, n_iter - done);
        PCS_CUDA(cudaMemcpyAsync(ctx->active, act.data(), S * sizeof(int), cudaMemcpyHostToDevice, ctx->stream),
                 "flags upload");
        st = launch_solve(ctx, field, mask, S, lambda, tau, sigma, k, chi_out, nullptr, e, ncl, done > 0 ? 1 : 0,
                          ctx->active);
        if (st != PCS_OK) return st;
        done += k;
        for (int s = 0; s < S; ++s)
            if (act[s]) iters[s] = done;
        // FP64 diagnostics of every slice (frozen slices keep their last state)
        std::vector<pcs_slice_report> r(S);
        st = pcs::ctx_report(ctx, field, mask, S, lambda, chi_out, r.data(), nullptr);
        if (st != PCS_OK) return st;
        int n_active = 0;
        for (int s = 0; s < S; ++s) {
            if (act[s]) rep[s] = r[s];
            rep[s].iters = iters[s];
            if (act[s] && rel_gap_tol > 0.0 && r[s].gap <= rel_gap_tol * std::max(r[s].objective, 1e-300)) act[s] = 0;
            n_active += act[s];
        }
        if (n_active == 0) break;
    }
    ctx->last_iters = done;
    return PCS_OK;
}

void pcs_destroy(pcs_ctx* ctx) { free_ctx(ctx); }

const char* pcs_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ------------------------------------------------------------------ uneven batches

struct pcs_batch {
    struct Class {
        int H = 0, W = 0;
        pcs_ctx* ctx = nullptr;  // holds the chosen variant; max_slices = capacity
        double L = 0.0;
        cudaStream_t stream = nullptr;
        cudaEvent_t done = nullptr;
        cudaEvent_t solved = nullptr;  // the class's solve finished (the next class's solve may start)
        float* pk_field = nullptr;  // packed inputs / outputs [capacity][H][W]
        unsigned char* pk_mask = nullptr;
        float* pk_chi = nullptr;
        float* inv_den = nullptr;  // [capacity]
        int capacity = 0;
        pcs_tuning tuning{};
        bool tuned = false;
    };
    pcs_options opt{};
    int autotune = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    cudaEvent_t fork = nullptr;
    std::vector<Class> classes;
    std::mutex mu;
};

namespace {

void free_class(pcs_batch::Class& c) {
    if (c.ctx) pcs_destroy(c.ctx);
    void* ptrs[] = {c.pk_field, c.pk_mask, c.pk_chi, c.inv_den};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (c.stream) cudaStreamDestroy(c.stream);
    if (c.done) cudaEventDestroy(c.done);
    if (c.solved) cudaEventDestroy(c.solved);
    c = pcs_batch::Class();
}

// Time every compiled variant of H x W on S zero-field slices (trial_iters
// iterations each, after one untimed run) and record them in c.tuning.
pcs_status tune_class(pcs_batch* b, pcs_batch::Class& c, int S, int trial_iters) {
    const size_t n = (size_t)S * c.H * c.W;
    float *f = nullptr, *chi = nullptr;
    unsigned char* m = nullptr;
    PCS_CUDA(cudaMalloc(&f, n * sizeof(float)), "cudaMalloc tuning");
    PCS_CUDA(cudaMalloc(&chi, n * sizeof(float)), "cudaMalloc tuning");
    PCS_CUDA(cudaMalloc(&m, n), "cudaMalloc tuning");
    PCS_CUDA(cudaMemsetAsync(f, 0, n * sizeof(float), c.stream), "memset");
    PCS_CUDA(cudaMemsetAsync(m, 1, n, c.stream), "memset");
    cudaEvent_t e0, e1;
    PCS_CUDA(cudaEventCreate(&e0), "event");
    PCS_CUDA(cudaEventCreate(&e1), "event");
    pcs_tuning& t = c.tuning;
    t = pcs_tuning{};
    t.H = c.H;
    t.W = c.W;
    double best = 1e300;
    pcs_status st = PCS_OK;
    for (const auto& e : entries()) {
        if (e.H != c.H || e.W != c.W || t.n_candidates >= 8) continue;
        pcs_options o = b->opt;
        o.cluster_size = e.C;
        o.kernel = e.resident ? 2 : 1;
        o.threads = e.threads;
        o.tile = e.tile;
        o.use_graph = 0;
        pcs_ctx* tc = nullptr;
        st = pcs_create(&tc, c.H, c.W, S, &o, c.stream);
        if (st != PCS_OK) break;
        float ms = 0.f;
        st = launch_solve(tc, f, m, S, 1.0, 0.35, 0.35, 2, chi);  // untimed warm-up
        if (st == PCS_OK) {
            cudaEventRecord(e0, c.stream);
            st = launch_solve(tc, f, m, S, 1.0, 0.35, 0.35, trial_iters, chi);
            cudaEventRecord(e1, c.stream);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
        }
        pcs_destroy(tc);
        if (st != PCS_OK) break;
        const int k = t.n_candidates++;
        t.ns_per_voxel_iter[k] = 1e6 * ms / ((double)n * trial_iters);
        t.cand_cluster_size[k] = e.C;
        t.cand_kernel[k] = e.resident ? 2 : 1;
        t.cand_threads[k] = e.threads;
        t.cand_tile[k] = e.tile;
        if (t.ns_per_voxel_iter[k] < best) {
            best = t.ns_per_voxel_iter[k];
            t.cluster_size = e.C;
            t.kernel = e.resident ? 2 : 1;
            t.threads = e.threads;
            t.tile = e.tile;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(f);
    cudaFree(chi);
    cudaFree(m);
    if (st != PCS_OK) return st;
    c.tuned = true;
    return PCS_OK;
}

// Make class c ready for S slices: variant chosen, context and packed buffers
// large enough, L known.
pcs_status prepare_class(pcs_batch* b, pcs_batch::Class& c, int S) {
    if (!c.stream) {
        PCS_CUDA(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking), "cudaStreamCreate");
        PCS_CUDA(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming), "cudaEventCreate");
        PCS_CUDA(cudaEventCreateWithFlags(&c.solved, cudaEventDisableTiming), "cudaEventCreate");
    }
    if (b->autotune && !c.tuned) {
        pcs_status st = tune_class(b, c, S < 128 ? S : 128, 40);
        if (st != PCS_OK) return st;
    }
    if (c.ctx && c.capacity >= S) return PCS_OK;
    const int cap = S > 2 * c.capacity ? S : 2 * c.capacity;
    if (c.ctx) pcs_destroy(c.ctx);
    c.ctx = nullptr;
    void* old[] = {c.pk_field, c.pk_mask, c.pk_chi, c.inv_den};
    for (void* q : old)
        if (q) cudaFree(q);
    c.pk_field = nullptr;
    c.pk_mask = nullptr;
    c.pk_chi = nullptr;
    c.inv_den = nullptr;
    pcs_options o = b->opt;
    o.use_graph = 0;
    if (c.tuned) {
        o.cluster_size = c.tuning.cluster_size;
        o.kernel = c.tuning.kernel;
        o.threads = c.tuning.threads;
        o.tile = c.tuning.tile;
    }
    pcs_status st = pcs_create(&c.ctx, c.H, c.W, cap, &o, c.stream);
    if (st != PCS_OK) return st;
    const size_t n = (size_t)cap * c.H * c.W;
    PCS_CUDA(cudaMalloc(&c.pk_field, n * sizeof(float)), "cudaMalloc batch");
    PCS_CUDA(cudaMalloc(&c.pk_mask, n), "cudaMalloc batch");
    PCS_CUDA(cudaMalloc(&c.pk_chi, n * sizeof(float)), "cudaMalloc batch");
    PCS_CUDA(cudaMalloc(&c.inv_den, (size_t)cap * sizeof(float)), "cudaMalloc batch");
    c.capacity = cap;
    if (c.L == 0.0) {  // full-mask operator norm of this size (pseudocode step 1)
        PCS_CUDA(cudaMemsetAsync(c.pk_mask, 1, (size_t)c.H * c.W, c.stream), "memset");
        st = pcs::ctx_opnorm(c.ctx, c.pk_mask, 1, 300, &c.L);
        if (st != PCS_OK) return st;
    }
    return PCS_OK;
}

}  // namespace

extern "C" {

pcs_status pcs_batch_create(pcs_batch** out, const pcs_options* opt, int autotune, void* cuda_stream) {
    if (!out) return fail(PCS_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1) return fail(PCS_ECUDA, "no CUDA device (%s)", cudaGetErrorString(e));
    pcs_batch* b = new pcs_batch();
    if (opt) b->opt = *opt;
    b->autotune = autotune;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    if ((e = cudaGetDevice(&b->device)) != cudaSuccess || (e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) {
        delete b;
        return cuda_fail(e, "batch set-up");
    }
    *out = b;
    return PCS_OK;
}

pcs_status pcs_batch_solve(pcs_batch* b, const pcs_volume* vols, int n_vols, int n_iter) {
    PCS_TRACE("pcs_batch_solve");
    if (!b) return fail(PCS_EINVAL, "batch is NULL");
    if (n_vols < 0 || (n_vols > 0 && !vols)) return fail(PCS_EINVAL, "bad volume list");
    if (n_iter < 0) return fail(PCS_EINVAL, "n_iter must be >= 0");
    std::unique_lock<std::mutex> lk(b->mu, std::try_to_lock);
    if (!lk.owns_lock()) return fail(PCS_EBUSY, "batch in use by another thread");
    // validate and group by slice size
    std::vector<int> cls_of(n_vols, -1);
    std::vector<int> cls_S;
    for (int v = 0; v < n_vols; ++v) {
        const pcs_volume& V = vols[v];
        if (V.S < 0) return fail(PCS_EINVAL, "volume %d: S < 0", v);
        if (V.S == 0) continue;
        if (!V.field || !V.mask || !V.chi_out) return fail(PCS_EINVAL, "volume %d: NULL buffer", v);
        if (!(V.lambda > 0.0) || !std::isfinite(V.lambda)) return fail(PCS_EINVAL, "volume %d: lambda must be > 0", v);
        if (!find_entry(V.H, V.W, 0) && !pcs::gen_supported(V.H, V.W))
            return fail(PCS_EUNSUPPORTED, "volume %d: no kernel for %d x %d", v, V.H, V.W);
        int k = -1;
        for (size_t c = 0; c < b->classes.size(); ++c)
            if (b->classes[c].H == V.H && b->classes[c].W == V.W) k = (int)c;
        if (k < 0) {
            b->classes.emplace_back();
            b->classes.back().H = V.H;
            b->classes.back().W = V.W;
            k = (int)b->classes.size() - 1;
        }
        cls_of[v] = k;
        if ((int)cls_S.size() < (int)b->classes.size()) cls_S.resize(b->classes.size(), 0);
        cls_S[k] += V.S;
    }
    cls_S.resize(b->classes.size(), 0);
    PCS_CUDA(cudaSetDevice(b->device), "cudaSetDevice");
    for (size_t c = 0; c < b->classes.size(); ++c) {
        if (cls_S[c] == 0) continue;
        pcs_status st = prepare_class(b, b->classes[c], cls_S[c]);
        if (st != PCS_OK) return st;
    }
    // fork: every class stream waits for the work already on the batch stream and packs its
    // inputs at once; the solves run one size class after another, the most work first (each
    // persistent launch balances its slices over all resident clusters, so concurrent launches of
    // different sizes would only contend for the SMs)
    PCS_CUDA(cudaEventRecord(b->fork, b->stream), "fork record");
    std::vector<size_t> order;
    for (size_t c = 0; c < b->classes.size(); ++c)
        if (cls_S[c] > 0) order.push_back(c);
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        return (double)cls_S[x] * b->classes[x].H * b->classes[x].W > (double)cls_S[y] * b->classes[y].H * b->classes[y].W;
    });
    const pcs_batch::Class* prev = nullptr;
    for (size_t c : order) {
        pcs_batch::Class& C = b->classes[c];
        PCS_CUDA(cudaStreamWaitEvent(C.stream, b->fork, 0), "fork wait");
        const size_t sl = (size_t)C.H * C.W;
        const double tau = 1.0 / C.L, sigma = 1.0 / C.L;
        std::vector<float> inv(cls_S[c]);
        int off = 0;
        for (int v = 0; v < n_vols; ++v) {
            if (cls_of[v] != (int)c) continue;
            const pcs_volume& V = vols[v];
            PCS_CUDA(cudaMemcpyAsync(C.pk_field + off * sl, V.field, V.S * sl * sizeof(float), cudaMemcpyDeviceToDevice, C.stream), "pack field");
            PCS_CUDA(cudaMemcpyAsync(C.pk_mask + off * sl, V.mask, V.S * sl, cudaMemcpyDeviceToDevice, C.stream), "pack mask");
            for (int s = 0; s < V.S; ++s) inv[off + s] = (float)(1.0 / (1.0 + sigma / V.lambda));
            off += V.S;
        }
        PCS_CUDA(cudaMemcpyAsync(C.inv_den, inv.data(), inv.size() * sizeof(float), cudaMemcpyHostToDevice, C.stream), "lambda upload");
        if (prev) PCS_CUDA(cudaStreamWaitEvent(C.stream, prev->solved, 0), "wait for the previous class");
        pcs_status st = launch_solve(C.ctx, C.pk_field, C.pk_mask, cls_S[c], 1.0, tau, sigma, n_iter, C.pk_chi, C.inv_den);
        if (st != PCS_OK) return st;
        PCS_CUDA(cudaEventRecord(C.solved, C.stream), "solved record");
        prev = &C;
        off = 0;
        for (int v = 0; v < n_vols; ++v) {
            if (cls_of[v] != (int)c) continue;
            const pcs_volume& V = vols[v];
            PCS_CUDA(cudaMemcpyAsync(V.chi_out, C.pk_chi + off * sl, V.S * sl * sizeof(float), cudaMemcpyDeviceToDevice, C.stream), "unpack chi");
            off += V.S;
        }
        PCS_CUDA(cudaEventRecord(C.done, C.stream), "join record");
        PCS_CUDA(cudaStreamWaitEvent(b->stream, C.done, 0), "join wait");
    }
    return PCS_OK;
}

pcs_status pcs_batch_tuning(pcs_batch* b, int H, int W, pcs_tuning* out) {
    if (!b || !out) return fail(PCS_EINVAL, "NULL argument");
    for (const auto& c : b->classes)
        if (c.H == H && c.W == W) {
            if (!c.tuned) {
                const pcs::KernelEntry* e = c.ctx ? c.ctx->entry : find_entry(H, W, 0);
                *out = pcs_tuning{};
                out->H = H;
                out->W = W;
                out->cluster_size = e ? e->C : 0;
                out->kernel = e ? (e->resident ? 2 : 1) : 0;
                out->threads = e ? e->threads : 0;
                out->tile = e ? e->tile : 0;
                out->L = c.L;
                return PCS_OK;
            }
            *out = c.tuning;
            out->L = c.L;
            return PCS_OK;
        }
    return fail(PCS_EINVAL, "size %d x %d not solved by this batch", H, W);
}

pcs_status pcs_batch_check(pcs_batch* b) {
    if (!b) return fail(PCS_EINVAL, "batch is NULL");
    std::unique_lock<std::mutex> lk(b->mu, std::try_to_lock);
    if (!lk.owns_lock()) return fail(PCS_EBUSY, "batch in use by another thread");
    PCS_CUDA(cudaSetDevice(b->device), "cudaSetDevice");
    PCS_CUDA(cudaStreamSynchronize(b->stream), "stream sync");
    pcs_status ret = PCS_OK;
    for (auto& c : b->classes) {
        if (!c.ctx) continue;
        pcs_status st = check_err_word(c.ctx);  // every size class: read (and clear) its word
        if (ret == PCS_OK) ret = st;
    }
    return ret;
}

void pcs_batch_destroy(pcs_batch* b) {
    if (!b) return;
    for (auto& c : b->classes) free_class(c);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

}  // extern "C"

// ------------------------------------------------------------------ all-FP64 solve (precision study)

extern "C" pcs_status pcs_solve_slices_f64(const double* field, const unsigned char* mask, int H, int W, int S,
                                           double lambda, double tau, double sigma, int n_iter, double* chi_out,
                                           int b0_axis, void* cuda_stream) {
    PCS_TRACE("pcs_solve_slices_f64");
    if (S < 0 || n_iter < 0) return fail(PCS_EINVAL, "S and n_iter must be >= 0");
    const pcs::KernelEntryF64* entry = nullptr;
    int ne = 0;
    const pcs::KernelEntryF64* es = pcs::entries_f64(&ne);
    for (int k = 0; k < ne; ++k)
        if (es[k].H == H && es[k].W == W) entry = &es[k];
    if (!entry) return fail(PCS_EUNSUPPORTED, "no FP64 kernel for %d x %d slices", H, W);
    if (S == 0) return PCS_OK;
    if (!field || !mask || !chi_out || (const void*)field == (const void*)chi_out)
        return fail(PCS_EINVAL, "NULL or aliased buffer");
    if (!(lambda > 0.0) || !(tau > 0.0) || !(sigma > 0.0)) return fail(PCS_EINVAL, "lambda, tau, sigma must be > 0");
    if (b0_axis != 0 && b0_axis != 1) return fail(PCS_EINVAL, "b0_axis must be 0 or 1");
    if (!aligned16(field) || !aligned16(mask) || !aligned16(chi_out)) return fail(PCS_EINVAL, "16-byte alignment");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<double> dtab, ddtab;
    std::vector<double2> tw;
    pcs::build_dipole_tables_t<double>(H, W, b0_axis, dtab, ddtab);
    pcs::build_twiddles_t<double2>(H > W ? H : W, tw);
    const size_t n = (size_t)S * H * W;
    double* scratch = nullptr;
    const size_t tab = dtab.size() + ddtab.size() + 2 * tw.size();
    PCS_CUDA(cudaMalloc(&scratch, (4 * n + tab) * sizeof(double)), "cudaMalloc FP64 scratch");
    double* dt = scratch + 4 * n;
    double* ddt = dt + dtab.size();
    double2* twd = reinterpret_cast<double2*>(ddt + ddtab.size());
    pcs_status ret = PCS_OK;
    cudaError_t e;
    int ncl = 0;
    if ((e = cudaMemcpyAsync(dt, dtab.data(), dtab.size() * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(ddt, ddtab.data(), ddtab.size() * sizeof(double), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(twd, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = entry->prepare(&ncl)) != cudaSuccess) {
        ret = cuda_fail(e, "FP64 set-up");
    } else {
        pcs::PDParamsT<double> prm;
        std::memset(&prm, 0, sizeof(prm));
        prm.field = field;
        prm.mask = mask;
        prm.chi = chi_out;
        prm.chibar = scratch;
        prm.p = scratch + n;
        prm.qx = scratch + 2 * n;
        prm.qy = scratch + 3 * n;
        prm.dtab = dt;
        prm.ddtab = ddt;
        prm.twid = twd;
        prm.S = S;
        prm.n_iter = n_iter;
        prm.sigma = sigma;
        prm.tau = tau;
        prm.inv_den = 1.0 / (1.0 + sigma / lambda);
        prm.inv_den_slice = nullptr;
        if (ncl > S) ncl = S;
        if (ncl < 1) ncl = 1;
        if ((e = entry->launch(prm, ncl, st)) != cudaSuccess) ret = cuda_fail(e, "FP64 kernel launch");
    }
    // the call is synchronous: it owns its scratch
    e = cudaStreamSynchronize(st);
    if (ret == PCS_OK && e != cudaSuccess) ret = cuda_fail(e, "stream sync");
    cudaFree(scratch);
    return ret;
}
