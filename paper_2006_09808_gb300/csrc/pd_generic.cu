// pd_generic.cu -- C-ABI entry of the any-size per-slice solver
// (pcs_solve_slices_generic; kernels in pd_generic.cuh).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/pcs.h"
#include "pd_generic.cuh"

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
    int tile;  // columns per CTA
};
template <int H>
constexpr ColEntry col_entry() {
    return ColEntry{H, pcs::GeoCol<H>::SMEM_BYTES, &pcs::gen_cols_fft_kernel<H>, pcs::GeoCol<H>::TY};
}
const ColEntry k_cols[] = {col_entry<64>(),  col_entry<128>(), col_entry<192>(),
                           col_entry<256>(), col_entry<384>(), col_entry<512>()};

size_t rows_smem(int W) { return sizeof(float2) * (size_t)W * (1 + 2 * pcs::kGenRowWarps); }
size_t cols_smem(int H) { return sizeof(float2) * ((size_t)H + (size_t)(2 * H + 1) * pcs::kGenColTile); }

}  // namespace

extern "C" {

int pcs_supported_generic(int H, int W) {
    GenPlan a, b;
    return (H % 2 == 0 && W % 2 == 0 && gen_plan(H, &a) && gen_plan(W, &b)) ? 1 : 0;
}

pcs_status pcs_solve_slices_generic(const float* field, const unsigned char* mask, const float* weight, int S,
                                    int H, int W, int b0_axis, double lambda, double tau, double sigma, int n_iter,
                                    int tv, float* chi_out, void* cuda_stream) {
    if (S < 0) return failg(PCS_EINVAL, "S must be >= 0");
    if (!(lambda > 0.0) || !(tau > 0.0) || !(sigma > 0.0)) return failg(PCS_EINVAL, "lambda, tau, sigma must be > 0");
    if (n_iter < 0) return failg(PCS_EINVAL, "n_iter must be >= 0");
    if (tv != 0 && tv != 1) return failg(PCS_EINVAL, "tv must be 0 or 1");
    if (b0_axis != 0 && b0_axis != 1) return failg(PCS_EINVAL, "b0_axis must be 0 or 1");
    GenParams g;
    std::memset(&g, 0, sizeof(g));
    if (H % 2 != 0 || W % 2 != 0 || !gen_plan(W, &g.prow) || !gen_plan(H, &g.pcol))
        return failg(PCS_EUNSUPPORTED, "H and W must be even, in [8, 512], with prime factors <= 61");
    if (S == 0) return PCS_OK;
    if (!field || !mask || !chi_out) return failg(PCS_EINVAL, "NULL argument");
    if (field == chi_out) return failg(PCS_EINVAL, "chi_out must not alias field");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t n = (size_t)S * H * W;
    const int M1 = W / 2 + 1;
    const size_t nspec = (size_t)S * H * M1;
    std::vector<float2> tw_r, tw_c;
    pcs::build_twiddles(W, tw_r);
    pcs::build_twiddles(H, tw_c);

    float* state = nullptr;  // chibar, p, qx, qy
    float2* spec = nullptr;
    float2* tabs = nullptr;  // row twiddles, then column twiddles
    cudaError_t e;
    pcs_status ret = PCS_OK;
    const ColEntry* ce = nullptr;
    for (const auto& c : k_cols)
        if (c.H == H) ce = &c;
    void (*cols_kern)(GenParams) = ce ? ce->kern : pcs::gen_cols_kernel;
    const int col_tile = ce ? ce->tile : pcs::kGenColTile;
    const int col_threads = ce ? 256 : pcs::kGenColTile * 32;
    const size_t srows = rows_smem(W), scols = ce ? ce->smem : cols_smem(H);
    if ((e = cudaMalloc(&state, 4 * n * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&spec, nspec * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&tabs, (size_t)(W + H) * sizeof(float2))) != cudaSuccess) {
        ret = failg(PCS_ECUDA, "cudaMalloc", e);
    } else if ((e = cudaMemcpyAsync(tabs, tw_r.data(), W * sizeof(float2), cudaMemcpyHostToDevice, st)) !=
                   cudaSuccess ||
               (e = cudaMemcpyAsync(tabs + W, tw_c.data(), H * sizeof(float2), cudaMemcpyHostToDevice, st)) !=
                   cudaSuccess ||
               (e = cudaMemsetAsync(state, 0, 4 * n * sizeof(float), st)) != cudaSuccess ||
               (e = cudaMemsetAsync(chi_out, 0, n * sizeof(float), st)) != cudaSuccess ||
               (e = cudaMemsetAsync(spec, 0, nspec * sizeof(float2), st)) != cudaSuccess ||
               (e = cudaFuncSetAttribute(pcs::gen_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)srows)) != cudaSuccess ||
               (e = cudaFuncSetAttribute(cols_kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scols)) !=
                   cudaSuccess) {
        ret = failg(PCS_ECUDA, "set-up", e);
    } else {
        g.field = field;
        g.mask = mask;
        g.weight = weight;
        g.chi = chi_out;
        g.chibar = state;
        g.p = state + n;
        g.qx = state + 2 * n;
        g.qy = state + 3 * n;
        g.spec = spec;
        g.trow = tabs;
        g.tcol = tabs + W;
        g.S = S;
        g.H = H;
        g.W = W;
        g.M1 = M1;
        g.sigma = (float)sigma;
        g.tau = (float)tau;
        g.inv_den = (float)(1.0 / (1.0 + sigma / lambda));
        g.tv_iso = tv;
        g.b0_axis = b0_axis;
        const int pairs = S * (H / 2);
        const dim3 grid_r((pairs + pcs::kGenRowWarps - 1) / pcs::kGenRowWarps);
        const dim3 grid_c((M1 + col_tile - 1) / col_tile, S);
        // iteration n: dual step from the spectrum D F chibar_n (zero at n = 0), column pass
        // (spectrum of W p), primal step, column pass (spectrum of chibar_{n+1}; not after the last)
        for (int it = 0; it < n_iter; ++it) {
            g.phase = 0;
            g.store = 1;
            pcs::gen_rows_kernel<<<grid_r, pcs::kGenRowWarps * 32, srows, st>>>(g);
            cols_kern<<<grid_c, col_threads, scols, st>>>(g);
            g.phase = 1;
            g.store = it + 1 < n_iter;
            pcs::gen_rows_kernel<<<grid_r, pcs::kGenRowWarps * 32, srows, st>>>(g);
            if (g.store) cols_kern<<<grid_c, col_threads, scols, st>>>(g);
            if ((e = cudaGetLastError()) != cudaSuccess) {
                ret = failg(PCS_ECUDA, "launch", e);
                break;
            }
        }
    }
    // synchronous: the call owns its scratch
    cudaError_t se = cudaStreamSynchronize(st);
    if (ret == PCS_OK && se != cudaSuccess) ret = failg(PCS_ECUDA, "stream sync", se);
    cudaFree(state);
    cudaFree(spec);
    cudaFree(tabs);
    return ret;
}

}  // extern "C"
