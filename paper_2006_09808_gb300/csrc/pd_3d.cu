// pd_3d.cu -- instances and the C-ABI entry point of the 3-D variant
// (pcs_solve_volume_3d; kernels in pd_3d.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/pcs.h"
#include "pd_3d.cuh"
#include "pd_launch.cuh"
#include "pcs_trace.h"

namespace pcs {
void build_twiddles(int n, std::vector<float2>& tw);
pcs_status set_last_error(pcs_status st, const char* msg);
}  // namespace pcs

namespace {

using pcs::Geo;
using pcs::GeoZ;
using pcs::P3Params;
using pcs::P3Report;

struct Slice3Entry {
    int H, W, C;
    size_t smem;
    cudaError_t (*prepare)(int* max_clusters);
    cudaError_t (*launch)(const P3Params& a, int n_clusters, cudaStream_t st, bool pdl);
    cudaError_t (*prepare_report)(int* max_clusters);
    cudaError_t (*launch_report)(const P3Report& r, int n_clusters, cudaStream_t st);
};

template <class G>
cudaError_t prepare3(int* mc) {
    return pcs::prepare_cluster<G>(pcs::pd3_slice_kernel<G>, G::SMEM_BYTES, mc);
}
// pdl: programmatic dependent launch (the kernel waits for the previous grid before it
// touches memory; its launch overlaps the end of that grid)
template <class G>
cudaError_t launch3(const P3Params& a, int ncl, cudaStream_t st, bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncl * G::C, 1, 1);
    cfg.blockDim = dim3(G::NT, 1, 1);
    cfg.dynamicSmemBytes = G::SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, pcs::pd3_slice_kernel<G>, a);
}
template <class G>
cudaError_t prepare3_report(int* mc) {
    return pcs::prepare_cluster<G>(pcs::pd3_report_kernel<G>, pcs::aux_smem<G>(), mc);
}
template <class G>
cudaError_t launch3_report(const P3Report& r, int ncl, cudaStream_t st) {
    return pcs::launch_cluster<G>(pcs::pd3_report_kernel<G>, r, pcs::aux_smem<G>(), ncl, st);
}
template <class G>
constexpr Slice3Entry slice3_entry() {
    return Slice3Entry{G::H, G::W, G::C, G::SMEM_BYTES, &prepare3<G>, &launch3<G>, &prepare3_report<G>,
                       &launch3_report<G>};
}

const Slice3Entry k_slice3[] = {
    slice3_entry<Geo<64, 64, 1>>(),
    slice3_entry<Geo<128, 128, 2>>(),
    slice3_entry<Geo<256, 256, 4, 2>>(),
    // one 512-thread CTA per SM: 36 clusters, two slices per cluster for 64 slices (the last entry
    // of a size is the one used)
    slice3_entry<Geo<256, 256, 4, 1, 512>>(),
};

struct Z3Entry {
    int NZ, H, W;
    cudaError_t (*launch)(float2* spec, const float2* twid, int ntw, float3 iv, cudaStream_t st, bool pdl);
};

// z pass: one CTA per tile of pencils
template <int NZ, int H, int W>
cudaError_t launch_z(float2* spec, const float2* twid, int ntw, float3 iv, cudaStream_t st, bool pdl) {
    using GZ = GeoZ<NZ, H, W>;
    auto kern = pcs::pd3_z_kernel<GZ, NZ, H, W>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(GZ::NTILES, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = GZ::SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, spec, static_cast<const float2*>(twid), ntw, iv);
}

const Z3Entry k_z3[] = {
    {32, 64, 64, &launch_z<32, 64, 64>},      {64, 64, 64, &launch_z<64, 64, 64>},
    {32, 128, 128, &launch_z<32, 128, 128>},  {64, 128, 128, &launch_z<64, 128, 128>},
    {128, 128, 128, &launch_z<128, 128, 128>}, {32, 256, 256, &launch_z<32, 256, 256>},
    {64, 256, 256, &launch_z<64, 256, 256>},  {128, 256, 256, &launch_z<128, 256, 256>},
};

// Pencil form (pd_3d.cuh): row kernel geometry per slice size (one row pass per CTA, two
// 256-thread CTAs per SM) and plane kernel per (S, H) (1024 threads where the plane, its z
// scratch and tables fit in shared memory, else 512).
template <int H>
using GeoRows3 = Geo<H, H, H / ((256 / 32) * (32 / (H / 2 / pcs::default_elems(H / 2)))), 2, 256>;

struct Pencil3Entry {
    int S, H, W;
    cudaError_t (*prepare)();
    cudaError_t (*launch_rows)(const P3Params& a, cudaStream_t st, bool pdl);
    cudaError_t (*launch_planes)(float2* spec, const float2* twid, int ntw, float3 iv, cudaStream_t st, bool pdl);
};

cudaError_t launch_dep3(const void* kern, void** args, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                        bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelExC(&cfg, kern, args);
}

template <int S, int H, int NT>
cudaError_t prepare_pencil() {
    using GR = GeoRows3<H>;
    using GP = pcs::GeoPlane<S, H, H, NT>;
    cudaError_t e = cudaFuncSetAttribute(pcs::pd3p_rows_kernel<GR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pcs::pencil_rows_smem<GR>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(pcs::pd3p_plane_kernel<GP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)GP::SMEM_BYTES);
}
template <int S, int H, int NT>
cudaError_t launch_pencil_rows(const P3Params& a, cudaStream_t st, bool pdl) {
    using GR = GeoRows3<H>;
    P3Params arg = a;
    void* args[] = {&arg};
    return launch_dep3(reinterpret_cast<const void*>(pcs::pd3p_rows_kernel<GR>), args, dim3(S * GR::C), dim3(GR::NT),
                       pcs::pencil_rows_smem<GR>(), st, pdl);
}
template <int S, int H, int NT>
cudaError_t launch_pencil_planes(float2* spec, const float2* twid, int ntw, float3 iv, cudaStream_t st, bool pdl) {
    using GP = pcs::GeoPlane<S, H, H, NT>;
    void* args[] = {&spec, &twid, &ntw, &iv};
    return launch_dep3(reinterpret_cast<const void*>(pcs::pd3p_plane_kernel<GP>), args, dim3(GP::M + 1), dim3(NT),
                       GP::SMEM_BYTES, st, pdl);
}
template <int S, int H, int NT>
constexpr Pencil3Entry pencil3_entry() {
    return Pencil3Entry{S, H, H, &prepare_pencil<S, H, NT>, &launch_pencil_rows<S, H, NT>,
                        &launch_pencil_planes<S, H, NT>};
}

const Pencil3Entry k_pencil3[] = {
    pencil3_entry<32, 64, 1024>(),  pencil3_entry<64, 64, 1024>(),  pencil3_entry<32, 128, 1024>(),
    pencil3_entry<64, 128, 1024>(), pencil3_entry<128, 128, 512>(), pencil3_entry<32, 256, 1024>(),
    pencil3_entry<64, 256, 1024>(),
};

pcs_status fail3(pcs_status st, const char* what, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess) {
        snprintf(buf, sizeof(buf), "pcs_solve_volume_3d: %s: %s", what, cudaGetErrorString(e));
    } else {
        snprintf(buf, sizeof(buf), "pcs_solve_volume_3d: %s", what);
    }
    return pcs::set_last_error(st, buf);
}

bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

}  // namespace

extern "C" {

int pcs_supported_volume_3d(int S, int H, int W) {
    bool slice = false, z = false;
    for (const auto& e : k_slice3) slice = slice || (e.H == H && e.W == W);
    for (const auto& e : k_z3) z = z || (e.NZ == S && e.H == H && e.W == W);
    return (slice && z) ? 1 : 0;
}

pcs_status pcs_solve_volume_3d(const float* field, const unsigned char* mask, const float* weight, int S, int H,
                               int W, double lambda, double tau, double sigma, int n_iter, int tv, const double* voxel,
                               float* chi_out, pcs_slice_report* rep, void* cuda_stream) {
    PCS_TRACE("pcs_solve_volume_3d");
    if (!field || !mask || !chi_out) return fail3(PCS_EINVAL, "NULL argument");
    if (!aligned16(weight)) return fail3(PCS_EINVAL, "weight must be 16-byte aligned");
    if (!(lambda > 0.0) || !(tau > 0.0) || !(sigma > 0.0)) return fail3(PCS_EINVAL, "lambda, tau, sigma must be > 0");
    if (n_iter < 0) return fail3(PCS_EINVAL, "n_iter must be >= 0");
    if (tv != 0 && tv != 1) return fail3(PCS_EINVAL, "tv must be 0 or 1");
    float3 iv = make_float3(1.f, 1.f, 1.f);  // inverse voxel edges (x, y, z), relative to the smallest
    if (voxel) {
        for (int a = 0; a < 3; ++a)
            if (!(voxel[a] > 0.0) || !std::isfinite(voxel[a])) return fail3(PCS_EINVAL, "voxel edges must be > 0");
        const double vmin = std::min(voxel[0], std::min(voxel[1], voxel[2]));
        iv = make_float3((float)(vmin / voxel[2]), (float)(vmin / voxel[1]), (float)(vmin / voxel[0]));
    }
    if (!aligned16(field) || !aligned16(mask) || !aligned16(chi_out))
        return fail3(PCS_EINVAL, "device buffers must be 16-byte aligned");
    if (field == chi_out) return fail3(PCS_EINVAL, "chi_out must not alias field");
    const Slice3Entry* se = nullptr;
    const Z3Entry* ze = nullptr;
    for (const auto& e : k_slice3)
        if (e.H == H && e.W == W) se = &e;
    for (const auto& e : k_z3)
        if (e.NZ == S && e.H == H && e.W == W) ze = &e;
    if (!se || !ze) return fail3(PCS_EUNSUPPORTED, "no 3-D kernel for this volume shape");
    const Pencil3Entry* pe = nullptr;  // the pencil form where the plane fits in shared memory
    for (const auto& e : k_pencil3)
        if (e.S == S && e.H == H && e.W == W) pe = &e;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t n = (size_t)S * H * W;
    const size_t nspec = (size_t)S * (W / 2 + 1) * H;
    const int ntw = H > W ? H : W;
    std::vector<float2> tw;
    pcs::build_twiddles(ntw, tw);

    float* state = nullptr;  // chibar, p, qx, qy, qz
    float2* spec = nullptr;
    float2* twid = nullptr;
    double* partial = nullptr;  // [S][C][kReportSums] when rep is set
    const size_t npart = (size_t)S * se->C * pcs::kReportSums;
    cudaError_t e;
    int ncl = 0;
    pcs_status ret = PCS_OK;
    if ((e = cudaMalloc(&state, 5 * n * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&spec, nspec * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&twid, tw.size() * sizeof(float2))) != cudaSuccess ||
        (rep && (e = cudaMalloc(&partial, npart * sizeof(double))) != cudaSuccess)) {
        ret = fail3(PCS_ECUDA, "cudaMalloc", e);
    } else if ((e = cudaMemcpyAsync(twid, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st)) !=
                   cudaSuccess ||
               (e = cudaMemsetAsync(state, 0, 5 * n * sizeof(float), st)) != cudaSuccess ||
               (e = cudaMemsetAsync(chi_out, 0, n * sizeof(float), st)) != cudaSuccess ||
               (e = se->prepare(&ncl)) != cudaSuccess) {
        ret = fail3(PCS_ECUDA, "set-up", e);
    } else {
        P3Params a;
        std::memset(&a, 0, sizeof(a));
        a.pd.field = field;
        a.pd.mask = mask;
        a.pd.chi = chi_out;
        a.pd.chibar = state;
        a.pd.p = state + n;
        a.pd.qx = state + 2 * n;
        a.pd.qy = state + 3 * n;
        a.pd.qz = state + 4 * n;
        a.pd.twid = twid;
        a.pd.S = S;
        a.pd.n_iter = n_iter;
        a.pd.sigma = (float)sigma;
        a.pd.tau = (float)tau;
        a.pd.inv_den = (float)(1.0 / (1.0 + sigma / lambda));
        a.pd.tv_iso = tv;
        a.pd.weight = weight;
        a.spec = spec;
        if (ncl > S) ncl = S;
        if (ncl < 1) ncl = 1;
        if (pe && (e = pe->prepare()) != cudaSuccess) ret = fail3(PCS_ECUDA, "pencil set-up", e);
        // pencil form: rows (dual) -> planes -> rows (primal) -> planes; the spectrum buffer holds
        // the planes [kx][s][y] between the launches
        for (int it = 0; pe && it < n_iter && ret == PCS_OK; ++it) {
            a.phase = 0;
            a.load = it > 0;
            a.store = 1;
            if ((e = pe->launch_rows(a, st, it > 0)) != cudaSuccess ||
                (e = pe->launch_planes(spec, twid, ntw, iv, st, true)) != cudaSuccess) {
                ret = fail3(PCS_ECUDA, "launch", e);
                break;
            }
            a.phase = 1;
            a.load = 1;
            a.store = it + 1 < n_iter;
            if ((e = pe->launch_rows(a, st, true)) != cudaSuccess ||
                (a.store && (e = pe->launch_planes(spec, twid, ntw, iv, st, true)) != cudaSuccess)) {
                ret = fail3(PCS_ECUDA, "launch", e);
                break;
            }
        }
        // slice kernel and z pass (shapes whose plane does not fit in shared memory):
        // iteration n: dual step from the spectrum of chibar_n (zero at n = 0), z pass,
        // primal step, z pass (the spectrum of chibar_{n+1}; not after the last)
        for (int it = 0; !pe && it < n_iter && ret == PCS_OK; ++it) {
            // serpentine slice order: each launch starts on the slices the one before ended on,
            // whose state is the most likely to be still in L2
            a.phase = 0;
            a.load = it > 0;
            a.store = 1;
            a.reverse = 0;
            if ((e = se->launch(a, ncl, st, it > 0)) != cudaSuccess ||
                (e = ze->launch(spec, twid, ntw, iv, st, true)) != cudaSuccess) {
                ret = fail3(PCS_ECUDA, "launch", e);
                break;
            }
            a.phase = 1;
            a.load = 1;
            a.store = it + 1 < n_iter;
            a.reverse = 1;
            if ((e = se->launch(a, ncl, st, true)) != cudaSuccess ||
                (a.store && (e = ze->launch(spec, twid, ntw, iv, st, true)) != cudaSuccess)) {
                ret = fail3(PCS_ECUDA, "launch", e);
                break;
            }
        }
        // FP64 diagnostics at the final (chi, p, q): spectrum of chi, z pass, data and
        // TV terms + spectrum of W p, z pass, stationarity
        int ncl_rep = 0;
        if (ret == PCS_OK && rep) {
            if ((e = se->prepare_report(&ncl_rep)) != cudaSuccess) {
                ret = fail3(PCS_ECUDA, "report set-up", e);
            } else {
                if (ncl_rep > S) ncl_rep = S;
                if (ncl_rep < 1) ncl_rep = 1;
                P3Report r;
                std::memset(&r, 0, sizeof(r));
                r.a = a;
                r.partial = partial;
                r.lam = lambda;
                for (int mode = 0; mode < 3 && ret == PCS_OK; ++mode) {
                    r.mode = mode;
                    if ((e = se->launch_report(r, ncl_rep, st)) != cudaSuccess ||
                        (mode < 2 && (e = ze->launch(spec, twid, ntw, iv, st, false)) != cudaSuccess))
                        ret = fail3(PCS_ECUDA, "report launch", e);
                }
            }
        }
    }
    // synchronous: the call owns its scratch
    cudaError_t se2 = cudaStreamSynchronize(st);
    if (ret == PCS_OK && se2 != cudaSuccess) ret = fail3(PCS_ECUDA, "stream sync", se2);
    if (ret == PCS_OK && rep) {
        std::vector<double> h(npart);
        if ((e = cudaMemcpy(h.data(), partial, npart * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess) {
            ret = fail3(PCS_ECUDA, "report copy", e);
        } else {
            // fixed-order sums: slice by slice, CTA by CTA
            double t[pcs::kReportSums] = {0, 0, 0, 0, 0};
            for (size_t k = 0; k < npart; ++k) t[k % pcs::kReportSums] += h[k];
            rep->objective = 0.5 * lambda * t[0] + t[1];
            rep->gap = t[2] / (2.0 * lambda) + t[3];
            rep->stationarity = std::sqrt(t[4]);
            rep->data_residual = std::sqrt(t[0]);
            rep->iters = n_iter;
            rep->pad = 0;
        }
    }
    cudaFree(state);
    cudaFree(spec);
    cudaFree(twid);
    cudaFree(partial);
    return ret;
}

}  // extern "C"
