// pcs_noalloc.cu -- a solve entry point that allocates no device memory.
//
// Who needs it: callers that are not allowed to call cudaMalloc once they are
// running -- e.g. a reconstruction plug-in inside a scanner or interventional
// host application that owns the GPU's memory budget and forbids allocations
// after start-up, or code that runs inside another framework's memory pool.
// pcs_create allocates its scratch, so such callers cannot use it.
//
// This entry point runs the same fused iteration kernel as pcs_solve_slices,
// but its scratch state (chibar, p, qx, qy) and its D(k) / twiddle tables
// live in file-scope static __device__ arrays of a fixed maximum size.  Every
// GPU that loads this library holds those arrays (about 16.5 MiB) until the
// process exits.  The caller still passes the field, the mask and chi_out.
//
// Per-device set-up happens on the first call on each device (with that
// device current): the arrays' device addresses are looked up with
// cudaGetSymbolAddress and the kernel attributes are set.  Each compiled
// slice size and B0 axis has its own fixed region of the table arrays,
// uploaded by the first call of that size and axis on the device (that call
// waits for the upload on its stream) and never rewritten, so a call of one
// size can never read another size's tables.  Make the first call of every
// size and axis before any stream capture.
//
// All calls share the state arrays and each call leaves its state behind;
// the kernel zeroes the state of every slice before iterating, so nothing
// needs clearing between calls.  Calls that overlap on the GPU (from two
// streams or two threads) race on the state arrays and must be serialised
// by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/pcs.h"
#include "pd_launch.cuh"
#include "pcs_trace.h"

namespace pcs {
void build_dipole_tables(int H, int W, int b0_axis, std::vector<float>& dtab, std::vector<float>& ddtab);
void build_twiddles(int n, std::vector<float2>& tw);
pcs_status set_last_error(pcs_status st, const char* msg);
}  // namespace pcs

namespace {

constexpr size_t kMaxVoxels = PCS_NOALLOC_MAX_VOXELS;  // S * H * W per call

// The compiled slice sizes (square) and their table regions: dtab [n/2][n] and ddtab [n] per
// (size, B0 axis), twiddles [n] per size.
constexpr int kSizes[] = {64, 128, 192, 256, 384, 512};
constexpr int kNumSizes = 6;
constexpr size_t dtab_offset(int k, int b0) {
    size_t o = 0;
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < kNumSizes; ++j) {
            if (a == b0 && j == k) return o;
            o += (size_t)(kSizes[j] / 2) * kSizes[j];
        }
    return o;
}
constexpr size_t line_offset(int k, int b0) {  // ddtab per (size, axis); twiddles use b0 = 0
    size_t o = 0;
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < kNumSizes; ++j) {
            if (a == b0 && j == k) return o;
            o += (size_t)kSizes[j];
        }
    return o;
}
constexpr size_t kDtabFloats = dtab_offset(kNumSizes, 1);  // past the last region: the total
constexpr size_t kLineFloats = line_offset(kNumSizes, 1);

// scratch state: chibar, p, qx, qy, kMaxVoxels floats each
static __device__ __align__(256) float g_noalloc_state[4 * kMaxVoxels];
// D tables of every (size, axis) region (about 2 MB), packed-column tables, twiddles
static __device__ __align__(256) float g_noalloc_dtab[kDtabFloats];
static __device__ __align__(256) float g_noalloc_ddtab[kLineFloats];
static __device__ __align__(256) float2 g_noalloc_twid[kLineFloats / 2];  // sum of the sizes

struct DeviceSetup {
    bool ready = false;
    float* state = nullptr;
    float* dtab = nullptr;
    float* ddtab = nullptr;
    float2* twid = nullptr;
    bool tables[kNumSizes][2] = {};   // (size, axis) region uploaded
    bool twiddles[kNumSizes] = {};    // size's twiddle region uploaded
    const pcs::KernelEntry* prepared[16] = {};
    int max_clusters[16] = {};
};

constexpr int kMaxDevices = 64;
DeviceSetup g_dev[kMaxDevices];
std::mutex g_mu;

pcs_status err(pcs_status st, const char* what, cudaError_t e) {
    char buf[256];
    snprintf(buf, sizeof(buf), "pcs_solve_slices_noalloc: %s: %s", what, cudaGetErrorString(e));
    return pcs::set_last_error(st, buf);
}

const pcs::KernelEntry* default_entry(int H, int W) {
    const pcs::KernelEntry* (*fns[])(int*) = {pcs::entries_64,  pcs::entries_128, pcs::entries_192,
                                               pcs::entries_256, pcs::entries_384, pcs::entries_512};
    for (auto fn : fns) {
        int n = 0;
        const pcs::KernelEntry* e = fn(&n);
        for (int k = 0; k < n; ++k)
            if (e[k].H == H && e[k].W == W) return &e[k];
    }
    return nullptr;
}

}  // namespace

extern "C" pcs_status pcs_solve_slices_noalloc(const float* field, const unsigned char* mask, int H, int W,
                                               int S, double lambda, double tau, double sigma, int n_iter,
                                               float* chi_out, int b0_axis, void* cuda_stream) {
    PCS_TRACE("pcs_solve_slices_noalloc");
    if (S < 0 || n_iter < 0) return pcs::set_last_error(PCS_EINVAL, "pcs_solve_slices_noalloc: S and n_iter must be >= 0");
    const pcs::KernelEntry* entry = default_entry(H, W);
    if (!entry) return pcs::set_last_error(PCS_EUNSUPPORTED, "pcs_solve_slices_noalloc: unsupported slice size");
    if ((size_t)S * (size_t)H * (size_t)W > kMaxVoxels) {
        char buf[200];
        snprintf(buf, sizeof(buf),
                 "pcs_solve_slices_noalloc: S*H*W = %zu exceeds the static scratch of %zu voxels; "
                 "split the batch or use pcs_create/pcs_solve_slices",
                 (size_t)S * H * W, kMaxVoxels);
        return pcs::set_last_error(PCS_EINVAL, buf);
    }
    if (S == 0) return PCS_OK;
    if (!field || !mask || !chi_out || field == chi_out)
        return pcs::set_last_error(PCS_EINVAL, "pcs_solve_slices_noalloc: NULL or aliased buffer");
    if (!(lambda > 0.0) || !(tau > 0.0) || !(sigma > 0.0) || !std::isfinite(lambda) || !std::isfinite(tau) ||
        !std::isfinite(sigma))
        return pcs::set_last_error(PCS_EINVAL, "pcs_solve_slices_noalloc: lambda, tau, sigma must be > 0");
    if (b0_axis != 0 && b0_axis != 1) return pcs::set_last_error(PCS_EINVAL, "pcs_solve_slices_noalloc: b0_axis");
    if (((reinterpret_cast<uintptr_t>(field) | reinterpret_cast<uintptr_t>(mask) |
          reinterpret_cast<uintptr_t>(chi_out)) & 15u) != 0)
        return pcs::set_last_error(PCS_EINVAL, "pcs_solve_slices_noalloc: buffers must be 16-byte aligned");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(PCS_ECUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return pcs::set_last_error(PCS_EUNSUPPORTED, "pcs_solve_slices_noalloc: device index");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    std::lock_guard<std::mutex> lk(g_mu);
    DeviceSetup& d = g_dev[dev];
    if (!d.ready) {  // once per device, with that device current
        if ((e = cudaGetSymbolAddress((void**)&d.state, g_noalloc_state)) != cudaSuccess)
            return err(PCS_ECUDA, "cudaGetSymbolAddress(state)", e);
        if ((e = cudaGetSymbolAddress((void**)&d.dtab, g_noalloc_dtab)) != cudaSuccess)
            return err(PCS_ECUDA, "cudaGetSymbolAddress(dtab)", e);
        if ((e = cudaGetSymbolAddress((void**)&d.ddtab, g_noalloc_ddtab)) != cudaSuccess)
            return err(PCS_ECUDA, "cudaGetSymbolAddress(ddtab)", e);
        if ((e = cudaGetSymbolAddress((void**)&d.twid, g_noalloc_twid)) != cudaSuccess)
            return err(PCS_ECUDA, "cudaGetSymbolAddress(twid)", e);
        d.ready = true;
    }
    int slot = -1;
    for (int k = 0; k < 16; ++k)
        if (d.prepared[k] == entry || d.prepared[k] == nullptr) {
            slot = k;
            break;
        }
    if (slot < 0) return pcs::set_last_error(PCS_EUNSUPPORTED, "pcs_solve_slices_noalloc: too many sizes");
    if (d.prepared[slot] == nullptr) {
        int a = 0;
        if ((e = entry->prepare(&d.max_clusters[slot], &a)) != cudaSuccess) return err(PCS_ECUDA, "kernel attributes", e);
        d.prepared[slot] = entry;
    }
    int k_size = -1;
    for (int k = 0; k < kNumSizes; ++k)
        if (kSizes[k] == H && H == W) k_size = k;
    if (k_size < 0) return pcs::set_last_error(PCS_EUNSUPPORTED, "pcs_solve_slices_noalloc: no table region");
    float* dtab_r = d.dtab + dtab_offset(k_size, b0_axis);
    float* ddtab_r = d.ddtab + line_offset(k_size, b0_axis);
    float2* twid_r = d.twid + line_offset(k_size, 0);  // float2 entries: the sizes before this one
    if (!d.tables[k_size][b0_axis] || !d.twiddles[k_size]) {
        // first call of this size (or axis) on this device: fill the regions not yet filled, once
        std::vector<float> dtab, ddtab;
        std::vector<float2> tw;
        pcs::build_dipole_tables(H, W, b0_axis, dtab, ddtab);
        pcs::build_twiddles(H, tw);
        if (dtab.size() != (size_t)(H / 2) * H || ddtab.size() != (size_t)H || tw.size() != (size_t)H)
            return pcs::set_last_error(PCS_ECUDA, "pcs_solve_slices_noalloc: table size mismatch");
        if (!d.tables[k_size][b0_axis] &&
            ((e = cudaMemcpyAsync(dtab_r, dtab.data(), dtab.size() * sizeof(float), cudaMemcpyHostToDevice,
                                  stream)) != cudaSuccess ||
             (e = cudaMemcpyAsync(ddtab_r, ddtab.data(), ddtab.size() * sizeof(float), cudaMemcpyHostToDevice,
                                  stream)) != cudaSuccess))
            return err(PCS_ECUDA, "table upload", e);
        if (!d.twiddles[k_size] &&
            (e = cudaMemcpyAsync(twid_r, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, stream)) !=
                cudaSuccess)
            return err(PCS_ECUDA, "table upload", e);
        // the host vectors die at scope exit: wait for the copies to read them
        if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return err(PCS_ECUDA, "stream sync", e);
        d.tables[k_size][b0_axis] = true;
        d.twiddles[k_size] = true;
    }

    const size_t n = (size_t)S * H * W;
    pcs::PDParams prm;
    std::memset(&prm, 0, sizeof(prm));
    prm.field = field;
    prm.mask = mask;
    prm.chi = chi_out;
    prm.chibar = d.state;
    prm.p = d.state + n;
    prm.qx = d.state + 2 * n;
    prm.qy = d.state + 3 * n;
    prm.dtab = dtab_r;
    prm.ddtab = ddtab_r;
    prm.twid = twid_r;
    prm.S = S;
    prm.n_iter = n_iter;
    prm.sigma = (float)sigma;
    prm.tau = (float)tau;
    prm.inv_den = (float)(1.0 / (1.0 + sigma / lambda));
    prm.inv_den_slice = nullptr;
    int ncl = d.max_clusters[slot];
    if (ncl > S) ncl = S;
    if (ncl < 1) ncl = 1;
    if ((e = entry->launch(prm, ncl, stream)) != cudaSuccess) return err(PCS_ECUDA, "kernel launch", e);
    return PCS_OK;
}
