// pcs_fieldmap.cu -- the preprocessing step of Sec. II.B (1): local field,
// magnitude weighting and mask from the two acquisitions without and with the
// readout shift T_shift (pcs_field_map).
//
// Two launches on the caller's stream: per-CTA maxima of |S0|^2 over a
// grid-stride range, then one pointwise pass (each CTA first reduces those
// maxima; max is order-independent, so deterministic) writing
// dB = arg(S1 conj S0) / (2 pi gamma_bar B0 T_shift) (ppm; zero outside the
// mask), W = |S0| / max |S0| and mask = (|S0|^2 >= t^2 max |S0|^2).  Two
// voxels per thread and step (16-byte loads).  The
// mask decision uses round-to-nearest float32 products and sums without
// contraction, so it is reproducible bit for bit.  Memory bound: 8 bytes in
// per voxel for the maximum, 16 in and 9 out for the map.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>

#include "../../include/pcs.h"
#include "pcs_trace.h"

namespace pcs {
pcs_status set_last_error(pcs_status st, const char* msg);
}  // namespace pcs

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float mag2_rn(float2 a) { return __fadd_rn(__fmul_rn(a.x, a.x), __fmul_rn(a.y, a.y)); }

// Per-CTA maxima of |S0|^2 over a grid-stride range, two voxels (one 16-byte load) per step.
__global__ void __launch_bounds__(kThreads) fm_max_kernel(const float4* __restrict__ s0, size_t n_pairs,
                                                          const float2* __restrict__ tail, int has_tail,
                                                          float* __restrict__ partial) {
    float m = 0.f;
    for (size_t k = (size_t)blockIdx.x * kThreads + threadIdx.x; k < n_pairs; k += (size_t)gridDim.x * kThreads) {
        const float4 a = __ldcs(s0 + k);
        m = fmaxf(m, fmaxf(mag2_rn(make_float2(a.x, a.y)), mag2_rn(make_float2(a.z, a.w))));
    }
    if (has_tail && blockIdx.x == 0 && threadIdx.x == 0) m = fmaxf(m, mag2_rn(*tail));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    __shared__ float red[kThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w) m = fmaxf(m, red[w]);
        partial[blockIdx.x] = m;
    }
}

__device__ __forceinline__ void fm_voxel(float2 a, float2 b, float cut, float inv_max, float ppm_per_rad,
                                         float& field, float& weight, unsigned char& mask) {
    const float m2 = mag2_rn(a);
    const bool in = m2 >= cut;
    const float re = b.x * a.x + b.y * a.y;  // S1 conj(S0)
    const float im = b.y * a.x - b.x * a.y;
    field = in ? atan2f(im, re) * ppm_per_rad : 0.f;
    weight = fminf(1.f, sqrtf(m2) * inv_max);
    mask = in ? 1 : 0;
}

// The map: every CTA first reduces the per-CTA maxima (max is order-independent).
__global__ void __launch_bounds__(kThreads) fm_map_kernel(const float4* __restrict__ s0, const float4* __restrict__ s1,
                                                          size_t n, const float* __restrict__ partial, int n_partial,
                                                          float thr2, float ppm_per_rad, float* __restrict__ field,
                                                          float* __restrict__ weight,
                                                          unsigned char* __restrict__ mask) {
    __shared__ float s_max;
    float m = 0.f;
    for (int k = threadIdx.x; k < n_partial; k += kThreads) m = fmaxf(m, __ldcg(partial + k));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    __shared__ float red[kThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w) m = fmaxf(m, red[w]);
        s_max = m;
    }
    __syncthreads();
    const float max2 = s_max;
    const float cut = __fmul_rn(thr2, max2);
    const float inv_max = max2 > 0.f ? 1.0f / sqrtf(max2) : 0.f;
    const size_t n_pairs = n / 2;
    for (size_t k = (size_t)blockIdx.x * kThreads + threadIdx.x; k < n_pairs; k += (size_t)gridDim.x * kThreads) {
        const float4 a = __ldcs(s0 + k), b = __ldcs(s1 + k);
        float2 f, w;
        uchar2 mk;
        fm_voxel(make_float2(a.x, a.y), make_float2(b.x, b.y), cut, inv_max, ppm_per_rad, f.x, w.x, mk.x);
        fm_voxel(make_float2(a.z, a.w), make_float2(b.z, b.w), cut, inv_max, ppm_per_rad, f.y, w.y, mk.y);
        __stcs(reinterpret_cast<float2*>(field) + k, f);
        __stcs(reinterpret_cast<float2*>(weight) + k, w);
        reinterpret_cast<uchar2*>(mask)[k] = mk;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {  // odd count: the last voxel
        const float2* a = reinterpret_cast<const float2*>(s0) + (n - 1);
        const float2* b = reinterpret_cast<const float2*>(s1) + (n - 1);
        fm_voxel(*a, *b, cut, inv_max, ppm_per_rad, field[n - 1], weight[n - 1], mask[n - 1]);
    }
}

pcs_status fm_fail(pcs_status st, const char* what, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess) {
        snprintf(buf, sizeof(buf), "pcs_field_map: %s: %s", what, cudaGetErrorString(e));
    } else {
        snprintf(buf, sizeof(buf), "pcs_field_map: %s", what);
    }
    return pcs::set_last_error(st, buf);
}

}  // namespace

extern "C" pcs_status pcs_field_map(const float* s0, const float* s1, size_t n_voxels, double t_shift_s,
                                    double b0_tesla, double threshold, float* field_out, float* weight_out,
                                    unsigned char* mask_out, void* cuda_stream) {
    PCS_TRACE("pcs_field_map");
    if (n_voxels == 0) return PCS_OK;
    if (!s0 || !s1 || !field_out || !weight_out || !mask_out) return fm_fail(PCS_EINVAL, "NULL argument");
    if (!(t_shift_s > 0.0) || !(b0_tesla > 0.0) || !(threshold >= 0.0))
        return fm_fail(PCS_EINVAL, "t_shift and b0 must be > 0, threshold >= 0");
    if ((reinterpret_cast<uintptr_t>(s0) | reinterpret_cast<uintptr_t>(s1)) & 15u)
        return fm_fail(PCS_EINVAL, "s0, s1 must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(field_out) | reinterpret_cast<uintptr_t>(weight_out)) & 7u ||
        (reinterpret_cast<uintptr_t>(mask_out) & 1u))
        return fm_fail(PCS_EINVAL, "field_out, weight_out must be 8-byte and mask_out 2-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return fm_fail(PCS_ECUDA, "device query", e);
    const double ppm_per_rad = 1e6 / (2.0 * M_PI * 42.577478518e6 * b0_tesla * t_shift_s);
    const float thr2 = (float)(threshold * threshold);
    const size_t n_pairs = n_voxels / 2;
    const size_t blocks_needed = (n_pairs + kThreads - 1) / kThreads;
    size_t g = blocks_needed < (size_t)sms * 4 ? blocks_needed : (size_t)sms * 4;
    const int grid = g < 1 ? 1 : (int)g;
    float* partial = nullptr;
    if ((e = cudaMallocAsync(&partial, (size_t)grid * sizeof(float), st)) != cudaSuccess)
        return fm_fail(PCS_ECUDA, "cudaMallocAsync", e);
    pcs_status ret = PCS_OK;
    const float4* a = reinterpret_cast<const float4*>(s0);
    const float4* b = reinterpret_cast<const float4*>(s1);
    fm_max_kernel<<<grid, kThreads, 0, st>>>(a, n_pairs, reinterpret_cast<const float2*>(s0) + (n_voxels - 1),
                                             (int)(n_voxels & 1), partial);
    fm_map_kernel<<<grid, kThreads, 0, st>>>(a, b, n_voxels, partial, grid, thr2, (float)ppm_per_rad, field_out,
                                             weight_out, mask_out);
    if ((e = cudaGetLastError()) != cudaSuccess) ret = fm_fail(PCS_ECUDA, "launch", e);
    cudaFreeAsync(partial, st);
    return ret;
}
