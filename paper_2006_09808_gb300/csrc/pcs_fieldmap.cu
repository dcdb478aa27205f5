// pcs_fieldmap.cu -- the preprocessing step of Sec. II.B (1): local field,
// magnitude weighting and mask from the two acquisitions without and with the
// readout shift T_shift (pcs_field_map).
//
// Two launches on the caller's stream: a grid-stride maximum of |S0|^2 over
// the volume (order-independent, so deterministic), then one pointwise pass
// writing dB = arg(S1 conj S0) / (2 pi gamma_bar B0 T_shift) (ppm; zero outside
// the mask), W = |S0| / max |S0| and mask = (|S0|^2 >= t^2 max |S0|^2).  The
// mask decision uses round-to-nearest float32 products and sums without
// contraction, so it is reproducible bit for bit.  Memory bound: 16 bytes in
// for the maximum, 16 in and 9 out per voxel for the map.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>

#include "../../include/pcs.h"

namespace pcs {
pcs_status set_last_error(pcs_status st, const char* msg);
}  // namespace pcs

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float mag2_rn(float2 a) { return __fadd_rn(__fmul_rn(a.x, a.x), __fmul_rn(a.y, a.y)); }

__global__ void __launch_bounds__(kThreads) fm_max_kernel(const float2* __restrict__ s0, size_t n,
                                                          unsigned* __restrict__ max_bits) {
    float m = 0.f;
    for (size_t k = (size_t)blockIdx.x * kThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kThreads)
        m = fmaxf(m, mag2_rn(__ldcs(s0 + k)));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    __shared__ float red[kThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w) m = fmaxf(m, red[w]);
        atomicMax(max_bits, __float_as_uint(m));  // non-negative floats order like their bit patterns
    }
}

__global__ void __launch_bounds__(kThreads) fm_map_kernel(const float2* __restrict__ s0, const float2* __restrict__ s1,
                                                          size_t n, const unsigned* __restrict__ max_bits,
                                                          float thr2, float ppm_per_rad, float* __restrict__ field,
                                                          float* __restrict__ weight,
                                                          unsigned char* __restrict__ mask) {
    const float max2 = __uint_as_float(*max_bits);
    const float cut = __fmul_rn(thr2, max2);
    const float inv_max = max2 > 0.f ? 1.0f / sqrtf(max2) : 0.f;
    for (size_t k = (size_t)blockIdx.x * kThreads + threadIdx.x; k < n; k += (size_t)gridDim.x * kThreads) {
        const float2 a = __ldcs(s0 + k), b = __ldcs(s1 + k);
        const float m2 = mag2_rn(a);
        const bool in = m2 >= cut;
        const float re = b.x * a.x + b.y * a.y;  // S1 conj(S0)
        const float im = b.y * a.x - b.x * a.y;
        __stcs(field + k, in ? atan2f(im, re) * ppm_per_rad : 0.f);
        __stcs(weight + k, fminf(1.f, sqrtf(m2) * inv_max));
        mask[k] = in ? 1 : 0;
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
    if (n_voxels == 0) return PCS_OK;
    if (!s0 || !s1 || !field_out || !weight_out || !mask_out) return fm_fail(PCS_EINVAL, "NULL argument");
    if (!(t_shift_s > 0.0) || !(b0_tesla > 0.0) || !(threshold >= 0.0))
        return fm_fail(PCS_EINVAL, "t_shift and b0 must be > 0, threshold >= 0");
    if ((reinterpret_cast<uintptr_t>(s0) | reinterpret_cast<uintptr_t>(s1)) & 7u)
        return fm_fail(PCS_EINVAL, "s0, s1 must be 8-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return fm_fail(PCS_ECUDA, "device query", e);
    const double ppm_per_rad = 1e6 / (2.0 * M_PI * 42.577478518e6 * b0_tesla * t_shift_s);
    const float thr2 = (float)(threshold * threshold);
    const size_t blocks_needed = (n_voxels + kThreads - 1) / kThreads;
    const int grid = (int)(blocks_needed < (size_t)sms * 8 ? blocks_needed : (size_t)sms * 8);
    unsigned* max_bits = nullptr;
    if ((e = cudaMallocAsync(&max_bits, sizeof(unsigned), st)) != cudaSuccess)
        return fm_fail(PCS_ECUDA, "cudaMallocAsync", e);
    pcs_status ret = PCS_OK;
    if ((e = cudaMemsetAsync(max_bits, 0, sizeof(unsigned), st)) != cudaSuccess) {
        ret = fm_fail(PCS_ECUDA, "memset", e);
    } else {
        fm_max_kernel<<<grid, kThreads, 0, st>>>(reinterpret_cast<const float2*>(s0), n_voxels, max_bits);
        fm_map_kernel<<<grid, kThreads, 0, st>>>(reinterpret_cast<const float2*>(s0),
                                                 reinterpret_cast<const float2*>(s1), n_voxels, max_bits, thr2,
                                                 (float)ppm_per_rad, field_out, weight_out, mask_out);
        if ((e = cudaGetLastError()) != cudaSuccess) ret = fm_fail(PCS_ECUDA, "launch", e);
    }
    cudaFreeAsync(max_bits, st);
    return ret;
}
