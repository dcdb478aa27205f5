// pd_launch.cuh -- launch glue shared by the per-size translation units.
#pragma once

#include <cuda_runtime.h>

#include "pd_aux.cuh"
#include "pd_cluster.cuh"
#include "pd_resident.cuh"

namespace pcs {

// One compiled (H, W, cluster size) variant: the iteration kernel and its
// diagnostics / step-size companions.
struct KernelEntry {
    int H, W, C;
    int resident;  // 1: state held on chip (pd_resident_kernel); 0: state streamed (pd_cluster_kernel)
    size_t smem;
    int threads;
    int tile;      // FFT tile shape: 100 x (elements per lane of the row transforms) + those of the columns
    // Sets function attributes; returns how many clusters of the iteration
    // kernel and of the auxiliary kernels can be resident.
    cudaError_t (*prepare)(int* max_clusters, int* max_clusters_aux);
    cudaError_t (*launch)(const PDParams& prm, int n_clusters, cudaStream_t stream);
    cudaError_t (*launch_report)(const AuxParams& prm, int n_clusters, cudaStream_t stream);
    cudaError_t (*launch_opnorm)(const AuxParams& prm, int n_clusters, cudaStream_t stream);
    // the balanced-schedule instantiation of the iteration kernel (NULL for the resident kernel)
    cudaError_t (*launch_sched)(const PDParams& prm, int n_clusters, cudaStream_t stream);
};

template <class G>
constexpr size_t aux_smem() {
    return G::SMEM_BYTES + 64 * sizeof(double);
}

template <class G, class P>
cudaError_t launch_cluster(void (*kern)(P), const P& prm, size_t smem, int n_clusters, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_clusters * G::C, 1, 1);
    cfg.blockDim = dim3(G::NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, prm);
}

template <class G, class P>
cudaError_t prepare_cluster(void (*kern)(P), size_t smem, int* max_clusters) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (G::C > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G::C, 1, 1);
    cfg.blockDim = dim3(G::NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(max_clusters, kern, &cfg);
}

template <class G>
cudaError_t launch_pd(const PDParams& prm, int n_clusters, cudaStream_t stream) {
    return launch_cluster<G>(pd_cluster_kernel<G>, prm, G::SMEM_BYTES, n_clusters, stream);
}
template <class G>
cudaError_t launch_pd_sched(const PDParams& prm, int n_clusters, cudaStream_t stream) {
    return launch_cluster<G>(pd_cluster_kernel<G, true>, prm, G::SMEM_BYTES, n_clusters, stream);
}
template <class G>
cudaError_t launch_report(const AuxParams& prm, int n_clusters, cudaStream_t stream) {
    return launch_cluster<G>(aux_report_kernel<G>, prm, aux_smem<G>(), n_clusters, stream);
}
template <class G>
cudaError_t launch_opnorm(const AuxParams& prm, int n_clusters, cudaStream_t stream) {
    return launch_cluster<G>(aux_opnorm_kernel<G>, prm, aux_smem<G>(), n_clusters, stream);
}

template <class G>
cudaError_t prepare_all(int* max_clusters, int* max_clusters_aux) {
    cudaError_t e = prepare_cluster<G>(pd_cluster_kernel<G>, G::SMEM_BYTES, max_clusters);
    if (e != cudaSuccess) return e;
    int a = 0, b = 0, c = 0;
    if ((e = prepare_cluster<G>(pd_cluster_kernel<G, true>, G::SMEM_BYTES, &c)) != cudaSuccess) return e;
    if (c < *max_clusters) *max_clusters = c;
    if ((e = prepare_cluster<G>(aux_report_kernel<G>, aux_smem<G>(), &a)) != cudaSuccess) return e;
    if ((e = prepare_cluster<G>(aux_opnorm_kernel<G>, aux_smem<G>(), &b)) != cudaSuccess) return e;
    *max_clusters_aux = a < b ? a : b;
    return cudaSuccess;
}

template <class G>
constexpr KernelEntry make_entry() {
    return KernelEntry{G::H,           G::W,           G::C,       0,
                       G::SMEM_BYTES,  G::NT,          100 * G::ER + G::EC, &prepare_all<G>,
                       &launch_pd<G>,  &launch_report<G>, &launch_opnorm<G>, &launch_pd_sched<G>};
}

// Resident variant: the iteration kernel keeps the state on chip; the
// diagnostics and power iteration use the streaming geometry's kernels.
template <class GR>
cudaError_t launch_res(const PDParams& prm, int n_clusters, cudaStream_t stream) {
    return launch_cluster<GR>(pd_resident_kernel<GR>, prm, GR::SMEM_BYTES, n_clusters, stream);
}
template <class GR>
cudaError_t prepare_res(int* max_clusters, int* max_clusters_aux) {
    using G = typename GR::B;
    cudaError_t e = prepare_cluster<GR>(pd_resident_kernel<GR>, GR::SMEM_BYTES, max_clusters);
    if (e != cudaSuccess) return e;
    int a = 0, b = 0;
    if ((e = prepare_cluster<G>(aux_report_kernel<G>, aux_smem<G>(), &a)) != cudaSuccess) return e;
    if ((e = prepare_cluster<G>(aux_opnorm_kernel<G>, aux_smem<G>(), &b)) != cudaSuccess) return e;
    *max_clusters_aux = a < b ? a : b;
    return cudaSuccess;
}
template <class GR>
constexpr KernelEntry make_resident_entry() {
    using G = typename GR::B;
    return KernelEntry{GR::H,           GR::W,          GR::C,       1,
                       GR::SMEM_BYTES,  GR::NT,         100 * GR::ER + GR::EC, &prepare_res<GR>,
                       &launch_res<GR>, &launch_report<G>, &launch_opnorm<G>, nullptr};
}

// FP64 variant (precision study): iteration kernel only.
struct KernelEntryF64 {
    int H, W, C;
    size_t smem;
    cudaError_t (*prepare)(int* max_clusters);
    cudaError_t (*launch)(const PDParamsT<double>& prm, int n_clusters, cudaStream_t stream);
};
template <class G>
cudaError_t launch_pd64(const PDParamsT<double>& prm, int n_clusters, cudaStream_t stream) {
    return launch_cluster<G>(pd_cluster_kernel<G>, prm, G::SMEM_BYTES, n_clusters, stream);
}
template <class G>
cudaError_t prepare_pd64(int* max_clusters) {
    return prepare_cluster<G>(pd_cluster_kernel<G>, G::SMEM_BYTES, max_clusters);
}
template <class G>
constexpr KernelEntryF64 make_f64_entry() {
    return KernelEntryF64{G::H, G::W, G::C, G::SMEM_BYTES, &prepare_pd64<G>, &launch_pd64<G>};
}
const KernelEntryF64* entries_f64(int* n);

// Per-size translation units define these (pd_<size>.cu).
const KernelEntry* entries_64(int* n);
const KernelEntry* entries_128(int* n);
const KernelEntry* entries_192(int* n);
const KernelEntry* entries_256(int* n);
const KernelEntry* entries_384(int* n);
const KernelEntry* entries_512(int* n);

}  // namespace pcs
