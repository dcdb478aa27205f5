// Fused primal-dual kernel instances for 256 x 256 slices (spectrum spread over a cluster).
#include "pd_launch.cuh"

namespace pcs {
static const KernelEntry k_entries[] = {
    // default: 4-CTA clusters, one 512-thread CTA per SM (more slices than its resident clusters
    // run on the balanced schedule)
    make_entry<Geo<256, 256, 4, 1, 512>>(),
    make_entry<Geo<256, 256, 4, 2>>(),
    make_resident_entry<GeoRes<256, 256, 8>>(),
    make_entry<Geo<256, 256, 2, 1>>(),
    make_entry<Geo<256, 256, 8, 2>>(),
    // eight elements per lane, 512-thread CTAs (more warps per SM)
    make_resident_entry<GeoRes<256, 256, 8, 512, 8, 8>>(),
    // other FFT tile shapes of the default geometry (the autotuner's choice): rows with 8
    // elements per lane (16 lanes per row, two row passes), or columns with 8 (32 lanes per column)
    make_entry<Geo<256, 256, 4, 1, 512, 8, 16>>(),
    make_entry<Geo<256, 256, 4, 1, 512, 16, 8>>(),
};
const KernelEntry* entries_256(int* n) {
    *n = (int)(sizeof(k_entries) / sizeof(k_entries[0]));
    return k_entries;
}
}  // namespace pcs
