// Fused primal-dual kernel instances for 256 x 256 slices (spectrum spread over a cluster).
#include "pd_launch.cuh"

namespace pcs {
static const KernelEntry k_entries[] = {
    make_entry<Geo<256, 256, 4, 2>>(),
    make_resident_entry<GeoRes<256, 256, 8>>(),
    make_entry<Geo<256, 256, 2, 1>>(),
    make_entry<Geo<256, 256, 8, 2>>(),
    // eight elements per lane, 512-thread CTAs (more warps per SM)
    make_resident_entry<GeoRes<256, 256, 8, 512, 8, 8>>(),
    make_entry<Geo<256, 256, 4, 2, 512, 8, 8>>(),
};
const KernelEntry* entries_256(int* n) {
    *n = (int)(sizeof(k_entries) / sizeof(k_entries[0]));
    return k_entries;
}
}  // namespace pcs
