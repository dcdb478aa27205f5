// Fused primal-dual kernel instances for 64 x 64 slices (whole slice in one CTA).
#include "pd_launch.cuh"

namespace pcs {
static const KernelEntry k_entries[] = {
    make_resident_entry<GeoRes<64, 64, 1>>(),
    make_entry<Geo<64, 64, 1, 2>>(),
};
const KernelEntry* entries_64(int* n) {
    *n = (int)(sizeof(k_entries) / sizeof(k_entries[0]));
    return k_entries;
}
}  // namespace pcs
