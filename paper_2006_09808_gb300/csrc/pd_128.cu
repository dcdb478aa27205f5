// Fused primal-dual kernel instances for 128 x 128 slices.
#include "pd_launch.cuh"

namespace pcs {
static const KernelEntry k_entries[] = {
    make_resident_entry<GeoRes<128, 128, 4>>(),
    make_entry<Geo<128, 128, 1, 2>>(),
    make_entry<Geo<128, 128, 2, 2>>(),
};
const KernelEntry* entries_128(int* n) {
    *n = (int)(sizeof(k_entries) / sizeof(k_entries[0]));
    return k_entries;
}
}  // namespace pcs
