// Fused primal-dual kernel instances for 512 x 512 slices.
#include "pd_launch.cuh"

namespace pcs {
static const KernelEntry k_entries[] = {
    make_entry<Geo<512, 512, 8, 1>>(),
    make_entry<Geo<512, 512, 8, 1, 512>>(),   // 16 warps per SM
    make_entry<Geo<512, 512, 16, 2>>(),       // 16-CTA clusters, two CTAs per SM
};
const KernelEntry* entries_512(int* n) {
    *n = (int)(sizeof(k_entries) / sizeof(k_entries[0]));
    return k_entries;
}
}  // namespace pcs
