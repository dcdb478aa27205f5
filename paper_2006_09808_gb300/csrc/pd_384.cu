// Fused primal-dual kernel instances for 384 x 384 slices (radix-3 stages).
#include "pd_launch.cuh"

namespace pcs {
static const KernelEntry k_entries[] = {
    make_entry<Geo<384, 384, 4, 1>>(),
    make_entry<Geo<384, 384, 4, 1, 384>>(),   // 12 warps per SM
};
const KernelEntry* entries_384(int* n) {
    *n = (int)(sizeof(k_entries) / sizeof(k_entries[0]));
    return k_entries;
}
}  // namespace pcs
