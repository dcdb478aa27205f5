// Fused primal-dual kernel instances for 192 x 192 slices (radix-3 stages).
#include "pd_launch.cuh"

namespace pcs {
static const KernelEntry k_entries[] = {
    make_entry<Geo<192, 192, 2, 2>>(),
};
const KernelEntry* entries_192(int* n) {
    *n = (int)(sizeof(k_entries) / sizeof(k_entries[0]));
    return k_entries;
}
}  // namespace pcs
