// FP64 instances of the fused iteration kernel (all-FP64 precision study):
// the same kernel template with double state, double transforms and double tables.
#include "pd_launch.cuh"

namespace pcs {
static const KernelEntryF64 k_entries[] = {
    make_f64_entry<Geo<64, 64, 1, 1, 256, 0, 0, double>>(),
    make_f64_entry<Geo<256, 256, 8, 1, 256, 0, 0, double>>(),
};
const KernelEntryF64* entries_f64(int* n) {
    *n = (int)(sizeof(k_entries) / sizeof(k_entries[0]));
    return k_entries;
}
}  // namespace pcs
