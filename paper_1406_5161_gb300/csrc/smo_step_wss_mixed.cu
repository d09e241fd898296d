// Instantiations of the persistent SMO step with the second-order choice of
// i_low, mixed row pass.
#include "smo_step.cuh"

namespace svmgb {
namespace smo {
void *smo_kernel_wss_mixed(int lpr, int resident) { return kernel_pick<MODE_MIXED, true>(lpr, resident); }
}  // namespace smo
}  // namespace svmgb
