// Instantiations of the persistent SMO step with the second-order choice of
// i_low, binary row pass.
#include "smo_step.cuh"

namespace svmgb {
namespace smo {
void *smo_kernel_wss_binary(int lpr, int resident) { return kernel_pick<MODE_BINARY, true>(lpr, resident); }
}  // namespace smo
}  // namespace svmgb
