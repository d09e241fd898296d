// Instantiations of the persistent SMO step with the second-order choice of
// i_low, fp64 row pass.
#include "smo_step.cuh"

namespace svmgb {
namespace smo {
void *smo_kernel_wss_fp64(int lpr, int resident) { return kernel_pick<MODE_FP64, true>(lpr, resident); }
}  // namespace smo
}  // namespace svmgb
