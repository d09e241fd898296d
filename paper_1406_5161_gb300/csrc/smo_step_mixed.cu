// Instantiations of the persistent SMO step for the mixed row pass.
#include "smo_step.cuh"

namespace svmgb {
cudaError_t launch_smo_mixed(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st)
{
    return smo::launch_mode<MODE_MIXED>(lpr, a, smem, st);
}
}  // namespace svmgb
