// Instantiations of the persistent SMO step for the fp64 row pass.
#include "smo_step.cuh"

namespace svmgb {
cudaError_t launch_smo_fp64(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st)
{
    return smo::launch_mode<MODE_FP64>(lpr, a, smem, st);
}
}  // namespace svmgb
