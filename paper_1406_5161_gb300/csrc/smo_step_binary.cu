// Instantiations of the persistent SMO step for the binary row pass.
#include "smo_step.cuh"

namespace svmgb {
cudaError_t launch_smo_binary(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st)
{
    return smo::launch_mode<MODE_BINARY>(lpr, a, smem, st);
}
}  // namespace svmgb
