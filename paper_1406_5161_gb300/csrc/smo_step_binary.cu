// Instantiations of the persistent SMO step for the binary row pass.
#include "smo_step.cuh"

namespace svmgb {
cudaError_t launch_smo_binary(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st, int cs)
{
    return smo::launch_mode<MODE_BINARY>(lpr, a, smem, st, cs);
}
int max_clusters_binary(int lpr, int resident, size_t smem, int cs)
{
    return smo::max_clusters<MODE_BINARY>(lpr, resident, smem, cs);
}
}  // namespace svmgb
