// Instantiations of the persistent SMO step for the fp64 row pass.
#include "smo_step.cuh"

namespace svmgb {
cudaError_t launch_smo_fp64(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st, int cs)
{
    return smo::launch_mode<MODE_FP64>(lpr, a, smem, st, cs);
}
int max_clusters_fp64(int lpr, int resident, size_t smem, int cs)
{
    return smo::max_clusters<MODE_FP64>(lpr, resident, smem, cs);
}
}  // namespace svmgb
