// Instantiations of the persistent SMO step for the mixed row pass.
#include "smo_step.cuh"

namespace svmgb {
cudaError_t launch_smo_mixed(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st, int cs)
{
    return smo::launch_mode<MODE_MIXED>(lpr, a, smem, st, cs);
}
int max_clusters_mixed(int lpr, int resident, size_t smem, int cs)
{
    return smo::max_clusters<MODE_MIXED>(lpr, resident, smem, cs);
}
}  // namespace svmgb
