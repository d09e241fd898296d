// Instantiations of the persistent SMO step for binary rows held as bit
// masks (4 words for d <= 128, 8 words for d <= 256; one lane per row).
#include "smo_step.cuh"

namespace svmgb {
cudaError_t launch_smo_bits(int mode, int lpr, const SmoArgs &a, size_t smem, cudaStream_t st, int cs)
{
    if (mode == MODE_BITS4) return smo::launch_mode<MODE_BITS4>(lpr, a, smem, st, cs);
    if (mode == MODE_BITS8) return smo::launch_mode<MODE_BITS8>(lpr, a, smem, st, cs);
    return cudaErrorInvalidValue;
}
int max_clusters_bits(int mode, int lpr, int resident, size_t smem, int cs)
{
    if (mode == MODE_BITS4) return smo::max_clusters<MODE_BITS4>(lpr, resident, smem, cs);
    if (mode == MODE_BITS8) return smo::max_clusters<MODE_BITS8>(lpr, resident, smem, cs);
    return 0;
}
}  // namespace svmgb
