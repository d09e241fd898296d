// Dispatch of the persistent SMO step by row-pass arithmetic.
#include "smo_step.cuh"

namespace svmgb {

cudaError_t launch_smo_binary(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st);
cudaError_t launch_smo_fp64(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st);
cudaError_t launch_smo_mixed(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st);

int smo_threads() { return smo::kThreads; }
size_t smo_cand_bytes() { return sizeof(smo::CandFull); }
size_t smo_static_smem() { return sizeof(smo::Shared); }

cudaError_t launch_smo_persistent(int mode, int lpr, const SmoArgs &a, size_t smem, cudaStream_t st)
{
    switch (mode) {
    case MODE_BINARY: return launch_smo_binary(lpr, a, smem, st);
    case MODE_FP64: return launch_smo_fp64(lpr, a, smem, st);
    case MODE_MIXED: return launch_smo_mixed(lpr, a, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace svmgb
