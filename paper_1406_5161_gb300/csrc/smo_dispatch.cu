// Dispatch of the persistent SMO step by row-pass arithmetic.
#include "smo_step.cuh"

namespace svmgb {

cudaError_t launch_smo_binary(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st, int cs);
cudaError_t launch_smo_fp64(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st, int cs);
cudaError_t launch_smo_mixed(int lpr, const SmoArgs &a, size_t smem, cudaStream_t st, int cs);
int max_clusters_binary(int lpr, int resident, size_t smem, int cs);
int max_clusters_fp64(int lpr, int resident, size_t smem, int cs);
int max_clusters_mixed(int lpr, int resident, size_t smem, int cs);
cudaError_t launch_smo_bits(int mode, int lpr, const SmoArgs &a, size_t smem, cudaStream_t st, int cs);
int max_clusters_bits(int mode, int lpr, int resident, size_t smem, int cs);

// Failure-handling check: one thread waits, with the fused step's bounded
// wait, on an mbarrier that nothing completes.
__global__ void k_diag_wait(int64_t timeout_ns, const int *err, int *gave_up)
{
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) smo::mbar_init(smo::smem_u32(&bar), 1);
    __syncthreads();
    if (threadIdx.x == 0) *gave_up = smo::mbar_wait_bounded(smo::smem_u32(&bar), 0u, timeout_ns, err);
}

cudaError_t launch_diag_wait(int64_t timeout_ns, const int *err, int *gave_up, cudaStream_t st)
{
    k_diag_wait<<<1, 32, 0, st>>>(timeout_ns, err, gave_up);
    return cudaGetLastError();
}

int smo_threads() { return smo::kThreads; }
size_t smo_cand_bytes() { return smo::kCandStride; }
size_t smo_static_smem(int mode)
{
    return sizeof(smo::Shared) + sizeof(uint64_t) * (mode == MODE_FP64 ? kExpfxTabLen : 1);
}

cudaError_t launch_smo_persistent(int mode, int lpr, const SmoArgs &a, size_t smem, cudaStream_t st,
                                  int cs)
{
    switch (mode) {
    case MODE_BINARY: return launch_smo_binary(lpr, a, smem, st, cs);
    case MODE_FP64: return launch_smo_fp64(lpr, a, smem, st, cs);
    case MODE_MIXED: return launch_smo_mixed(lpr, a, smem, st, cs);
    case MODE_BITS4:
    case MODE_BITS8: return launch_smo_bits(mode, lpr, a, smem, st, cs);
    default: return cudaErrorInvalidValue;
    }
}

int smo_max_clusters(int mode, int lpr, int resident, size_t smem, int cs)
{
    switch (mode) {
    case MODE_BINARY: return max_clusters_binary(lpr, resident, smem, cs);
    case MODE_FP64: return max_clusters_fp64(lpr, resident, smem, cs);
    case MODE_MIXED: return max_clusters_mixed(lpr, resident, smem, cs);
    case MODE_BITS4:
    case MODE_BITS8: return max_clusters_bits(mode, lpr, resident, smem, cs);
    default: return 0;
    }
}

}  // namespace svmgb
