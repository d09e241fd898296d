// Instantiations of the persistent SMO step with the second-order choice of
// i_low, bit-mask rows; and the dispatch over the row-pass arithmetic.
#include "smo_step.cuh"

namespace svmgb {
namespace smo {
void *smo_kernel_wss_fp64(int lpr, int resident);
void *smo_kernel_wss_mixed(int lpr, int resident);
void *smo_kernel_wss_binary(int lpr, int resident);

void *smo_kernel_wss(int mode, int lpr, int resident)
{
    switch (mode) {
    case MODE_FP64: return smo_kernel_wss_fp64(lpr, resident);
    case MODE_MIXED: return smo_kernel_wss_mixed(lpr, resident);
    case MODE_BINARY: return smo_kernel_wss_binary(lpr, resident);
    case MODE_BITS4: return kernel_pick<MODE_BITS4, true>(lpr, resident);
    case MODE_BITS8: return kernel_pick<MODE_BITS8, true>(lpr, resident);
    default: return nullptr;
    }
}
}  // namespace smo
}  // namespace svmgb
