// kernels_tb.cu -- temporally blocked step (several steps per launch).
#include "rfa_internal.cuh"

namespace rfa {

bool tb_supported(const rfa_grid *, int, int) { return false; }

cudaError_t launch_step_tb(rfa_grid *, int, int, const void *, const void *, void *, void *, bool)
{
    return cudaErrorNotSupported;
}

}  // namespace rfa
