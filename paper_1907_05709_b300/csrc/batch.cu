// batch.cu -- batched persistent stepping of several grids.
#include "rfa_internal.cuh"

struct rfa_batch {
    int n = 0;
};

extern "C" {
rfa_status rfa_batch_create(rfa_grid *const *, int, rfa_batch **out)
{
    if (out) *out = nullptr;
    rfa::set_error("batched stepping not built yet");
    return RFA_E_UNSUPPORTED;
}
rfa_status rfa_batch_step(rfa_batch *, int64_t)
{
    rfa::set_error("batched stepping not built yet");
    return RFA_E_UNSUPPORTED;
}
rfa_status rfa_batch_destroy(rfa_batch *b)
{
    delete b;
    return RFA_OK;
}
}
