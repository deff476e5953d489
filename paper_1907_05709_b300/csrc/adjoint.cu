// adjoint.cu -- sqrt(N) checkpoint recording and the discrete adjoint.
#include "rfa_internal.cuh"

#include <cmath>

namespace rfa {

void record_free(rfa_grid *g)
{
    for (void *p : g->rec.ck_hi) cudaFree(p);
    for (void *p : g->rec.ck_lo) if (p) cudaFree(p);
    g->rec.ck_hi.clear();
    g->rec.ck_lo.clear();
    g->rec.valid = false;
    g->rec.seg = 0;
    g->rec.nsteps = 0;
}

rfa_status record_begin(rfa_grid *g, int64_t nsteps)
{
    record_free(g);
    g->rec.seg = (int64_t)std::ceil(std::sqrt((double)nsteps));
    if (g->rec.seg < 1) g->rec.seg = 1;
    g->rec.valid = true;
    return RFA_OK;
}

rfa_status record_checkpoint(rfa_grid *g, int64_t step_index)
{
    (void)step_index;
    void *hi = nullptr, *lo = nullptr;
    size_t bytes = g->nvp * g->state_elem();
    if (cudaMalloc(&hi, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("checkpoint allocation failed");
        return RFA_E_OOM;
    }
    if (g->sp == RFA_STATE_F32C && cudaMalloc(&lo, g->nvp * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(hi);
        set_error("checkpoint allocation failed");
        return RFA_E_OOM;
    }
    RFA_CUDA(cudaMemcpyAsync(hi, g->th[g->cur], bytes, cudaMemcpyDeviceToDevice, g->stream));
    if (lo) RFA_CUDA(cudaMemcpyAsync(lo, g->lo[g->cur], g->nvp * 4, cudaMemcpyDeviceToDevice, g->stream));
    g->rec.ck_hi.push_back(hi);
    g->rec.ck_lo.push_back(lo);
    return RFA_OK;
}

rfa_status backward_impl(rfa_grid *, const float *, double *)
{
    set_error("adjoint not built yet");
    return RFA_E_UNSUPPORTED;
}

}  // namespace rfa

extern "C" rfa_status rfa_backward(rfa_grid *g, const float *dLdT_final_dev, double *grads)
{
    if (!g || !dLdT_final_dev || !grads) {
        rfa::set_error("null argument");
        return RFA_E_INVALID;
    }
    return rfa::backward_impl(g, dLdT_final_dev, grads);
}
