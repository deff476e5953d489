// diag.cu -- diagnostic entry points for the failure-detection paths.
//
// Every device-side wait in this library (TMA mbarriers, the batch's grid
// barrier) spins with a clock64 limit and, when the limit passes, records
// kStatusTimeout instead of hanging.  rfa_selftest_wait_timeout exercises the
// same pattern on a flag that nothing sets, so the host-side reporting can be
// tested without faulting or hanging a GPU; rfa_set_wait_limits shortens the
// limits of the real waits so that a test can make them run out.
#include "rfa_internal.cuh"

namespace rfa {
namespace {

__global__ void k_wait_flag(const volatile unsigned *flag, long long limit, unsigned *status)
{
    const long long t0 = clock64();
    while (*flag == 0u) {
        if (clock64() - t0 > limit) {
            atomicOr(status, kStatusTimeout);
            return;
        }
        __nanosleep(256);
    }
}

}  // namespace
}  // namespace rfa

using namespace rfa;

extern "C" rfa_status rfa_selftest_wait_timeout(long long spin_limit_cycles)
{
    if (spin_limit_cycles < 1 || spin_limit_cycles > (1ll << 32)) {
        set_error("spin_limit_cycles must be in 1..2^32");
        return RFA_E_INVALID;
    }
    unsigned *buf = nullptr;  // [0] flag (never set), [1] status
    RFA_CUDA(cudaMalloc((void **)&buf, 2 * sizeof(unsigned)));
    cudaError_t e = cudaMemset(buf, 0, 2 * sizeof(unsigned));
    if (e == cudaSuccess) {
        k_wait_flag<<<1, 32>>>(buf, spin_limit_cycles, buf + 1);
        e = cudaGetLastError();
    }
    unsigned st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, buf + 1, sizeof st, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "rfa_selftest_wait_timeout");
    if (st & kStatusTimeout) {
        set_error("device-side wait gave up after its limit (self-test)");
        return RFA_E_TIMEOUT;
    }
    return RFA_OK;
}

extern "C" rfa_status rfa_set_wait_limits(long long mbarrier_cycles, long long grid_barrier_cycles)
{
    if (mbarrier_cycles < 1 || mbarrier_cycles > (1ll << 32) || grid_barrier_cycles < 1 ||
        grid_barrier_cycles > (1ll << 32)) {
        set_error("wait limits must be in 1..2^32 cycles");
        return RFA_E_INVALID;
    }
    RFA_CUDA(tb_set_wait_limits(mbarrier_cycles, grid_barrier_cycles));
    return RFA_OK;
}
