// noalloc.cu -- necrosis counts and smoothed volume through an entry point that
// allocates no memory at all.
//
// Who needs it: callers that must not allocate device memory while they run --
// a real-time loop (for example a VR renderer stepping the ablation every
// frame) where a cudaMalloc/cudaFree would synchronise the device and stall
// the frame, or a host application that pre-reserves its whole device memory
// budget and forbids any later allocation.  This entry point calls no allocator
// and, unlike rfa_necrosis_mask, neither copies to the host nor synchronises;
// its only scratch is the fixed array below.
//
// How: the per-block partial sums of the two-pass reduction live in one
// file-scope device array of fixed size (kNoAllocRecords records of 32 bytes,
// 512 KiB), which every GPU that loads the library holds until the process
// exits.  Host code must not use the array's name as a device pointer; its
// device address is looked up once per device with cudaGetSymbolAddress, on
// the first call made with that device current.
//
// Limits: one record (and one block) per 16384 padded voxels, so grids of
// more than kNoAllocRecords * 16384 padded voxels (268,435,456; e.g. 640^3)
// are rejected.  Records of 16384 voxels give a 256^3 grid 1024 blocks, about
// seven per SM, so the streaming loads have enough warps in flight.
// Every call shares the array: each call overwrites all the records it later
// reads, so nothing has to be cleared, but calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the records.
#include "rfa_internal.cuh"
#include "necrosis.cuh"

#include <cstdint>
#include <mutex>

namespace rfa {

namespace {

constexpr int kNoAllocRecords = 16384;
constexpr size_t kNoAllocVoxelsPerRecord = 16384;

struct NaRecord {
    unsigned long long n_thermal, n_arrh;
    double smooth;
    double pad;
};

// block of 256 threads: warp trees, then the 8 warp sums in order (fixed order)
template <typename T>
__device__ __forceinline__ T na_block_sum(T v)
{
    __shared__ T sh[8];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = T(0);
    for (int k = 0; k < 8; ++k) t += sh[k];
    return t;
}

static __device__ __align__(256) NaRecord g_noalloc_scratch[kNoAllocRecords];

std::mutex g_na_mu;
void *g_na_ptr[64] = {};  // device address of the scratch array, per device ordinal

// per-record partials over padded voxels [16384 r, 16384 (r + 1)): thermal
// latch, Arrhenius (Omega + carry >= 1), smoothed sigmoid sum, in the quads of
// rfa_necrosis_mask (4 x voxels from a multiple of 4: the same FP32 quad sums;
// records start at multiples of 4 and the padded pitch is one).  The grid
// limit keeps every padded index below 2^32.
template <int SP>
__global__ void __launch_bounds__(256) k_na_partials(const void *th, const float *lo,
                                                     const uint8_t *latch, const double *omega,
                                                     const float *carry, int nx, int ny, int nz,
                                                     int pitch, double off, double inv_width,
                                                     NaRecord *rec, unsigned *status)
{
    const unsigned nvp = (unsigned)((size_t)pitch * ny * nz);
    const unsigned begin = blockIdx.x * (unsigned)kNoAllocVoxelsPerRecord;
    const unsigned end = nvp - begin > (unsigned)kNoAllocVoxelsPerRecord ? begin + (unsigned)kNoAllocVoxelsPerRecord : nvp;
    const float offf = (float)off, iwf = (float)inv_width;
    unsigned n0 = 0, n1 = 0;
    double sm = 0.0;
    for (unsigned i = begin + 4u * threadIdx.x; i < end; i += 4u * blockDim.x) {
        const int x0 = (int)(i % (unsigned)pitch);
        if (x0 >= nx) continue;
        const int nin = nx - x0 < 4 ? nx - x0 : 4;
        uint8_t m[4];
        if (!RFA_CHECK_RANGE(i, (size_t)i + 4, nvp, i, 4, status)) continue;
        necro_quad<SP>(th, lo, latch, omega, carry, i, nin, off, inv_width, offf, iwf, n0, n1, sm, m);
    }
    const unsigned long long c0 = na_block_sum((unsigned long long)n0), c1 = na_block_sum((unsigned long long)n1);
    const double s = na_block_sum(sm);
    if (threadIdx.x == 0) rec[blockIdx.x] = NaRecord{c0, c1, s, 0.0};
}

// sum the records in a fixed order on one block of 256 threads;
// out = {count_thermal, count_arrhenius, smooth_volume_m3, 0}
__global__ void __launch_bounds__(256) k_na_final(const NaRecord *rec, int n, double h3, void *out)
{
    unsigned long long c0 = 0, c1 = 0;
    double sm = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        c0 += rec[k].n_thermal;
        c1 += rec[k].n_arrh;
        sm += rec[k].smooth;
    }
    c0 = na_block_sum(c0);
    c1 = na_block_sum(c1);
    sm = na_block_sum(sm);
    if (threadIdx.x == 0) {
        int64_t *o = (int64_t *)out;
        o[0] = (int64_t)c0;
        o[1] = (int64_t)c1;
        ((double *)out)[2] = h3 * sm;
        ((double *)out)[3] = 0.0;
    }
}

}  // namespace

}  // namespace rfa

using namespace rfa;

extern "C" rfa_status rfa_necrosis_reduce_noalloc(rfa_grid *g, double smooth_width_K, void *result_dev)
{
    if (!g || !result_dev) {
        set_error("null argument");
        return RFA_E_INVALID;
    }
    if (!(smooth_width_K > 0.0)) {
        set_error("smooth_width_K must be > 0");
        return RFA_E_INVALID;
    }
    if (((uintptr_t)result_dev & 7u) != 0) {  // the kernel stores int64 and double words
        set_error("result_dev must be 8-byte aligned");
        return RFA_E_INVALID;
    }
    const size_t nrec = (g->nvp + kNoAllocVoxelsPerRecord - 1) / kNoAllocVoxelsPerRecord;
    if (nrec > (size_t)kNoAllocRecords) {
        set_error("grid too large for rfa_necrosis_reduce_noalloc: at most 268435456 padded voxels "
                  "(16384 scratch records of 16384 voxels)");
        return RFA_E_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal out of range");
        return RFA_E_INVALID;
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            // first call on this device: look up the device address of the scratch array
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
            g_na_ptr[dev] = p;
        }
        scratch = g_na_ptr[dev];
    }
    NaRecord *rec = (NaRecord *)scratch;
    const void *th = g->th[g->cur];
    const float *lo = (const float *)g->lo[g->cur];
    const double off = g->T_thr - g->T_a, iw = 1.0 / smooth_width_K;
    const unsigned nb = (unsigned)nrec;
    if (g->sp == RFA_STATE_F64)
        k_na_partials<RFA_STATE_F64><<<nb, 256, 0, g->stream>>>(th, lo, g->latch, g->omega, g->omega_c, g->nx,
                                                                g->ny, g->nz, g->pitch, off, iw, rec, g->status);
    else if (g->sp == RFA_STATE_F32C)
        k_na_partials<RFA_STATE_F32C><<<nb, 256, 0, g->stream>>>(th, lo, g->latch, g->omega, g->omega_c, g->nx,
                                                                 g->ny, g->nz, g->pitch, off, iw, rec, g->status);
    else
        k_na_partials<RFA_STATE_F32><<<nb, 256, 0, g->stream>>>(th, lo, g->latch, g->omega, g->omega_c, g->nx,
                                                                g->ny, g->nz, g->pitch, off, iw, rec, g->status);
    k_na_final<<<1, 256, 0, g->stream>>>(rec, (int)nrec, g->h * g->h * g->h, result_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rfa_necrosis_reduce_noalloc launch");
    return RFA_OK;
}
