// kernels_reduce.cu -- necrosis mask and volumes, and conversions of the
// padded device state to dense host-layout arrays.
//
// Necrosis (Sec. "Introduction": instantaneous death above 60 C; Eq.
// eq-tissState for the Arrhenius criterion Omega >= 1) is reduced in two
// passes: a fixed grid of kReduceBlocks blocks writes per-block partials
// (warp shuffles, then shared memory), and one block sums the partials in a
// fixed order, so the counts and the FP64 smoothed volume are bit-reproducible.
#include "rfa_internal.cuh"
#include "necrosis.cuh"

namespace rfa {

namespace {

struct NecroPartial {
    unsigned long long n_thermal, n_arrh;
    double smooth;
    double pad;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T block_sum256(T v)
{
    // fixed order: warp tree, then the 8 warp sums in order
    __shared__ T sh[8];
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = T(0);
    for (int k = 0; k < 8; ++k) t += sh[k];
    return t;
}

// a warp per grid row, lanes along x in quads
template <int SP>
__global__ void __launch_bounds__(256) k_necrosis(const void *th, const float *lo,
                                                  const uint8_t *latch, const double *omega,
                                                  const float *carry,
                                                  int nx, int ny, int nz, int pitch, double T_a,
                                                  double T_thr, double inv_width,
                                                  uint8_t *mask_dense, NecroPartial *part, unsigned *status)
{
    const size_t nvp = (size_t)pitch * ny * nz;
    unsigned n0 = 0, n1 = 0;
    double sm = 0.0;
    const double off = T_thr - T_a;
    const float offf = (float)off, iwf = (float)inv_width;
    for (int row = blockIdx.x * 8 + (int)(threadIdx.x >> 5); row < ny * nz; row += gridDim.x * 8) {
        const size_t rb = (size_t)row * pitch;
        for (int x0 = 4 * (int)(threadIdx.x & 31); x0 < nx; x0 += 128) {
            const int nin = nx - x0 < 4 ? nx - x0 : 4;
            uint8_t m[4];
            if (!RFA_CHECK_RANGE(rb + x0, rb + x0 + 4, nvp, rb + x0, 4, status)) continue;
            necro_quad<SP>(th, lo, latch, omega, carry, rb + x0, nin, off, inv_width, offf, iwf, n0, n1, sm, m);
            if (mask_dense)
                for (int q = 0; q < nin; ++q) mask_dense[(size_t)row * nx + x0 + q] = m[q];
        }
    }
    const unsigned long long c0 = block_sum256((unsigned long long)n0), c1 = block_sum256((unsigned long long)n1);
    const double s = block_sum256(sm);
    if (threadIdx.x == 0) part[blockIdx.x] = NecroPartial{c0, c1, s, 0.0};
}

// the partials in a fixed order on one block of 256 threads
__global__ void __launch_bounds__(256) k_necrosis_final(const NecroPartial *part, int n, NecroPartial *out)
{
    unsigned long long a = 0, b = 0;
    double c = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        a += part[k].n_thermal;
        b += part[k].n_arrh;
        c += part[k].smooth;
    }
    a = block_sum256(a);
    b = block_sum256(b);
    c = block_sum256(c);
    if (threadIdx.x == 0) *out = NecroPartial{a, b, c, 0.0};
}

template <int SP>
__global__ void k_to_temperature(const void *th, const float *lo, int nx, int ny, int nz,
                                 int pitch, double T_a, void *dst, int as_f64)
{
    size_t n = (size_t)nx * ny * nz;
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n;
         j += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(j % nx);
        size_t r = j / nx;
        size_t i = r * pitch + x;
        double v;
        if (SP == RFA_STATE_F64) v = ((const double *)th)[i];
        else v = (double)((const float *)th)[i] + (SP == RFA_STATE_F32C ? (double)lo[i] : 0.0);
        v += T_a;
        if (as_f64) ((double *)dst)[j] = v;
        else ((float *)dst)[j] = (float)v;
    }
}

struct FieldView {
    int nx, ny, nz, pitch, sp, pp;
    const void *ab, *s;
    const uint8_t *latch;
    const double *omega;
    const float *carry;
};

__global__ void k_get_field(const FieldView G, const void *th, const float *lo, int field,
                            double *dst)
{
    size_t n = (size_t)G.nx * G.ny * G.nz;
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n;
         j += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(j % G.nx);
        size_t r = j / G.nx;
        size_t i = r * G.pitch + x;
        double v = 0.0;
        switch (field) {
        case RFA_FIELD_THETA:
            if (G.sp == RFA_STATE_F64) v = ((const double *)th)[i];
            else v = (double)((const float *)th)[i] + (G.sp == RFA_STATE_F32C ? (double)lo[i] : 0.0);
            break;
        case RFA_FIELD_THETA_LO:
            v = G.sp == RFA_STATE_F32C ? (double)lo[i] : 0.0;
            break;
        case RFA_FIELD_A:
        case RFA_FIELD_B: {
            int k = field == RFA_FIELD_A ? 0 : 1;
            if (G.pp == RFA_PARAM_BF16) {
                uint32_t u = ((const uint32_t *)G.ab)[i];
                v = bf16_to_float(k == 0 ? (u & 0xffffu) : (u >> 16));
            } else if (G.pp == RFA_PARAM_F32) {
                float2 t = ((const float2 *)G.ab)[i];
                v = k == 0 ? t.x : t.y;
            } else {
                double2 t = ((const double2 *)G.ab)[i];
                v = k == 0 ? t.x : t.y;
            }
            break;
        }
        case RFA_FIELD_S:
            v = G.sp == RFA_STATE_F64 ? ((const double *)G.s)[i] : (double)((const float *)G.s)[i];
            break;
        case RFA_FIELD_LATCH:
            v = G.latch[i];
            break;
        case RFA_FIELD_OMEGA:
            v = G.omega[i] + (double)G.carry[i];  // FP64 integral plus its FP32 carry
            break;
        default:
            break;
        }
        dst[j] = v;
    }
}

}  // namespace

cudaError_t launch_necrosis(rfa_grid *g, uint8_t *mask_dense_dev, double width_K, void *result_dev)
{
    NecroPartial *part = (NecroPartial *)g->red;
    const void *th = g->th[g->cur];
    const float *lo = (const float *)g->lo[g->cur];
    double iw = 1.0 / width_K;
    if (g->sp == RFA_STATE_F64)
        k_necrosis<RFA_STATE_F64><<<kReduceBlocks, 256, 0, g->stream>>>(
            th, lo, g->latch, g->omega, g->omega_c, g->nx, g->ny, g->nz, g->pitch, g->T_a, g->T_thr, iw,
            mask_dense_dev, part, g->status);
    else if (g->sp == RFA_STATE_F32C)
        k_necrosis<RFA_STATE_F32C><<<kReduceBlocks, 256, 0, g->stream>>>(
            th, lo, g->latch, g->omega, g->omega_c, g->nx, g->ny, g->nz, g->pitch, g->T_a, g->T_thr, iw,
            mask_dense_dev, part, g->status);
    else
        k_necrosis<RFA_STATE_F32><<<kReduceBlocks, 256, 0, g->stream>>>(
            th, lo, g->latch, g->omega, g->omega_c, g->nx, g->ny, g->nz, g->pitch, g->T_a, g->T_thr, iw,
            mask_dense_dev, part, g->status);
    k_necrosis_final<<<1, 256, 0, g->stream>>>(part, kReduceBlocks, (NecroPartial *)result_dev);
    return cudaGetLastError();
}

cudaError_t launch_to_temperature(rfa_grid *g, void *dst, int as_f64)
{
    const void *th = g->th[g->cur];
    const float *lo = (const float *)g->lo[g->cur];
    if (g->sp == RFA_STATE_F64)
        k_to_temperature<RFA_STATE_F64><<<148 * 8, 256, 0, g->stream>>>(th, lo, g->nx, g->ny, g->nz, g->pitch, g->T_a, dst, as_f64);
    else if (g->sp == RFA_STATE_F32C)
        k_to_temperature<RFA_STATE_F32C><<<148 * 8, 256, 0, g->stream>>>(th, lo, g->nx, g->ny, g->nz, g->pitch, g->T_a, dst, as_f64);
    else
        k_to_temperature<RFA_STATE_F32><<<148 * 8, 256, 0, g->stream>>>(th, lo, g->nx, g->ny, g->nz, g->pitch, g->T_a, dst, as_f64);
    return cudaGetLastError();
}

cudaError_t launch_get_field(rfa_grid *g, int field, double *dst)
{
    FieldView G{g->nx, g->ny, g->nz, g->pitch, g->sp, g->pp, g->ab, g->s, g->latch, g->omega, g->omega_c};
    k_get_field<<<148 * 8, 256, 0, g->stream>>>(G, g->th[g->cur], (const float *)g->lo[g->cur],
                                                field, dst);
    return cudaGetLastError();
}

}  // namespace rfa
