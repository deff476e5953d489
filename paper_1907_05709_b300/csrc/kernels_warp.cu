// kernels_warp.cu -- the breathing-motion resampling of the temperature field
// (Sec. "Consideration of Breathing Motion", Eq. breathing): the simulation
// runs in the reference space X, and the temperature shown in the moving space
// x at time t is T(x) = T_ref(x + u_inv(x, t)), with u_inv the inverse motion
// vector field.  T_ref is sampled by trilinear interpolation of the voxel
// values; sample positions are clamped to the grid (the nearest face value
// outside it).
//
// Precision: the fractional sample offset is formed from the displacement in
// voxels alone (x + d with x integer: floor(x + d) = x + floor(d)), so FP32
// keeps it to a few 1e-7 of the displacement.  Compensated states interpolate hi and lo
// separately in FP32 and add them in FP64 for an FP64 output; an FP32 output
// interpolates hi alone (|lo| <= ulp(hi)/2 is below its resolution).  FP64
// states interpolate in FP64.
#include "rfa_internal.cuh"

namespace rfa {
namespace {

template <class R>
struct Axis {
    int i0, i1;
    R f;
};

// sample coordinate c + d (c integer voxel index, d displacement in voxels),
// clamped to [0, n-1]: i = c + floor(d); below 0 -> voxel 0, at or past n-1 ->
// voxel n-1, else between i and i+1 with weight f = d - floor(d)
template <class R>
__device__ __forceinline__ Axis<R> axis_sample(int c, R d, int n)
{
    Axis<R> a;
    d = fmin(fmax(d, -(R)(n + 1)), (R)(n + 1));  // also maps NaN to the low face
    const R fl = floor(d);
    const int i = c + (int)fl;  // |fl| <= n + 1: no overflow
    if (i < 0) {
        a.i0 = a.i1 = 0;
        a.f = R(0);
    } else if (i >= n - 1) {
        a.i0 = a.i1 = n - 1;
        a.f = R(0);
    } else {
        a.i0 = i;
        a.i1 = i + 1;
        a.f = d - fl;
    }
    return a;
}

template <class R>
__device__ __forceinline__ R lerp_(R a, R b, R f)
{
    return a + f * (b - a);
}

// the 8 corners from one base pointer and the three axis steps (0 where an
// axis is clamped)
template <class R>
__device__ __forceinline__ R trilinear_at(const R *p, int dx, size_t dy, size_t dz, R fx, R fy, R fz)
{
    const R c00 = lerp_(__ldg(p), __ldg(p + dx), fx);
    const R c10 = lerp_(__ldg(p + dy), __ldg(p + dy + dx), fx);
    const R c01 = lerp_(__ldg(p + dz), __ldg(p + dz + dx), fx);
    const R c11 = lerp_(__ldg(p + dz + dy), __ldg(p + dz + dy + dx), fx);
    return lerp_(lerp_(c00, c10, fy), lerp_(c01, c11, fy), fz);
}

template <class R, class Load>
__device__ __forceinline__ R trilinear(const Axis<R> &ax, const Axis<R> &ay, const Axis<R> &az, const Load &v)
{
    const R c00 = lerp_(v(ax.i0, ay.i0, az.i0), v(ax.i1, ay.i0, az.i0), ax.f);
    const R c10 = lerp_(v(ax.i0, ay.i1, az.i0), v(ax.i1, ay.i1, az.i0), ax.f);
    const R c01 = lerp_(v(ax.i0, ay.i0, az.i1), v(ax.i1, ay.i0, az.i1), ax.f);
    const R c11 = lerp_(v(ax.i0, ay.i1, az.i1), v(ax.i1, ay.i1, az.i1), ax.f);
    return lerp_(lerp_(c00, c10, ay.f), lerp_(c01, c11, ay.f), az.f);
}

// a thread per output voxel: x across the 32 lanes, y across the block's 8
// rows, z across the grid (looping past 65535 planes); u is [3][nz][ny][nx]
template <int SP>
__global__ void __launch_bounds__(256) k_warp(const void *th, const float *lo, const float *u, int nx, int ny,
                                              int nz, int pitch, size_t plane, double h, double T_a, float rh,
                                              float T_af, void *dst, int as_f64)
{
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const size_t n = (size_t)nx * ny * nz;
    for (int z = blockIdx.z; z < nz; z += gridDim.z) {
        const size_t j = ((size_t)z * ny + y) * nx + x;
        if (SP == RFA_STATE_F64) {
            const Axis<double> ax = axis_sample<double>(x, (double)u[j] / h, nx);
            const Axis<double> ay = axis_sample<double>(y, (double)u[j + n] / h, ny);
            const Axis<double> az = axis_sample<double>(z, (double)u[j + 2 * n] / h, nz);
            const double *t = (const double *)th;
            const double T = trilinear<double>(ax, ay, az, [&](int i, int k, int l) {
                                 return t[(size_t)l * plane + (size_t)k * pitch + i];
                             }) + T_a;
            if (as_f64) ((double *)dst)[j] = T;
            else ((float *)dst)[j] = (float)T;
        } else {
            // displacement in voxels: u * rh with rh = 1/h rounded to FP32 on the
            // host (within 2 ulp of u/h: ~2e-7 relative)
            const Axis<float> ax = axis_sample<float>(x, __fmul_rn(__ldg(u + j), rh), nx);
            const Axis<float> ay = axis_sample<float>(y, __fmul_rn(__ldg(u + j + n), rh), ny);
            const Axis<float> az = axis_sample<float>(z, __fmul_rn(__ldg(u + j + 2 * n), rh), nz);
            const size_t o = (size_t)az.i0 * plane + (size_t)ay.i0 * pitch + ax.i0;
            const int dx = ax.i1 - ax.i0;
            const size_t dy = (size_t)(ay.i1 - ay.i0) * pitch, dz = (size_t)(az.i1 - az.i0) * plane;
            const float vh = trilinear_at<float>((const float *)th + o, dx, dy, dz, ax.f, ay.f, az.f);
            // the lo part of a compensated state is at most half an ulp of hi, below
            // the resolution of an FP32 temperature (theta >= 0 near the needle, so
            // ulp(hi) <= ulp(T)): only a double output interpolates it
            float vl = 0.f;
            if (SP == RFA_STATE_F32C && as_f64) vl = trilinear_at<float>(lo + o, dx, dy, dz, ax.f, ay.f, az.f);
            if (as_f64) ((double *)dst)[j] = ((double)vh + (double)vl) + T_a;
            else ((float *)dst)[j] = __fadd_rn(__fadd_rn(vh, vl), T_af);
        }
    }
}

}  // namespace
}  // namespace rfa

using namespace rfa;

extern "C" rfa_status rfa_warp_temperature(rfa_grid *g, const float *u_inv_dev, void *dst_dev, int as_f64)
{
    if (!g || !u_inv_dev || !dst_dev) {
        set_error("null argument");
        return RFA_E_INVALID;
    }
    if (!g->have_tissue) {
        set_error("rfa_set_tissue must come first");
        return RFA_E_STATE;
    }
    const void *th = g->th[g->cur];
    const float *lo = (const float *)g->lo[g->cur];
    const float rh = (float)(1.0 / g->h), T_af = (float)g->T_a;
    const dim3 blk(32, 8), grd((g->nx + 31) / 32, (g->ny + 7) / 8, g->nz < 65535 ? g->nz : 65535);
    if (g->sp == RFA_STATE_F64)
        k_warp<RFA_STATE_F64><<<grd, blk, 0, g->stream>>>(th, lo, u_inv_dev, g->nx, g->ny, g->nz, g->pitch, g->plane,
                                                         g->h, g->T_a, rh, T_af, dst_dev, as_f64);
    else if (g->sp == RFA_STATE_F32C)
        k_warp<RFA_STATE_F32C><<<grd, blk, 0, g->stream>>>(th, lo, u_inv_dev, g->nx, g->ny, g->nz, g->pitch, g->plane,
                                                          g->h, g->T_a, rh, T_af, dst_dev, as_f64);
    else
        k_warp<RFA_STATE_F32><<<grd, blk, 0, g->stream>>>(th, lo, u_inv_dev, g->nx, g->ny, g->nz, g->pitch, g->plane,
                                                         g->h, g->T_a, rh, T_af, dst_dev, as_f64);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rfa_warp_temperature launch");
    return RFA_OK;
}
