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

#include <climits>

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

// the same sample for FP32, without branches: a clamped axis samples one voxel
// (step 0) with weight 0, exactly as above (i1 = i0, f = 0)
struct AxisF {
    int i0, step;
    float f;
};
__device__ __forceinline__ AxisF axis_sample_f(int c, float d, int n, float lo, float hi)
{
    d = fminf(fmaxf(d, lo), hi);  // lo = -(n+1), hi = n+1; also maps NaN to the low face
    const float fl = floorf(d);
    const int i = c + (int)fl;
    const bool in = i >= 0 && i < n - 1;
    return {min(max(i, 0), n - 1), in ? 1 : 0, in ? d - fl : 0.f};
}

template <class R>
__device__ __forceinline__ R lerp_(R a, R b, R f)
{
    return a + f * (b - a);
}

// the 8 corners at offsets o (+ dx, dy, dz: the axis steps, 0 where an axis is
// clamped) from a base pointer, in the index type I
template <class R, class I>
__device__ __forceinline__ R trilinear_at(const R *p, I o, I dx, I dy, I dz, R fx, R fy, R fz)
{
    const R c00 = lerp_(__ldg(p + o), __ldg(p + o + dx), fx);
    const R c10 = lerp_(__ldg(p + o + dy), __ldg(p + o + dy + dx), fx);
    const R c01 = lerp_(__ldg(p + o + dz), __ldg(p + o + dz + dx), fx);
    const R c11 = lerp_(__ldg(p + o + dz + dy), __ldg(p + o + dz + dy + dx), fx);
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
// rows, z across the grid (looping past 65535 planes); u is [3][nz][ny][nx].
// I: the index type of the FP32 path (int where every index fits, which
// saves the 64-bit address arithmetic)
template <int SP, class I>
__global__ void __launch_bounds__(256) k_warp(const void *th, const float *lo, const float *u, int nx, int ny,
                                              int nz, int pitch, size_t plane, double h, double T_a, float rh,
                                              float T_af, void *dst, int as_f64)
{
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const I n = (I)nx * ny * nz;
    const float lx = -(float)(nx + 1), hx = (float)(nx + 1), ly = -(float)(ny + 1), hy = (float)(ny + 1);
    const float lz = -(float)(nz + 1), hz = (float)(nz + 1);
    for (int z = blockIdx.z; z < nz; z += gridDim.z) {
        const I j = ((I)z * ny + y) * nx + x;
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
            const AxisF ax = axis_sample_f(x, __fmul_rn(__ldg(u + j), rh), nx, lx, hx);
            const AxisF ay = axis_sample_f(y, __fmul_rn(__ldg(u + j + n), rh), ny, ly, hy);
            const AxisF az = axis_sample_f(z, __fmul_rn(__ldg(u + j + 2 * n), rh), nz, lz, hz);
            const I o = (I)az.i0 * (I)plane + (I)ay.i0 * (I)pitch + ax.i0;
            const I dx = ax.step, dy = ay.step ? (I)pitch : I(0), dz = az.step ? (I)plane : I(0);
            const float vh = trilinear_at<float, I>((const float *)th, o, dx, dy, dz, ax.f, ay.f, az.f);
            // the lo part of a compensated state is at most half an ulp of hi, below
            // the resolution of an FP32 temperature (theta >= 0 near the needle, so
            // ulp(hi) <= ulp(T)): only a double output interpolates it
            float vl = 0.f;
            if (SP == RFA_STATE_F32C && as_f64) vl = trilinear_at<float, I>(lo, o, dx, dy, dz, ax.f, ay.f, az.f);
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
    // 32-bit indices where u (3 nx ny nz values) and the padded state fit
    const size_t nvox = (size_t)g->nx * g->ny * g->nz;
    const bool idx32 = 3 * nvox <= (size_t)INT_MAX && g->nvp <= (size_t)INT_MAX;
#define WARP_ARGS                                                                                                  \
    th, lo, u_inv_dev, g->nx, g->ny, g->nz, g->pitch, g->plane, g->h, g->T_a, rh, T_af, dst_dev, as_f64
    if (g->sp == RFA_STATE_F64) k_warp<RFA_STATE_F64, size_t><<<grd, blk, 0, g->stream>>>(WARP_ARGS);
    else if (g->sp == RFA_STATE_F32C && idx32) k_warp<RFA_STATE_F32C, int><<<grd, blk, 0, g->stream>>>(WARP_ARGS);
    else if (g->sp == RFA_STATE_F32C) k_warp<RFA_STATE_F32C, size_t><<<grd, blk, 0, g->stream>>>(WARP_ARGS);
    else if (idx32) k_warp<RFA_STATE_F32, int><<<grd, blk, 0, g->stream>>>(WARP_ARGS);
    else k_warp<RFA_STATE_F32, size_t><<<grd, blk, 0, g->stream>>>(WARP_ARGS);
#undef WARP_ARGS
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rfa_warp_temperature launch");
    return RFA_OK;
}
