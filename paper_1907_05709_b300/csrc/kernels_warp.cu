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

#include <algorithm>
#include <climits>

namespace rfa {
namespace {

// sample coordinate c + d (c integer voxel index, d displacement in voxels),
// clamped to [0, n-1], without branches: i = c + floor(d); below 0 -> voxel 0,
// at or past n-1 -> voxel n-1 (both: one voxel, step 0, weight 0), else
// between i and i + 1 (step 1) with weight f = d - floor(d)
template <class R>
struct AxisS {
    int i0, step;
    R f;
};
__device__ __forceinline__ AxisS<float> axis_sample_f(int c, float d, int n, float lo, float hi)
{
    d = fminf(fmaxf(d, lo), hi);  // lo = -(n+1), hi = n+1; also maps NaN to the low face
    const float fl = floorf(d);
    const int i = c + (int)fl;    // |fl| <= n + 1: no overflow
    const bool in = i >= 0 && i < n - 1;
    return {min(max(i, 0), n - 1), in ? 1 : 0, in ? d - fl : 0.f};
}
__device__ __forceinline__ AxisS<double> axis_sample_d(int c, double d, int n)
{
    d = fmin(fmax(d, -(double)(n + 1)), (double)(n + 1));
    const double fl = floor(d);
    const int i = c + (int)fl;
    const bool in = i >= 0 && i < n - 1;
    return {min(max(i, 0), n - 1), in ? 1 : 0, in ? d - fl : 0.0};
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

// a thread per output voxel and plane: x across the 32 lanes, y across the
// block's 8 rows, z across the grid (planes z, z + gridDim.z, ...); u is
// [3][nz][ny][nx].  The FP32 path loads the displacement of its next plane
// before it gathers the current one, so the DRAM latency of u overlaps the
// corner loads.  I: the index type of the FP32 path (int where every index
// fits, which saves the 64-bit address arithmetic)
template <int SP, class I>
__global__ void __launch_bounds__(256) k_warp(const void *th, const float *lo, const float *u, int nx, int ny,
                                              int nz, int pitch, size_t plane, double rhd, double T_a, float rh,
                                              float T_af, void *dst, int as_f64)
{
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const I n = (I)nx * ny * nz;
    if constexpr (SP == RFA_STATE_F64) {
        for (int z = blockIdx.z; z < nz; z += gridDim.z) {
            const I j = ((I)z * ny + y) * nx + x;
            // displacement in voxels: u times 1/h in FP64 (within an ulp of u/h)
            const AxisS<double> ax = axis_sample_d(x, (double)__ldg(u + j) * rhd, nx);
            const AxisS<double> ay = axis_sample_d(y, (double)__ldg(u + j + n) * rhd, ny);
            const AxisS<double> az = axis_sample_d(z, (double)__ldg(u + j + 2 * n) * rhd, nz);
            const size_t o = (size_t)az.i0 * plane + (size_t)ay.i0 * (size_t)pitch + ax.i0;
            const size_t dx = ax.step, dy = ay.step ? (size_t)pitch : 0, dz = az.step ? plane : 0;
            const double T = trilinear_at<double, size_t>((const double *)th, o, dx, dy, dz, ax.f, ay.f, az.f) + T_a;
            if (as_f64) ((double *)dst)[j] = T;
            else ((float *)dst)[j] = (float)T;
        }
    } else {
        const float lx = -(float)(nx + 1), hx = (float)(nx + 1), ly = -(float)(ny + 1), hy = (float)(ny + 1);
        const float lz = -(float)(nz + 1), hz = (float)(nz + 1);
        const I pstep = (I)gridDim.z * ny * nx;  // index step between this thread's planes
        int z = blockIdx.z;
        if (z >= nz) return;
        I j = ((I)z * ny + y) * nx + x;
        float u0 = __ldg(u + j), u1 = __ldg(u + j + n), u2 = __ldg(u + j + 2 * n);
        for (;;) {
            const int zn = z + gridDim.z;
            const bool more = zn < nz;
            const I jn = j + pstep;
            float v0 = 0.f, v1 = 0.f, v2 = 0.f;
            if (more) {
                v0 = __ldg(u + jn);
                v1 = __ldg(u + jn + n);
                v2 = __ldg(u + jn + 2 * n);
            }
            // displacement in voxels: u * rh with rh = 1/h rounded to FP32 on the
            // host (within 2 ulp of u/h: ~2e-7 relative)
            const AxisS<float> ax = axis_sample_f(x, __fmul_rn(u0, rh), nx, lx, hx);
            const AxisS<float> ay = axis_sample_f(y, __fmul_rn(u1, rh), ny, ly, hy);
            const AxisS<float> az = axis_sample_f(z, __fmul_rn(u2, rh), nz, lz, hz);
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
            if (!more) break;
            z = zn;
            j = jn;
            u0 = v0;
            u1 = v1;
            u2 = v2;
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
    const double rhd = 1.0 / g->h;
    const float rh = (float)rhd, T_af = (float)g->T_a;
    // planes per thread: about four where the grid still has four waves of
    // blocks at 8 blocks per SM (the FP32 path prefetches the next plane's u)
    const int bxy = ((g->nx + 31) / 32) * ((g->ny + 7) / 8);
    const int waves4 = 4 * 8 * 148;
    int gz = (g->nz + 3) / 4;
    if ((long long)gz * bxy < waves4) gz = (int)std::min<long long>(g->nz, (waves4 + bxy - 1) / bxy);
    if (g->sp == RFA_STATE_F64) gz = g->nz;
    gz = std::min(gz, 65535);
    const dim3 blk(32, 8), grd((g->nx + 31) / 32, (g->ny + 7) / 8, gz);
    // 32-bit indices where u (3 nx ny nz values) and the padded state fit
    const size_t nvox = (size_t)g->nx * g->ny * g->nz;
    const bool idx32 = 3 * nvox <= (size_t)INT_MAX && g->nvp <= (size_t)INT_MAX;
#define WARP_ARGS                                                                                                  \
    th, lo, u_inv_dev, g->nx, g->ny, g->nz, g->pitch, g->plane, rhd, g->T_a, rh, T_af, dst_dev, as_f64
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
