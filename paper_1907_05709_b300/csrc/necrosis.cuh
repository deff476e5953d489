// necrosis.cuh -- the per-quad necrosis evaluation shared by the necrosis
// reductions (rfa_necrosis_mask and the allocation-free entry point), so that
// both form the same FP32 quad sums of the smoothed volume.
#pragma once
#include "rfa_internal.cuh"

namespace rfa {

// Omega + carry >= 1 (the Arrhenius criterion on the FP64 integral plus its
// FP32 carry) without the FP64 sum where the answer is fixed: both below 0.5
// (the high word of Omega) gives an FP64 sum below 1, a finite Omega of at
// least 2 with a carry above -1 one above 1; NaN and the rest take the sum.
__device__ __forceinline__ bool arrhenius_dead(double om, float c)
{
    const int hi = __double2hiint(om);
    if (hi < 0x3FE00000 && c < 0.5f) return false;
    if (hi >= 0x40000000 && hi < 0x7FF00000 && c > -1.0f) return true;
    return om + (double)c >= 1.0;
}

// One quad of 4 x voxels at padded index i (a multiple of 4; nin of them
// inside the grid): mask bits (bit 0 thermal latch, bit 1 Arrhenius), their
// counts, and the sigmoid sigma((T - T_thr) / width) summed over the quad in
// the state's precision, in the fixed order ((s0 + s1) + s2) + s3 (0 for
// voxels outside the grid), added to sm in FP64.  off = T_thr - T_a and
// inv_width come in FP64 and, for FP32 states, in FP32 (offf, iwf).
template <int SP>
__device__ __forceinline__ void necro_quad(const void *th, const float *lo, const uint8_t *latch,
                                           const double *omega, const float *carry, size_t i, int nin,
                                           double off, double inv_width, float offf, float iwf,
                                           unsigned &n0, unsigned &n1, double &sm, uint8_t m[4])
{
    using T = typename std::conditional<SP == RFA_STATE_F64, double, float>::type;
    const uchar4 l4 = *reinterpret_cast<const uchar4 *>(latch + i);
    const double2 oa = reinterpret_cast<const double2 *>(omega + i)[0], ob = reinterpret_cast<const double2 *>(omega + i)[1];
    const float4 c4 = *reinterpret_cast<const float4 *>(carry + i);
    const uint8_t lv[4] = {l4.x, l4.y, l4.z, l4.w};
    const double ov[4] = {oa.x, oa.y, ob.x, ob.y};
    const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
    T v[4];
    if (SP == RFA_STATE_F64) {
        const double2 ta = reinterpret_cast<const double2 *>(th)[i / 2], tb = reinterpret_cast<const double2 *>(th)[i / 2 + 1];
        v[0] = (T)ta.x, v[1] = (T)ta.y, v[2] = (T)tb.x, v[3] = (T)tb.y;
    } else {
        const float4 h4 = reinterpret_cast<const float4 *>(th)[i / 4];
        v[0] = (T)h4.x, v[1] = (T)h4.y, v[2] = (T)h4.z, v[3] = (T)h4.w;
        if (SP == RFA_STATE_F32C) {
            const float4 q4 = reinterpret_cast<const float4 *>(lo)[i / 4];
            v[0] = (T)__fadd_rn((float)v[0], q4.x), v[1] = (T)__fadd_rn((float)v[1], q4.y);
            v[2] = (T)__fadd_rn((float)v[2], q4.z), v[3] = (T)__fadd_rn((float)v[3], q4.w);
        }
    }
    T qs = T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        m[q] = 0;
        if (q >= nin) continue;
        m[q] = (lv[q] ? 1 : 0) | (arrhenius_dead(ov[q], cv[q]) ? 2 : 0);
        n0 += m[q] & 1;
        n1 += m[q] >> 1;
        T sg;
        if (SP == RFA_STATE_F64) {
            const double u = ((double)v[q] - off) * inv_width;
            sg = (T)(1.0 / (1.0 + exp(-u)));
        } else {
            const float u = ((float)v[q] - offf) * iwf;
            sg = (T)(1.0f / (1.0f + __expf(-u)));
        }
        qs = qs + sg;
    }
    sm += (double)qs;
}

}  // namespace rfa
