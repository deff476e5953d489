// rfa_update.cuh -- the per-voxel update of Eq. CUDAbioheat3d, shared by every
// forward kernel so that the one-step, temporally blocked and batched kernels
// produce bit-identical states (the adjoint recomputes the trajectory with the
// one-step kernel).  Every operation uses an explicitly rounded intrinsic so
// the compiler cannot contract or reorder differently in different kernels.
//
// theta' = theta + a * S - b * theta + s,   S = sum over the six neighbours of
// (theta_nb - theta), accumulated in the fixed order x-, x+, y-, y+, z-, z+;
// a neighbour outside the grid contributes +0.
#pragma once

#include <cuda_runtime.h>

namespace rfa {

// ----------------------------------------------------------- compensated FP32
// neighbour difference of the pair (nh + nl) - (c + cl)
__device__ __forceinline__ float cdiff(float nh, float nl, float c, float cl)
{
    return __fadd_rn(__fsub_rn(nh, c), __fsub_rn(nl, cl));
}

// New pair from the old pair and the difference sum S.  The increment is added
// to hi error-free (TwoSum), its rounding error joins lo, and the pair is
// renormalised (Fast2Sum) so |lo| stays within half an ulp of hi.
// (hi, lo) + delta: TwoSum of hi and delta, the error joins lo, Fast2Sum renormalises
__device__ __forceinline__ void cadd(float c, float cl, float delta, float &nh, float &nl)
{
    float s1 = __fadd_rn(c, delta);
    float bb = __fsub_rn(s1, c);
    float e1 = __fadd_rn(__fsub_rn(c, __fsub_rn(s1, bb)), __fsub_rn(delta, bb));
    float l1 = __fadd_rn(cl, e1);
    float s2 = __fadd_rn(s1, l1);
    nl = __fsub_rn(l1, __fsub_rn(s2, s1));
    nh = s2;
}

__device__ __forceinline__ void cupdate(float c, float cl, float S, float a, float b, float s,
                                        float &nh, float &nl)
{
    float th = __fadd_rn(c, cl);
    float delta = __fmaf_rn(a, S, __fmaf_rn(-b, th, s));
    cadd(c, cl, delta, nh, nl);
}

// ------------------------------------------------- compensated FP32, voxel pairs
// The same operations on two voxels at once with the paired FP32 instructions
// of sm_100+ (each lane rounds exactly like the scalar intrinsic, so results are
// bit-identical to cdiff / cupdate).  x - y is formed as x + (-y), which IEEE
// round-to-nearest defines identically.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }

__device__ __forceinline__ float2 cdiff2(float2 nh, float2 nl, float2 c, float2 cl)
{
    return add2(sub2(nh, c), sub2(nl, cl));
}

// (th returns the old value c + cl rounded to FP32, the operand of -b theta)
__device__ __forceinline__ void cupdate2(float2 c, float2 cl, float2 S, float2 a, float2 b, float2 s,
                                         float2 &nh, float2 &nl, float2 &th)
{
    th = add2(c, cl);
    float2 delta = __ffma2_rn(a, S, __ffma2_rn(neg2(b), th, s));
    float2 s1 = add2(c, delta);
    float2 bb = sub2(s1, c);
    float2 e1 = add2(sub2(c, sub2(s1, bb)), sub2(delta, bb));
    float2 l1 = add2(cl, e1);
    float2 s2 = add2(s1, l1);
    nl = sub2(l1, sub2(s2, s1));
    nh = s2;
}

// ----------------------------------------------------------------- plain FP32
__device__ __forceinline__ float pdiff(float n, float c) { return __fsub_rn(n, c); }
__device__ __forceinline__ float pupdate(float c, float S, float a, float b, float s)
{
    return __fadd_rn(c, __fmaf_rn(a, S, __fmaf_rn(-b, c, s)));
}

// ----------------------------------------------------------------------- FP64
__device__ __forceinline__ double pdiff(double n, double c) { return __dsub_rn(n, c); }
__device__ __forceinline__ double pupdate(double c, double S, double a, double b, double s)
{
    return __dadd_rn(c, __fma_rn(a, S, __fma_rn(-b, c, s)));
}

__device__ __forceinline__ float acc(float x, float y) { return __fadd_rn(x, y); }
__device__ __forceinline__ double acc(double x, double y) { return __dadd_rn(x, y); }

// ------------------------------------------------------------------- damage
// Arrhenius increment dt A exp(-Ea / (R T_K)) = exp2(c0 - c1 / T_K) in FP32
// (c0 = log2(A dt), c1 = Ea / (R ln 2)), with the hardware reciprocal-based
// division and base-2 exponential (relative error ~1e-6, far inside the
// damage tolerance; the exponent is formed in ln space so A = 7.39e39 and
// exp(-100) stay inside FP32 range).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float arrhenius_inc(float theta, float c0, float c1, float TK0)
{
    float tk = __fadd_rn(theta, TK0);
    return ex2_approx(__fsub_rn(c0, __fmul_rn(c1, rcp_approx(tk))));
}
__device__ __forceinline__ float2 arrhenius_inc2(float2 theta, float c0, float c1, float TK0)
{
    float2 tk = add2(theta, make_float2(TK0, TK0));
    float2 x = __fmul2_rn(make_float2(c1, c1), make_float2(rcp_approx(tk.x), rcp_approx(tk.y)));
    float2 e = sub2(make_float2(c0, c0), x);
    return make_float2(ex2_approx(e.x), ex2_approx(e.y));
}

// The damage integral is Omega + P: Omega in FP64 and P an FP32 carry that
// holds the not-yet-folded increments plus the rounding error of the last
// fold.  Increments are added to P in FP32; every few launches the carry is
// folded into Omega with an error-free TwoSum in FP64 and P keeps the
// rounding error.  Readers use Omega + P.
__device__ __forceinline__ void carry_fold(double &om, float &P)
{
    const double p = (double)P;
    const double s = __dadd_rn(om, p);
    const double bb = __dsub_rn(s, om);
    const double err = __dadd_rn(__dsub_rn(om, __dsub_rn(s, bb)), __dsub_rn(p, bb));
    om = s;
    P = (float)err;
}

}  // namespace rfa
