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
__device__ __forceinline__ void cupdate(float c, float cl, float S, float a, float b, float s,
                                        float &nh, float &nl)
{
    float th = __fadd_rn(c, cl);
    float delta = __fmaf_rn(a, S, __fmaf_rn(-b, th, s));
    float s1 = __fadd_rn(c, delta);
    float bb = __fsub_rn(s1, c);
    float e1 = __fadd_rn(__fsub_rn(c, __fsub_rn(s1, bb)), __fsub_rn(delta, bb));
    float l1 = __fadd_rn(cl, e1);
    float s2 = __fadd_rn(s1, l1);
    nl = __fsub_rn(l1, __fsub_rn(s2, s1));
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
__device__ __forceinline__ float arrhenius_inc(float theta, float c0, float c1, float TK0)
{
    float tk = __fadd_rn(theta, TK0);
    return exp2f(__fsub_rn(c0, __fdiv_rn(c1, tk)));
}

// Kahan step of the FP64 damage integral with an FP32-stored compensation
__device__ __forceinline__ void kahan_add(double &om, float &ck, double inc)
{
    double yk = __dsub_rn(inc, (double)ck);
    double tk = __dadd_rn(om, yk);
    ck = (float)__dsub_rn(__dsub_rn(tk, om), yk);
    om = tk;
}

}  // namespace rfa
