// kernels_cond.cu -- conservative conduction, div(K grad T) of Eq.
// 2675-eq1_Kath with the face conductance of two voxels the harmonic mean of
// their conductivities (the paper's scalar-K Eq. 2675-eq2 is the special case
// of uniform K).  For a free voxel i of label l and its in-grid neighbour j of
// label m:
//     theta'_i = theta_i + sum_j w(l, m) (theta_j - theta_i) - b_i theta_i + s_i,
//     w(l, m)  = dt / (rho_l c_l h^2) * 2 K_l K_m / (K_l + K_m).
// The weights depend on the label pair only, so they live in a label-pair table
// (FP32, or FP64 with FP64 coefficients); the per-voxel fields are the labels
// and the usual b, s.  Fixed voxels (a = 0: fixed labels, Dirichlet faces) keep
// their value and still set their neighbours' face conductances.
//
// One step per launch, one thread per voxel: the kernel of the model options
// (this form, and the perfusion weighted by the tissue state alpha = 1 /
// max(1, Omega) of Eq. eq-tissState with either form), not the benchmarked
// path.  Latch and damage integral as in the one-step kernel; with the centre
// form and alpha = 1 it performs the one-step kernel's operations exactly.
//
// The adjoint of the step: with lambda = dL/dtheta',
//     (A^T lambda)_j = A_jj lambda_j + sum_{i nb of j, i free} w(l_i, l_j) lambda_i,
//     A_jj = 1 - sum_nb w(l_j, l_nb) - b_j (free j), 1 (fixed j),
// and dL/dK_l collects lambda_i (theta_j - theta_i) dw(l_i, l_j)/dK_l through
// both labels of every face of a free voxel i.
#include "rfa_internal.cuh"
#include "rfa_update.cuh"

#include <cmath>
#include <cstdio>

namespace rfa {

namespace {

struct CondArgs {
    const void *th_in;
    const float *lo_in;
    void *th_out;
    float *lo_out;
    const void *ab, *s;
    const uint8_t *label;
    const void *wpair;  // [kCondLabels][kCondLabels], float (double for FP64 coefficients)
    uint8_t *latch;
    double *omega;
    float *omega_c;
    unsigned *status;
    int nx, ny, nz, pitch;
    size_t plane;
    double thr;
    DamageConst dc;
    int damage, latch_on, fold;
    int zchunk;
    int cond;   // 0: centre form (a_i * sum of differences), 1: harmonic face weights
    int alpha;  // perfusion weighted by 1 / max(1, Omega) of the step's start
};

template <typename T>
struct MQ {
    T v[4];
};
__device__ __forceinline__ MQ<float> mldq(const float *p)
{
    const float4 t = *reinterpret_cast<const float4 *>(p);
    return {{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ MQ<double> mldq(const double *p)
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    return {{a.x, a.y, b.x, b.y}};
}
template <typename T>
__device__ __forceinline__ MQ<T> mzq()
{
    return {{T(0), T(0), T(0), T(0)}};
}
// a and b of voxels i..i+3 (i a multiple of 4) in the parameter type's own
// precision: float for BF16/FP32 storage, double for FP64
template <int PP, typename W>
__device__ __forceinline__ void mld_ab(const void *ab, size_t i, W a[4], W b[4])
{
    if (PP == RFA_PARAM_BF16) {
        const uint4 w = *reinterpret_cast<const uint4 *>((const uint32_t *)ab + i);
        const uint32_t v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a[q] = (W)bf16_to_float(v[q] & 0xffffu);
            b[q] = (W)bf16_to_float(v[q] >> 16);
        }
    } else if (PP == RFA_PARAM_F32) {
        const float4 u = reinterpret_cast<const float4 *>((const float2 *)ab + i)[0];
        const float4 w = reinterpret_cast<const float4 *>((const float2 *)ab + i)[1];
        a[0] = (W)u.x, b[0] = (W)u.y, a[1] = (W)u.z, b[1] = (W)u.w;
        a[2] = (W)w.x, b[2] = (W)w.y, a[3] = (W)w.z, b[3] = (W)w.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 v = ((const double2 *)ab)[i + q];
            a[q] = (W)v.x;
            b[q] = (W)v.y;
        }
    }
}

__device__ __forceinline__ int byte_at(uint32_t w, int q) { return (int)((w >> (8 * q)) & 0xffu); }

// the cache line holding p into L2 (no register is written): a thread streaming z
// asks for its fields two planes ahead, so their HBM latency overlaps the planes
// in between
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// (hi, lo) + delta of two voxels at once with the paired FP32 instructions:
// every lane performs cadd's operations in cadd's order (bit-identical)
__device__ __forceinline__ void cadd2(float2 c, float2 cl, float2 delta, float2 &nh, float2 &nl)
{
    const float2 s1 = add2(c, delta);
    const float2 bb = sub2(s1, c);
    const float2 e1 = add2(sub2(c, sub2(s1, bb)), sub2(delta, bb));
    const float2 l1 = add2(cl, e1);
    const float2 s2 = add2(s1, l1);
    nl = sub2(l1, sub2(s2, s1));
    nh = s2;
}

// One step of the model options, a thread per quad of 4 consecutive x voxels
// streaming z (planes z-1, z, z+1 and their labels in registers); x neighbours
// and their labels by warp shuffles, y neighbours through L1.  Per voxel the
// centre form performs the one-step kernel's operations; the harmonic form
// weighs every neighbour difference with its face weight from the label-pair
// table; with the tissue-state coupling b is divided by max(1, Omega).
// Every form runs at 2 CTAs/SM: at 3 (80 registers) the conservative form spills
// and reloads its parameters, and was 13 % slower (measured at 256^3).  The fields
// are prefetched into L2 two planes ahead (one plane: 1 %, two: 3-9 % faster).
template <int SP, int PP, bool COND, bool ALPHA>
__global__ void __launch_bounds__(256, 2) k_step_model(const CondArgs A)
{
    using T = typename std::conditional<SP == RFA_STATE_F64, double, float>::type;
    using W = typename std::conditional<PP == RFA_PARAM_F64, double, float>::type;
    using IT = typename std::conditional<SP == RFA_STATE_F64, double, float>::type;
    // b after the tissue-state division: double where the state or the parameters are FP64
    using BT = typename std::conditional<SP == RFA_STATE_F64 || PP == RFA_PARAM_F64, double, float>::type;
    constexpr bool COMP = SP == RFA_STATE_F32C;
    const unsigned FULL = 0xffffffffu;
    __shared__ W wt[kCondLabels * kCondLabels];
    for (int k = threadIdx.y * blockDim.x + threadIdx.x; k < kCondLabels * kCondLabels; k += blockDim.x * blockDim.y)
        wt[k] = ((const W *)A.wpair)[k];
    __syncthreads();
    const int lane = threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (y >= A.ny) return;  // whole warp (blockDim.x == 32), after the only barrier
    const int x0 = 4 * (blockIdx.x * 32 + lane);
    const bool inrow = x0 < A.pitch;
    // Every lane takes part in every quad load and shuffle, with no branch and no
    // zero fill: a lane past the row's end reads the row's last quad and stores nothing,
    // and a neighbour outside the grid is read at the voxel's own place (its
    // difference is then dropped by the in-grid flags; a label read there equals
    // the voxel's own, so the one-label test still covers the in-grid faces alone).
    const int xq = inrow ? x0 : A.pitch - 4;
    const int zb = blockIdx.z * A.zchunk, ze = min(A.nz, zb + A.zchunk);
    const T *hin = (const T *)A.th_in;
    T *hout = (T *)A.th_out;
    const T thr = (T)A.thr;
    const size_t rowoff = (size_t)y * A.pitch + xq;
    const bool hasYm = y > 0, hasYp = y < A.ny - 1, hasL = x0 > 0, hasR = x0 + 4 < A.nx;
    const size_t dym = hasYm ? (size_t)A.pitch : 0, dyp = hasYp ? (size_t)A.pitch : 0;
    // lane 0 reads the voxel left of its quad and lane 31 the one right of it (those
    // two lanes alone: the same load from every lane made the one-step kernel 3 %
    // slower at 256^3); the other lanes take theirs from their neighbours by shuffles
    const ptrdiff_t dxe = lane == 0 ? (hasL && xq > 0 ? -1 : 0) : (lane == 31 && hasR ? 4 : 0);
    MQ<T> hm, hc, hp;
    MQ<float> lm = mzq<float>(), lc = mzq<float>(), lp = mzq<float>();
    uint32_t labm, labc, labp;
    {
        const size_t ic = (size_t)zb * A.plane + rowoff, im = zb > 0 ? ic - A.plane : ic;
#ifdef RFA_CHECK
        // checked build: the warp leaves when any lane's range falls outside the arrays
        if (!__all_sync(FULL, RFA_CHECK_RANGE(im, ic + 4, A.plane * A.nz, ic, 4, A.status))) return;
#endif
        hc = mldq(hin + ic);
        hm = mldq(hin + im);
        if (COMP) {
            lc = mldq(A.lo_in + ic);
            lm = mldq(A.lo_in + im);
        }
        labc = *reinterpret_cast<const uint32_t *>(A.label + ic);
        labm = *reinterpret_cast<const uint32_t *>(A.label + im);
    }
    bool bad = false;
    for (int z = zb; z < ze; ++z) {
        const size_t i = (size_t)z * A.plane + rowoff;
        const bool hasZp = z + 1 < A.nz, hasZm = z > 0;
        const size_t ip = hasZp ? i + A.plane : i;
#ifdef RFA_CHECK
        // checked build: every access of this iteration lies in [lo, hi) of arrays of
        // plane * nz elements, the quads 4-aligned; the warp stops at the first miss
        {
            const long long lo = std::min((long long)(i - dym), (long long)i + dxe);
            const long long hi = std::max((long long)std::max(ip, i + dyp) + 4, (long long)i + dxe + 1);
            if (!__all_sync(FULL, RFA_CHECK_RANGE(lo, hi, A.plane * A.nz, i, 4, A.status))) break;
        }
#endif
        if (z + 2 < A.nz) {  // the streamed fields two planes ahead into L2
            const size_t iq = i + 2 * A.plane;
            prefetch_l2(hin + iq);
            if (COMP) prefetch_l2(A.lo_in + iq);
            prefetch_l2(A.label + iq);
            prefetch_l2((const char *)A.ab + iq * (PP == RFA_PARAM_BF16 ? 4 : PP == RFA_PARAM_F32 ? 8 : 16));
            prefetch_l2((const T *)A.s + iq);
            if (A.damage || ALPHA) prefetch_l2(A.omega_c + iq);
            if (ALPHA || A.fold) prefetch_l2(A.omega + iq);
        }
        hp = mldq(hin + ip);
        const MQ<T> hym = mldq(hin + i - dym), hyp = mldq(hin + i + dyp);
        MQ<float> lym = mzq<float>(), lyp = mzq<float>();
        float le = 0.f;
        T he = T(0);
        uint32_t lbe = 0;
        const bool edge = lane == 0 || lane == 31;
        if (COMP) {
            lp = mldq(A.lo_in + ip);
            lym = mldq(A.lo_in + i - dym);
            lyp = mldq(A.lo_in + i + dyp);
            if (edge) le = A.lo_in[i + dxe];
        }
        labp = *reinterpret_cast<const uint32_t *>(A.label + ip);
        const uint32_t labym = *reinterpret_cast<const uint32_t *>(A.label + i - dym);
        const uint32_t labyp = *reinterpret_cast<const uint32_t *>(A.label + i + dyp);
        if (edge) {
            he = hin[i + dxe];
            lbe = A.label[i + dxe];
        }
        W aq[4], bq[4];
        mld_ab<PP, W>(A.ab, i, aq, bq);
        const MQ<T> sq = mldq((const T *)A.s + i);
        MQ<double> om4 = mzq<double>();
        float4 cc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (A.damage || ALPHA) {
            cc = *reinterpret_cast<const float4 *>(A.omega_c + i);
            if (ALPHA || A.fold || SP == RFA_STATE_F64) om4 = mldq(A.omega + i);
        }
        // x neighbours across quads (value, lo part, label)
        T left = __shfl_up_sync(FULL, hc.v[3], 1), right = __shfl_down_sync(FULL, hc.v[0], 1);
        float lleft = 0.f, lright = 0.f;
        if (COMP) {
            lleft = __shfl_up_sync(FULL, lc.v[3], 1);
            lright = __shfl_down_sync(FULL, lc.v[0], 1);
        }
        uint32_t labl = __shfl_up_sync(FULL, labc >> 24, 1), labr = __shfl_down_sync(FULL, labc & 0xffu, 1);
        if (lane == 0) {
            left = he;
            lleft = le;
            labl = lbe;
        }
        if (lane == 31) {
            right = he;
            lright = le;
            labr = lbe;
        }
        // the quad, its x neighbours and its y/z neighbour quads all of one label
        const uint32_t l0 = labc & 0xffu;
        const bool uni = labc == l0 * 0x01010101u && labym == labc && labyp == labc && labm == labc &&
                         labp == labc && labl == l0 && labr == l0;
        W wuni = W(0);
        if (COND && uni) wuni = wt[l0 * (kCondLabels + 1)];
        const float ccv[4] = {cc.x, cc.y, cc.z, cc.w};
        MQ<T> ho;
        MQ<float> lo;
        uint32_t latch_bits = 0;
        IT inc[4] = {0, 0, 0, 0};
        // b of a free voxel: with the tissue state, b / max(1, Omega) with Omega at the
        // start of the step.  Omega below 0.5 (the high word of the double) and a carry
        // below 0.5 give an FP64 sum below 1 exactly, so the FP64 sum and the division
        // are skipped there.
        auto bfree = [&](int q) -> BT {
            BT bd = (BT)bq[q];
            if (ALPHA && !(__double2hiint(om4.v[q]) < 0x3FE00000 && ccv[q] < 0.5f)) {
                const double om = om4.v[q] + (double)ccv[q];
                if (om > 1.0) bd = (BT)((double)bq[q] / om);
            }
            return bd;
        };
        if (COMP) {
            // compensated FP32 state: the voxels (0, 1) and (2, 3) of the quad at once with
            // the paired FP32 instructions; every lane performs the operations of cdiff,
            // cupdate and cadd in their order, so the results are bit-identical to the
            // one-voxel forms (the centre form's to the one-step kernel's)
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const int qa = 2 * p, qb = qa + 1;
                const int xa = x0 + qa, xb = x0 + qb;
                const float2 c2 = make_float2((float)hc.v[qa], (float)hc.v[qb]);
                const float2 cl2 = make_float2(lc.v[qa], lc.v[qb]);
                float2 nh2 = c2, nl2 = cl2;
                const bool ua = aq[qa] != W(0) && xa < A.nx, ub = aq[qb] != W(0) && xb < A.nx;
                if (ua || ub) {
                    const float2 b2 = make_float2((float)bfree(qa), (float)bfree(qb));
                    const float2 s2 = make_float2((float)sq.v[qa], (float)sq.v[qb]);
                    // neighbour pairs in the fixed order x-, x+, y-, y+, z-, z+
                    const float2 nb[6] = {
                        make_float2(qa == 0 ? (float)left : (float)hc.v[qa - 1], (float)hc.v[qa]),
                        make_float2((float)hc.v[qb], qb == 3 ? (float)right : (float)hc.v[qb + 1]),
                        make_float2((float)hym.v[qa], (float)hym.v[qb]),
                        make_float2((float)hyp.v[qa], (float)hyp.v[qb]),
                        make_float2((float)hm.v[qa], (float)hm.v[qb]),
                        make_float2((float)hp.v[qa], (float)hp.v[qb])};
                    const float2 nbl[6] = {make_float2(qa == 0 ? lleft : lc.v[qa - 1], lc.v[qa]),
                                           make_float2(lc.v[qb], qb == 3 ? lright : lc.v[qb + 1]),
                                           make_float2(lym.v[qa], lym.v[qb]),
                                           make_float2(lyp.v[qa], lyp.v[qb]),
                                           make_float2(lm.v[qa], lm.v[qb]),
                                           make_float2(lp.v[qa], lp.v[qb])};
                    const bool ina[6] = {xa > 0, xa + 1 < A.nx, hasYm, hasYp, hasZm, hasZp};
                    const bool inb[6] = {true, xb + 1 < A.nx, hasYm, hasYp, hasZm, hasZp};
                    float2 h2, l2;
                    if (!COND) {
                        float2 S = make_float2(0.f, 0.f);
#pragma unroll
                        for (int d = 0; d < 6; ++d) {
                            const float2 dd = cdiff2(nb[d], nbl[d], c2, cl2);
                            S = add2(S, make_float2(ina[d] ? dd.x : 0.f, inb[d] ? dd.y : 0.f));
                        }
                        float2 th;
                        cupdate2(c2, cl2, S, make_float2((float)aq[qa], (float)aq[qb]), b2, s2, h2, l2, th);
                    } else {
                        // face weights: one table entry where the quad and all its
                        // neighbours share a label, else one look-up per face and voxel
                        float2 w2[6];
                        if (uni) {
#pragma unroll
                            for (int d = 0; d < 6; ++d) w2[d] = make_float2((float)wuni, (float)wuni);
                        } else {
                            const int la = byte_at(labc, qa), lb = byte_at(labc, qb);
                            const int nla[6] = {qa == 0 ? (int)labl : byte_at(labc, qa - 1), byte_at(labc, qb),
                                                byte_at(labym, qa), byte_at(labyp, qa),
                                                byte_at(labm, qa), byte_at(labp, qa)};
                            const int nlb[6] = {byte_at(labc, qa), qb == 3 ? (int)labr : byte_at(labc, qb + 1),
                                                byte_at(labym, qb), byte_at(labyp, qb),
                                                byte_at(labm, qb), byte_at(labp, qb)};
#pragma unroll
                            for (int d = 0; d < 6; ++d)
                                w2[d] = make_float2((float)wt[la * kCondLabels + nla[d]],
                                                    (float)wt[lb * kCondLabels + nlb[d]]);
                        }
                        const float2 th = add2(c2, cl2);
                        float2 delta = __ffma2_rn(neg2(b2), th, s2);
#pragma unroll
                        for (int d = 0; d < 6; ++d) {
                            const float2 r = __ffma2_rn(w2[d], cdiff2(nb[d], nbl[d], c2, cl2), delta);
                            delta = make_float2(ina[d] ? r.x : delta.x, inb[d] ? r.y : delta.y);
                        }
                        cadd2(c2, cl2, delta, h2, l2);
                    }
                    nh2 = make_float2(ua ? h2.x : c2.x, ub ? h2.y : c2.y);
                    nl2 = make_float2(ua ? l2.x : cl2.x, ub ? l2.y : cl2.y);
                }
                if (xa >= A.nx) nh2.x = nl2.x = 0.f;
                if (xb >= A.nx) nh2.y = nl2.y = 0.f;
                bad |= (xa < A.nx && !isfinite(nh2.x)) || (xb < A.nx && !isfinite(nh2.y));
                ho.v[qa] = (T)nh2.x;
                ho.v[qb] = (T)nh2.y;
                lo.v[qa] = nl2.x;
                lo.v[qb] = nl2.y;
                if (A.latch_on) {
                    if (xa < A.nx && nh2.x + nl2.x >= (float)thr) latch_bits |= 1u << (8 * qa);
                    if (xb < A.nx && nh2.y + nl2.y >= (float)thr) latch_bits |= 1u << (8 * qb);
                }
                if (A.damage) {
                    const float2 e2 = arrhenius_inc2(add2(nh2, nl2), A.dc.c0, A.dc.c1, A.dc.TK0);
                    inc[qa] = (IT)e2.x;
                    inc[qb] = (IT)e2.y;
                }
            }
        }
        if (!COMP) {
            // plain FP32 or FP64 state, one voxel at a time
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int x = x0 + q;
                const T c = hc.v[q];
                T nh = c;
                if (aq[q] != W(0) && x < A.nx) {
                    const BT bd = bfree(q);
                    // neighbours in the fixed order x-, x+, y-, y+, z-, z+
                    const bool in[6] = {x > 0, x + 1 < A.nx, hasYm, hasYp, hasZm, hasZp};
                    const T nbh[6] = {q == 0 ? left : hc.v[q - 1], q == 3 ? right : hc.v[q + 1], hym.v[q],
                                      hyp.v[q], hm.v[q], hp.v[q]};
                    if (!COND) {
                        T S = T(0);
#pragma unroll
                        for (int d = 0; d < 6; ++d) S = acc(S, in[d] ? pdiff(nbh[d], c) : T(0));
                        nh = pupdate(c, S, (T)aq[q], (T)bd, sq.v[q]);
                    } else {
                        // face weights w(l, m): one table entry where the quad and all its
                        // neighbours share a label, else one look-up per face
                        W wv[6];
                        if (uni) {
#pragma unroll
                            for (int d = 0; d < 6; ++d) wv[d] = wuni;
                        } else {
                            const int l = byte_at(labc, q);
                            const int nbl_lab[6] = {q == 0 ? (int)labl : byte_at(labc, q - 1),
                                                    q == 3 ? (int)labr : byte_at(labc, q + 1),
                                                    byte_at(labym, q), byte_at(labyp, q),
                                                    byte_at(labm, q), byte_at(labp, q)};
#pragma unroll
                            for (int d = 0; d < 6; ++d) wv[d] = wt[l * kCondLabels + nbl_lab[d]];
                        }
                        T delta;
                        if (SP == RFA_STATE_F64) delta = (T)__fma_rn(-bd, (double)c, (double)sq.v[q]);
                        else delta = (T)__fmaf_rn(-(float)bd, (float)c, (float)sq.v[q]);
#pragma unroll
                        for (int d = 0; d < 6; ++d)
                            if (in[d]) {
                                const T w = (T)wv[d];
                                if (SP == RFA_STATE_F64)
                                    delta = (T)__fma_rn((double)w, __dsub_rn((double)nbh[d], (double)c), (double)delta);
                                else
                                    delta = (T)__fmaf_rn((float)w, __fsub_rn((float)nbh[d], (float)c), (float)delta);
                            }
                        nh = SP == RFA_STATE_F64 ? (T)__dadd_rn((double)c, (double)delta)
                                                 : (T)__fadd_rn((float)c, (float)delta);
                    }
                }
                if (x >= A.nx) nh = T(0);
                bad |= x < A.nx && !isfinite(nh);
                ho.v[q] = nh;
                lo.v[q] = 0.f;
                if (A.latch_on && x < A.nx && nh >= thr) latch_bits |= 1u << (8 * q);
                if (A.damage && x < A.nx) {
                    if (SP == RFA_STATE_F64) inc[q] = exp2(A.dc.c0d - A.dc.c1d / ((double)nh + A.dc.TK0d));
                    else inc[q] = arrhenius_inc(__fadd_rn((float)nh, 0.f), A.dc.c0, A.dc.c1, A.dc.TK0);
                }
            }
        }
        if (inrow) {
            if (SP == RFA_STATE_F64) {
                reinterpret_cast<double2 *>(hout + i)[0] = make_double2((double)ho.v[0], (double)ho.v[1]);
                reinterpret_cast<double2 *>(hout + i)[1] = make_double2((double)ho.v[2], (double)ho.v[3]);
            } else {
                *reinterpret_cast<float4 *>(hout + i) =
                    make_float4((float)ho.v[0], (float)ho.v[1], (float)ho.v[2], (float)ho.v[3]);
            }
            if (COMP) *reinterpret_cast<float4 *>(A.lo_out + i) = make_float4(lo.v[0], lo.v[1], lo.v[2], lo.v[3]);
            if (A.latch_on && latch_bits) {
                uint32_t *lp32 = reinterpret_cast<uint32_t *>(A.latch + i);
                const uint32_t old = *lp32;
                if ((old | latch_bits) != old) *lp32 = old | latch_bits;
            }
            if (A.damage) {
                float P[4] = {cc.x, cc.y, cc.z, cc.w};
                double om[4] = {om4.v[0], om4.v[1], om4.v[2], om4.v[3]};
                if (SP == RFA_STATE_F64) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (x0 + q >= A.nx) continue;
                        const double sm = __dadd_rn(om[q], (double)inc[q]);
                        const double bb = __dsub_rn(sm, om[q]);
                        const double er =
                            __dadd_rn(__dsub_rn(om[q], __dsub_rn(sm, bb)), __dsub_rn((double)inc[q], bb));
                        om[q] = sm;
                        P[q] = __fadd_rn(P[q], (float)er);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (x0 + q < A.nx) P[q] = __fadd_rn(P[q], (float)inc[q]);
                    if (A.fold)
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (x0 + q < A.nx) carry_fold(om[q], P[q]);
                }
                if (SP == RFA_STATE_F64 || A.fold) {
                    reinterpret_cast<double2 *>(A.omega + i)[0] = make_double2(om[0], om[1]);
                    reinterpret_cast<double2 *>(A.omega + i)[1] = make_double2(om[2], om[3]);
                }
                *reinterpret_cast<float4 *>(A.omega_c + i) = make_float4(P[0], P[1], P[2], P[3]);
            }
        }
        hm = hc;
        hc = hp;
        labm = labc;
        labc = labp;
        if (COMP) {
            lm = lc;
            lc = lp;
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(A.status, kStatusNonfinite);
}

struct CondAdjArgs {
    const float *lam_in, *th;
    float *lam_out, *Lam;
    const void *ab;
    const uint8_t *label;
    const LabelCoef *tab;          // a != 0 marks the labels whose voxels are updated
    const float *wpair, *dA, *dB;  // [kCondLabels][kCondLabels]: w, dw/dK_l, dw/dK_m
    float gw[kCondLabels];         // d b / d w_b of each label
    int nx, ny, nz, pitch, zchunk, face, n_labels;
    size_t plane;
    double *acc;                   // [0..7] dL/dK, [8..15] dL/dw_b
};

// One adjoint step of the conservative form: lam_out = A^T lam_in, Lam +=
// lam_in, and the contractions dL/dK (through both labels of every face of a
// free voxel) and dL/dw_b.  A thread per quad of 4 x voxels streaming z
// (lambda, theta and labels of planes z-1, z, z+1 in registers), x neighbours
// by warp shuffles.  A voxel is updated by the forward step exactly when its
// stored a is nonzero, i.e. when its label's a is nonzero and it is not a
// Dirichlet face voxel: the voxel itself is tested on its stored a, its
// neighbours on their label and position (no coefficient loads for them).
// Row j of the step matrix holds w(l_j, l_i) for its neighbour i, so
// lam_out_i = diag_i lam_i + sum over free neighbours j of w(l_j, l_i) lam_j,
// diag_i = 1 - b_i - sum_j w(l_i, l_j) for a free i (1 otherwise).  The label
// sums stay in registers and leave the block with one FP64 atomic per label.
template <int PP>
__global__ void __launch_bounds__(256, 2) k_adjoint_cond(const CondAdjArgs A)
{
    constexpr int NL = 8;  // the backward pass admits at most 8 labels
    const unsigned FULL = 0xffffffffu;
    // per label pair (l, m) of a voxel and its neighbour, the four weights a face
    // uses, in one 16-byte entry: w(l, m), dw(l, m)/dK_l, and w(m, l), dw(m, l)/dK_l
    // where label m is updated by the step (0 where it is fixed, so that a fixed
    // neighbour's terms vanish without a test)
    __shared__ float4 pair[kCondLabels * kCondLabels];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int k = tid; k < kCondLabels * kCondLabels; k += blockDim.x * blockDim.y) {
        const int l = k / kCondLabels, m = k % kCondLabels, km = m * kCondLabels + l;
        const bool mfree = m < A.n_labels && A.tab[m].a != 0.0;
        pair[k] = make_float4(A.wpair[k], A.dA[k], mfree ? A.wpair[km] : 0.f, mfree ? A.dB[km] : 0.f);
    }
    __syncthreads();
    float accK[NL], accW[NL];
#pragma unroll
    for (int L = 0; L < NL; ++L) accK[L] = accW[L] = 0.f;
    auto add_label = [&](float (&acc)[NL], int lab, float v) {
#pragma unroll
        for (int L = 0; L < NL; ++L) acc[L] += lab == L ? v : 0.f;
    };
    const int lane = threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (y < A.ny) {  // whole warp (blockDim.x == 32)
        const int x0 = 4 * (blockIdx.x * 32 + lane);
        const bool inrow = x0 < A.pitch;
        const int zb = blockIdx.z * A.zchunk, ze = min(A.nz, zb + A.zchunk);
        const size_t rowoff = (size_t)y * A.pitch + x0;
        const bool hasYm = y > 0, hasYp = y + 1 < A.ny;
        const bool dir = A.face == RFA_FACE_DIRICHLET;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 lm = z4, lc = z4, lp = z4, tm = z4, tc = z4, tp = z4;
        uint32_t labm = 0, labc = 0, labp = 0;
        if (inrow) {
            const size_t i = (size_t)zb * A.plane + rowoff;
            lc = *reinterpret_cast<const float4 *>(A.lam_in + i);
            tc = *reinterpret_cast<const float4 *>(A.th + i);
            labc = *reinterpret_cast<const uint32_t *>(A.label + i);
            if (zb > 0) {
                lm = *reinterpret_cast<const float4 *>(A.lam_in + i - A.plane);
                tm = *reinterpret_cast<const float4 *>(A.th + i - A.plane);
                labm = *reinterpret_cast<const uint32_t *>(A.label + i - A.plane);
            }
        }
        for (int z = zb; z < ze; ++z) {
            const size_t i = (size_t)z * A.plane + rowoff;
            const bool hasZm = z > 0, hasZp = z + 1 < A.nz;
            float4 lym = z4, lyp = z4, tym = z4, typ = z4, Lc = z4;
            uint32_t labym = 0, labyp = 0;
            float aq[4] = {0.f, 0.f, 0.f, 0.f}, bq[4] = {0.f, 0.f, 0.f, 0.f};
            if (inrow) {
                lp = tp = z4;
                labp = 0;
                if (hasZp) {
                    lp = *reinterpret_cast<const float4 *>(A.lam_in + i + A.plane);
                    tp = *reinterpret_cast<const float4 *>(A.th + i + A.plane);
                    labp = *reinterpret_cast<const uint32_t *>(A.label + i + A.plane);
                }
                if (hasYm) {
                    lym = *reinterpret_cast<const float4 *>(A.lam_in + i - A.pitch);
                    tym = *reinterpret_cast<const float4 *>(A.th + i - A.pitch);
                    labym = *reinterpret_cast<const uint32_t *>(A.label + i - A.pitch);
                }
                if (hasYp) {
                    lyp = *reinterpret_cast<const float4 *>(A.lam_in + i + A.pitch);
                    typ = *reinterpret_cast<const float4 *>(A.th + i + A.pitch);
                    labyp = *reinterpret_cast<const uint32_t *>(A.label + i + A.pitch);
                }
                mld_ab<PP, float>(A.ab, i, aq, bq);
                Lc = *reinterpret_cast<const float4 *>(A.Lam + i);
            }
            // x neighbours across quads: lambda, theta, label
            float lamL = __shfl_up_sync(FULL, lc.w, 1), lamR = __shfl_down_sync(FULL, lc.x, 1);
            float thL = __shfl_up_sync(FULL, tc.w, 1), thR = __shfl_down_sync(FULL, tc.x, 1);
            int labL = (int)__shfl_up_sync(FULL, labc >> 24, 1), labR = (int)__shfl_down_sync(FULL, labc & 0xffu, 1);
            if (inrow && lane == 0 && x0 > 0) {
                lamL = A.lam_in[i - 1];
                thL = A.th[i - 1];
                labL = A.label[i - 1];
            }
            if (inrow && lane == 31 && x0 + 4 < A.nx) {
                lamR = A.lam_in[i + 4];
                thR = A.th[i + 4];
                labR = A.label[i + 4];
            }
            if (inrow) {
                const float lcv[4] = {lc.x, lc.y, lc.z, lc.w}, tcv[4] = {tc.x, tc.y, tc.z, tc.w};
                const float lmv[4] = {lm.x, lm.y, lm.z, lm.w}, tmv[4] = {tm.x, tm.y, tm.z, tm.w};
                const float lpv[4] = {lp.x, lp.y, lp.z, lp.w}, tpv[4] = {tp.x, tp.y, tp.z, tp.w};
                const float lymv[4] = {lym.x, lym.y, lym.z, lym.w}, tymv[4] = {tym.x, tym.y, tym.z, tym.w};
                const float lypv[4] = {lyp.x, lyp.y, lyp.z, lyp.w}, typv[4] = {typ.x, typ.y, typ.z, typ.w};
                const float Lcv[4] = {Lc.x, Lc.y, Lc.z, Lc.w};
                float lo_[4], Lo_[4], gkq[4], gwq[4];
                // the neighbours on a Dirichlet face: the y- / y+ / z- / z+ neighbour rows
                // are fixed for the quad; the x neighbours share the quad's row and plane
                const bool rowface = dir && (y == 0 || y == A.ny - 1 || z == 0 || z == A.nz - 1);
                const bool fyz[4] = {dir && (y - 1 == 0 || z == 0 || z == A.nz - 1),
                                     dir && (y + 1 == A.ny - 1 || z == 0 || z == A.nz - 1),
                                     dir && (z - 1 == 0 || y == 0 || y == A.ny - 1),
                                     dir && (z + 1 == A.nz - 1 || y == 0 || y == A.ny - 1)};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int x = x0 + q;
                    const bool valid = x < A.nx;
                    const int l = byte_at(labc, q);
                    const float lam = lcv[q], t = tcv[q];
                    const bool fr = valid && aq[q] != 0.f;  // the forward's own test on the stored a
                    // neighbours in the order x-, x+, y-, y+, z-, z+
                    const bool in[6] = {x > 0, x + 1 < A.nx, hasYm, hasYp, hasZm, hasZp};
                    const float nl[6] = {q == 0 ? lamL : lcv[q - 1], q == 3 ? lamR : lcv[q + 1], lymv[q], lypv[q],
                                         lmv[q], lpv[q]};
                    const float nt[6] = {q == 0 ? thL : tcv[q - 1], q == 3 ? thR : tcv[q + 1], tymv[q], typv[q],
                                         tmv[q], tpv[q]};
                    const int nlab[6] = {q == 0 ? labL : byte_at(labc, q - 1), q == 3 ? labR : byte_at(labc, q + 1),
                                         byte_at(labym, q), byte_at(labyp, q), byte_at(labm, q), byte_at(labp, q)};
                    const bool nface[6] = {rowface || (dir && (x - 1 == 0 || x - 1 == A.nx - 1)),
                                           rowface || (dir && (x + 1 == 0 || x + 1 == A.nx - 1)),
                                           fyz[0] || (dir && (x == 0 || x == A.nx - 1)),
                                           fyz[1] || (dir && (x == 0 || x == A.nx - 1)),
                                           fyz[2] || (dir && (x == 0 || x == A.nx - 1)),
                                           fyz[3] || (dir && (x == 0 || x == A.nx - 1))};
                    // dL/dK: the face (i, j) of a free voxel i gives da[l_i][l_j] lam_i (theta_j -
                    // theta_i) to label l_i and db[l_i][l_j] lam_i (theta_j - theta_i) to label
                    // l_j; the second is collected here by the receiving voxel, so every term
                    // lands on this voxel's own label
                    // (the two dL/dK terms in separate sums: shorter dependent chains)
                    float diag = fr ? 1.f - bq[q] : 1.f, nsum = 0.f, g_in = 0.f, g_out = 0.f;
#pragma unroll
                    for (int d = 0; d < 6; ++d) {
                        if (!in[d]) continue;
                        const int m = nlab[d];
                        const float4 c = pair[l * kCondLabels + m];
                        if (!nface[d]) {  // (a fixed neighbour's entry holds zeros)
                            nsum += c.z * nl[d];
                            g_in += c.w * (nl[d] * (t - nt[d]));
                        }
                        if (fr) {
                            diag -= c.x;
                            g_out += c.y * (nt[d] - t);
                        }
                    }
                    const float gk = g_in + lam * g_out;
                    lo_[q] = valid ? diag * lam + nsum : 0.f;
                    Lo_[q] = valid ? Lcv[q] + lam : 0.f;
                    gkq[q] = valid ? gk : 0.f;
                    gwq[q] = fr ? lam * t : 0.f;
                }
                // label sums: once per quad where its voxels share a label
                if (labc == (labc & 0xffu) * 0x01010101u) {
                    add_label(accK, (int)(labc & 0xffu), (gkq[0] + gkq[1]) + (gkq[2] + gkq[3]));
                    add_label(accW, (int)(labc & 0xffu), (gwq[0] + gwq[1]) + (gwq[2] + gwq[3]));
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        add_label(accK, byte_at(labc, q), gkq[q]);
                        add_label(accW, byte_at(labc, q), gwq[q]);
                    }
                }
                *reinterpret_cast<float4 *>(A.lam_out + i) = make_float4(lo_[0], lo_[1], lo_[2], lo_[3]);
                *reinterpret_cast<float4 *>(A.Lam + i) = make_float4(Lo_[0], Lo_[1], Lo_[2], Lo_[3]);
            }
            lm = lc;
            lc = lp;
            tm = tc;
            tc = tp;
            labm = labc;
            labc = labp;
        }
    }
    // block reduction of the label sums, then one FP64 atomic per label and block
    __shared__ float sK[8][NL], sW[8][NL];
    const int w = threadIdx.y;
#pragma unroll
    for (int L = 0; L < NL; ++L) {
        float k = accK[L], v = accW[L];
        for (int o = 16; o > 0; o >>= 1) {
            k += __shfl_xor_sync(FULL, k, o);
            v += __shfl_xor_sync(FULL, v, o);
        }
        if (lane == 0) {
            sK[w][L] = k;
            sW[w][L] = v;
        }
    }
    __syncthreads();
    if (w == 0 && lane < NL) {
        double k = 0.0, v = 0.0;
        for (int j = 0; j < (int)blockDim.y; ++j) {
            k += sK[j][lane];
            v += sW[j][lane];
        }
        if (k != 0.0) atomicAdd(&A.acc[lane], k);
        if (v != 0.0) atomicAdd(&A.acc[8 + lane], -v * (double)A.gw[lane]);
    }
}

}  // namespace

// label-pair tables of the conservative form (host, FP64; the same expression
// order as any other FP64 evaluation of w(l, m), so the FP32 rounding agrees)
rfa_status cond_build_tables(rfa_grid *g, const rfa_tissue *table, int L)
{
    if (L > kCondLabels) {
        set_error("conservative conduction supports at most 16 labels");
        return RFA_E_UNSUPPORTED;
    }
    std::vector<double> W(kCondLabels * kCondLabels, 0.0), DA(W), DB(W);
    for (int l = 0; l < L; ++l) {
        const rfa_tissue &tl = table[l];
        const double gl = g->dt / (tl.rho * tl.c * g->h * g->h);
        for (int m = 0; m < L; ++m) {
            const rfa_tissue &tm = table[m];
            const double Ks = tl.k + tm.k;
            if (Ks > 0.0) {
                W[l * kCondLabels + m] = gl * (2.0 * tl.k * tm.k / Ks);
                DA[l * kCondLabels + m] = gl * 2.0 * tm.k * tm.k / (Ks * Ks);
                DB[l * kCondLabels + m] = gl * 2.0 * tl.k * tl.k / (Ks * Ks);
            }
        }
    }
    // positivity: 1 - deg * max_m w(l, m) - b_l >= 0 for every free label
    const double deg = 2.0 * ((g->nx > 1) + (g->ny > 1) + (g->nz > 1));
    for (int l = 0; l < L; ++l) {
        if (table[l].fixed) continue;
        double wmax = 0.0;
        for (int m = 0; m < L; ++m) {
            const double w = g->pp == RFA_PARAM_F64 ? W[l * kCondLabels + m] : (double)(float)W[l * kCondLabels + m];
            wmax = std::fmax(wmax, w);
        }
        LabelCoef c{};
        const rfa_tissue &t = table[l];
        c.k = t.k; c.rho = t.rho; c.c = t.c; c.w_b = t.w_b; c.rho_b = t.rho_b; c.c_b = t.c_b;
        const double b = round_coef(coef_b(c, g->dt), g->pp);
        if (1.0 - deg * wmax - b < 0.0) {
            char buf[192];
            std::snprintf(buf, sizeof buf, "label %d: 1 - %g max w - b = %.6g < 0 (conservative form); reduce dt", l,
                          deg, 1.0 - deg * wmax - b);
            set_error(buf);
            return RFA_E_UNSTABLE;
        }
    }
    if (g->pp == RFA_PARAM_F64) {
        RFA_CUDA(cudaMemcpyAsync(g->d_wpair, W.data(), W.size() * 8, cudaMemcpyHostToDevice, g->stream));
    } else {
        std::vector<float> Wf(W.begin(), W.end());
        RFA_CUDA(cudaMemcpyAsync(g->d_wpair, Wf.data(), Wf.size() * 4, cudaMemcpyHostToDevice, g->stream));
    }
    std::vector<float> Wa(3 * kCondLabels * kCondLabels);
    for (int k = 0; k < kCondLabels * kCondLabels; ++k) {
        Wa[k] = (float)W[k];
        Wa[kCondLabels * kCondLabels + k] = (float)DA[k];
        Wa[2 * kCondLabels * kCondLabels + k] = (float)DB[k];
    }
    RFA_CUDA(cudaMemcpyAsync(g->d_wadj, Wa.data(), Wa.size() * 4, cudaMemcpyHostToDevice, g->stream));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    return RFA_OK;
}

cudaError_t launch_step_model(rfa_grid *g, const void *th_in, const void *lo_in, void *th_out, void *lo_out,
                              bool damage, bool latch, bool fold)
{
    CondArgs A;
    A.cond = g->cond == RFA_COND_HARMONIC ? 1 : 0;
    A.alpha = g->alpha_perf;
    if (!A.cond && !A.alpha) return cudaErrorInvalidValue;  // the one-step kernel serves this model
    A.th_in = th_in;
    A.lo_in = (const float *)lo_in;
    A.th_out = th_out;
    A.lo_out = (float *)lo_out;
    A.ab = g->ab;
    A.s = g->s;
    A.label = g->label;
    A.wpair = g->d_wpair;
    A.latch = g->latch;
    A.omega = g->omega;
    A.omega_c = g->omega_c;
    A.status = g->status;
    A.nx = g->nx;
    A.ny = g->ny;
    A.nz = g->nz;
    A.pitch = g->pitch;
    A.plane = g->plane;
    A.thr = g->T_thr - g->T_a;
    A.dc = damage_consts(g);
    A.damage = damage ? 1 : 0;
    A.latch_on = latch ? 1 : 0;
    A.fold = fold ? 1 : 0;
    A.zchunk = choose_zchunk(g, 3);
    const dim3 blk(32, 8), grd = plain_grid_dims(g, A.zchunk);
#define COND_CASE(SPV, PPV)                                                                                  \
    if (g->sp == SPV && g->pp == PPV) {                                                                      \
        if (A.cond && A.alpha) k_step_model<SPV, PPV, true, true><<<grd, blk, 0, g->stream>>>(A);            \
        else if (A.cond) k_step_model<SPV, PPV, true, false><<<grd, blk, 0, g->stream>>>(A);                 \
        else k_step_model<SPV, PPV, false, true><<<grd, blk, 0, g->stream>>>(A);                             \
    }
    COND_CASE(RFA_STATE_F32, RFA_PARAM_BF16)
    COND_CASE(RFA_STATE_F32, RFA_PARAM_F32)
    COND_CASE(RFA_STATE_F32, RFA_PARAM_F64)
    COND_CASE(RFA_STATE_F32C, RFA_PARAM_BF16)
    COND_CASE(RFA_STATE_F32C, RFA_PARAM_F32)
    COND_CASE(RFA_STATE_F32C, RFA_PARAM_F64)
    COND_CASE(RFA_STATE_F64, RFA_PARAM_BF16)
    COND_CASE(RFA_STATE_F64, RFA_PARAM_F32)
    COND_CASE(RFA_STATE_F64, RFA_PARAM_F64)
#undef COND_CASE
    return cudaGetLastError();
}

cudaError_t launch_adjoint_cond(rfa_grid *g, const float *lam_in, float *lam_out, float *Lam, const float *th,
                                double *acc)
{
    CondAdjArgs A;
    A.lam_in = lam_in;
    A.lam_out = lam_out;
    A.Lam = Lam;
    A.th = th;
    A.ab = g->ab;
    A.label = g->label;
    A.wpair = g->d_wadj;
    A.dA = g->d_wadj + kCondLabels * kCondLabels;
    A.dB = g->d_wadj + 2 * kCondLabels * kCondLabels;
    for (int l = 0; l < kCondLabels; ++l) {
        A.gw[l] = 0.f;
        if (l < g->n_labels && !g->table[l].fixed) {
            const rfa_tissue &t = g->table[l];
            A.gw[l] = (float)((t.rho_b * t.c_b / (t.rho * t.c)) * g->dt);
        }
    }
    A.nx = g->nx;
    A.ny = g->ny;
    A.nz = g->nz;
    A.pitch = g->pitch;
    A.plane = g->plane;
    A.acc = acc;
    A.tab = g->d_table;
    A.face = g->face;
    A.n_labels = g->n_labels;
    A.zchunk = choose_zchunk_waves(g, 2);
    const dim3 blk(32, 8), grd = plain_grid_dims(g, A.zchunk);
    if (g->pp == RFA_PARAM_BF16) k_adjoint_cond<RFA_PARAM_BF16><<<grd, blk, 0, g->stream>>>(A);
    else if (g->pp == RFA_PARAM_F32) k_adjoint_cond<RFA_PARAM_F32><<<grd, blk, 0, g->stream>>>(A);
    else k_adjoint_cond<RFA_PARAM_F64><<<grd, blk, 0, g->stream>>>(A);
    return cudaGetLastError();
}

}  // namespace rfa

using namespace rfa;

extern "C" rfa_status rfa_set_perfusion_coupling(rfa_grid *g, int mode)
{
    if (!g) {
        set_error("null grid");
        return RFA_E_INVALID;
    }
    if (mode != RFA_PERF_CONSTANT && mode != RFA_PERF_TISSUE_STATE) {
        set_error("unknown perfusion coupling");
        return RFA_E_INVALID;
    }
    if (mode != g->alpha_perf && g->steps > 0) g->rec.valid = false;
    g->alpha_perf = mode;
    return RFA_OK;
}

extern "C" rfa_status rfa_set_conduction(rfa_grid *g, int mode)
{
    if (!g) {
        set_error("null grid");
        return RFA_E_INVALID;
    }
    if (mode != RFA_COND_CENTRE && mode != RFA_COND_HARMONIC) {
        set_error("unknown conduction mode");
        return RFA_E_INVALID;
    }
    if (mode == RFA_COND_HARMONIC && g->tip_on) {
        set_error("the conservative form does not run with a FIXED_TIP needle");
        return RFA_E_UNSUPPORTED;
    }
    if (mode == RFA_COND_HARMONIC && g->have_tissue) {
        const rfa_status st = cond_build_tables(g, g->table.data(), g->n_labels);
        if (st != RFA_OK) return st;
    }
    if (mode != g->cond && g->steps > 0) g->rec.valid = false;  // the recorded steps used the other form
    g->cond = mode;
    return RFA_OK;
}
