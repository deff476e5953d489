// kernels_step.cu -- one explicit step per launch (Eq. CUDAbioheat3d), fused
// with the necrosis latch and the Arrhenius damage update.
//
// Per free voxel (theta = T - T_a; a, b, s as in rfa_internal.cuh):
//     theta' = theta + a * sum_nb (theta_nb - theta) - b * theta + s
// a neighbour outside the grid contributes nothing; fixed voxels have
// a = b = s = 0.  The difference form keeps the FP32 stencil free of the
// cancellation in sum_nb theta_nb - 6 theta.
//
// Thread mapping: one thread owns 4 consecutive x voxels (a float4 "quad") of
// one row and streams along z over a chunk of planes, keeping the planes
// z-1, z, z+1 of its quad in registers (2.5D streaming).  A warp covers 128
// consecutive x voxels; the x neighbours across quads come from warp shuffles,
// the y neighbours from the rows above/below (L1/L2 hits).
//
// Compensated state (F32C): the value is hi + lo.  Neighbour differences are
// taken as (hi_nb - hi) + (lo_nb - lo), the increment is added to hi with an
// error-free TwoSum, the rounding error goes to lo, and (hi, lo) is
// renormalised with Fast2Sum.
//
// Damage: inc = dt A exp(-Ea / (R T_K)) is evaluated in FP32 as
// exp2(c0 - c1 / T_K) with c0 = log2(A dt), c1 = Ea / (R ln 2) (ln-space keeps
// A = 7.39e39 and exp(-100) inside FP32 range).  The integral is kept as an
// FP64 value plus an FP32 carry: increments go into the carry, which is folded
// into the FP64 value with an error-free TwoSum on launches flagged `fold`
// (every few launches); the FP64 state adds every increment in FP64 directly.
#include "rfa_internal.cuh"
#include "rfa_update.cuh"

#include <cmath>

namespace rfa {

namespace {

template <typename T>
struct Q4 {
    T v[4];
};

__device__ __forceinline__ Q4<float> ldq(const float *p)
{
    float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    return {{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ Q4<double> ldq(const double *p)
{
    double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void stq(float *p, const Q4<float> &q)
{
    *reinterpret_cast<float4 *>(p) = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
}
__device__ __forceinline__ void stq(double *p, const Q4<double> &q)
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(q.v[0], q.v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(q.v[2], q.v[3]);
}
template <typename T>
__device__ __forceinline__ Q4<T> zq()
{
    return {{T(0), T(0), T(0), T(0)}};
}

// coefficients of 4 consecutive voxels, converted to the arithmetic type
template <int PP, typename R>
__device__ __forceinline__ void load_ab(const void *ab, size_t i, R a[4], R b[4])
{
    if (PP == RFA_PARAM_BF16) {
        uint4 u = __ldg(reinterpret_cast<const uint4 *>((const uint32_t *)ab + i));
        uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a[q] = (R)bf16_to_float(w[q] & 0xffffu);
            b[q] = (R)bf16_to_float(w[q] >> 16);
        }
    } else if (PP == RFA_PARAM_F32) {
        const float4 *p = reinterpret_cast<const float4 *>((const float2 *)ab + i);
        float4 u = __ldg(p), v = __ldg(p + 1);
        a[0] = (R)u.x; b[0] = (R)u.y; a[1] = (R)u.z; b[1] = (R)u.w;
        a[2] = (R)v.x; b[2] = (R)v.y; a[3] = (R)v.z; b[3] = (R)v.w;
    } else {
        const double2 *p = (const double2 *)ab + i;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double2 t = __ldg(p + q);
            a[q] = (R)t.x;
            b[q] = (R)t.y;
        }
    }
}

// the cache line holding p into L2 (no register is written): a thread streaming z
// asks for its fields two planes ahead, so their HBM latency overlaps the planes
// in between (256^3: 0.80 -> 0.84 of HBM; the 96^3-192^3 grids of the batch's
// per-needle loop: 18 % faster)
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

struct PlainArgs {
    const void *th_in, *lo_in, *ab, *s;
    void *th_out, *lo_out;
    uint8_t *latch;
    double *omega;
    float *omega_c;
    unsigned *status;
    int nx, ny, nz, pitch, zchunk;
    size_t plane;
    double thr;  // latch threshold on theta
    DamageConst dc;
    int fold;    // fold the FP32 damage carry into the FP64 integral this launch
};

template <int SP, int PP, bool DMG, bool LATCH, bool FOLD>
__global__ void __launch_bounds__(256) k_step_plain(const PlainArgs A)
{
    using T = typename std::conditional<SP == RFA_STATE_F64, double, float>::type;
    constexpr bool COMP = (SP == RFA_STATE_F32C);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (y >= A.ny) return;  // whole warp: blockDim.x == 32
    const int x0 = 4 * (blockIdx.x * 32 + lane);
    const bool inrow = x0 < A.pitch;
    const int zb = blockIdx.z * A.zchunk;
    const int ze = min(A.nz, zb + A.zchunk);
    const T *hin = (const T *)A.th_in;
    const float *lin = (const float *)A.lo_in;
    T *hout = (T *)A.th_out;
    float *lout = (float *)A.lo_out;
    const bool hasYm = y > 0, hasYp = y < A.ny - 1;
    const bool hasL = x0 > 0, hasR = x0 + 4 < A.nx;
    const T thr = (T)A.thr;
    // Every lane takes part in every quad load and shuffle, with no branch and no
    // zero fill: a lane past the row's end reads the row's last quad and stores nothing,
    // and a neighbour outside the grid is read at the voxel's own place (its
    // difference is then dropped by the in-grid flags).
    const int xq = inrow ? x0 : A.pitch - 4;
    const size_t rowoff = (size_t)y * A.pitch + xq;
    const size_t dym = hasYm ? (size_t)A.pitch : 0, dyp = hasYp ? (size_t)A.pitch : 0;
    // lane 0 reads the voxel left of its quad and lane 31 the one right of it (those
    // two lanes alone: the same load from every lane made the one-step kernel 3 %
    // slower at 256^3); the other lanes take theirs from their neighbours by shuffles
    const ptrdiff_t dxe = lane == 0 ? (hasL && xq > 0 ? -1 : 0) : (lane == 31 && hasR ? 4 : 0);

    Q4<T> hm, hc, hp;
    Q4<float> lm = zq<float>(), lc = zq<float>(), lp = zq<float>();
    {
        const size_t ic = (size_t)zb * A.plane + rowoff, im = zb > 0 ? ic - A.plane : ic;
#ifdef RFA_CHECK
        // checked build: the warp leaves when any lane's range falls outside the arrays
        if (!__all_sync(FULL, RFA_CHECK_RANGE(im, ic + 4, A.plane * A.nz, ic, 4, A.status))) return;
#endif
        hc = ldq(hin + ic);
        hm = ldq(hin + im);
        if (COMP) {
            lc = ldq(lin + ic);
            lm = ldq(lin + im);
        }
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
        if (inrow && z + 2 < A.nz) {  // the streamed fields two planes ahead into L2
            const size_t iq = i + 2 * A.plane;
            prefetch_l2(hin + iq);
            if (COMP) prefetch_l2(lin + iq);
            prefetch_l2((const char *)A.ab + iq * (PP == RFA_PARAM_BF16 ? 4 : PP == RFA_PARAM_F32 ? 8 : 16));
            prefetch_l2((const T *)A.s + iq);
            if (LATCH) prefetch_l2(A.latch + iq);
            if (DMG) prefetch_l2(A.omega_c + iq);
            if (DMG && FOLD) prefetch_l2(A.omega + iq);
        }
        hp = ldq(hin + ip);
        const Q4<T> hym = ldq(hin + i - dym), hyp = ldq(hin + i + dyp);
        Q4<float> lym = zq<float>(), lyp = zq<float>();
        float le = 0.f;
        T he = T(0);
        const bool edge = lane == 0 || lane == 31;
        if (COMP) {
            lp = ldq(lin + ip);
            lym = ldq(lin + i - dym);
            lyp = ldq(lin + i + dyp);
            if (edge) le = lin[i + dxe];
        }
        if (edge) he = hin[i + dxe];
        T aq[4], bq[4];
        load_ab<PP, T>(A.ab, i, aq, bq);
        const Q4<T> sv = ldq((const T *)A.s + i);
        // x neighbours across quads
        T left = __shfl_up_sync(FULL, hc.v[3], 1), right = __shfl_down_sync(FULL, hc.v[0], 1);
        float lleft = 0.f, lright = 0.f;
        if (COMP) {
            lleft = __shfl_up_sync(FULL, lc.v[3], 1);
            lright = __shfl_down_sync(FULL, lc.v[0], 1);
        }
        if (lane == 0) {
            left = he;
            lleft = le;
        }
        if (lane == 31) {
            right = he;
            lright = le;
        }
        Q4<T> ho;
        Q4<float> lo;
        uint32_t latch_bits = 0;
        double Sd[4];
        if (COMP) {
            // the voxels (0, 1) and (2, 3) of the quad at once with the paired FP32
            // instructions: every lane performs the operations of cdiff and cupdate in
            // their order, bit-identical to the one-voxel forms
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const int qa = 2 * p, qb = qa + 1;
                const int xa = x0 + qa, xb = x0 + qb;
                const float2 c2 = make_float2((float)hc.v[qa], (float)hc.v[qb]);
                const float2 cl2 = make_float2(lc.v[qa], lc.v[qb]);
                // neighbour pairs in the fixed order x-, x+, y-, y+, z-, z+ (Eq. 2675-eq3)
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
                float2 S = make_float2(0.f, 0.f);
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    const float2 dd = cdiff2(nb[d], nbl[d], c2, cl2);
                    S = add2(S, make_float2(ina[d] ? dd.x : 0.f, inb[d] ? dd.y : 0.f));
                }
                float2 h2, l2, th;
                cupdate2(c2, cl2, S, make_float2((float)aq[qa], (float)aq[qb]),
                         make_float2((float)bq[qa], (float)bq[qb]), make_float2((float)sv.v[qa], (float)sv.v[qb]),
                         h2, l2, th);
                if (xa >= A.nx) h2.x = l2.x = 0.f;
                if (xb >= A.nx) h2.y = l2.y = 0.f;
                bad |= (xa < A.nx && !isfinite(h2.x)) || (xb < A.nx && !isfinite(h2.y));
                ho.v[qa] = (T)h2.x;
                ho.v[qb] = (T)h2.y;
                lo.v[qa] = l2.x;
                lo.v[qb] = l2.y;
                if (LATCH) {
                    if (xa < A.nx && h2.x + l2.x >= (float)thr) latch_bits |= 1u << (8 * qa);
                    if (xb < A.nx && h2.y + l2.y >= (float)thr) latch_bits |= 1u << (8 * qb);
                }
                if (DMG) {
                    const float2 e2 = arrhenius_inc2(add2(h2, l2), A.dc.c0, A.dc.c1, A.dc.TK0);
                    Sd[qa] = (double)e2.x;
                    Sd[qb] = (double)e2.y;
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int x = x0 + q;
                const T c = hc.v[q];
                const T xm = q == 0 ? left : hc.v[q - 1];
                const T xp = q == 3 ? right : hc.v[q + 1];
                // sum of neighbour differences (Eq. 2675-eq3 in x, y, z), fixed order
                T S = T(0);
                S = acc(S, x > 0 ? pdiff(xm, c) : T(0));
                S = acc(S, x + 1 < A.nx ? pdiff(xp, c) : T(0));
                S = acc(S, hasYm ? pdiff(hym.v[q], c) : T(0));
                S = acc(S, hasYp ? pdiff(hyp.v[q], c) : T(0));
                S = acc(S, hasZm ? pdiff(hm.v[q], c) : T(0));
                S = acc(S, hasZp ? pdiff(hp.v[q], c) : T(0));
                T nh = pupdate(c, S, aq[q], bq[q], sv.v[q]);
                if (x >= A.nx) nh = T(0);
                bad |= (x < A.nx) && !isfinite((double)nh);
                ho.v[q] = nh;
                lo.v[q] = 0.f;
                if (LATCH && x < A.nx && nh + T(0) >= thr) latch_bits |= 1u << (8 * q);
                if (DMG) {
                    if (SP == RFA_STATE_F64) {
                        double tk = (double)nh + A.dc.TK0d;
                        Sd[q] = exp2(A.dc.c0d - A.dc.c1d / tk);
                    } else {
                        Sd[q] = (double)arrhenius_inc(__fadd_rn((float)nh, 0.f), A.dc.c0, A.dc.c1, A.dc.TK0);
                    }
                }
            }
        }
        if (inrow) {
            stq(hout + i, ho);
            if (COMP) stq(lout + i, lo);
            if (LATCH && latch_bits) {
                uint32_t *lp32 = reinterpret_cast<uint32_t *>(A.latch + i);
                uint32_t old = *lp32;
                if ((old | latch_bits) != old) *lp32 = old | latch_bits;
            }
            if (DMG) {
                // Omega + P: FP64 integral plus FP32 carry (see carry_fold)
                float4 *cp = reinterpret_cast<float4 *>(A.omega_c + i);
                float4 cc = *cp;
                float P[4] = {cc.x, cc.y, cc.z, cc.w};
                double2 *op = reinterpret_cast<double2 *>(A.omega + i);
                if (SP == RFA_STATE_F64) {
                    // FP64 state: every increment is added in FP64, error-free, the
                    // rounding error joining the carry
                    double2 o01 = op[0], o23 = op[1];
                    double om[4] = {o01.x, o01.y, o23.x, o23.y};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (x0 + q >= A.nx) continue;
                        const double sm = __dadd_rn(om[q], Sd[q]);
                        const double bb = __dsub_rn(sm, om[q]);
                        const double er = __dadd_rn(__dsub_rn(om[q], __dsub_rn(sm, bb)), __dsub_rn(Sd[q], bb));
                        om[q] = sm;
                        P[q] = __fadd_rn(P[q], (float)er);
                    }
                    op[0] = make_double2(om[0], om[1]);
                    op[1] = make_double2(om[2], om[3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (x0 + q < A.nx) P[q] = __fadd_rn(P[q], (float)Sd[q]);
                    if (FOLD) {
                        double2 o01 = op[0], o23 = op[1];
                        double om[4] = {o01.x, o01.y, o23.x, o23.y};
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (x0 + q < A.nx) carry_fold(om[q], P[q]);
                        op[0] = make_double2(om[0], om[1]);
                        op[1] = make_double2(om[2], om[3]);
                    }
                }
                *cp = make_float4(P[0], P[1], P[2], P[3]);
            }
        }
        hm = hc;
        hc = hp;
        if (COMP) {
            lm = lc;
            lc = lp;
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(A.status, kStatusNonfinite);
}

}  // namespace

DamageConst damage_consts(const rfa_grid *g)
{
    DamageConst d;
    double c0 = std::log2(g->A * g->dt);
    double c1 = g->Ea / (g->R * std::log(2.0));
    double TK0 = g->T_a + 273.15;
    d.c0 = (float)c0;
    d.c1 = (float)c1;
    d.TK0 = (float)TK0;
    d.c0d = c0;
    d.c1d = c1;
    d.TK0d = TK0;
    return d;
}

cudaError_t launch_step_plain(rfa_grid *g, const void *th_in, const void *lo_in, void *th_out,
                              void *lo_out, bool damage, bool latch, bool fold)
{
    PlainArgs A;
    A.fold = fold ? 1 : 0;
    A.th_in = th_in;
    A.lo_in = lo_in;
    A.th_out = th_out;
    A.lo_out = lo_out;
    A.ab = g->ab;
    A.s = g->s;
    A.latch = g->latch;
    A.omega = g->omega;
    A.omega_c = g->omega_c;
    A.status = g->status;
    A.nx = g->nx;
    A.ny = g->ny;
    A.nz = g->nz;
    A.pitch = g->pitch;
    A.plane = g->plane;
    A.zchunk = choose_zchunk(g, 3);
    A.thr = g->T_thr - g->T_a;
    A.dc = damage_consts(g);
    dim3 blk(32, 8);
    dim3 grd = plain_grid_dims(g, A.zchunk);
#define PLAIN_CASE(SPV, PPV)                                                                       \
    if (g->sp == SPV && g->pp == PPV) {                                                           \
        if (damage && latch && fold) k_step_plain<SPV, PPV, true, true, true><<<grd, blk, 0, g->stream>>>(A);   \
        else if (damage && latch) k_step_plain<SPV, PPV, true, true, false><<<grd, blk, 0, g->stream>>>(A);     \
        else if (latch) k_step_plain<SPV, PPV, false, true, false><<<grd, blk, 0, g->stream>>>(A);              \
        else if (damage && fold) k_step_plain<SPV, PPV, true, false, true><<<grd, blk, 0, g->stream>>>(A);      \
        else if (damage) k_step_plain<SPV, PPV, true, false, false><<<grd, blk, 0, g->stream>>>(A);             \
        else k_step_plain<SPV, PPV, false, false, false><<<grd, blk, 0, g->stream>>>(A);                        \
    }
    PLAIN_CASE(RFA_STATE_F32, RFA_PARAM_BF16)
    PLAIN_CASE(RFA_STATE_F32, RFA_PARAM_F32)
    PLAIN_CASE(RFA_STATE_F32, RFA_PARAM_F64)
    PLAIN_CASE(RFA_STATE_F32C, RFA_PARAM_BF16)
    PLAIN_CASE(RFA_STATE_F32C, RFA_PARAM_F32)
    PLAIN_CASE(RFA_STATE_F32C, RFA_PARAM_F64)
    PLAIN_CASE(RFA_STATE_F64, RFA_PARAM_BF16)
    PLAIN_CASE(RFA_STATE_F64, RFA_PARAM_F32)
    PLAIN_CASE(RFA_STATE_F64, RFA_PARAM_F64)
#undef PLAIN_CASE
    return cudaGetLastError();
}

}  // namespace rfa
