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

template <int PP>
__device__ __forceinline__ void cond_ab(const void *ab, size_t i, double &a, double &b)
{
    if (PP == RFA_PARAM_BF16) {
        const uint32_t w = ((const uint32_t *)ab)[i];
        a = bf16_to_float(w & 0xffffu);
        b = bf16_to_float(w >> 16);
    } else if (PP == RFA_PARAM_F32) {
        const float2 v = ((const float2 *)ab)[i];
        a = v.x;
        b = v.y;
    } else {
        const double2 v = ((const double2 *)ab)[i];
        a = v.x;
        b = v.y;
    }
}

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
    int cond;   // 0: centre form (a_i * sum of differences), 1: harmonic face weights
    int alpha;  // perfusion weighted by 1 / max(1, Omega) of the step's start
};

template <int SP, int PP>
__global__ void __launch_bounds__(256) k_step_model(const CondArgs A)
{
    using T = typename std::conditional<SP == RFA_STATE_F64, double, float>::type;
    using W = typename std::conditional<PP == RFA_PARAM_F64, double, float>::type;
    __shared__ W wt[kCondLabels * kCondLabels];
    for (int k = threadIdx.y * blockDim.x + threadIdx.x; k < kCondLabels * kCondLabels; k += blockDim.x * blockDim.y)
        wt[k] = ((const W *)A.wpair)[k];
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= A.pitch || y >= A.ny) return;
    const size_t i = (size_t)z * A.plane + (size_t)y * A.pitch + x;
    const T *hin = (const T *)A.th_in;
    T *hout = (T *)A.th_out;
    if (x >= A.nx) {  // row padding stays zero
        hout[i] = T(0);
        if (SP == RFA_STATE_F32C) A.lo_out[i] = 0.f;
        return;
    }
    double ad, bd;
    cond_ab<PP>(A.ab, i, ad, bd);
    const T c = hin[i];  // (ad, bd: the voxel's a and b as stored)
    const float cl = SP == RFA_STATE_F32C ? A.lo_in[i] : 0.f;
    T nh = c;
    float nl = cl;
    if (ad != 0.0) {
        const int l = A.label[i];
        const W *wl = wt + l * kCondLabels;
        // neighbours in the fixed order x-, x+, y-, y+, z-, z+
        const bool in[6] = {x > 0, x + 1 < A.nx, y > 0, y + 1 < A.ny, z > 0, z + 1 < A.nz};
        const long long off[6] = {-1, 1, -(long long)A.pitch, (long long)A.pitch, -(long long)A.plane,
                                  (long long)A.plane};
        const T sv = ((const T *)A.s)[i];
        if (A.alpha) {  // tissue state: alpha = 1 / max(1, Omega) with Omega before this step
            const double om = A.omega[i] + (double)A.omega_c[i];
            if (om > 1.0) bd = bd / om;
        }
        if (!A.cond) {
            // centre form: the one-step kernel's operations (bit-identical to it when alpha = 1)
            if (SP == RFA_STATE_F32C) {
                float S = 0.f;
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    const size_t j = (size_t)((long long)i + (in[d] ? off[d] : 0));
                    S = acc(S, in[d] ? cdiff((float)hin[j], A.lo_in[j], (float)c, cl) : 0.f);
                }
                float h2, l2;
                cupdate((float)c, cl, S, (float)ad, (float)bd, (float)sv, h2, l2);
                nh = (T)h2;
                nl = l2;
            } else {
                T S = T(0);
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    const size_t j = (size_t)((long long)i + (in[d] ? off[d] : 0));
                    S = acc(S, in[d] ? pdiff(hin[j], c) : T(0));
                }
                nh = pupdate(c, S, (T)ad, (T)bd, sv);
            }
        } else if (SP == RFA_STATE_F32C) {
            const float th = __fadd_rn((float)c, cl);
            float delta = __fmaf_rn(-(float)bd, th, (float)sv);
#pragma unroll
            for (int d = 0; d < 6; ++d)
                if (in[d]) {
                    const size_t j = (size_t)((long long)i + off[d]);
                    const float w = (float)wl[A.label[j]];
                    delta = __fmaf_rn(w, cdiff((float)hin[j], A.lo_in[j], (float)c, cl), delta);
                }
            float h2, l2;
            cadd((float)c, cl, delta, h2, l2);
            nh = (T)h2;
            nl = l2;
        } else {
            T delta;
            if (SP == RFA_STATE_F64) delta = (T)__fma_rn(-bd, (double)c, (double)sv);
            else delta = (T)__fmaf_rn(-(float)bd, (float)c, (float)sv);
#pragma unroll
            for (int d = 0; d < 6; ++d)
                if (in[d]) {
                    const size_t j = (size_t)((long long)i + off[d]);
                    const T w = (T)wl[A.label[j]];
                    if (SP == RFA_STATE_F64) delta = (T)__fma_rn((double)w, __dsub_rn((double)hin[j], (double)c), (double)delta);
                    else delta = (T)__fmaf_rn((float)w, __fsub_rn((float)hin[j], (float)c), (float)delta);
                }
            nh = SP == RFA_STATE_F64 ? (T)__dadd_rn((double)c, (double)delta) : (T)__fadd_rn((float)c, (float)delta);
        }
    }
    hout[i] = nh;
    if (SP == RFA_STATE_F32C) A.lo_out[i] = nl;
    if (!isfinite((double)nh)) atomicOr(A.status, kStatusNonfinite);
    if (A.latch_on && nh + (T)nl >= (T)A.thr) A.latch[i] = 1;
    if (A.damage) {
        if (SP == RFA_STATE_F64) {
            const double inc = exp2(A.dc.c0d - A.dc.c1d / ((double)nh + A.dc.TK0d));
            const double om = A.omega[i];
            const double sm = __dadd_rn(om, inc);
            const double bb = __dsub_rn(sm, om);
            const double er = __dadd_rn(__dsub_rn(om, __dsub_rn(sm, bb)), __dsub_rn(inc, bb));
            A.omega[i] = sm;
            A.omega_c[i] = __fadd_rn(A.omega_c[i], (float)er);
        } else {
            float P = __fadd_rn(A.omega_c[i], arrhenius_inc(__fadd_rn((float)nh, nl), A.dc.c0, A.dc.c1, A.dc.TK0));
            if (A.fold) {
                double om = A.omega[i];
                carry_fold(om, P);
                A.omega[i] = om;
            }
            A.omega_c[i] = P;
        }
    }
}

struct CondAdjArgs {
    const float *lam_in, *th;
    float *lam_out, *Lam;
    const void *ab;
    const uint8_t *label;
    const float *wpair, *dA, *dB;  // [kCondLabels][kCondLabels]: w, dw/dK_l, dw/dK_m
    float gw[kCondLabels];         // d b / d w_b of each label
    int nx, ny, nz, pitch;
    size_t plane;
    double *acc;                   // [0..7] dL/dK, [8..15] dL/dw_b
};

template <int PP>
__global__ void __launch_bounds__(256) k_adjoint_cond(const CondAdjArgs A)
{
    __shared__ float wt[kCondLabels * kCondLabels], da[kCondLabels * kCondLabels], db[kCondLabels * kCondLabels];
    __shared__ float sK[kCondLabels], sW[kCondLabels];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
    for (int k = tid; k < kCondLabels * kCondLabels; k += nthr) {
        wt[k] = A.wpair[k];
        da[k] = A.dA[k];
        db[k] = A.dB[k];
    }
    if (tid < kCondLabels) sK[tid] = sW[tid] = 0.f;
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x < A.pitch && y < A.ny) {
        const size_t j = (size_t)z * A.plane + (size_t)y * A.pitch + x;
        if (x >= A.nx) {
            A.lam_out[j] = 0.f;
        } else {
            double ad, bd;
            cond_ab<PP>(A.ab, j, ad, bd);
            const bool free_j = ad != 0.0;
            const int lj = A.label[j];
            const float lam = A.lam_in[j], tj = A.th[j];
            const bool in[6] = {x > 0, x + 1 < A.nx, y > 0, y + 1 < A.ny, z > 0, z + 1 < A.nz};
            const long long off[6] = {-1, 1, -(long long)A.pitch, (long long)A.pitch, -(long long)A.plane,
                                      (long long)A.plane};
            float diag = 1.f, nsum = 0.f, gk_own = 0.f;
            if (free_j) diag = 1.f - (float)bd;
#pragma unroll
            for (int d = 0; d < 6; ++d)
                if (in[d]) {
                    const size_t i = (size_t)((long long)j + off[d]);
                    const int li = A.label[i];
                    double ai, bi;
                    cond_ab<PP>(A.ab, i, ai, bi);
                    if (ai != 0.0) nsum += wt[li * kCondLabels + lj] * A.lam_in[i];  // row i of A holds w(l_i, l_j)
                    if (free_j) {
                        diag -= wt[lj * kCondLabels + li];
                        const float v = lam * (A.th[i] - tj);
                        gk_own += da[lj * kCondLabels + li] * v;
                        if (li == lj) gk_own += db[lj * kCondLabels + li] * v;
                        else atomicAdd(&sK[li], db[lj * kCondLabels + li] * v);
                    }
                }
            A.lam_out[j] = diag * lam + nsum;
            A.Lam[j] += lam;
            if (free_j) {
                atomicAdd(&sK[lj], gk_own);
                atomicAdd(&sW[lj], lam * tj);
            }
        }
    }
    __syncthreads();
    if (tid < 8) {  // the backward pass admits at most 8 labels (acc: [0..7] K, [8..15] w_b)
        if (sK[tid] != 0.f) atomicAdd(&A.acc[tid], (double)sK[tid]);
        if (sW[tid] != 0.f) atomicAdd(&A.acc[8 + tid], -(double)sW[tid] * (double)A.gw[tid]);
    }
}

dim3 cond_grid(const rfa_grid *g) { return dim3((unsigned)((g->pitch + 31) / 32), (unsigned)((g->ny + 7) / 8), (unsigned)g->nz); }

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
    const dim3 blk(32, 8), grd = cond_grid(g);
#define COND_CASE(SPV, PPV) \
    if (g->sp == SPV && g->pp == PPV) k_step_model<SPV, PPV><<<grd, blk, 0, g->stream>>>(A);
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
    const dim3 blk(32, 8), grd = cond_grid(g);
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
    if (mode == RFA_COND_HARMONIC && g->have_tissue) {
        const rfa_status st = cond_build_tables(g, g->table.data(), g->n_labels);
        if (st != RFA_OK) return st;
    }
    if (mode != g->cond && g->steps > 0) g->rec.valid = false;  // the recorded steps used the other form
    g->cond = mode;
    return RFA_OK;
}
