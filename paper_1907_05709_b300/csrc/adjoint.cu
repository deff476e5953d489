// adjoint.cu -- sqrt(N) checkpoint recording and the discrete adjoint of the
// explicit step (the paper has no adjoint; this differentiates the scheme of
// Eq. CUDAbioheat3d as implemented by the forward kernels).
//
// Forward step (free voxel i):  theta'_i = theta_i + a_i sum_nb (theta_j - theta_i) - b_i theta_i + s_i
// Its transpose applied to lambda, with mu = a * lambda (a = b = 0 on fixed voxels):
//     (A^T lambda)_i = lambda_i + sum_nb (mu_j - mu_i) - b_i lambda_i
// Gradients over the recorded steps n = 0..N-1 (lambda^{n+1} = dL/dtheta^{n+1}):
//     dL/dK_l   = sum_n sum_{i in l, free} lambda^{n+1}_i * dt/(rho c_l h^2) * (L theta^n)_i
//     dL/dw_b,l = -sum_n sum_{i in l, free} lambda^{n+1}_i * rho_b c_b dt/(rho c_l) * theta^n_i
//     Lambda_i  = sum_{n=1..N} lambda^n_i,  then with s_i = c_i w_i / W, c_i = P dt/(h^3 rho c_i):
//     dL/dP     = sum_i Lambda_i c_i w_i / (P W)
//     dL/dtip   = sum_i Lambda_i c_i dw_i / W - (dW / W^2) sum_i Lambda_i c_i w_i
// with dw_i/dtip = 4 d_i^-6 (x_i - p*_i) outside the clamp radius (every
// segment moves rigidly with the tip) and W = sum_free w, dW = sum_free dw.
//
// Lambda is accumulated once per pair of reverse steps (the second step of a
// pair adds both inputs; the first input is still in its ping-pong buffer when
// the second step reads it), which halves its read-modify-write traffic.
//
// Trajectory: checkpoints (hi, lo) every ceil(sqrt(N)) steps are taken while
// rfa_step records; the backward pass replays each segment -- two steps per
// launch with the blocked kernel in replay mode, which also stores the
// intermediate state, else one step per launch (both bit-identical to the
// forward kernels) -- writing the hi part of every state straight into a
// segment buffer, then runs the adjoint steps of the segment in reverse.
#include "rfa_internal.cuh"

#include <cmath>
#include <vector>

namespace rfa {

// ------------------------------------------------------------------ recording
void record_reset(rfa_grid *g)
{
    g->rec.used = 0;
    g->rec.valid = false;
    g->rec.seg = 0;
    g->rec.nsteps = 0;
}

void record_free(rfa_grid *g)
{
    for (void *p : g->rec.ck_hi) cudaFree(p);
    for (void *p : g->rec.ck_lo)
        if (p) cudaFree(p);
    g->rec.ck_hi.clear();
    g->rec.ck_lo.clear();
    record_reset(g);
}

rfa_status record_begin(rfa_grid *g, int64_t nsteps)
{
    record_reset(g);
    g->rec.seg = (int64_t)std::ceil(std::sqrt((double)nsteps));
    if (g->rec.seg < 1) g->rec.seg = 1;
    g->rec.valid = true;
    return RFA_OK;
}

rfa_status record_checkpoint(rfa_grid *g, int64_t step_index)
{
    (void)step_index;
    const size_t bytes = g->nvp * g->state_elem();
    if (g->rec.used == g->rec.ck_hi.size()) {  // the pool grows by one
        void *hi = nullptr, *lo = nullptr;
        if (cudaMalloc(&hi, bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("checkpoint allocation failed");
            return RFA_E_OOM;
        }
        if (g->sp == RFA_STATE_F32C && cudaMalloc(&lo, g->nvp * 4) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(hi);
            set_error("checkpoint allocation failed");
            return RFA_E_OOM;
        }
        g->rec.ck_hi.push_back(hi);
        g->rec.ck_lo.push_back(lo);
    }
    void *hi = g->rec.ck_hi[g->rec.used], *lo = g->rec.ck_lo[g->rec.used];
    RFA_CUDA(cudaMemcpyAsync(hi, g->th[g->cur], bytes, cudaMemcpyDeviceToDevice, g->stream));
    if (lo) RFA_CUDA(cudaMemcpyAsync(lo, g->lo[g->cur], g->nvp * 4, cudaMemcpyDeviceToDevice, g->stream));
    ++g->rec.used;
    return RFA_OK;
}

namespace {

constexpr int kMaxGradLabels = 8;

struct AdjArgs {
    const float *lam_in, *th;
    float *lam_out, *Lam;
    const void *ab;
    const uint8_t *label;
    const LabelCoef *tab;
    int nx, ny, nz, pitch, zchunk, face;
    // Lambda update of this step: 0 none, 1 Lambda += lambda_in + lambda_prev (the
    // previous step's input, still in lam_out until this step overwrites it), 2
    // Lambda += lambda_in.  Pairing the steps halves Lambda's read-modify-write.
    int lam_mode;
    size_t plane;
    float fk[kMaxGradLabels], gw[kMaxGradLabels];
    double *acc;  // [2 * kMaxGradLabels]: sum lambda f L(theta), -sum lambda g theta
    unsigned *status;  // the grid's status word (index checks of the checked build)
};

template <int PP>
__device__ __forceinline__ void adj_load_ab(const void *ab, size_t i, float a[4], float b[4])
{
    if (PP == RFA_PARAM_BF16) {
        uint4 u = __ldg(reinterpret_cast<const uint4 *>((const uint32_t *)ab + i));
        uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a[q] = bf16_to_float(w[q] & 0xffffu);
            b[q] = bf16_to_float(w[q] >> 16);
        }
    } else if (PP == RFA_PARAM_F32) {
        const float4 *p = reinterpret_cast<const float4 *>((const float2 *)ab + i);
        float4 u = __ldg(p), v = __ldg(p + 1);
        a[0] = u.x; b[0] = u.y; a[1] = u.z; b[1] = u.w;
        a[2] = v.x; b[2] = v.y; a[3] = v.z; b[3] = v.w;
    } else {
        const double2 *p = (const double2 *)ab + i;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double2 t = __ldg(p + q);
            a[q] = (float)t.x;
            b[q] = (float)t.y;
        }
    }
}

__device__ __forceinline__ float4 ld4g(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
// the cache line holding p into L2 (no register is written): a thread streaming z
// asks for its fields two planes ahead, so their HBM latency overlaps the planes
// in between
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// the coefficient a of one voxel
template <int PP>
__device__ __forceinline__ float adj_load_a1(const void *ab, size_t i)
{
    if (PP == RFA_PARAM_BF16) return bf16_to_float(__ldg((const uint32_t *)ab + i) & 0xffffu);
    if (PP == RFA_PARAM_F32) return __ldg((const float2 *)ab + i).x;
    return (float)__ldg((const double2 *)ab + i).x;
}

// one adjoint step: lam_out = A^T lam_in, Lam += lam_in, per-label contractions.
// Every lane of a row takes part in every quad load, with no branch and no zero fill:
// a lane past the row's end reads the row's last quad and stores nothing, and a
// neighbour outside the grid is read at the voxel's own place and dropped by the
// in-grid flags.
template <int PP, int NL>
__global__ void __launch_bounds__(256, 2) k_adjoint_step(const AdjArgs A)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    float accK[NL], accW[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) accK[l] = accW[l] = 0.f;
    float runK = 0.f, runW = 0.f;  // open run of quads of label run_lab (255: none)
    unsigned run_lab = 255u;
    const bool wvalid = y < A.ny;  // warp-uniform (blockDim.x == 32)
    const int x0 = 4 * (blockIdx.x * 32 + lane);
    const bool inrow = wvalid && x0 < A.pitch;
    const int xq = x0 < A.pitch ? x0 : A.pitch - 4;
    const int zb = blockIdx.z * A.zchunk;
    const int ze = min(A.nz, zb + A.zchunk);
    const size_t rowoff = (size_t)(wvalid ? y : 0) * A.pitch + xq;
    const bool hasYm = y > 0, hasYp = y < A.ny - 1;
    const size_t dym = hasYm ? (size_t)A.pitch : 0, dyp = hasYp ? (size_t)A.pitch : 0;
    // lane 0 reads the voxel left of its quad and lane 31 the one right of it (those
    // two lanes alone: the same loads from every lane made the step 3.5 % slower);
    // the other lanes take theirs from their neighbours by shuffles
    const ptrdiff_t dxe = lane == 0 ? (x0 > 0 && xq > 0 ? -1 : 0) : (lane == 31 && x0 + 4 < A.nx ? 4 : 0);

    if (wvalid) {
        float4 lm, lc, lp, tm, tc, tp;                            // lambda and theta at z-1, z, z+1
        float am[4], ac[4], ap[4], bc[4], bp[4], bdum[4];
        bool run = true;
        {
            const size_t ic = (size_t)zb * A.plane + rowoff, im = zb > 0 ? ic - A.plane : ic;
#ifdef RFA_CHECK
            // checked build: the warp skips its chunk when any lane's range falls outside
            run = __all_sync(FULL, RFA_CHECK_RANGE(im, ic + 4, A.plane * A.nz, ic, 4, A.status));
#endif
            if (run) {
                lm = ld4g(A.lam_in + im);
                tm = ld4g(A.th + im);
                adj_load_ab<PP>(A.ab, im, am, bdum);
                lc = ld4g(A.lam_in + ic);
                tc = ld4g(A.th + ic);
                adj_load_ab<PP>(A.ab, ic, ac, bc);
            }
        }
        for (int z = zb; run && z < ze; ++z) {
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
                prefetch_l2(A.lam_in + iq);
                prefetch_l2(A.th + iq);
                prefetch_l2((const char *)A.ab + iq * (PP == RFA_PARAM_BF16 ? 4 : PP == RFA_PARAM_F32 ? 8 : 16));
                if (A.lam_mode != 0) prefetch_l2(A.Lam + iq);
                if (A.lam_mode == 1) prefetch_l2(A.lam_out + iq);
            }
            lp = ld4g(A.lam_in + ip);
            tp = ld4g(A.th + ip);
            adj_load_ab<PP>(A.ab, ip, ap, bp);
            const float4 lym = ld4g(A.lam_in + i - dym), tym = ld4g(A.th + i - dym);
            const float4 lyp = ld4g(A.lam_in + i + dyp), typ = ld4g(A.th + i + dyp);
            float aym[4], ayp[4];
            adj_load_ab<PP>(A.ab, i - dym, aym, bdum);
            adj_load_ab<PP>(A.ab, i + dyp, ayp, bdum);
            const uint32_t lab4 = __ldg(reinterpret_cast<const uint32_t *>(A.label + i));
            float4 Lc = make_float4(0, 0, 0, 0), Lp = Lc;
            if (A.lam_mode != 0) Lc = *reinterpret_cast<const float4 *>(A.Lam + i);
            if (A.lam_mode == 1) Lp = *reinterpret_cast<const float4 *>(A.lam_out + i);
            float ae = 0.f, le = 0.f, te = 0.f;
            if (lane == 0 || lane == 31) {
                ae = adj_load_a1<PP>(A.ab, i + dxe);
                le = __ldg(A.lam_in + i + dxe);
                te = __ldg(A.th + i + dxe);
            }
            const float lcv[4] = {lc.x, lc.y, lc.z, lc.w}, tcv[4] = {tc.x, tc.y, tc.z, tc.w};
            const float lmv[4] = {lm.x, lm.y, lm.z, lm.w}, tmv[4] = {tm.x, tm.y, tm.z, tm.w};
            const float lpv[4] = {lp.x, lp.y, lp.z, lp.w}, tpv[4] = {tp.x, tp.y, tp.z, tp.w};
            const float lymv[4] = {lym.x, lym.y, lym.z, lym.w}, tymv[4] = {tym.x, tym.y, tym.z, tym.w};
            const float lypv[4] = {lyp.x, lyp.y, lyp.z, lyp.w}, typv[4] = {typ.x, typ.y, typ.z, typ.w};
            float mu[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) mu[q] = ac[q] * lcv[q];
            // x neighbours across quads: mu and theta
            float muL = __shfl_up_sync(FULL, mu[3], 1), muR = __shfl_down_sync(FULL, mu[0], 1);
            float thL = __shfl_up_sync(FULL, tcv[3], 1), thR = __shfl_down_sync(FULL, tcv[0], 1);
            if (lane == 0) {
                muL = ae * le;
                thL = te;
            }
            if (lane == 31) {
                muR = ae * le;
                thR = te;
            }
            if (inrow) {
                float lo_[4], Lo_[4], vk4[4], vw4[4];
                const float Lcv[4] = {Lc.x, Lc.y, Lc.z, Lc.w}, Lpv[4] = {Lp.x, Lp.y, Lp.z, Lp.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int x = x0 + q;
                    const float l = lcv[q], t = tcv[q], m = mu[q];
                    const float muxm = q == 0 ? muL : mu[q - 1], muxp = q == 3 ? muR : mu[q + 1];
                    const float txm = q == 0 ? thL : tcv[q - 1], txp = q == 3 ? thR : tcv[q + 1];
                    float smu = 0.f, lt = 0.f;
                    if (x > 0) { smu += muxm - m; lt += txm - t; }
                    if (x + 1 < A.nx) { smu += muxp - m; lt += txp - t; }
                    if (hasYm) { smu += aym[q] * lymv[q] - m; lt += tymv[q] - t; }
                    if (hasYp) { smu += ayp[q] * lypv[q] - m; lt += typv[q] - t; }
                    if (hasZm) { smu += am[q] * lmv[q] - m; lt += tmv[q] - t; }
                    if (hasZp) { smu += ap[q] * lpv[q] - m; lt += tpv[q] - t; }
                    const bool valid = x < A.nx;
                    lo_[q] = valid ? l + smu - bc[q] * l : 0.f;
                    Lo_[q] = valid ? Lcv[q] + (A.lam_mode == 1 ? Lpv[q] + l : l) : 0.f;
                    // free voxels are exactly those with a > 0 (fixed labels and Dirichlet
                    // faces carry a = 0; every tissue has K > 0)
                    const bool free_vox = valid && ac[q] > 0.f;
                    vk4[q] = free_vox ? l * lt : 0.f;
                    vw4[q] = free_vox ? l * t : 0.f;
                }
                // per-label sums: a run of quads of one label adds into (runK, runW);
                // other quads flush the run and go voxel by voxel
                if (lab4 == run_lab * 0x01010101u) {
                    runK += (vk4[0] + vk4[1]) + (vk4[2] + vk4[3]);
                    runW += (vw4[0] + vw4[1]) + (vw4[2] + vw4[3]);
                } else {
#pragma unroll
                    for (int L = 0; L < NL; ++L) {
                        accK[L] += run_lab == (unsigned)L ? runK : 0.f;
                        accW[L] += run_lab == (unsigned)L ? runW : 0.f;
                    }
                    runK = runW = 0.f;
                    run_lab = 255u;
                    if (lab4 == (lab4 & 0xffu) * 0x01010101u) {
                        run_lab = lab4 & 0xffu;
                        runK = (vk4[0] + vk4[1]) + (vk4[2] + vk4[3]);
                        runW = (vw4[0] + vw4[1]) + (vw4[2] + vw4[3]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const unsigned lab = (lab4 >> (8 * q)) & 0xffu;
#pragma unroll
                            for (int L = 0; L < NL; ++L) {
                                accK[L] += lab == (unsigned)L ? vk4[q] : 0.f;
                                accW[L] += lab == (unsigned)L ? vw4[q] : 0.f;
                            }
                        }
                    }
                }
                *reinterpret_cast<float4 *>(A.lam_out + i) = make_float4(lo_[0], lo_[1], lo_[2], lo_[3]);
                if (A.lam_mode != 0)
                    *reinterpret_cast<float4 *>(A.Lam + i) = make_float4(Lo_[0], Lo_[1], Lo_[2], Lo_[3]);
            }
            lm = lc; lc = lp; tm = tc; tc = tp;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                am[q] = ac[q];
                ac[q] = ap[q];
                bc[q] = bp[q];
            }
        }
    }
#pragma unroll
    for (int L = 0; L < NL; ++L) {  // close the last run
        accK[L] += run_lab == (unsigned)L ? runK : 0.f;
        accW[L] += run_lab == (unsigned)L ? runW : 0.f;
    }
    // block reduction of the per-label sums, then one FP64 atomic per label and block
    __shared__ float sK[8][NL], sW[8][NL];
    const int w = threadIdx.y;
#pragma unroll
    for (int L = 0; L < NL; ++L) {
        float k = accK[L] * A.fk[L], v = accW[L] * A.gw[L];
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
        if (v != 0.0) atomicAdd(&A.acc[kMaxGradLabels + lane], -v);
    }
}

// padded lambda^N from the caller's dense dL/dT; zero Lambda
__global__ void k_adj_init(const float *dLdT, float *lam, float *Lam, int nx, int ny, int nz, int pitch)
{
    size_t nvp = (size_t)pitch * ny * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nvp; i += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(i % pitch);
        size_t r = i / pitch;
        lam[i] = x < nx ? dLdT[r * nx + x] : 0.f;
        Lam[i] = 0.f;
    }
}

__device__ double adj_needle_distance(const NeedleGeom &g, double px, double py, double pz, double q[3])
{
    double best = 1e300;
    for (int k = 0; k < g.nseg; ++k) {
        const Segment &sg = g.seg[k];
        double ux = sg.p1[0] - sg.p0[0], uy = sg.p1[1] - sg.p0[1], uz = sg.p1[2] - sg.p0[2];
        double wx = px - sg.p0[0], wy = py - sg.p0[1], wz = pz - sg.p0[2];
        double uu = ux * ux + uy * uy + uz * uz;
        double t = uu > 0.0 ? (wx * ux + wy * uy + wz * uz) / uu : 0.0;
        t = fmin(fmax(t, 0.0), 1.0);
        double cx = sg.p0[0] + t * ux, cy = sg.p0[1] + t * uy, cz = sg.p0[2] + t * uz;
        double d2 = (px - cx) * (px - cx) + (py - cy) * (py - cy) + (pz - cz) * (pz - cz);
        if (d2 < best) {
            best = d2;
            q[0] = cx;
            q[1] = cy;
            q[2] = cz;
        }
    }
    return sqrt(best);
}

// partial sums over free voxels: [W, dW(3), sum Lam c w, sum Lam c dw(3)]
__global__ void k_src_grad_partials(NeedleGeom geom, const float *Lam, const uint8_t *label,
                                    const LabelCoef *tab, int nx, int ny, int nz, int pitch, double h,
                                    double dt, int face, double *part)
{
    size_t nvp = (size_t)pitch * ny * nz;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nvp; i += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(i % pitch);
        if (x >= nx) continue;
        size_t r = i / pitch;
        int y = (int)(r % ny), z = (int)(r / ny);
        bool face_vox = (x == 0 || y == 0 || z == 0 || x == nx - 1 || y == ny - 1 || z == nz - 1);
        const LabelCoef t = tab[label[i]];
        if (t.fixed || (face == RFA_FACE_DIRICHLET && face_vox)) continue;
        double p[3] = {x * h, y * h, z * h}, q[3] = {0, 0, 0};
        double d = adj_needle_distance(geom, p[0], p[1], p[2], q);
        double rr = fmax(d, geom.r0);
        double w = 1.0 / (rr * rr * rr * rr);
        double dw[3] = {0, 0, 0};
        if (d > geom.r0) {
            double d6 = d * d * d * d * d * d;
            for (int c = 0; c < 3; ++c) dw[c] = 4.0 * (p[c] - q[c]) / d6;
        }
        double cL = (double)Lam[i] * geom.P * dt / (h * h * h * t.rho * t.c);
        acc[0] += w;
        for (int c = 0; c < 3; ++c) acc[1 + c] += dw[c];
        acc[4] += cL * w;
        for (int c = 0; c < 3; ++c) acc[5 + c] += cL * dw[c];
    }
    __shared__ double sh[8][8];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = 0; k < 8; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double v = 0.0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) v += sh[j][threadIdx.x];
        part[(size_t)blockIdx.x * 8 + threadIdx.x] = v;
    }
}

__global__ void k_src_grad_final(const double *part, int nblocks, double *out)
{
    if (threadIdx.x < 8) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += part[(size_t)b * 8 + threadIdx.x];
        out[threadIdx.x] = v;
    }
}

cudaError_t launch_adjoint_step(rfa_grid *g, const AdjArgs &A0, const float *lam_in, float *lam_out,
                                const float *th, int lam_mode)
{
    AdjArgs A = A0;
    A.lam_in = lam_in;
    A.lam_out = lam_out;
    A.th = th;
    A.lam_mode = lam_mode;
    dim3 blk(32, 8);
    dim3 grd = plain_grid_dims(g, A.zchunk);
    const bool few = g->n_labels <= 4;
    if (g->pp == RFA_PARAM_BF16) {
        if (few) k_adjoint_step<RFA_PARAM_BF16, 4><<<grd, blk, 0, g->stream>>>(A);
        else k_adjoint_step<RFA_PARAM_BF16, 8><<<grd, blk, 0, g->stream>>>(A);
    } else if (g->pp == RFA_PARAM_F32) {
        if (few) k_adjoint_step<RFA_PARAM_F32, 4><<<grd, blk, 0, g->stream>>>(A);
        else k_adjoint_step<RFA_PARAM_F32, 8><<<grd, blk, 0, g->stream>>>(A);
    } else {
        if (few) k_adjoint_step<RFA_PARAM_F64, 4><<<grd, blk, 0, g->stream>>>(A);
        else k_adjoint_step<RFA_PARAM_F64, 8><<<grd, blk, 0, g->stream>>>(A);
    }
    return cudaGetLastError();
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

}  // namespace

rfa_status read_status(rfa_grid *g);  // runtime.cu: the grid's status word, after a synchronize

rfa_status backward_impl(rfa_grid *g, const float *dLdT, double *grads)
{
    if (g->sp == RFA_STATE_F64) {
        set_error("rfa_backward supports FP32 and compensated FP32 states");
        return RFA_E_UNSUPPORTED;
    }
    if (!g->have_tissue || !g->rec.valid || g->rec.nsteps != g->steps || g->rec.used == 0) {
        set_error("rfa_backward needs every step since rfa_set_tissue recorded (rfa_step(..., 1))");
        return RFA_E_STATE;
    }
    if (g->src_mode != 0) {
        set_error("rfa_backward supports the max(d, r0)^-4 needle source only");
        return RFA_E_UNSUPPORTED;
    }
    if (g->alpha_perf) {
        set_error("rfa_backward does not differentiate the tissue-state perfusion coupling");
        return RFA_E_UNSUPPORTED;
    }
    if (g->tip_on) {
        set_error("rfa_backward does not differentiate a FIXED_TIP needle (no RF source)");
        return RFA_E_UNSUPPORTED;
    }
    if (g->n_labels > kMaxGradLabels) {
        set_error("rfa_backward supports at most 8 labels");
        return RFA_E_UNSUPPORTED;
    }
    const int64_t N = g->rec.nsteps, seg = g->rec.seg;
    const size_t nvp = g->nvp;
    DevBuf segbuf, lob, lam, Lam, acc, part;
    const size_t seg_bytes = (size_t)seg * nvp * 4;
    if (cudaMalloc(&segbuf.p, seg_bytes) != cudaSuccess || cudaMalloc(&lob.p, 2 * nvp * 4) != cudaSuccess ||
        cudaMalloc(&lam.p, 2 * nvp * 4) != cudaSuccess || cudaMalloc(&Lam.p, nvp * 4) != cudaSuccess ||
        cudaMalloc(&acc.p, 64 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&part.p, (size_t)kReduceBlocks * 8 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        set_error("backward workspace allocation failed");
        return RFA_E_OOM;
    }
    float *sb = (float *)segbuf.p, *lo2 = (float *)lob.p, *lam2 = (float *)lam.p;
    double *accd = (double *)acc.p;
    RFA_CUDA(cudaMemsetAsync(accd, 0, 64 * sizeof(double), g->stream));
    k_adj_init<<<148 * 8, 256, 0, g->stream>>>(dLdT, lam2, (float *)Lam.p, g->nx, g->ny, g->nz, g->pitch);
    RFA_CUDA(cudaGetLastError());

    AdjArgs A{};
    A.Lam = (float *)Lam.p;
    A.ab = g->ab;
    A.label = g->label;
    A.tab = g->d_table;
    A.nx = g->nx;
    A.ny = g->ny;
    A.nz = g->nz;
    A.pitch = g->pitch;
    A.plane = g->plane;
    A.zchunk = choose_zchunk_waves(g, 2);
    A.face = g->face;
    A.acc = accd;
    A.status = g->status;
    for (int l = 0; l < kMaxGradLabels; ++l) {
        A.fk[l] = A.gw[l] = 0.f;
        if (l < g->n_labels && !g->table[l].fixed) {
            const rfa_tissue &t = g->table[l];
            A.fk[l] = (float)((1.0 / (t.rho * t.c)) * g->dt / (g->h * g->h));
            A.gw[l] = (float)((t.rho_b * t.c_b / (t.rho * t.c)) * g->dt);
        }
    }
    // replay schedule: the depth-2 blocked kernel (the grid's tile if it runs depth 2)
    int replay_variant = -1;
    if (g->sched.tb_depth == 2 && tb_supported(g, 2, g->sched.tile_variant)) replay_variant = g->sched.tile_variant;
    else if (tb_supported(g, 2, 0)) replay_variant = 0;
    int lcur = 0;  // lambda ping-pong index holding lambda^{n+1}
    int64_t kadj = 0;  // adjoint steps done (the centre form pairs their Lambda updates)
    const int64_t nck = (int64_t)g->rec.used;
    for (int64_t c = nck - 1; c >= 0; --c) {
        const int64_t s0 = c * seg, s1 = (s0 + seg < N) ? s0 + seg : N;
        // recompute theta^{s0} .. theta^{s1-1}; hi parts land in the segment buffer
        RFA_CUDA(cudaMemcpyAsync(sb, g->rec.ck_hi[c], nvp * 4, cudaMemcpyDeviceToDevice, g->stream));
        if (g->sp == RFA_STATE_F32C)
            RFA_CUDA(cudaMemcpyAsync(lo2, g->rec.ck_lo[c], nvp * 4, cudaMemcpyDeviceToDevice, g->stream));
        // two steps per launch with the blocked kernel where it applies (it also
        // stores the intermediate state), the remainder one step at a time
        const int64_t nstate = s1 - s0;
        int64_t j = 0;
        int lc = 0;  // lo buffer of state j
        while (j + 1 < nstate) {
            const float *lin = g->sp == RFA_STATE_F32C ? lo2 + (size_t)lc * nvp : nullptr;
            float *lout = g->sp == RFA_STATE_F32C ? lo2 + (size_t)(lc ^ 1) * nvp : nullptr;
            if (replay_variant >= 0 && j + 2 < nstate) {
                RFA_CUDA(launch_step_tb_rec(g, 2, replay_variant, sb + (size_t)j * nvp, lin,
                                            sb + (size_t)(j + 2) * nvp, lout, sb + (size_t)(j + 1) * nvp));
                j += 2;
            } else if (g->cond == RFA_COND_HARMONIC) {
                RFA_CUDA(launch_step_model(g, sb + (size_t)j * nvp, lin, sb + (size_t)(j + 1) * nvp, lout, false,
                                          false, false));
                j += 1;
            } else {
                RFA_CUDA(launch_step_plain(g, sb + (size_t)j * nvp, lin, sb + (size_t)(j + 1) * nvp, lout, false,
                                           false, false));
                j += 1;
            }
            lc ^= 1;
        }
        for (int64_t st = s1 - 1; st >= s0; --st) {
            const float *th = sb + (size_t)(st - s0) * nvp;
            if (g->cond == RFA_COND_HARMONIC)
                RFA_CUDA(launch_adjoint_cond(g, lam2 + (size_t)lcur * nvp, lam2 + (size_t)(lcur ^ 1) * nvp,
                                             (float *)Lam.p, th, accd));
            else
                RFA_CUDA(launch_adjoint_step(g, A, lam2 + (size_t)lcur * nvp, lam2 + (size_t)(lcur ^ 1) * nvp, th,
                                             (kadj & 1) ? 1 : (kadj == N - 1 ? 2 : 0)));
            lcur ^= 1;
            ++kadj;
        }
    }
    // source contractions
    k_src_grad_partials<<<kReduceBlocks, 256, 0, g->stream>>>(g->geom, (const float *)Lam.p, g->label,
                                                               g->d_table, g->nx, g->ny, g->nz, g->pitch,
                                                               g->h, g->dt, g->face, (double *)part.p);
    k_src_grad_final<<<1, 32, 0, g->stream>>>((const double *)part.p, kReduceBlocks, accd + 32);
    RFA_CUDA(cudaGetLastError());
    double host[64];
    RFA_CUDA(cudaMemcpyAsync(host, accd, sizeof host, cudaMemcpyDeviceToHost, g->stream));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    tb_forget_maps(g);  // tensor maps of the segment buffers, freed on return
    // a replay or reverse step that recorded a fault (a non-finite value, a timed-out
    // wait, an index check of the checked build) fails the call
    const rfa_status st = read_status(g);
    if (st != RFA_OK) return st;
    const double W = host[32], A1 = host[36];
    const double *dW = host + 33, *A2 = host + 37;
    const double P = g->geom.P;
    grads[0] = (W > 0.0 && P > 0.0) ? A1 / (P * W) : 0.0;
    for (int c = 0; c < 3; ++c) grads[1 + c] = W > 0.0 ? A2[c] / W - dW[c] * A1 / (W * W) : 0.0;
    for (int l = 0; l < g->n_labels; ++l) {
        grads[4 + l] = host[l];
        grads[4 + g->n_labels + l] = host[kMaxGradLabels + l];
    }
    return RFA_OK;
}

}  // namespace rfa

extern "C" rfa_status rfa_backward(rfa_grid *g, const float *dLdT_final_dev, double *grads)
{
    if (!g || !dLdT_final_dev || !grads) {
        rfa::set_error("null argument");
        return RFA_E_INVALID;
    }
    return rfa::backward_impl(g, dLdT_final_dev, grads);
}
