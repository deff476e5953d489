// kernels_setup.cu -- tissue set-up and RF source placement (run once per
// set-up / needle placement).
//
// Tissue set-up follows Sec. "Implementation": the segmented label image is
// turned into the start temperature image; vessel (fixed) labels keep their
// temperature (Eq. 2675-eq6 and Alg. 1's else-branch).  Per voxel the update
// coefficients of Eq. CUDAbioheat3d divided by rho c_p are formed in FP64 and
// rounded once to the storage precision.
//
// The RF source: the paper gives the resistive heating sigma |grad V|^2 of Eq.
// 2675-eq1_Linte only symbolically; around an electrode |grad V|^2 falls off as
// 1/r^4, so q_i ~ max(d_i, r0)^-4 with d_i the distance to the nearest active
// needle segment, normalised so that sum_free q_i h^3 = P exactly.
#include "rfa_internal.cuh"

#include <algorithm>
#include <cmath>

namespace rfa {

namespace {

// rounded update coefficients of every free label (one thread per label)
__global__ void k_label_coef(LabelCoef *tab, int n_labels, double dt, double h, int pp)
{
    const int l = threadIdx.x;
    if (l >= n_labels) return;
    LabelCoef t = tab[l];
    t.a = t.fixed ? 0.0 : round_coef(coef_a(t, dt, h), pp);
    t.b = t.fixed ? 0.0 : round_coef(coef_b(t, dt), pp);
    t.dt_rhoc = dt / (t.rho * t.c);
    tab[l] = t;
}

// Every value k_setup writes follows from the voxel's label (or is 0 on a
// Dirichlet face voxel of a free label), so each block first forms, per label,
// the stored coefficient pair and the start value (hi, and for compensated
// states the exact lo) with the per-voxel expressions, then a warp per grid row
// writes them (no per-voxel FP64 and no 64-bit index division).
template <int SP, int PP>
__global__ void __launch_bounds__(256) k_setup(const uint8_t *__restrict__ labels,
                                               const LabelCoef *__restrict__ tab, int nx, int ny, int nz,
                                               int pitch, double h, double dt, double T_a, int face, void *th0,
                                               void *th1, void *lo0, void *lo1, void *ab, void *s,
                                               uint8_t *label_pad, uint8_t *latch, double *omega,
                                               float *omega_c, int n_labels, unsigned *status)
{
    using T = typename std::conditional<SP == RFA_STATE_F64, double, float>::type;
    using AB = typename std::conditional<PP == RFA_PARAM_BF16, uint32_t,
                                         typename std::conditional<PP == RFA_PARAM_F32, float2, double2>::type>::type;
    __shared__ AB sab[256];
    __shared__ T sth[256];
    __shared__ float slo[256];
    __shared__ uint8_t sfixed[256];
    for (int l = threadIdx.x; l < n_labels; l += blockDim.x) {
        const LabelCoef t = tab[l];
        const double a = t.fixed ? 0.0 : t.a, b = t.fixed ? 0.0 : t.b;
        const double th = t.fixed ? t.T_fixed - T_a : 0.0;
        if (PP == RFA_PARAM_BF16) {
            *reinterpret_cast<uint32_t *>(&sab[l]) = (uint32_t)bf16_bits_rne(a) | ((uint32_t)bf16_bits_rne(b) << 16);
        } else if (PP == RFA_PARAM_F32) {
            *reinterpret_cast<float2 *>(&sab[l]) = make_float2((float)a, (float)b);
        } else {
            *reinterpret_cast<double2 *>(&sab[l]) = make_double2(a, b);
        }
        sth[l] = (T)th;
        // the pair (hi, lo) represents th exactly
        slo[l] = SP == RFA_STATE_F32C ? (float)(th - (double)(float)th) : 0.f;
        sfixed[l] = t.fixed ? 1 : 0;
    }
    __syncthreads();
    const AB zero_ab{};
    for (int row = blockIdx.x * 8 + (int)(threadIdx.x >> 5); row < ny * nz; row += gridDim.x * 8) {
        const int y = row % ny, z = row / ny;
        const bool face_row = y == 0 || z == 0 || y == ny - 1 || z == nz - 1;
        const size_t rb = (size_t)row * pitch;
        for (int x = threadIdx.x & 31; x < pitch; x += 32) {
            const size_t i = rb + x;
            AB abv = zero_ab;
            T th = T(0);
            float lo = 0.f;
            uint8_t l = 0;
            if (!RFA_CHECK_RANGE(i, i + 1, (size_t)pitch * ny * nz, 0, 1, status) ||
                (x < nx && !RFA_CHECK_RANGE((size_t)row * nx + x, (size_t)row * nx + x + 1, (size_t)nx * ny * nz, 0, 1,
                                            status)))
                continue;
            if (x < nx) {
                l = labels[(size_t)row * nx + x];
                if (l >= n_labels) {
                    atomicOr(status, kStatusBadLabel);
                    l = 0;
                }
                const bool face_vox = face_row || x == 0 || x == nx - 1;
                if (sfixed[l]) {
                    th = sth[l];
                    lo = slo[l];
                } else if (!(face == RFA_FACE_DIRICHLET && face_vox)) {
                    abv = sab[l];
                }
            }
            ((T *)th0)[i] = th;
            ((T *)th1)[i] = th;
            if (SP == RFA_STATE_F32C) {
                ((float *)lo0)[i] = lo;
                ((float *)lo1)[i] = lo;
            }
            ((AB *)ab)[i] = abv;
            ((T *)s)[i] = T(0);
            label_pad[i] = l;
            latch[i] = 0;
            omega[i] = 0.0;
            omega_c[i] = 0.0f;
        }
    }
}

// w = max(d, r0)^-4 = 1 / max(d^2, r0^2)^2
__device__ inline double needle_weight2(const NeedleGeom &g, double d2)
{
    double r2 = fmax(d2, g.r0 * g.r0);
    return 1.0 / (r2 * r2);
}

// block-wide FP64 sum; every thread gets the result
__device__ double block_sum(double v)
{
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// pass 1: per-block sums of w over free voxels
__global__ void k_source_sum(NeedleGeom geom, const uint8_t *__restrict__ label,
                             const LabelCoef *__restrict__ tab, int nx, int ny, int nz,
                             int pitch, double h, int face, float margin, double *partial, double *wbuf,
                             unsigned *status)
{
    __shared__ float s32[kMaxSegments][7];
    load_seg32(geom, s32);
    __syncthreads();
    const float hf = (float)h;
    size_t nvp = (size_t)pitch * ny * nz;
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nvp;
         i += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(i % pitch);
        if (x >= nx) continue;
        size_t r = i / pitch;
        int y = (int)(r % ny);
        int z = (int)(r / ny);
        bool face_vox = (x == 0 || y == 0 || z == 0 || x == nx - 1 || y == ny - 1 || z == nz - 1);
        if (tab[label[i]].fixed || (face == RFA_FACE_DIRICHLET && face_vox)) continue;
        if (!RFA_CHECK_RANGE(i, i + 1, nvp, 0, 1, status)) continue;
        const double w = needle_weight2(
            geom, needle_dist2_pruned(geom, s32, x * h, y * h, z * h, x * hf, y * hf, z * hf, margin));
        wbuf[i] = w;
        acc += w;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// pass 2: W = sum of the partials in fixed order (out[0]) and the scale
// P / (h^3 W) of the weights (out[1]; 0 without a needle or weight)
__global__ void k_source_scale(const double *partial, int n, double P, double h, int nseg, double *out)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) {
        out[0] = acc;
        out[1] = (acc > 0.0 && nseg > 0) ? P / (h * h * h * acc) : 0.0;
    }
}

// pass 3: s_i = (P w_i / (h^3 W) + Q_m) dt / (rho c)_i on free voxels, 0
// elsewhere; a warp per grid row, the per-label values in shared memory
template <int SP>
__global__ void __launch_bounds__(256) k_source_write(const uint8_t *__restrict__ label,
                                                      const LabelCoef *__restrict__ tab, int n_labels, int nx,
                                                      int ny, int nz, int pitch, int face, const double *Wp,
                                                      const double *wbuf, void *s, unsigned *status)
{
    using T = typename std::conditional<SP == RFA_STATE_F64, double, float>::type;
    __shared__ double qm[256], dtrc[256];
    __shared__ uint8_t fixed[256];
    for (int l = threadIdx.x; l < n_labels; l += blockDim.x) {
        qm[l] = tab[l].Q_m;
        dtrc[l] = tab[l].dt_rhoc;
        fixed[l] = tab[l].fixed ? 1 : 0;
    }
    __syncthreads();
    const double scale = Wp[1];
    for (int row = blockIdx.x * 8 + (int)(threadIdx.x >> 5); row < ny * nz; row += gridDim.x * 8) {
        const int y = row % ny, z = row / ny;
        const bool face_row = y == 0 || z == 0 || y == ny - 1 || z == nz - 1;
        const size_t rb = (size_t)row * pitch;
        for (int x = threadIdx.x & 31; x < pitch; x += 32) {
            const size_t i = rb + x;
            if (!RFA_CHECK_RANGE(i, i + 1, (size_t)pitch * ny * nz, 0, 1, status)) continue;
            double v = 0.0;
            if (x < nx) {
                const int l = label[i];
                const bool face_vox = face_row || x == 0 || x == nx - 1;
                if (!(fixed[l] || (face == RFA_FACE_DIRICHLET && face_vox)))
                    v = fma(scale, wbuf[i], qm[l]) * dtrc[l];
            }
            ((T *)s)[i] = (T)v;
        }
    }
}

// The paper's hot tip (Sec. "Evaluation Methods"): a voxel hemisphere five
// voxels across and three deep, held at a fixed temperature.  One thread per
// candidate offset (u, v across the axis in -2..2, w = 0..2 along it); a voxel
// belongs to the hemisphere when (u/2.5)^2 + (v/2.5)^2 + (w/3)^2 <= 1, tested
// exactly as 36 u^2 + 36 v^2 + 25 w^2 <= 225.
//   paint:   a = b = s = 0, theta = theta_tip (hi and the exact lo of a pair);
//   restore: a, b as the set-up stores them for the voxel's label (0 for fixed
//            labels and Dirichlet face voxels), theta of fixed voxels back to
//            their held value; free voxels keep their current temperature
//            (their source is rewritten by the next placement).
struct TipGeom {
    int c[3];
    int ax, sgn;
};

template <int SP, int PP>
__global__ void k_tip(TipGeom t, const uint8_t *__restrict__ label, const LabelCoef *__restrict__ tab, int nx,
                      int ny, int nz, int pitch, int face, double T_a, double th_tip, bool paint, void *th,
                      void *lo, void *ab, void *s, unsigned *status)
{
    using T = typename std::conditional<SP == RFA_STATE_F64, double, float>::type;
    using AB = typename std::conditional<PP == RFA_PARAM_BF16, uint32_t,
                                         typename std::conditional<PP == RFA_PARAM_F32, float2, double2>::type>::type;
    const int k = threadIdx.x;
    if (k >= 75) return;
    const int u = k % 5 - 2, v = (k / 5) % 5 - 2, w = k / 25;
    if (36 * u * u + 36 * v * v + 25 * w * w > 225) return;
    int p[3] = {t.c[0], t.c[1], t.c[2]};
    p[t.ax] += t.sgn * w;
    p[(t.ax + 1) % 3] += u;
    p[(t.ax + 2) % 3] += v;
    if (p[0] < 0 || p[1] < 0 || p[2] < 0 || p[0] >= nx || p[1] >= ny || p[2] >= nz) return;
    const size_t i = ((size_t)p[2] * ny + p[1]) * pitch + p[0];
    if (!RFA_CHECK_RANGE(i, i + 1, (size_t)pitch * ny * nz, 0, 1, status)) return;
    double a = 0.0, b = 0.0, thv = th_tip;
    bool set_theta = paint;
    if (paint) {
        ((T *)s)[i] = T(0);
    } else {
        const LabelCoef c = tab[label[i]];
        const bool face_vox = p[0] == 0 || p[1] == 0 || p[2] == 0 || p[0] == nx - 1 || p[1] == ny - 1 ||
                              p[2] == nz - 1;
        if (c.fixed) {
            set_theta = true;
            thv = c.T_fixed - T_a;
        } else if (face == RFA_FACE_DIRICHLET && face_vox) {
            set_theta = true;
            thv = 0.0;
        } else {
            a = c.a;
            b = c.b;
        }
    }
    if (PP == RFA_PARAM_BF16)
        ((uint32_t *)ab)[i] = (uint32_t)bf16_bits_rne(a) | ((uint32_t)bf16_bits_rne(b) << 16);
    else if (PP == RFA_PARAM_F32)
        ((float2 *)ab)[i] = make_float2((float)a, (float)b);
    else
        ((double2 *)ab)[i] = make_double2(a, b);
    if (set_theta) {
        ((T *)th)[i] = (T)thv;
        if (SP == RFA_STATE_F32C) ((float *)lo)[i] = (float)(thv - (double)(float)thv);
    }
}

}  // namespace

cudaError_t launch_tip(rfa_grid *g, bool paint, double T_tip_C)
{
    TipGeom t;
    for (int d = 0; d < 3; ++d) t.c[d] = g->tip_c[d];
    t.ax = g->tip_ax;
    t.sgn = g->tip_sgn;
    const double th_tip = T_tip_C - g->T_a;
    void *th = g->th[g->cur], *lo = g->lo[g->cur];
#define TIP_CASE(SPV, PPV)                                                                                       \
    if (g->sp == SPV && g->pp == PPV)                                                                           \
        k_tip<SPV, PPV><<<1, 96, 0, g->stream>>>(t, g->label, g->d_table, g->nx, g->ny, g->nz, g->pitch, g->face, \
                                                 g->T_a, th_tip, paint, th, lo, g->ab, g->s, g->status);
    TIP_CASE(RFA_STATE_F32, RFA_PARAM_BF16)
    TIP_CASE(RFA_STATE_F32, RFA_PARAM_F32)
    TIP_CASE(RFA_STATE_F32, RFA_PARAM_F64)
    TIP_CASE(RFA_STATE_F32C, RFA_PARAM_BF16)
    TIP_CASE(RFA_STATE_F32C, RFA_PARAM_F32)
    TIP_CASE(RFA_STATE_F32C, RFA_PARAM_F64)
    TIP_CASE(RFA_STATE_F64, RFA_PARAM_BF16)
    TIP_CASE(RFA_STATE_F64, RFA_PARAM_F32)
    TIP_CASE(RFA_STATE_F64, RFA_PARAM_F64)
#undef TIP_CASE
    return cudaGetLastError();
}

cudaError_t launch_setup(rfa_grid *g, const uint8_t *labels_dense_dev, int n_labels)
{
    dim3 blk(256), grd(148 * 8);
    k_label_coef<<<1, 256, 0, g->stream>>>(g->d_table, n_labels, g->dt, g->h, g->pp);
#define SETUP_CASE(SPV, PPV)                                                                     \
    if (g->sp == SPV && g->pp == PPV)                                                           \
        k_setup<SPV, PPV><<<grd, blk, 0, g->stream>>>(                                          \
            labels_dense_dev, g->d_table, g->nx, g->ny, g->nz, g->pitch, g->h, g->dt, g->T_a,   \
            g->face, g->th[0], g->th[1], g->lo[0], g->lo[1], g->ab, g->s, g->label, g->latch,   \
            g->omega, g->omega_c, n_labels, g->status);
    SETUP_CASE(RFA_STATE_F32, RFA_PARAM_BF16)
    SETUP_CASE(RFA_STATE_F32, RFA_PARAM_F32)
    SETUP_CASE(RFA_STATE_F32, RFA_PARAM_F64)
    SETUP_CASE(RFA_STATE_F32C, RFA_PARAM_BF16)
    SETUP_CASE(RFA_STATE_F32C, RFA_PARAM_F32)
    SETUP_CASE(RFA_STATE_F32C, RFA_PARAM_F64)
    SETUP_CASE(RFA_STATE_F64, RFA_PARAM_BF16)
    SETUP_CASE(RFA_STATE_F64, RFA_PARAM_F32)
    SETUP_CASE(RFA_STATE_F64, RFA_PARAM_F64)
#undef SETUP_CASE
    return cudaGetLastError();
}

cudaError_t launch_source_write(rfa_grid *g, const double *partial, int npartial)
{
    double *W = (double *)g->red + kReduceBlocks;
    k_source_scale<<<1, 1024, 0, g->stream>>>(partial, npartial, g->geom.P, g->h, g->geom.nseg, W);
    if (g->sp == RFA_STATE_F64)
        k_source_write<RFA_STATE_F64><<<148 * 8, 256, 0, g->stream>>>(
            g->label, g->d_table, g->n_labels, g->nx, g->ny, g->nz, g->pitch, g->face, W, (const double *)g->stage,
            g->s, g->status);
    else
        k_source_write<RFA_STATE_F32><<<148 * 8, 256, 0, g->stream>>>(
            g->label, g->d_table, g->n_labels, g->nx, g->ny, g->nz, g->pitch, g->face, W, (const double *)g->stage,
            g->s, g->status);
    return cudaGetLastError();
}

cudaError_t launch_source(rfa_grid *g)
{
    double *partial = (double *)g->red;
    const float margin = needle_margin(g);
    k_source_sum<<<kReduceBlocks, 256, 0, g->stream>>>(g->geom, g->label, g->d_table, g->nx,
                                                       g->ny, g->nz, g->pitch, g->h, g->face, margin,
                                                       partial, (double *)g->stage, g->status);
    return launch_source_write(g, partial, kReduceBlocks);
}

}  // namespace rfa
