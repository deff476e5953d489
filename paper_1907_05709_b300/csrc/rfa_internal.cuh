// rfa_internal.cuh -- internal declarations of the B300 bioheat library.
//
// Layout in HBM (every per-voxel field of a grid): [nz][ny][pitch] with x
// fastest and pitch = nx rounded up to a multiple of 4, so every row starts on a
// 16-byte boundary (float4 / TMA friendly).  Padding voxels (x >= nx) hold zero
// and are never read as neighbours.
//
// State theta = T - T_a:
//   F32  : float  th[2]                     (ping-pong)
//   F32C : float  th[2] + float lo[2]       (compensated pair, value = hi + lo)
//   F64  : double th[2]
// Coefficients a = K dt / (rho c h^2) and b = w_b rho_b c_b dt / (rho c):
//   BF16 : one uint32 per voxel, a in the low 16 bits, b in the high 16 bits
//   F32  : float2 (a, b);  F64 : double2 (a, b)
// Source s = (q + Q_m) dt / (rho c): float (F32/F32C) or double (F64).
// Fixed voxels (vessels, Dirichlet faces) carry a = b = s = 0, so the update
// leaves them unchanged without a branch.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rfa.h"

namespace rfa {

constexpr unsigned kStatusNonfinite = 1u;
constexpr unsigned kStatusTimeout = 2u;
constexpr unsigned kStatusBadLabel = 4u;
constexpr unsigned kStatusGridTimeout = 8u;  // with kStatusTimeout: the batch's grid barrier ran out
constexpr unsigned kStatusBadIndex = 16u;    // an index check of the checked build failed

// Index checks of the checked build (compiled with -DRFA_CHECK, librfa_check.so):
// an access range [lo, hi) outside [0, n), or a vector access whose first index
// is not a multiple of `align`, records kStatusBadIndex in the grid's status
// word and the access is skipped.  The ordinary build compiles every check to
// `true`.  No check traps.
#ifdef RFA_CHECK
__device__ __forceinline__ bool check_range(long long lo, long long hi, long long n, long long first, int align,
                                            unsigned *status)
{
    const bool ok = lo >= 0 && hi <= n && lo <= hi && (first % align) == 0;
    if (!ok && status) atomicOr(status, kStatusBadIndex);
    return ok;
}
#define RFA_CHECK_RANGE(lo, hi, n, first, align, status)                                                     \
    ::rfa::check_range((long long)(lo), (long long)(hi), (long long)(n), (long long)(first), (align), (status))
#else
#define RFA_CHECK_RANGE(lo, hi, n, first, align, status) true
#endif
constexpr int kMaxSegments = 17;
constexpr int kReduceBlocks = 592;  // 4 per SM on 148 SMs; fixed => deterministic reductions
constexpr int kCarrySteps = 256;   // fold the FP32 damage carry into the FP64 integral every 256 steps

struct LabelCoef {
    double k, rho, c, w_b, rho_b, c_b, Q_m, T_fixed;
    int fixed;
    double a, b;   // stored (rounded) update coefficients, filled on the device by k_label_coef
    double dt_rhoc;  // dt / (rho c), filled there too
};

struct Segment {
    double p0[3], p1[3];
    double inv_uu;  // 1 / |p1 - p0|^2 (0 for a point)
};

struct NeedleGeom {
    Segment seg[kMaxSegments];
    int nseg;
    double r0, P;
};

// -------------------------------------------------------------- BF16 rounding
// Round a double to the nearest bfloat16 (8 significant bits, ties to even)
// and return its bit pattern.  Magnitudes below 2^-126 flush to signed zero.
__host__ __device__ inline uint16_t bf16_bits_rne(double x)
{
    uint64_t u;
#ifdef __CUDA_ARCH__
    u = (uint64_t)__double_as_longlong(x);
#else
    std::memcpy(&u, &x, 8);
#endif
    uint64_t sign = u & 0x8000000000000000ull;
    uint64_t mag = u & 0x7fffffffffffffffull;
    if (mag < (uint64_t)(1023 - 126) << 52) return (uint16_t)(sign >> 48);
    uint64_t lsb = (mag >> 45) & 1ull;
    mag += (1ull << 44) - 1ull + lsb;       // half of the dropped range, ties to even
    mag &= ~((1ull << 45) - 1ull);          // keep 7 fraction bits
    // re-bias the exponent from binary64 (1023) to binary32 / bfloat16 (127)
    uint64_t e = (mag >> 52) - 1023 + 127;
    if (e >= 255) return (uint16_t)((sign >> 48) | 0x7f80u);   // overflow -> inf
    uint32_t f = (uint32_t)(e << 7) | (uint32_t)((mag >> 45) & 0x7fu);
    return (uint16_t)((sign >> 48) | f);
}

__host__ __device__ inline float bf16_to_float(uint32_t bits16)
{
    uint32_t u = bits16 << 16;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, 4);
    return f;
#endif
}

__host__ __device__ inline double round_coef(double x, int param_prec)
{
    if (param_prec == RFA_PARAM_BF16) return (double)bf16_to_float(bf16_bits_rne(x));
    if (param_prec == RFA_PARAM_F32) return (double)(float)x;
    return x;
}

// coefficient expressions (Eq. CUDAbioheat3d divided through by rho c_p)
__host__ __device__ inline double coef_a(const LabelCoef &t, double dt, double h)
{
    return (t.k / (t.rho * t.c)) * dt / (h * h);
}
__host__ __device__ inline double coef_b(const LabelCoef &t, double dt)
{
    return (t.w_b * t.rho_b * t.c_b / (t.rho * t.c)) * dt;
}

// ------------------------------------------------------------ backward record
struct Record {
    bool valid = false;        // every step since set-up was recorded
    int64_t seg = 0;           // checkpoint spacing
    int64_t nsteps = 0;        // steps recorded
    // checkpoint states (hi, lo) every seg steps: the first `used` of a pool of
    // buffers that later recordings reuse (freed with the grid), so recording
    // allocates nothing once the pool is large enough
    std::vector<void *> ck_hi;
    std::vector<void *> ck_lo;
    size_t used = 0;
};

// Schedules of the step
struct Schedule {
    int tb_depth = 1;      // steps per launch
    int tile_variant = 0;  // blocked-kernel tile shape
};

}  // namespace rfa

struct rfa_grid {
    int nx = 0, ny = 0, nz = 0, pitch = 0;
    size_t plane = 0, nvp = 0;  // pitch*ny, pitch*ny*nz
    double h = 0, dt = 0, T_a = 37.0;
    int sp = 0, pp = 0, face = 0;
    cudaStream_t stream = nullptr;

    void *th[2] = {nullptr, nullptr};
    void *lo[2] = {nullptr, nullptr};
    int cur = 0;
    void *ab = nullptr;
    void *s = nullptr;
    uint8_t *label = nullptr;
    uint8_t *latch = nullptr;
    double *omega = nullptr;
    float *omega_c = nullptr;
    unsigned *status = nullptr;     // device status word
    unsigned *status_host = nullptr;  // pinned mirror
    void *red = nullptr;            // reduction partials (kReduceBlocks * 32 B)
    void *stage = nullptr;          // staging buffer (nvox * 8 B)
    rfa::LabelCoef *d_table = nullptr;
    std::vector<rfa_tissue> table;
    int n_labels = 0;

    bool have_tissue = false, have_needle = false;
    rfa_needle needle{};
    rfa::NeedleGeom geom{};
    // the hemisphere of a placed FIXED_TIP needle: voxel nearest the tip,
    // axis index (0 x, 1 y, 2 z) and direction of the dome
    bool tip_on = false;
    int tip_c[3] = {0, 0, 0};
    int tip_ax = 2, tip_sgn = 1;
    int dmg = 0;
    double A = 7.39e39, Ea = 2.577e5, R = 8.31, T_thr = 60.0;
    int64_t steps = 0;
    int64_t carry_steps = 0;  // steps accumulated in the FP32 damage carry since the last fold
    rfa::Schedule sched;
    rfa::Record rec;
    int cond = 0;              // RFA_COND_CENTRE or RFA_COND_HARMONIC
    int src_mode = 0;          // 0: max(d, r0)^-4 weights; 1: potential solve (sigma |grad V|^2)
    int alpha_perf = 0;        // 1: perfusion weighted by 1 / max(1, Omega)
    std::vector<double> sigma; // electrical conductivity per label (potential solve)
    int pot_max_iters = 0, pot_iters = 0;
    int pot_precond = 0;       // RFA_PRECOND_MULTIGRID or RFA_PRECOND_JACOBI
    double pot_tol = 0.0, pot_res = 0.0;
    void *d_wpair = nullptr;   // conservative form: label-pair weights (float, double for FP64 coefficients)
    float *d_wadj = nullptr;   // FP32 weights and their K derivatives for the adjoint (3 tables)

    size_t state_elem() const { return sp == RFA_STATE_F64 ? 8 : 4; }
    size_t ab_elem() const { return pp == RFA_PARAM_BF16 ? 4 : (pp == RFA_PARAM_F32 ? 8 : 16); }
    size_t nvox() const { return (size_t)nx * ny * nz; }
};

namespace rfa {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
rfa_status cuda_fail(cudaError_t e, const char *what);
#define RFA_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return rfa::cuda_fail(e_, #call); \
    } while (0)

// squared distance from a voxel centre to the nearest active segment
__device__ inline double needle_dist2(const NeedleGeom &g, double px, double py, double pz)
{
    double best = 1e300;
    for (int k = 0; k < g.nseg; ++k) {
        const Segment &sg = g.seg[k];
        double ux = sg.p1[0] - sg.p0[0], uy = sg.p1[1] - sg.p0[1], uz = sg.p1[2] - sg.p0[2];
        double wx = px - sg.p0[0], wy = py - sg.p0[1], wz = pz - sg.p0[2];
        double t = (wx * ux + wy * uy + wz * uz) * sg.inv_uu;
        t = fmin(fmax(t, 0.0), 1.0);
        double ex = wx - t * ux, ey = wy - t * uy, ez = wz - t * uz;
        best = fmin(best, ex * ex + ey * ey + ez * ez);
    }
    return best;
}

// The segments in FP32 for the pruned distance below, one per thread of the
// block's first nseg threads (the caller synchronises): p0 (3), p1 - p0 (3),
// 1 / |p1 - p0|^2.
__device__ __forceinline__ void load_seg32(const NeedleGeom &g, float (*s32)[7])
{
    if (threadIdx.x < (unsigned)g.nseg) {
        const Segment &sg = g.seg[threadIdx.x];
        for (int c = 0; c < 3; ++c) {
            s32[threadIdx.x][c] = (float)sg.p0[c];
            s32[threadIdx.x][3 + c] = (float)(sg.p1[c] - sg.p0[c]);
        }
        s32[threadIdx.x][6] = (float)sg.inv_uu;
    }
}

// squared distance to the nearest segment in FP32 (within e of the FP64 value,
// see needle_margin)
__device__ __forceinline__ float needle_dist2_f32(const NeedleGeom &g, const float (*s32)[7], float pxf, float pyf,
                                                  float pzf)
{
    float m32 = 3.0e38f;
    for (int k = 0; k < g.nseg; ++k) {
        const float *q = s32[k];
        const float wx = pxf - q[0], wy = pyf - q[1], wz = pzf - q[2];
        const float t = fminf(fmaxf((wx * q[3] + wy * q[4] + wz * q[5]) * q[6], 0.f), 1.f);
        const float ex = wx - t * q[3], ey = wy - t * q[4], ez = wz - t * q[5];
        m32 = fminf(m32, ex * ex + ey * ey + ez * ez);
    }
    return m32;
}

// needle_dist2 with the same FP64 value, evaluating in FP64 only the segments
// that can be the nearest.  An FP32 pass over all segments gives each squared
// distance to within e (bounded by the coordinates' magnitude); the nearest
// segment's FP32 value is then within 2e of the FP32 minimum, so every segment
// within margin >= 2e of it is evaluated with needle_dist2's FP64 expression
// and the minimum of those is needle_dist2's minimum.  s32 holds the segments
// in FP32: p0 (3), p1 - p0 (3), 1 / |p1 - p0|^2.
__device__ __forceinline__ double needle_dist2_pruned(const NeedleGeom &g, const float (*s32)[7], double px,
                                                      double py, double pz, float pxf, float pyf, float pzf,
                                                      float margin)
{
    auto d32 = [&](int k) {
        const float *q = s32[k];
        const float wx = pxf - q[0], wy = pyf - q[1], wz = pzf - q[2];
        const float t = fminf(fmaxf((wx * q[3] + wy * q[4] + wz * q[5]) * q[6], 0.f), 1.f);
        const float ex = wx - t * q[3], ey = wy - t * q[4], ez = wz - t * q[5];
        return ex * ex + ey * ey + ez * ez;
    };
    float m32 = 3.0e38f;
    for (int k = 0; k < g.nseg; ++k) m32 = fminf(m32, d32(k));
    double best = 1e300;
    for (int k = 0; k < g.nseg; ++k) {
        if (!(d32(k) <= m32 + margin)) continue;
        const Segment &sg = g.seg[k];
        double ux = sg.p1[0] - sg.p0[0], uy = sg.p1[1] - sg.p0[1], uz = sg.p1[2] - sg.p0[2];
        double wx = px - sg.p0[0], wy = py - sg.p0[1], wz = pz - sg.p0[2];
        double t = (wx * ux + wy * uy + wz * uz) * sg.inv_uu;
        t = fmin(fmax(t, 0.0), 1.0);
        double ex = wx - t * ux, ey = wy - t * uy, ez = wz - t * uz;
        best = fmin(best, ex * ex + ey * ey + ez * ez);
    }
    return best;
}

// With coordinates of magnitude at most L, the FP32 squared distance is off by
// at most e = ~110 u L d + 3 u d^2 <= 2.3e-5 L^2 (u = 2^-24, d <= 2 sqrt(3) L:
// roundings of the coordinates, the projection t and the difference e).  The
// nearest segment is then within 2e <= 4.6e-5 L^2 of the FP32 minimum, and the
// FP64 minimum within e of it; the margin is 2e-4 L^2.
inline float needle_margin(const rfa_grid *g)
{
    double L = std::max({g->nx, g->ny, g->nz}) * g->h;
    for (int k = 0; k < g->geom.nseg; ++k)
        for (int c = 0; c < 3; ++c)
            L = std::max({L, std::fabs(g->geom.seg[k].p0[c]), std::fabs(g->geom.seg[k].p1[c])});
    return (float)(2e-4 * L * L);
}

// ---------------------------------------------------------------- launchers
// setup / source (kernels_setup.cu)
cudaError_t launch_setup(rfa_grid *g, const uint8_t *labels_dense_dev, int n_labels);
cudaError_t launch_source(rfa_grid *g);
// FIXED_TIP hemisphere (g->tip_*): paint holds its voxels at theta_tip with
// a = b = s = 0; otherwise its voxels get back what their labels define
cudaError_t launch_tip(rfa_grid *g, bool paint, double T_tip_C);
// s from source weights already in g->stage (FP64 per padded voxel) and their
// per-block partial sums over the free voxels
cudaError_t launch_source_write(rfa_grid *g, const double *partial, int npartial);
// the RF source from the electric potential (kernels_potential.cu); uses g->geom,
// g->sigma, g->pot_max_iters, g->pot_tol; sets g->pot_iters, g->pot_res
rfa_status potential_place(rfa_grid *g);
// plain one-step-per-launch kernel (kernels_step.cu)
struct DamageConst {
    float c0, c1, TK0;     // inc = exp2(c0 - c1 / (theta + TK0)), FP32 path
    double c0d, c1d, TK0d; // same constants for the FP64 state
};
DamageConst damage_consts(const rfa_grid *g);
cudaError_t launch_step_plain(rfa_grid *g, const void *th_in, const void *lo_in, void *th_out,
                              void *lo_out, bool damage, bool latch, bool fold);
// conservative conduction (kernels_cond.cu): label-pair tables of at most kCondLabels labels
constexpr int kCondLabels = 16;
rfa_status cond_build_tables(rfa_grid *g, const rfa_tissue *table, int n_labels);
// one step of the model options (harmonic conduction and/or tissue-state perfusion)
cudaError_t launch_step_model(rfa_grid *g, const void *th_in, const void *lo_in, void *th_out, void *lo_out,
                              bool damage, bool latch, bool fold);
cudaError_t launch_adjoint_cond(rfa_grid *g, const float *lam_in, float *lam_out, float *Lam, const float *th,
                                double *acc);
// temporal-blocked TMA kernel (kernels_tb.cu)
bool tb_supported(const rfa_grid *g, int depth, int variant);
// spin limits (SM cycles) of the blocked kernels' mbarrier waits and of the
// batch's grid barrier, for kernels launched afterwards on the current device
cudaError_t tb_set_wait_limits(long long mbar_cycles, long long grid_cycles);
// true while limits other than the default are set (kernels then read them at start)
bool tb_limits_set();
void tb_forget_maps(const rfa_grid *g);
cudaError_t launch_step_tb(rfa_grid *g, int depth, int variant, const void *th_in,
                           const void *lo_in, void *th_out, void *lo_out, bool damage, bool fold);
// replay for the adjoint: depth steps without latch or damage; the hi parts of
// the depth - 1 intermediate states go to rec_hi + (k - 1) * nvp (k = 1 .. depth-1)
cudaError_t launch_step_tb_rec(rfa_grid *g, int depth, int variant, const void *th_in, const void *lo_in,
                               void *th_out, void *lo_out, float *rec_hi);
// blocked stepping geometry (kernels_tb.cu): outputs and tiling of one grid;
// `maps` points at the tensor maps (hi, lo, ab, s) of the input state
struct TBTile {
    const CUtensorMap *maps;
    float *hi_out, *lo_out;
    uint8_t *latch;
    double *omega;
    float *omega_c;
    int nx, ny, nz, pitch;
    size_t plane;
    int xt, yt, zc;  // tiles in x and y, z chunks; work items = xt * yt * zc
    float thr;
    float c0, c1, TK0;
    float *rec_hi;  // replay: hi of the intermediate states (stage k at rec_hi + (k - 1) * rec_stride)
    size_t rec_stride;
};
// a batch member on the host: tiles and tensor maps for both ping-pong parities
struct TBMemberHost {
    TBTile tile[2];
    CUtensorMap maps[8];
    int items = 0;
};
bool tb_batch_member(const rfa_grid *g, int depth, int variant, int max_chunk, TBMemberHost &out);
size_t tb_member_bytes();
void tb_pack_member(const TBMemberHost &h, const CUtensorMap *maps_dev, int item_begin, int cur0, void *dst);
cudaError_t prepare_batch_tb(int depth, int variant, bool damage, int nitems, int *grid);
cudaError_t graph_batch_tb(int depth, int variant, bool damage, const void *members_dev, int nmem, int nitems,
                           int ntime, unsigned *gbar, unsigned *status, int grid, cudaGraphExec_t *exec);
cudaError_t launch_batch_tb(int depth, int variant, bool damage, const void *members_dev, int nmem,
                            int nitems, int ntime, unsigned *gbar, unsigned *status, cudaStream_t stream, int grid);
// reductions and conversions (kernels_reduce.cu)
cudaError_t launch_necrosis(rfa_grid *g, uint8_t *mask_dense_dev, double width_K,
                            void *result_dev);
cudaError_t launch_to_temperature(rfa_grid *g, void *dst_dense_dev, int as_f64);
cudaError_t launch_get_field(rfa_grid *g, int field, double *dst_dense_dev);

// adjoint (adjoint.cu)
rfa_status backward_impl(rfa_grid *g, const float *dLdT, double *grads);
void record_free(rfa_grid *g);   // release the checkpoint pool (grid destruction)
void record_reset(rfa_grid *g);  // forget the recording, keep the pool
rfa_status record_begin(rfa_grid *g, int64_t nsteps);
rfa_status record_checkpoint(rfa_grid *g, int64_t step_index);

// forward stepping used by rfa_step and the adjoint recompute (runtime.cu)
rfa_status advance(rfa_grid *g, int64_t nsteps, bool damage, bool latch);

// z planes per block of the z-streaming kernels (blocks of 32 x 8 quads): short
// enough that at least two waves of resident blocks fill the 148 SMs, long
// enough (>= 4) that the two extra planes a chunk reads stay a small overhead
inline int choose_zchunk(const rfa_grid *g, int blocks_per_sm)
{
    const int quads = (g->pitch + 3) / 4;
    const long long bxy = (long long)((quads + 31) / 32) * ((g->ny + 7) / 8);
    const long long target = 2LL * 148 * blocks_per_sm;
    const long long nchunks = (target + bxy - 1) / bxy;
    long long zc = (g->nz + nchunks - 1) / nchunks;
    if (zc < 4) zc = 4;
    if (zc > 32) zc = 32;
    if (zc > g->nz) zc = g->nz;
    return (int)zc;
}

// z chunk for a latency-bound kernel (the adjoint step, whose fields sit in L2
// at the sizes it runs): fewest waves of blocks_per_sm x 148 resident CTAs times
// the planes each CTA streams (its chunk plus 2 halo planes).  At 128^3 this
// takes 8-plane chunks in one wave where choose_zchunk's 4-plane chunks took
// 1.7 waves (measured: 5 % less backward time).  HBM-bound kernels keep
// choose_zchunk: a partial last wave still saturates their bandwidth.
inline int choose_zchunk_waves(const rfa_grid *g, int blocks_per_sm)
{
    const int quads = (g->pitch + 3) / 4;
    const long long bxy = (long long)((quads + 31) / 32) * ((g->ny + 7) / 8);
    const long long slots = 148LL * blocks_per_sm;
    int best = 1;
    long long best_cost = -1;
    for (int zc = 1; zc <= g->nz && zc <= 64; ++zc) {
        const long long blocks = bxy * ((g->nz + zc - 1) / zc);
        const long long cost = ((blocks + slots - 1) / slots) * (zc + 2);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = zc;
        }
    }
    return best;
}

inline dim3 plain_grid_dims(const rfa_grid *g, int zchunk)
{
    int quads = (g->pitch + 3) / 4;
    return dim3((unsigned)((quads + 31) / 32), (unsigned)((g->ny + 7) / 8),
                (unsigned)((g->nz + zchunk - 1) / zchunk));
}

}  // namespace rfa
