// kernels_tb.cu -- temporally blocked explicit step: M steps of Eq.
// CUDAbioheat3d per launch (compensated FP32 state, BF16 coefficients),
// fused with the 60 C latch and the FP64 Arrhenius integral.
//
// Prior art is the paper's one-step shared-memory kernel (Alg. 1, Table
// 2675-runtimes); on B300 the step is HBM- and FP64-bound, so this kernel
// re-reads nothing from HBM across M steps and touches the FP64 damage
// integral once per launch instead of once per step.
//
// Tiling.  A CTA owns an output tile of 64 (x) by TY = EY - 2M (y) voxels and a
// chunk of z planes.  It loads the tile plus a 4-voxel x halo and an M-voxel y
// halo (72 x EY columns) plane by plane with TMA (cp.async.bulk.tensor, one
// mbarrier per ring slot, zero fill outside the grid) and streams along z:
// stage k (1 <= k <= M) computes step k on plane p0 - k when stage-0 plane p0
// has arrived, reading the three planes q-1, q, q+1 of stage k-1 from a
// 3-plane shared-memory ring.  The last stage writes the output tile to HBM.
// The valid region shrinks by one voxel per stage in x and y (trapezoid).
//
// Numerics.  Every stage uses the same update (rfa_update.cuh) and the same
// neighbour order as the one-step kernel, so a launch of depth M produces
// bit-identical states to M one-step launches.  The latch takes the maximum
// of the M new values; the M Arrhenius increments are summed in FP32
// registers and added to the FP32 carry of the FP64 integral; on launches
// flagged `fold` the carry is folded into the FP64 value (error-free TwoSum).
//
// Waits on mbarriers are bounded (clock64); on timeout the kernel records
// kStatusTimeout in the grid's status word and every thread leaves.
#include "rfa_internal.cuh"
#include "rfa_update.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <array>
#include <map>
#include <mutex>
#include <tuple>

namespace rfa {

namespace {

constexpr int TB_EX = 72;       // loaded tile width: 64 output + 4 halo on each side
constexpr int TB_TX = 64;       // output tile width
constexpr int TB_HX = 4;        // x halo (keeps the TMA x coordinate 16-byte aligned)
constexpr int TB_TR = 8;        // thread rows; a CTA has TB_EX * TB_TR = 576 threads
constexpr int TB_THREADS = TB_EX * TB_TR;

template <int M, int EY>
struct Cfg {
    static constexpr int RY = EY / TB_TR;        // tile rows per thread
    static constexpr int TY = EY - 2 * M;        // output rows per tile
    static constexpr int S0 = M + 2;             // stage-0 ring slots (planes p0-M .. p0+1)
    static constexpr int PLANE = TB_EX * EY;     // elements per tile plane
    static constexpr int SLOT0 = 4 * PLANE;      // floats per stage-0 slot: hi, lo, ab, s
    static constexpr int RINGK = 2 * PLANE;      // floats per stage-k slot: (hi, lo) pairs
    static constexpr int RING_OFF = S0 * SLOT0;  // float offset of the stage rings
    static constexpr int BAR_OFF = RING_OFF + (M - 1) * 3 * RINGK;
    static constexpr int SMEM = BAR_OFF * 4 + 8 * S0;
    static constexpr int MINB = SMEM <= 110 * 1024 ? 2 : 1;
    static_assert(EY % TB_TR == 0 && TY > 0 && M <= TB_HX, "bad tile");
};

struct TBArgs {
    float *hi_out, *lo_out;
    uint8_t *latch;
    double *omega;
    float *omega_c;
    unsigned *status;
    int nx, ny, nz, pitch, zchunk;
    size_t plane;
    float thr;
    float c0, c1, TK0;
    int fold;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bounded wait for the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1ll << 32)) return false;  // ~2 s at 2 GHz
    }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

template <int M, int EY, bool DMG>
__global__ void __launch_bounds__(TB_THREADS, Cfg<M, EY>::MINB)
    k_step_tb(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
              const __grid_constant__ CUtensorMap tm_ab, const __grid_constant__ CUtensorMap tm_s,
              const TBArgs A)
{
    using C = Cfg<M, EY>;
    constexpr int RY = C::RY, S0 = C::S0, PLANE = C::PLANE;
    extern __shared__ __align__(128) float sm[];
    const uint32_t sm_base = smem_u32(sm);
    if (sm_base & 127u) {  // TMA destinations need 128-byte alignment
        if (threadIdx.x == 0) atomicOr(A.status, kStatusTimeout);
        return;
    }
    const uint32_t bar_base = sm_base + 4u * C::BAR_OFF;

    const int tid = threadIdx.x;
    const int xl = tid % TB_EX, tr = tid / TB_EX;
    const int X0 = blockIdx.x * TB_TX;
    const int Y0 = blockIdx.y * C::TY;
    const int zb = blockIdx.z * A.zchunk;
    const int ze = min(A.nz, zb + A.zchunk);
    const int L = ze - zb + 2 * M;   // stage-0 planes zb-M .. ze+M-1
    const int xg = X0 - TB_HX + xl;
    const bool colok = xl >= 1 && xl < TB_EX - 1 && xg >= 0 && xg < A.nx;
    const bool outcol = xl >= TB_HX && xl < TB_HX + TB_TX && xg < A.nx;
    const bool xm_ok = xg > 0, xp_ok = xg + 1 < A.nx;

    // per-row constants of this thread
    int yg[RY], id[RY];
    bool rowok[RY], ym_ok[RY], yp_ok[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int yl = tr * RY + r;
        yg[r] = Y0 - M + yl;
        id[r] = yl * TB_EX + xl;
        rowok[r] = colok && yg[r] >= 0 && yg[r] < A.ny;
        ym_ok[r] = yg[r] > 0;
        yp_ok[r] = yg[r] + 1 < A.ny;
    }

    if (tid == 0) {
        for (int j = 0; j < S0; ++j) mbar_init(bar_base + 8u * j, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int itp) {  // stage-0 plane zb - M + itp into slot itp % S0
        const int j = itp % S0;
        const uint32_t dst = sm_base + 4u * (uint32_t)(j * C::SLOT0);
        const uint32_t bar = bar_base + 8u * j;
        const int z = zb - M + itp;
        mbar_expect_tx(bar, (uint32_t)(C::SLOT0 * 4));
        tma_load_3d(dst, &tm_hi, X0 - TB_HX, Y0 - M, z, bar);
        tma_load_3d(dst + 4u * PLANE, &tm_lo, X0 - TB_HX, Y0 - M, z, bar);
        tma_load_3d(dst + 8u * PLANE, &tm_ab, X0 - TB_HX, Y0 - M, z, bar);
        tma_load_3d(dst + 12u * PLANE, &tm_s, X0 - TB_HX, Y0 - M, z, bar);
    };
    if (tid == 0) issue(0);

    float part[M + 1][RY], mx[M + 1][RY];
#pragma unroll
    for (int k = 0; k <= M; ++k)
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            part[k][r] = 0.f;
            mx[k][r] = -3.0e38f;
        }
    bool bad = false;
    // ring slot of plane p: ring0 (p - zb + M) % S0, stage rings (p - zb + M) % 3
    int s0_cur = 0, s3_cur = 0;  // slots of stage-0 plane p0 (it % S0, it % 3)

    for (int it = 0; it < L; ++it) {
        const int p0 = zb - M + it;
        if (tid == 0 && it + 1 < L) issue(it + 1);
#pragma unroll
        for (int k = M; k >= 2; --k)
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                part[k][r] = part[k - 1][r];
                mx[k][r] = mx[k - 1][r];
            }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            part[1][r] = 0.f;
            mx[1][r] = -3.0e38f;
        }
        const bool ok = mbar_wait(bar_base + 8u * s0_cur, (uint32_t)((it / S0) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(A.status, kStatusTimeout);
                if (it + 1 < L) mbar_wait(bar_base + 8u * ((it + 1) % S0), (uint32_t)(((it + 1) / S0) & 1));
            }
            return;
        }
#pragma unroll
        for (int k = 1; k <= M; ++k) {
            const int q = p0 - k;
            if (it >= 2 * k && q >= 0 && q < A.nz) {
                // slots of planes q-1, q, q+1 (stage k-1) and of the coefficients of q
                const int sq0 = (s0_cur + S0 - k) % S0;              // ring0 slot of plane q
                const int s3q = (s3_cur + 3 * M - k) % 3;            // stage-ring slot of plane q
                const int cb = sq0 * C::SLOT0;                        // coefficients of plane q
                const bool zm_ok = q > 0, zp_ok = q + 1 < A.nz;
#pragma unroll
                for (int r = 0; r < RY; ++r) {
                    const int yl = tr * RY + r;
                    if (!(rowok[r] && yl >= k && yl < EY - k)) continue;
                    const int i = id[r];
                    float c, cl, S = 0.f;
                    if (k == 1) {
                        const int bc = cb, bm = ((sq0 + S0 - 1) % S0) * C::SLOT0, bp = ((sq0 + 1) % S0) * C::SLOT0;
                        c = sm[bc + i];
                        cl = sm[bc + PLANE + i];
                        S = acc(S, xm_ok ? cdiff(sm[bc + i - 1], sm[bc + PLANE + i - 1], c, cl) : 0.f);
                        S = acc(S, xp_ok ? cdiff(sm[bc + i + 1], sm[bc + PLANE + i + 1], c, cl) : 0.f);
                        S = acc(S, ym_ok[r] ? cdiff(sm[bc + i - TB_EX], sm[bc + PLANE + i - TB_EX], c, cl) : 0.f);
                        S = acc(S, yp_ok[r] ? cdiff(sm[bc + i + TB_EX], sm[bc + PLANE + i + TB_EX], c, cl) : 0.f);
                        S = acc(S, zm_ok ? cdiff(sm[bm + i], sm[bm + PLANE + i], c, cl) : 0.f);
                        S = acc(S, zp_ok ? cdiff(sm[bp + i], sm[bp + PLANE + i], c, cl) : 0.f);
                    } else {
                        const float2 *R = reinterpret_cast<const float2 *>(sm + C::RING_OFF + ((k - 2) * 3 + s3q) * C::RINGK);
                        const float2 *Rm = reinterpret_cast<const float2 *>(sm + C::RING_OFF + ((k - 2) * 3 + (s3q + 2) % 3) * C::RINGK);
                        const float2 *Rp = reinterpret_cast<const float2 *>(sm + C::RING_OFF + ((k - 2) * 3 + (s3q + 1) % 3) * C::RINGK);
                        const float2 cc = R[i];
                        c = cc.x;
                        cl = cc.y;
                        float2 v;
                        v = R[i - 1];      S = acc(S, xm_ok ? cdiff(v.x, v.y, c, cl) : 0.f);
                        v = R[i + 1];      S = acc(S, xp_ok ? cdiff(v.x, v.y, c, cl) : 0.f);
                        v = R[i - TB_EX];  S = acc(S, ym_ok[r] ? cdiff(v.x, v.y, c, cl) : 0.f);
                        v = R[i + TB_EX];  S = acc(S, yp_ok[r] ? cdiff(v.x, v.y, c, cl) : 0.f);
                        v = Rm[i];         S = acc(S, zm_ok ? cdiff(v.x, v.y, c, cl) : 0.f);
                        v = Rp[i];         S = acc(S, zp_ok ? cdiff(v.x, v.y, c, cl) : 0.f);
                    }
                    const uint32_t w = __float_as_uint(sm[cb + 2 * PLANE + i]);
                    float nh, nl;
                    cupdate(c, cl, S, bf16_to_float(w & 0xffffu), bf16_to_float(w >> 16), sm[cb + 3 * PLANE + i], nh, nl);
                    const float val = __fadd_rn(nh, nl);
                    mx[k][r] = fmaxf(mx[k][r], val);
                    if (DMG) part[k][r] = __fadd_rn(part[k][r], arrhenius_inc(val, A.c0, A.c1, A.TK0));
                    if (k < M) {
                        float2 *O = reinterpret_cast<float2 *>(sm + C::RING_OFF + ((k - 1) * 3 + s3q) * C::RINGK);
                        O[i] = make_float2(nh, nl);
                    } else if (outcol && yl >= M && yl < EY - M) {
                        const size_t gi = (size_t)q * A.plane + (size_t)yg[r] * A.pitch + xg;
                        A.hi_out[gi] = nh;
                        A.lo_out[gi] = nl;
                        bad |= !isfinite(nh);
                        if (mx[k][r] >= A.thr && A.latch[gi] == 0) A.latch[gi] = 1;
                        if (DMG) {
                            float P = __fadd_rn(A.omega_c[gi], part[k][r]);
                            if (A.fold) {
                                double om = A.omega[gi];
                                carry_fold(om, P);
                                A.omega[gi] = om;
                            }
                            A.omega_c[gi] = P;
                        }
                    }
                }
            }
            __syncthreads();
        }
        s0_cur = s0_cur + 1 == S0 ? 0 : s0_cur + 1;
        s3_cur = s3_cur + 1 == 3 ? 0 : s3_cur + 1;
    }
    if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(A.status, kStatusNonfinite);
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

bool make_map(CUtensorMap *m, const void *base, CUtensorMapDataType dt, const rfa_grid *g, int ey)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)g->nx, (cuuint64_t)g->ny, (cuuint64_t)g->nz};
    cuuint64_t strides[2] = {(cuuint64_t)g->pitch * 4, (cuuint64_t)g->plane * 4};
    cuuint32_t box[3] = {(cuuint32_t)TB_EX, (cuuint32_t)ey, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, dt, 3, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int variant_ey(int variant) { return variant == 1 ? 24 : 16; }

template <int M, int EY, bool DMG>
cudaError_t launch_inst(rfa_grid *g, const CUtensorMap *maps, const TBArgs &A0)
{
    using C = Cfg<M, EY>;
    cudaError_t e = cudaFuncSetAttribute(k_step_tb<M, EY, DMG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    TBArgs A = A0;
    const int xt = (g->nx + TB_TX - 1) / TB_TX;
    const int yt = (g->ny + C::TY - 1) / C::TY;
    const int resident = 148 * C::MINB;
    int zc = (2 * resident + xt * yt - 1) / (xt * yt);
    int maxzc = g->nz / (4 * M) > 0 ? g->nz / (4 * M) : 1;
    if (zc > maxzc) zc = maxzc;
    if (zc < 1) zc = 1;
    A.zchunk = (g->nz + zc - 1) / zc;
    dim3 grd((unsigned)xt, (unsigned)yt, (unsigned)((g->nz + A.zchunk - 1) / A.zchunk));
    k_step_tb<M, EY, DMG><<<grd, TB_THREADS, C::SMEM, g->stream>>>(maps[0], maps[1], maps[2], maps[3], A);
    return cudaGetLastError();
}

// tensor maps per (grid, input buffers, tile height); erased when the grid is destroyed
struct MapCache {
    std::map<std::tuple<const rfa_grid *, const void *, const void *, int>, std::array<CUtensorMap, 4>> m;
    std::mutex mu;
};
MapCache &map_cache()
{
    static MapCache c;
    return c;
}

}  // namespace

bool tb_supported(const rfa_grid *g, int depth, int variant)
{
    if (g->sp != RFA_STATE_F32C || g->pp != RFA_PARAM_BF16) return false;
    if (variant < 0 || variant > 1) return false;
    if (variant == 0 && (depth < 2 || depth > 4)) return false;
    if (variant == 1 && (depth < 2 || depth > 3)) return false;
    return encode_fn() != nullptr;
}

void tb_forget_maps(const rfa_grid *g)
{
    auto &c = map_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    for (auto it = c.m.begin(); it != c.m.end();) {
        if (std::get<0>(it->first) == g) it = c.m.erase(it);
        else ++it;
    }
}

cudaError_t launch_step_tb(rfa_grid *g, int depth, int variant, const void *th_in, const void *lo_in,
                           void *th_out, void *lo_out, bool damage, bool fold)
{
    const int ey = variant_ey(variant);
    std::array<CUtensorMap, 4> maps;
    {
        auto &c = map_cache();
        std::lock_guard<std::mutex> lk(c.mu);
        auto key = std::make_tuple((const rfa_grid *)g, th_in, lo_in, ey);
        auto it = c.m.find(key);
        if (it == c.m.end()) {
            if (!make_map(&maps[0], th_in, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g, ey) ||
                !make_map(&maps[1], lo_in, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g, ey) ||
                !make_map(&maps[2], g->ab, CU_TENSOR_MAP_DATA_TYPE_UINT32, g, ey) ||
                !make_map(&maps[3], g->s, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g, ey))
                return cudaErrorInvalidValue;
            c.m[key] = maps;
        } else {
            maps = it->second;
        }
    }
    TBArgs A;
    A.hi_out = (float *)th_out;
    A.lo_out = (float *)lo_out;
    A.latch = g->latch;
    A.omega = g->omega;
    A.omega_c = g->omega_c;
    A.status = g->status;
    A.nx = g->nx;
    A.ny = g->ny;
    A.nz = g->nz;
    A.pitch = g->pitch;
    A.plane = g->plane;
    A.zchunk = g->nz;
    A.thr = (float)(g->T_thr - g->T_a);
    DamageConst dc = damage_consts(g);
    A.c0 = dc.c0;
    A.c1 = dc.c1;
    A.TK0 = dc.TK0;
    A.fold = fold ? 1 : 0;
#define TB_CASE(MV, EYV)                                                                 \
    if (depth == MV && ey == EYV)                                                        \
        return damage ? launch_inst<MV, EYV, true>(g, maps.data(), A)                   \
                      : launch_inst<MV, EYV, false>(g, maps.data(), A);
    TB_CASE(2, 16)
    TB_CASE(3, 16)
    TB_CASE(4, 16)
    TB_CASE(2, 24)
    TB_CASE(3, 24)
#undef TB_CASE
    return cudaErrorInvalidValue;
}

}  // namespace rfa
