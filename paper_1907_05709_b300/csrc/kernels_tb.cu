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
// mbarrier per ring slot, zero fill outside the grid) and streams along z.
// A thread works on quads of 4 consecutive x voxels of one tile row (paired
// FP32 instructions on voxels (0,1) and (2,3)): stage k (1 <= k <= M) computes
// step k on plane p0 - k when stage-0 plane p0 has arrived, reading the three
// planes q-1, q, q+1 of stage k-1 from a 3-plane shared-memory ring.  The
// valid region shrinks by one voxel per stage in x and y (trapezoid); stage
// k < M covers tile rows k .. EY-1-k, the last stage only the output tile, and
// writes it to HBM.  CTA barriers follow stages 1 .. M-1 only (one per plane
// at M = 2): the last stage's coefficients are taken to registers before the
// last barrier and its input ring has a fourth slot, so the next plane's early
// stages overlap it; the next stage-0 plane is requested two planes ahead, right
// after the last barrier.
//
// Numerics.  Every stage uses the same update (rfa_update.cuh) and the same
// neighbour order as the one-step kernel, so a launch of depth M produces
// bit-identical states to M one-step launches.  The latch takes the maximum
// of the M new values; the M Arrhenius increments are summed in FP32 and
// added to the FP32 carry of the FP64 integral; on launches flagged `fold`
// the carry is folded into the FP64 value (error-free TwoSum).
//
// Waits on mbarriers are bounded (clock64); on timeout the kernel records
// kStatusTimeout in the grid's status word and every thread leaves.
#include "rfa_internal.cuh"
#include "rfa_update.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

namespace rfa {

namespace {

constexpr int TB_EX = 72;       // loaded tile width: 64 output + 4 halo on each side
constexpr int TB_TX = 64;       // output tile width
constexpr int TB_HX = 4;        // x halo (keeps the TMA x coordinate 16-byte aligned)
constexpr int TB_QX = TB_EX / 4;  // quads (4 consecutive x voxels) per tile row

// Tile variants (height EY of the loaded tile):
//   0: EY = 16 (2 CTAs per SM at depth 2)
//   1: EY = 32 (1 CTA per SM)
__host__ __device__ constexpr int tile_ey(int v) { return v == 1 ? 32 : 16; }

template <int M, int V>
struct Cfg {
    static constexpr int EY = tile_ey(V);
    static constexpr int TY = EY - 2 * M;                 // output rows per tile
    static constexpr int NQ1 = (EY - 2) * TB_QX;          // quads of stage 1 (tile rows 1 .. EY-2)
    static constexpr int NQO = TY * (TB_QX - 2);          // quads of the last stage (the output tile)
    static constexpr int THREADS = (NQ1 + 31) / 32 * 32;  // one thread per stage-1 quad
    // stage-0 ring: planes p0-M .. p0+1, and p0+2 requested into the slot of p0-M
    // once the last barrier of the plane has passed
    static constexpr int S0 = M + 2;
    static constexpr int BOX = TB_EX * EY;                // floats of one TMA box (a tile plane)
    // stride of the planes in shared memory: TMA destinations need 128-byte alignment
    static constexpr int PLANE = (BOX + 31) / 32 * 32;
    static constexpr int SLOT0 = 4 * PLANE;               // stage-0 slot: hi, lo, ab, s planes
    // ring of stage k (1 <= k < M): slots of hi, lo; from stage 2 on also the
    // running Arrhenius sum and the running maximum of the voxel's values.  3 slots;
    // the last ring (read by the last stage, after which there is no barrier) 4.
    __host__ __device__ static constexpr int ring_planes(int k) { return k >= 2 ? 4 : 2; }
    __host__ __device__ static constexpr int ring_slots(int k) { return k == M - 1 ? 4 : 3; }
    __host__ __device__ static constexpr int ring_off(int k)
    {
        int o = S0 * SLOT0;
        for (int j = 1; j < k; ++j) o += ring_slots(j) * ring_planes(j) * PLANE;
        return o;
    }
    static constexpr int BAR_OFF = ring_off(M);
    static constexpr int SMEM = BAR_OFF * 4 + 8 * S0;
    static constexpr int MINB = SMEM <= 110 * 1024 ? 2 : 1;
    static_assert(TY > 0 && M >= 2 && M <= TB_HX && SMEM <= 227 * 1024, "bad tile");
    static_assert((PLANE * 4) % 128 == 0 && (SLOT0 * 4) % 128 == 0, "TMA destinations must be 128-byte aligned");
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

// Spin limits of the bounded waits in SM clock cycles: the TMA (mbarrier) waits
// and the batch's grid barrier.  kDefaultLimit (2^32 cycles, about 2 s at
// 2 GHz) is compiled into the kernels; while a test has set other limits through
// rfa_set_wait_limits, the host launches the instantiations with LIM = true,
// which read them from these globals at start.
constexpr long long kDefaultLimit = 1ll << 32;
__device__ long long g_wait_limit_mbar = kDefaultLimit;
__device__ long long g_wait_limit_grid = kDefaultLimit;
// the wait for a CTA's own copies in flight before it leaves after a timeout
// keeps the full limit whatever the limits above are
constexpr long long kDrainLimit = 1ll << 32;

// bounded wait for the phase with the given parity; false on timeout.  Each
// try_wait may suspend the thread for up to `hint` ns (it resumes as soon as
// the phase completes), so waiting warps do not spin on the issue slots.  The
// kernels pass kSuspendNs, or 0 for limits below kSuspendMin (set only by
// tests), which polls with test_wait, so that a short limit is not hidden
// inside one suspended try_wait.
constexpr uint32_t kSuspendNs = 100000;
constexpr long long kSuspendMin = 1ll << 20;
__device__ __forceinline__ uint32_t suspend_hint(long long limit) { return limit >= kSuspendMin ? kSuspendNs : 0u; }
// mbarrier phase test: a suspending try_wait, or with hint 0 the non-blocking test_wait
__device__ __forceinline__ uint32_t mbar_test(uint32_t bar, uint32_t parity, uint32_t hint)
{
    uint32_t done;
    if (hint)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity), "r"(hint)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
    return done;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit, uint32_t hint)
{
    const long long t0 = clock64();
    while (true) {
        if (mbar_test(bar, parity, hint)) return true;
        if (clock64() - t0 > limit) return false;
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

__device__ __forceinline__ float4 ld4(const float *sm, int off)
{
    return *reinterpret_cast<const float4 *>(sm + off);
}

// per-CTA pipeline state, kept across work items and time blocks
struct TBPipe {
    float *sm;
    uint32_t sm_base, bar_base;
    long long nload;   // stage-0 planes consumed so far (ring slot and mbarrier phase)
    long long limit;   // spin limit of the mbarrier waits (kernels instantiated with LIM)
    uint32_t hint;     // suspend-time hint of their try_wait (ns)
};

template <int M, int V>
__device__ __forceinline__ void tb_item_geom(const TBTile &T, int item, int &X0, int &Y0, int &zb, int &ze)
{
    const int tx = item % T.xt, r = item / T.xt;
    const int ty = r % T.yt, zi = r / T.yt;
    X0 = tx * TB_TX;
    Y0 = ty * Cfg<M, V>::TY;
    zb = (int)((long long)zi * T.nz / T.zc);
    ze = (int)((long long)(zi + 1) * T.nz / T.zc);
}

// stage-0 plane z of the tile at (X0, Y0) into ring slot j
template <int M, int V>
__device__ __forceinline__ void tb_issue(TBPipe &P, int j, const CUtensorMap *maps, int X0, int Y0, int z)
{
    using C = Cfg<M, V>;
    const uint32_t dst = P.sm_base + 4u * (uint32_t)(j * C::SLOT0);
    const uint32_t bar = P.bar_base + 8u * j;
    mbar_expect_tx(bar, (uint32_t)(4 * C::BOX * 4));   // four boxes of 4-byte elements
    tma_load_3d(dst, &maps[0], X0 - TB_HX, Y0 - M, z, bar);
    tma_load_3d(dst + 4u * C::PLANE, &maps[1], X0 - TB_HX, Y0 - M, z, bar);
    tma_load_3d(dst + 8u * C::PLANE, &maps[2], X0 - TB_HX, Y0 - M, z, bar);
    tma_load_3d(dst + 12u * C::PLANE, &maps[3], X0 - TB_HX, Y0 - M, z, bar);
}

// The work items a CTA advances: a fixed stride (items of one grid are alike),
// or claimed from a counter (batch members differ in size, so CTAs that finish
// early take more).  start() gives the first item, after(cur) the next one.
struct StrideItems {
    int first, stride;
    __device__ int start() const { return first; }
    __device__ int after(int cur) const { return cur + stride; }
};
struct ClaimedItems {
    unsigned *ctr;
    __device__ int start() const { return (int)atomicAdd(ctr, 1u); }
    __device__ int after(int) const { return (int)atomicAdd(ctr, 1u); }
};

// Checked build: every shared-memory word stage k reads or writes for the quad at
// plane offset id lies inside the rings (below the mbarriers).  The ordinary build
// compiles this to true.
template <int M, int V>
__device__ __forceinline__ bool tb_stage_smem_ok(int k, const int *r0, const int *e, const int *f, int id,
                                                 unsigned *status)
{
#ifdef RFA_CHECK
    using C = Cfg<M, V>;
    constexpr int PLANE = C::PLANE;
    int lo = r0[k], hi = r0[k] + 4 * PLANE;  // coefficients (ab, s) of the stage's plane
    if (k == 1) {
        lo = min(lo, min(r0[0], min(r0[1], r0[2])));
        hi = max(hi, max(r0[0], max(r0[1], r0[2])) + 2 * PLANE);
    } else {
        const int rk = C::ring_off(k - 1), sl = C::ring_planes(k - 1) * PLANE;
        const int nsl = C::ring_slots(k - 1);
        for (int d = 0; d < nsl; ++d) {
            const int b = rk + (nsl == 4 ? f[d] : e[d % 3]) * sl;
            lo = min(lo, b);
            hi = max(hi, b + sl);
        }
    }
    if (k < M) {
        const int ro = C::ring_off(k), sl = C::ring_planes(k) * PLANE;
        lo = min(lo, ro);
        hi = max(hi, ro + C::ring_slots(k) * sl);
    }
    // words id - TB_EX .. id + TB_EX + 3 of every plane in [lo, hi) (the x neighbours
    // id - 1 and id + 4 lie between: a quad in the tile's outer column reads itself)
    return RFA_CHECK_RANGE((long long)lo + id - TB_EX, (long long)hi - PLANE + id + TB_EX + 4, C::BAR_OFF, id, 4,
                           status) &&
           RFA_CHECK_RANGE(lo, hi, C::BAR_OFF, 0, 1, status);
#else
    return true;
#endif
}

// Advance the work items of `items` (< nitems) by M steps.
// get(item, local, maps) returns the item's TBTile (a reference to kernel
// parameters for one grid; a register copy for the batch), its index in that
// tile and the tensor maps of the tile's input state.
// Returns false if a wait timed out (kStatusTimeout recorded, CTA must leave).
//
// Thread -> quad maps (fixed for the kernel): stage k < M covers tile rows
// k .. EY-1-k with all TB_QX quads (thread t takes quad t + k TB_QX); the last
// stage covers only the output tile (thread t takes row M + t / 16, quad
// 1 + t % 16), so no warp of the last stage works on halo columns.
//
// Faces: the kernel is used with Dirichlet faces only, where every face voxel
// is fixed (a = b = s = 0) and its neighbour sum is multiplied by a = 0; voxels
// outside the grid are loaded as zeros (TMA zero fill, a = b = s = 0) and
// compute to exact zeros.  So no neighbour needs an in-grid test: every sum
// that reaches a free voxel has only in-grid terms.
//
// Latch and damage: stage k >= 2 receives the values of stage k-1 as its
// centre operand, so it evaluates the Arrhenius increment and the latch
// maximum of those; the last stage adds those of its own result.  For M = 2
// nothing is carried between planes; for M = 3 the running sum and maximum
// travel with the values through the stage-2 ring.  The sums keep the order
// ((inc_1 + inc_2) + ...) of the per-step evaluation.
template <int M, int V, bool DMG, bool FOLD, bool REC, bool LIM, class Items, class Get>
__device__ bool tb_run(TBPipe &P, const Items &items, int nitems, const Get &get, unsigned *status, bool &bad)
{
    static_assert(!(REC && DMG), "the replay has no damage integral");
    using C = Cfg<M, V>;
    constexpr int S0 = C::S0, PLANE = C::PLANE;
    float *sm = P.sm;
    const uint32_t bar_base = P.bar_base;
    const int tid = threadIdx.x;

    // per-stage quad of this thread: plane offset, x-neighbour offsets, active
    int mid[M + 1], mxl[M + 1], mxh[M + 1];
    bool mact[M + 1];
#pragma unroll
    for (int k = 1; k < M; ++k) {
        const int u = tid + k * TB_QX;
        const int yl = u / TB_QX, qx = u - yl * TB_QX;
        mact[k] = tid < (C::EY - 2 * k) * TB_QX;
        mid[k] = yl * TB_EX + 4 * qx;
        mxl[k] = qx > 0 ? -1 : 0;             // the tile's outer columns read themselves
        mxh[k] = qx < TB_QX - 1 ? 4 : 3;      // (their results are never used)
    }
    // replay: stage k < M also stores its quads that lie in the output tile
    bool mrec[M + 1];
    int mxo[M + 1], myo[M + 1];  // tile column of the quad's first voxel minus the x halo, row minus M
#pragma unroll
    for (int k = 0; k <= M; ++k) {
        const int u = tid + k * TB_QX;
        const int yl = u / TB_QX, qx = u - yl * TB_QX;
        mrec[k] = REC && k >= 1 && k < M && tid < (C::EY - 2 * k) * TB_QX && yl >= M && yl < C::EY - M &&
                  qx >= 1 && qx < TB_QX - 1;
        mxo[k] = 4 * qx - TB_HX;
        myo[k] = yl - M;
    }
    mact[M] = tid < C::NQO;
    mid[M] = (M + tid / 16) * TB_EX + 4 * (1 + tid % 16);
    mxl[M] = -1;
    mxh[M] = 4;
    mid[0] = mxl[0] = mxh[0] = 0;
    mact[0] = false;

    constexpr int PD = 2;  // stage-0 planes requested ahead of the one consumed
    // item queue: the current item and the next one, both known to every thread;
    // thread 0 takes the one after next during the current item (after its first
    // barrier, when every thread has read the current entry) and the next item's
    // first planes are requested before the current one ends
    __shared__ int s_q[2];
    if (tid == 0) {
        const int i0 = items.start();
        s_q[0] = i0;
        s_q[1] = i0 < nitems ? items.after(i0) : nitems;
        if (i0 < nitems) {  // the first PD planes of the first item
            int local;
            const CUtensorMap *mp;
            const TBTile &T = get(i0, local, mp);
            int X0, Y0, zb, ze;
            tb_item_geom<M, V>(T, local, X0, Y0, zb, ze);
#pragma unroll
            for (int j = 0; j < PD; ++j) tb_issue<M, V>(P, (int)((P.nload + j) % S0), mp, X0, Y0, zb - M + j);
        }
    }
    __syncthreads();
    int qk = 0;
    int item = s_q[0], nxt = s_q[1];
    while (item < nitems) {
        int local;
        const CUtensorMap *maps;
        decltype(auto) A = get(item, local, maps);
        int X0, Y0, zb, ze;
        tb_item_geom<M, V>(A, local, X0, Y0, zb, ze);
        const int L = ze - zb + 2 * M;   // stage-0 planes zb-M .. ze+M-1
        // output quad of this thread
        const int xg0 = X0 + 4 * (tid % 16);
        const int yg = Y0 + tid / 16;
        const bool out_quad = mact[M] && yg < A.ny && xg0 < A.nx;
        const int nin = A.nx - xg0;      // voxels of the quad inside the grid (>= 4: all)

        // ring-0 slot offsets of planes p0 - d (d = 0 .. S0-1); stage-ring slots of
        // planes p0 - d: e[d % 3] (3-slot rings), f[d % 4] (the last ring); all
        // rotate once per plane
        int s0_cur = (int)(P.nload % S0);
        uint32_t phase = (uint32_t)((P.nload / S0) & 1);
        int r0[S0];
#pragma unroll
        for (int d = 0; d < S0; ++d) r0[d] = ((s0_cur - d + S0) % S0) * C::SLOT0;
        int e[3] = {0, 2, 1};
        int f[4] = {0, 3, 2, 1};
        float4 k1ch = make_float4(0.f, 0.f, 0.f, 0.f), k1cl = k1ch, k1mh = k1ch, k1ml = k1ch;

        for (int it = 0; it < L; ++it, ++P.nload) {
            const int p0 = zb - M + it;
            const int s0_next = s0_cur + 1 == S0 ? 0 : s0_cur + 1;
            // output-stage operands of plane p0 - M, loaded early to hide their latency
            const int qo = p0 - M;
            // (checked build: the output quad's global words lie in the grid's arrays)
            const bool out_now =
                out_quad && it >= 2 * M && qo >= 0 && qo < A.nz &&
                RFA_CHECK_RANGE((size_t)qo * A.plane + (size_t)yg * A.pitch + xg0,
                                (size_t)qo * A.plane + (size_t)yg * A.pitch + xg0 + 4, A.plane * A.nz, xg0, 4, status);
            const size_t gio = out_now ? (size_t)qo * A.plane + (size_t)yg * A.pitch + xg0 : 0;
            float4 carry4 = make_float4(0.f, 0.f, 0.f, 0.f);
            uint32_t latch4 = 0;
            double2 om01 = make_double2(0.0, 0.0), om23 = om01;
            if (out_now && !REC) {
                latch4 = *reinterpret_cast<const uint32_t *>(A.latch + gio);
                if (DMG) carry4 = *reinterpret_cast<const float4 *>(A.omega_c + gio);
                if (DMG && FOLD) {
                    om01 = reinterpret_cast<const double2 *>(A.omega + gio)[0];
                    om23 = reinterpret_cast<const double2 *>(A.omega + gio)[1];
                }
            }
            const bool ok = mbar_wait(bar_base + 8u * s0_cur, phase, LIM ? P.limit : kDefaultLimit,
                                      LIM ? P.hint : kSuspendNs);
            // the last stage's coefficients (plane p0 - M) go to registers before the
            // last barrier: its ring-0 slot is then refilled right after that barrier
            uint4 wM = make_uint4(0u, 0u, 0u, 0u);
            float4 sM = make_float4(0.f, 0.f, 0.f, 0.f);
            if (mact[M] && it >= 2 * M) {
                wM = *reinterpret_cast<const uint4 *>(sm + r0[M] + 2 * PLANE + mid[M]);
                sM = ld4(sm, r0[M] + 3 * PLANE + mid[M]);
            }
#pragma unroll
            for (int k = 1; k <= M; ++k) {
                if (it >= 2 * k && mact[k] && tb_stage_smem_ok<M, V>(k, r0, e, f, mid[k], status)) {
                    const int id = mid[k];
                    const int cb = r0[k];                     // coefficients of plane q = p0 - k
                    int bc, bm, bp;                           // planes q, q - 1, q + 1 of stage k - 1
                    if (k == 1) {
                        bc = r0[1];
                        bm = r0[2];
                        bp = r0[0];
                    } else {
                        const int rk = C::ring_off(k - 1), sl = C::ring_planes(k - 1) * PLANE;
                        if (k == M) {  // the last ring: 4 slots
                            bc = rk + f[k % 4] * sl;
                            bm = rk + f[(k + 1) % 4] * sl;
                            bp = rk + f[(k - 1) % 4] * sl;
                        } else {
                            bc = rk + e[k % 3] * sl;
                            bm = rk + e[(k + 1) % 3] * sl;
                            bp = rk + e[(k - 1) % 3] * sl;
                        }
                    }
                    float4 ch, cl, zmh, zml;
                    if (k == 1 && it > 2) {  // this column's planes p0-2, p0-1, kept from the last iteration
                        ch = k1ch; cl = k1cl; zmh = k1mh; zml = k1ml;
                    } else {
                        ch = ld4(sm, bc + id); cl = ld4(sm, bc + PLANE + id);
                        zmh = ld4(sm, bm + id); zml = ld4(sm, bm + PLANE + id);
                    }
                    const float4 ymh = ld4(sm, bc + id - TB_EX), yml = ld4(sm, bc + PLANE + id - TB_EX);
                    const float4 yph = ld4(sm, bc + id + TB_EX), ypl = ld4(sm, bc + PLANE + id + TB_EX);
                    const float4 zph = ld4(sm, bp + id), zpl = ld4(sm, bp + PLANE + id);
                    if (k == 1) { k1mh = ch; k1ml = cl; k1ch = zph; k1cl = zpl; }
                    const float lh = sm[bc + id + mxl[k]], ll = sm[bc + PLANE + id + mxl[k]];
                    const float rh = sm[bc + id + mxh[k]], rl = sm[bc + PLANE + id + mxh[k]];
                    const uint4 w4 = k == M ? wM : *reinterpret_cast<const uint4 *>(sm + cb + 2 * PLANE + id);
                    const float4 s4 = k == M ? sM : ld4(sm, cb + 3 * PLANE + id);
                    // voxel pairs (0,1) and (2,3) of the quad
                    const float2 C01 = make_float2(ch.x, ch.y), C23 = make_float2(ch.z, ch.w);
                    const float2 L01 = make_float2(cl.x, cl.y), L23 = make_float2(cl.z, cl.w);
                    // neighbour differences in the fixed order x-, x+, y-, y+, z-, z+; the x
                    // differences voxel by voxel, written into the halves of the pairs
                    const float xh[6] = {lh, ch.x, ch.y, ch.z, ch.w, rh}, xl[6] = {ll, cl.x, cl.y, cl.z, cl.w, rl};
                    float dm[4], dp[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        dm[j] = cdiff(xh[j], xl[j], xh[j + 1], xl[j + 1]);
                        dp[j] = cdiff(xh[j + 2], xl[j + 2], xh[j + 1], xl[j + 1]);
                    }
                    float2 S01 = add2(make_float2(dm[0], dm[1]), make_float2(dp[0], dp[1]));
                    float2 S23 = add2(make_float2(dm[2], dm[3]), make_float2(dp[2], dp[3]));
                    S01 = add2(S01, cdiff2(make_float2(ymh.x, ymh.y), make_float2(yml.x, yml.y), C01, L01));
                    S23 = add2(S23, cdiff2(make_float2(ymh.z, ymh.w), make_float2(yml.z, yml.w), C23, L23));
                    S01 = add2(S01, cdiff2(make_float2(yph.x, yph.y), make_float2(ypl.x, ypl.y), C01, L01));
                    S23 = add2(S23, cdiff2(make_float2(yph.z, yph.w), make_float2(ypl.z, ypl.w), C23, L23));
                    S01 = add2(S01, cdiff2(make_float2(zmh.x, zmh.y), make_float2(zml.x, zml.y), C01, L01));
                    S23 = add2(S23, cdiff2(make_float2(zmh.z, zmh.w), make_float2(zml.z, zml.w), C23, L23));
                    S01 = add2(S01, cdiff2(make_float2(zph.x, zph.y), make_float2(zpl.x, zpl.y), C01, L01));
                    S23 = add2(S23, cdiff2(make_float2(zph.z, zph.w), make_float2(zpl.z, zpl.w), C23, L23));
                    const float2 a01 = make_float2(bf16_to_float(w4.x & 0xffffu), bf16_to_float(w4.y & 0xffffu));
                    const float2 a23 = make_float2(bf16_to_float(w4.z & 0xffffu), bf16_to_float(w4.w & 0xffffu));
                    const float2 b01 = make_float2(bf16_to_float(w4.x >> 16), bf16_to_float(w4.y >> 16));
                    const float2 b23 = make_float2(bf16_to_float(w4.z >> 16), bf16_to_float(w4.w >> 16));
                    float2 H01, H23, N01, N23, T01, T23;
                    cupdate2(C01, L01, S01, a01, b01, make_float2(s4.x, s4.y), H01, N01, T01);
                    cupdate2(C23, L23, S23, a23, b23, make_float2(s4.z, s4.w), H23, N23, T23);
                    // running Arrhenius sum and maximum of the values of stages 1 .. k-1
                    float2 P01 = make_float2(0.f, 0.f), P23 = P01, X01 = T01, X23 = T23;
                    if (k >= 2) {
                        if (DMG) {
                            P01 = arrhenius_inc2(T01, A.c0, A.c1, A.TK0);
                            P23 = arrhenius_inc2(T23, A.c0, A.c1, A.TK0);
                        }
                        if (k >= 3) {  // earlier stages' sum and maximum, stored with the values
                            const float4 pp = ld4(sm, bc + 2 * PLANE + id), pm = ld4(sm, bc + 3 * PLANE + id);
                            if (DMG) {
                                P01 = add2(make_float2(pp.x, pp.y), P01);
                                P23 = add2(make_float2(pp.z, pp.w), P23);
                            }
                            X01 = make_float2(fmaxf(pm.x, T01.x), fmaxf(pm.y, T01.y));
                            X23 = make_float2(fmaxf(pm.z, T23.x), fmaxf(pm.w, T23.y));
                        }
                    }
                    if (k < M) {
                        const int ro = C::ring_off(k), sl = C::ring_planes(k) * PLANE;
                        const int bo = ro + (k == M - 1 ? f[k % 4] : e[k % 3]) * sl;
                        *reinterpret_cast<float4 *>(sm + bo + id) = make_float4(H01.x, H01.y, H23.x, H23.y);
                        *reinterpret_cast<float4 *>(sm + bo + PLANE + id) = make_float4(N01.x, N01.y, N23.x, N23.y);
                        if (k >= 2) {
                            *reinterpret_cast<float4 *>(sm + bo + 2 * PLANE + id) =
                                make_float4(P01.x, P01.y, P23.x, P23.y);
                            *reinterpret_cast<float4 *>(sm + bo + 3 * PLANE + id) =
                                make_float4(X01.x, X01.y, X23.x, X23.y);
                        }
                        if (REC && mrec[k]) {
                            const int q = p0 - k, xr = X0 + mxo[k], yr = Y0 + myo[k];
                            const size_t ro_ = (size_t)(k - 1) * A.rec_stride + (size_t)(q > 0 ? q : 0) * A.plane +
                                               (size_t)yr * A.pitch + (xr > 0 ? xr : 0);
                            if (q >= zb && q < ze && yr < A.ny && xr < A.nx &&  // this item's planes only
                                RFA_CHECK_RANGE(ro_, ro_ + 4, (size_t)(M - 1) * A.rec_stride, ro_, 4, status)) {
                                float *dst = A.rec_hi + (size_t)(k - 1) * A.rec_stride + (size_t)q * A.plane +
                                             (size_t)yr * A.pitch + xr;
                                *reinterpret_cast<float4 *>(dst) = make_float4(H01.x, H01.y, H23.x, H23.y);
                            }
                        }
                    } else if (out_now) {
                        // last stage: this step's own value, then the output quad (16-byte
                        // aligned: X0 % 64 == 0, pitch % 4 == 0; padding voxels compute to 0)
                        const float2 V01 = add2(H01, N01), V23 = add2(H23, N23);
                        *reinterpret_cast<float4 *>(A.hi_out + gio) = make_float4(H01.x, H01.y, H23.x, H23.y);
                        *reinterpret_cast<float4 *>(A.lo_out + gio) = make_float4(N01.x, N01.y, N23.x, N23.y);
                        bad |= !(isfinite(H01.x) && isfinite(H01.y) && isfinite(H23.x) && isfinite(H23.y));
                        if (!REC) {  // latch and damage (the replay leaves them alone)
                            const float mx[4] = {fmaxf(X01.x, V01.x), fmaxf(X01.y, V01.y), fmaxf(X23.x, V23.x),
                                                 fmaxf(X23.y, V23.y)};
                            uint32_t lbits = 0;
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if (j < nin && mx[j] >= A.thr) lbits |= 1u << (8 * j);
                            if ((latch4 | lbits) != latch4)
                                *reinterpret_cast<uint32_t *>(A.latch + gio) = latch4 | lbits;
                            if (DMG) {
                                P01 = add2(P01, arrhenius_inc2(V01, A.c0, A.c1, A.TK0));
                                P23 = add2(P23, arrhenius_inc2(V23, A.c0, A.c1, A.TK0));
                                const float part[4] = {P01.x, P01.y, P23.x, P23.y};
                                float Pc[4] = {carry4.x, carry4.y, carry4.z, carry4.w};
#pragma unroll
                                for (int j = 0; j < 4; ++j)
                                    if (j < nin) Pc[j] = __fadd_rn(Pc[j], part[j]);
                                if (FOLD) {
                                    double om[4] = {om01.x, om01.y, om23.x, om23.y};
#pragma unroll
                                    for (int j = 0; j < 4; ++j)
                                        if (j < nin) carry_fold(om[j], Pc[j]);
                                    double2 *op = reinterpret_cast<double2 *>(A.omega + gio);
                                    op[0] = make_double2(om[0], om[1]);
                                    op[1] = make_double2(om[2], om[3]);
                                }
                                *reinterpret_cast<float4 *>(A.omega_c + gio) = make_float4(Pc[0], Pc[1], Pc[2], Pc[3]);
                            }
                        }
                    }
                }
                // a barrier after every stage but the last: the next plane's stages
                // 1 .. M-1 touch no slot the last stage still reads (4-slot last ring,
                // its coefficients already in registers), so warps without a quad in
                // the last stage go straight on to the next plane
                if (k == 1) {
                    // the stage-1 barrier also agrees on the stage-0 wait: a CTA whose
                    // wait timed out leaves (stage 1 only wrote shared memory)
                    if (__syncthreads_or(!ok)) {
                        if (tid == 0) {
                            // let every request in flight land before the CTA's shared
                            // memory is released (bounded): this plane, and the next one,
                            // requested one iteration ago if it exists
                            atomicOr(status, kStatusTimeout);
                            const long long last = P.nload + ((it + 1 < L || nxt < nitems) ? 1 : 0);
                            for (long long q = P.nload; q <= last; ++q)
                                mbar_wait(bar_base + 8u * (uint32_t)(q % S0), (uint32_t)((q / S0) & 1),
                                          kDrainLimit, kSuspendNs);
                        }
                        return false;
                    }
                } else if (k < M) {
                    __syncthreads();
                }
                if (k == 1 && it == 0 && tid == 0) s_q[qk] = nxt < nitems ? items.after(nxt) : nitems;
                if (k == M - 1 && tid == 0) {
                    // every read of plane p0 - M's slot is done: request plane p0 + PD
                    // into it (of this item, else of the next one)
                    const int s0_pd = s0_cur + PD >= S0 ? s0_cur + PD - S0 : s0_cur + PD;
                    if (it + PD < L) {
                        tb_issue<M, V>(P, s0_pd, maps, X0, Y0, p0 + PD);
                    } else if (nxt < nitems) {
                        int local1;
                        const CUtensorMap *maps1;
                        decltype(auto) T1 = get(nxt, local1, maps1);
                        int X1, Y1, zb1, ze1;
                        tb_item_geom<M, V>(T1, local1, X1, Y1, zb1, ze1);
                        tb_issue<M, V>(P, s0_pd, maps1, X1, Y1, zb1 - M + (it + PD - L));
                    }
                }
            }
            // rotate the ring slots by one plane
            const int t0 = r0[S0 - 1];
#pragma unroll
            for (int d = S0 - 1; d > 0; --d) r0[d] = r0[d - 1];
            r0[0] = t0;
            const int t1 = e[2];
            e[2] = e[1];
            e[1] = e[0];
            e[0] = t1;
            const int t2 = f[3];
            f[3] = f[2];
            f[2] = f[1];
            f[1] = f[0];
            f[0] = t2;
            if (s0_next == 0) phase ^= 1u;
            s0_cur = s0_next;
        }
        item = nxt;
        nxt = s_q[qk];
        qk ^= 1;
    }
    return true;
}

template <int M, int V>
__device__ __forceinline__ bool tb_setup(TBPipe &P, unsigned *status)
{
    using C = Cfg<M, V>;
    extern __shared__ __align__(128) float sm[];
    P.sm = sm;
    P.sm_base = smem_u32(sm);
    P.bar_base = P.sm_base + 4u * C::BAR_OFF;
    P.nload = 0;
    P.limit = g_wait_limit_mbar;
    P.hint = suspend_hint(P.limit);
    if (P.sm_base & 127u) {  // TMA destinations need 128-byte alignment
        if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
        return false;
    }
    if (threadIdx.x == 0) {
        for (int j = 0; j < C::S0; ++j) mbar_init(P.bar_base + 8u * j, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    return true;
}

struct TBMaps {
    CUtensorMap m[4];
};

// one grid, M steps
template <int M, int V, bool DMG, bool FOLD, bool REC, bool LIM>
__global__ void __launch_bounds__(Cfg<M, V>::THREADS, Cfg<M, V>::MINB)
    k_step_tb(const __grid_constant__ TBMaps maps, const TBTile T0, unsigned *status)
{
    TBPipe P;
    if (!tb_setup<M, V>(P, status)) return;
    // the descriptor stays in kernel-parameter space (constant-bank operands).
    // The reference returned is to the kernel's own parameter, which outlives
    // every call of the lambda; the compiler's "reference to local" note does
    // not apply (a pointer to a __grid_constant__ copy instead cost 3 % more
    // instructions).
#pragma nv_diag_suppress 836
    auto get = [&](int item, int &local, const CUtensorMap *&mp) -> const TBTile & {
        local = item;
        mp = maps.m;
        return T0;
    };
#pragma nv_diag_default 836
    bool bad = false;
    tb_run<M, V, DMG, FOLD, REC, LIM>(P, StrideItems{(int)blockIdx.x, (int)gridDim.x}, T0.xt * T0.yt * T0.zc, get,
                                      status, bad);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusNonfinite);
}

// ------------------------------------------------------------------ batch
// A batch member: tile descriptors for both ping-pong parities (tile[p] reads
// state p and writes state p ^ 1), its first work item and its parity at t = 0.
struct TBMember {
    TBTile tile[2];
    int item_begin, cur0;
};

// Software grid barrier for a cooperative (co-resident) grid; bounded spin
// (limit in SM cycles).  bar[0] counts arrivals, bar[1] is the generation.
__device__ bool grid_sync(unsigned *bar, unsigned nblocks, long long limit)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        int ok = 1;
        if (arrived == nblocks) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g) {
                if (clock64() - t0 > limit) {
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// every member, ntime blocks of M steps, one persistent launch
template <int M, int V, bool DMG, bool LIM>
__global__ void __launch_bounds__(Cfg<M, V>::THREADS, Cfg<M, V>::MINB)
    k_batch_tb(const TBMember *mem, int nmem, int nitems, int ntime, int fold_every, unsigned *gbar,
               unsigned *status)
{
    TBPipe P;
    if (!tb_setup<M, V>(P, status)) return;
    const long long glimit = LIM ? g_wait_limit_grid : kDefaultLimit;
    bool bad = false;
    for (int t = 0; t < ntime; ++t) {
        auto get = [&](int item, int &local, const CUtensorMap *&mp) -> TBTile {
            int lo = 0, hi = nmem - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (mem[mid].item_begin <= item) lo = mid;
                else hi = mid - 1;
            }
            local = item - mem[lo].item_begin;
            const TBTile T = mem[lo].tile[(mem[lo].cur0 + t) & 1];  // register copy of the global descriptor
            mp = T.maps;
            return T;
        };
        const bool fold = DMG && ((t + 1) % fold_every == 0 || t == ntime - 1);
        const ClaimedItems items{gbar + 2 + t};  // one counter per time block, zeroed before the launch
        const bool ok = fold ? tb_run<M, V, DMG, true, false, LIM>(P, items, nitems, get, status, bad)
                             : tb_run<M, V, DMG, false, false, LIM>(P, items, nitems, get, status, bad);
        if (!ok) break;
        if (!grid_sync(gbar, gridDim.x, glimit)) {
            if (threadIdx.x == 0) atomicOr(status, kStatusTimeout | kStatusGridTimeout);
            break;
        }
        // the next block's TMA (async proxy) reads what other CTAs just stored
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusNonfinite);
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

int variant_ey(int variant) { return tile_ey(variant); }

// tiles and balanced z chunks of one grid: the busiest of `resident` persistent
// CTAs should stream as few planes as possible (each item costs chunk + 2M planes)
template <int M, int V>
void tile_plan(const rfa_grid *g, int resident, int max_chunk, TBTile &T)
{
    using C = Cfg<M, V>;
    T.xt = (g->nx + TB_TX - 1) / TB_TX;
    T.yt = (g->ny + C::TY - 1) / C::TY;
    const long long tiles = (long long)T.xt * T.yt;
    int best_zc = 1;
    double best = 1e300;
    for (int zc = 1; zc <= g->nz; ++zc) {
        const long long items = tiles * zc;
        const long long per_cta = (items + resident - 1) / resident;
        const double cost = (double)per_cta * ((double)g->nz / zc + 2.0 * M);
        if ((double)g->nz / zc <= max_chunk && cost < best * 0.999) {
            best = cost;
            best_zc = zc;
        }
        if ((double)g->nz / zc < 2.0 * M) break;
    }
    T.zc = best_zc;
}

void fill_tile(const rfa_grid *g, int parity, TBTile &T)
{
    T.maps = nullptr;
    T.hi_out = (float *)g->th[parity ^ 1];
    T.lo_out = (float *)g->lo[parity ^ 1];
    T.latch = g->latch;
    T.omega = g->omega;
    T.omega_c = g->omega_c;
    T.nx = g->nx;
    T.ny = g->ny;
    T.nz = g->nz;
    T.pitch = g->pitch;
    T.plane = g->plane;
    T.thr = (float)(g->T_thr - g->T_a);
    DamageConst dc = damage_consts(g);
    T.c0 = dc.c0;
    T.c1 = dc.c1;
    T.TK0 = dc.TK0;
    T.rec_hi = nullptr;
    T.rec_stride = g->nvp;
}

// set while rfa_set_wait_limits has set limits other than the default (process-wide)
std::atomic<bool> g_limits_set{false};

template <int M, int V, bool DMG, bool FOLD, bool REC, bool LIM>
cudaError_t launch_inst_lim(rfa_grid *g, const TBMaps &maps, TBTile T)
{
    using C = Cfg<M, V>;
    cudaError_t e = cudaFuncSetAttribute(k_step_tb<M, V, DMG, FOLD, REC, LIM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    const int resident = 148 * C::MINB;
    tile_plan<M, V>(g, resident, 1 << 30, T);
    const long long items = (long long)T.xt * T.yt * T.zc;
    const unsigned grid = (unsigned)(items < resident ? items : resident);
    k_step_tb<M, V, DMG, FOLD, REC, LIM><<<grid, C::THREADS, C::SMEM, g->stream>>>(maps, T, g->status);
    return cudaGetLastError();
}

template <int M, int V, bool DMG, bool FOLD, bool REC = false>
cudaError_t launch_inst(rfa_grid *g, const TBMaps &maps, TBTile T)
{
    return g_limits_set.load() ? launch_inst_lim<M, V, DMG, FOLD, REC, true>(g, maps, T)
                               : launch_inst_lim<M, V, DMG, FOLD, REC, false>(g, maps, T);
}

// shared-memory opt-in and the co-resident grid size of the batch kernel
// (host-side queries, kept outside stream capture)
template <int M, int V, bool DMG>
cudaError_t prepare_batch_inst(int nitems, int *grid)
{
    using C = Cfg<M, V>;
    // both instantiations (default and test wait limits): shared-memory opt-in, and the
    // co-resident grid of the one with the lower occupancy
    cudaError_t e = cudaFuncSetAttribute(k_batch_tb<M, V, DMG, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_batch_tb<M, V, DMG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             C::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per_sm = 0, per_sm_lim = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_tb<M, V, DMG, false>, C::THREADS, C::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_lim, k_batch_tb<M, V, DMG, true>, C::THREADS,
                                                      C::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm_lim < per_sm) per_sm = per_sm_lim;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid = nsm * per_sm < nitems ? nsm * per_sm : nitems;
    return cudaSuccess;
}

template <int M, int V, bool DMG>
cudaError_t launch_batch_inst(const TBMember *mem, int nmem, int nitems, int ntime, int fold_every,
                              unsigned *gbar, unsigned *status, cudaStream_t stream, int grid)
{
    using C = Cfg<M, V>;
    // cooperative launch: every CTA is resident at once, which the grid barrier needs
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)C::THREADS);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (g_limits_set.load())
        return cudaLaunchKernelEx(&cfg, k_batch_tb<M, V, DMG, true>, mem, nmem, nitems, ntime, fold_every, gbar, status);
    return cudaLaunchKernelEx(&cfg, k_batch_tb<M, V, DMG, false>, mem, nmem, nitems, ntime, fold_every, gbar, status);
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

cudaError_t tb_set_wait_limits(long long mbar_cycles, long long grid_cycles)
{
    cudaError_t e = cudaMemcpyToSymbol(g_wait_limit_mbar, &mbar_cycles, sizeof mbar_cycles);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbol(g_wait_limit_grid, &grid_cycles, sizeof grid_cycles);
    if (e != cudaSuccess) return e;
    g_limits_set.store(mbar_cycles != kDefaultLimit || grid_cycles != kDefaultLimit);
    return cudaSuccess;
}

bool tb_limits_set() { return g_limits_set.load(); }

bool tb_supported(const rfa_grid *g, int depth, int variant)
{
    if (g->sp != RFA_STATE_F32C || g->pp != RFA_PARAM_BF16) return false;
    if (variant < 0 || variant > 1) return false;
    if (g->face != RFA_FACE_DIRICHLET) return false;  // insulated faces: one-step kernel
    if (g->cond != RFA_COND_CENTRE || g->alpha_perf) return false;  // model options: their own kernel
    if (variant == 0 && (depth < 2 || depth > 3)) return false;
    if (variant >= 1 && depth != 2) return false;
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

bool tb_make_maps(const rfa_grid *g, int variant, const void *th_in, const void *lo_in, CUtensorMap out[4])
{
    const int ey = variant_ey(variant);
    auto &c = map_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto key = std::make_tuple((const rfa_grid *)g, th_in, lo_in, ey);
    auto it = c.m.find(key);
    if (it == c.m.end()) {
        std::array<CUtensorMap, 4> maps;
        if (!make_map(&maps[0], th_in, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g, ey) ||
            !make_map(&maps[1], lo_in, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g, ey) ||
            !make_map(&maps[2], g->ab, CU_TENSOR_MAP_DATA_TYPE_UINT32, g, ey) ||
            !make_map(&maps[3], g->s, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g, ey))
            return false;
        it = c.m.emplace(key, maps).first;
    }
    for (int k = 0; k < 4; ++k) out[k] = it->second[k];
    return true;
}

cudaError_t launch_step_tb(rfa_grid *g, int depth, int variant, const void *th_in, const void *lo_in,
                           void *th_out, void *lo_out, bool damage, bool fold)
{
    TBMaps maps;
    if (!tb_make_maps(g, variant, th_in, lo_in, maps.m)) return cudaErrorInvalidValue;
    TBTile T;
    fill_tile(g, g->th[0] == th_in ? 0 : 1, T);
    T.hi_out = (float *)th_out;
    T.lo_out = (float *)lo_out;
#define TB_CASE(MV, VV)                                                                 \
    if (depth == MV && variant == VV)                                                        \
        return !damage ? launch_inst<MV, VV, false, false>(g, maps, T)                 \
               : fold  ? launch_inst<MV, VV, true, true>(g, maps, T)                   \
                       : launch_inst<MV, VV, true, false>(g, maps, T);
    TB_CASE(2, 0)
    TB_CASE(3, 0)
    TB_CASE(2, 1)
#undef TB_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_tb_rec(rfa_grid *g, int depth, int variant, const void *th_in, const void *lo_in,
                               void *th_out, void *lo_out, float *rec_hi)
{
    TBMaps maps;
    if (!tb_make_maps(g, variant, th_in, lo_in, maps.m)) return cudaErrorInvalidValue;
    TBTile T;
    fill_tile(g, 0, T);
    T.hi_out = (float *)th_out;
    T.lo_out = (float *)lo_out;
    T.rec_hi = rec_hi;
    if (depth == 2 && variant == 0) return launch_inst<2, 0, false, false, true>(g, maps, T);
    if (depth == 3 && variant == 0) return launch_inst<3, 0, false, false, true>(g, maps, T);
    if (depth == 2 && variant == 1) return launch_inst<2, 1, false, false, true>(g, maps, T);
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ batch host side
// Descriptor of one member for both parities; `maps_dev` receives 8 tensor maps
// (parity 0 then 1) that the caller copies to device memory at `maps_dev_addr`.
bool tb_batch_member(const rfa_grid *g, int depth, int variant, int max_chunk, TBMemberHost &out)
{
    TBTile T;
    fill_tile(g, 0, T);
    const int ey = variant_ey(variant);
    // batch items: every member's tiles with z chunks of at most max_chunk planes
    // (the persistent grid balances the many items of all members)
    T.xt = (g->nx + TB_TX - 1) / TB_TX;
    T.yt = (g->ny + (ey - 2 * depth) - 1) / (ey - 2 * depth);
    T.zc = (g->nz + max_chunk - 1) / max_chunk;
    for (int p = 0; p < 2; ++p) {
        if (!tb_make_maps(g, variant, g->th[p], g->lo[p], out.maps + 4 * p)) return false;
        fill_tile(g, p, out.tile[p]);
        out.tile[p].xt = T.xt;
        out.tile[p].yt = T.yt;
        out.tile[p].zc = T.zc;
    }
    out.items = T.xt * T.yt * T.zc;
    return true;
}

size_t tb_member_bytes() { return sizeof(TBMember); }

void tb_pack_member(const TBMemberHost &h, const CUtensorMap *maps_dev, int item_begin, int cur0, void *dst)
{
    TBMember m;
    for (int p = 0; p < 2; ++p) {
        m.tile[p] = h.tile[p];
        m.tile[p].maps = maps_dev + 4 * p;
    }
    m.item_begin = item_begin;
    m.cur0 = cur0;
    std::memcpy(dst, &m, sizeof m);
}

cudaError_t prepare_batch_tb(int depth, int variant, bool damage, int nitems, int *grid)
{
#define PREP_CASE(MV, VV)                                                              \
    if (depth == MV && variant == VV)                                                       \
        return damage ? prepare_batch_inst<MV, VV, true>(nitems, grid)                 \
                      : prepare_batch_inst<MV, VV, false>(nitems, grid);
    PREP_CASE(2, 0)
    PREP_CASE(3, 0)
    PREP_CASE(2, 1)
#undef PREP_CASE
    return cudaErrorInvalidValue;
}

// A two-node graph (barrier reset, then the batch kernel as a cooperative
// kernel node): stream capture does not accept cooperative launches.
template <int M, int V, bool DMG>
cudaError_t graph_batch_inst(const TBMember *mem, int nmem, int nitems, int ntime, int fold_every,
                             unsigned *gbar, unsigned *status, int grid, cudaGraphExec_t *exec)
{
    using C = Cfg<M, V>;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    cudaGraphNode_t nmemset = nullptr, nkernel = nullptr;
    cudaMemsetParams mp = {};
    mp.dst = gbar;
    mp.value = 0;
    mp.elementSize = sizeof(unsigned);
    mp.width = 2 + (size_t)ntime;  // grid barrier and one item counter per time block
    mp.height = 1;
    mp.pitch = 0;
    e = cudaGraphAddMemsetNode(&nmemset, graph, nullptr, 0, &mp);
    void *args[] = {(void *)&mem, (void *)&nmem, (void *)&nitems, (void *)&ntime, (void *)&fold_every,
                    (void *)&gbar, (void *)&status};
    if (e == cudaSuccess) {
        cudaKernelNodeParams kp = {};
        kp.func = g_limits_set.load() ? (void *)k_batch_tb<M, V, DMG, true> : (void *)k_batch_tb<M, V, DMG, false>;
        kp.gridDim = dim3((unsigned)grid);
        kp.blockDim = dim3((unsigned)C::THREADS);
        kp.sharedMemBytes = C::SMEM;
        kp.kernelParams = args;
        e = cudaGraphAddKernelNode(&nkernel, graph, &nmemset, 1, &kp);
    }
    if (e == cudaSuccess) {
        cudaLaunchAttributeValue v = {};
        v.cooperative = 1;
        e = cudaGraphKernelNodeSetAttribute(nkernel, cudaLaunchAttributeCooperative, &v);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

cudaError_t graph_batch_tb(int depth, int variant, bool damage, const void *members_dev, int nmem, int nitems,
                           int ntime, unsigned *gbar, unsigned *status, int grid, cudaGraphExec_t *exec)
{
    const int fold_every = kCarrySteps / depth > 0 ? kCarrySteps / depth : 1;
    const TBMember *mem = (const TBMember *)members_dev;
#define GRAPH_CASE(MV, VV)                                                                                        \
    if (depth == MV && variant == VV)                                                                                  \
        return damage ? graph_batch_inst<MV, VV, true>(mem, nmem, nitems, ntime, fold_every, gbar, status, grid, exec) \
                      : graph_batch_inst<MV, VV, false>(mem, nmem, nitems, ntime, fold_every, gbar, status, grid, exec);
    GRAPH_CASE(2, 0)
    GRAPH_CASE(3, 0)
    GRAPH_CASE(2, 1)
#undef GRAPH_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_tb(int depth, int variant, bool damage, const void *members_dev, int nmem,
                            int nitems, int ntime, unsigned *gbar, unsigned *status, cudaStream_t stream, int grid)
{
    const int fold_every = kCarrySteps / depth > 0 ? kCarrySteps / depth : 1;
    const TBMember *mem = (const TBMember *)members_dev;
#define BATCH_CASE(MV, VV)                                                                                           \
    if (depth == MV && variant == VV)                                                                                     \
        return damage ? launch_batch_inst<MV, VV, true>(mem, nmem, nitems, ntime, fold_every, gbar, status, stream, grid) \
                      : launch_batch_inst<MV, VV, false>(mem, nmem, nitems, ntime, fold_every, gbar, status, stream, grid);
    BATCH_CASE(2, 0)
    BATCH_CASE(3, 0)
    BATCH_CASE(2, 1)
#undef BATCH_CASE
    return cudaErrorInvalidValue;
}

}  // namespace rfa
