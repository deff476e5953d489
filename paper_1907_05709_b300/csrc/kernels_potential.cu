// kernels_potential.cu -- the RF heat source of Linte's model, sigma |grad V|^2
// of Eq. 2675-eq1_Linte, from the electric potential of the needle: the second
// stencil of the path.
//
//   div(sigma grad V) = 0 on the free voxels, V = 1 on the electrode (voxels
//   within r0 of the needle's active segments, the geometry of the 1/r^4
//   source) and V = 0 on the outer faces (ground); face conductances are the
//   harmonic mean of the two voxels' sigma (per label).  Discretely, for a
//   free voxel i:  sum_nb sigma_f (V_i - V_nb) = 0, a symmetric positive
//   definite system in the free unknowns.
//
// Solver: preconditioned conjugate gradients (a multigrid V-cycle, below, or
// the inverse diagonal), matrix-free, to an FP64 relative residual (the source sets the heating of every later step;
// FP64 keeps the solve far below the FP32 state's resolution).  B300's FP64
// pipe is narrow, so the iterations run in FP32, with the residual replaced
// by the true FP64 one every time the FP32 residual has fallen by kInnerEta
// (CG with residual replacement, "reliable updates": van der Vorst and Ye's
// residual replacement for Krylov methods).  At a replacement the FP32
// correction e is added to the FP64 iterate x, r = b - A x is formed in FP64,
// and the Jacobi iteration goes on from the kept search direction with beta =
// (r.z)_new / (r.z)_old, so it keeps its Krylov information instead of
// restarting (the multigrid iteration restarts: see the host loop).  A cycle also ends when its FP32 residual has made no new 1 %
// low for kFlatChecks reads (FP32 stagnation).  A cycle that gains less than a
// factor 2 (FP32 at its attainable accuracy, about cond(A) * 2^-24) hands over
// to Jacobi-preconditioned FP64 conjugate gradients from the current x.  The
// stopping rule is the FP64 one either way: ||b - A x|| <= tol ||b||.  The diagonal and its inverse are stored once (no
// per-iteration division).  Scalars stay on the device; the host reads the
// residual every kCheck (Jacobi) or kCheckMg (multigrid) iterations.
//
// Heating: q_i = sum_nb sigma_f (V_nb - V_i)^2 / (2 h^2), each face's
// dissipation split between its two voxels, so that sum_i q_i h^3 equals the
// network's dissipated power; then q is scaled so that the free voxels receive
// the needle power P, exactly like the 1/r^4 weights (launch_source_write).
#include "rfa_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace rfa {

namespace {

constexpr int kCheck = 20;       // Jacobi iterations between host reads of the residual
constexpr int kCheckMg = 4;      // multigrid iterations between host reads (each costs several Jacobi ones)
constexpr int kFlatChecks = 10;  // a cycle ends early after this many reads without a 1 % lower FP32 residual
constexpr double kInnerEta = 1e-2;  // FP32 residual reduction between residual replacements
enum { CLS_FREE = 0, CLS_ELECTRODE = 1, CLS_GROUND = 2, CLS_PAD = 3 };
// scalars: rz, alpha, beta, rr, bb
enum { SC_RZ = 0, SC_ALPHA, SC_BETA, SC_RR, SC_BB, SC_N };

struct PotGrid {
    const uint8_t *cls, *label;
    const uint8_t *quni;  // per quad: 1 + the label shared by the quad and its neighbours, 0 if mixed
    const double *S;  // [kCondLabels][kCondLabels] face conductances
    int nx, ny, nz, pitch;
    size_t plane, nvp;
};

__device__ double pot_block_sum(double v)
{
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// neighbour index in direction d (x-, x+, y-, y+, z-, z+); false outside the grid
__device__ __forceinline__ bool pot_nb(const PotGrid &G, size_t i, int x, int y, int z, int d, size_t &j)
{
    switch (d) {
    case 0: j = i - 1; return x > 0;
    case 1: j = i + 1; return x + 1 < G.nx;
    case 2: j = i - G.pitch; return y > 0;
    case 3: j = i + G.pitch; return y + 1 < G.ny;
    case 4: j = i - G.plane; return z > 0;
    default: j = i + G.plane; return z + 1 < G.nz;
    }
}

__device__ __forceinline__ void pot_xyz(const PotGrid &G, size_t i, int &x, int &y, int &z)
{
    x = (int)(i % G.pitch);
    const size_t r = i / G.pitch;
    y = (int)(r % G.ny);
    z = (int)(r / G.ny);
}

// the per-iteration kernels: a warp per grid row (one 32-bit division per row
// instead of 64-bit ones per voxel), lanes along x; padding voxels untouched
#define POT_ROWS(G)                                                                                                 \
    for (int row = blockIdx.x * 8 + (int)(threadIdx.x >> 5); row < (G).ny * (G).nz; row += gridDim.x * 8)         \
        for (int y = row % (G).ny, z = row / (G).ny, x = threadIdx.x & 31; x < (G).nx; x += 32)

__device__ __forceinline__ size_t pot_at(const PotGrid &G, int x, int y, int z)
{
    return (size_t)z * G.plane + (size_t)y * G.pitch + x;
}

// Electrode: the voxels whose FP64 squared distance to the needle is at most
// r0^2.  The FP32 distance decides where it lies more than the margin from r0^2
// (the FP64 value is within the margin of it); the voxels near r0^2 take the
// FP64 value (needle_dist2_pruned equals needle_dist2), so the classes are those
// of the FP64 test everywhere.  A warp per grid row, lanes along x (padding
// included).
__global__ void __launch_bounds__(256) k_pot_class(NeedleGeom geom, PotGrid G, double h, float margin, uint8_t *cls)
{
    __shared__ float s32[kMaxSegments][7];
    load_seg32(geom, s32);
    __syncthreads();
    const double r02 = geom.r0 * geom.r0;
    const float r02f = (float)r02, hf = (float)h;
    for (int row = blockIdx.x * 8 + (int)(threadIdx.x >> 5); row < G.ny * G.nz; row += gridDim.x * 8) {
        const int y = row % G.ny, z = row / G.ny;
        for (int x = threadIdx.x & 31; x < G.pitch; x += 32) {
            uint8_t c = CLS_FREE;
            if (x >= G.nx) {
                c = CLS_PAD;
            } else if (x == 0 || y == 0 || z == 0 || x == G.nx - 1 || y == G.ny - 1 || z == G.nz - 1) {
                c = CLS_GROUND;
            } else {
                const float d32 = needle_dist2_f32(geom, s32, x * hf, y * hf, z * hf);
                bool el;
                if (d32 > r02f + margin) el = false;
                else if (d32 + margin < r02f) el = true;
                else el = needle_dist2_pruned(geom, s32, x * h, y * h, z * h, x * hf, y * hf, z * hf, margin) <= r02;
                if (el) c = CLS_ELECTRODE;
            }
            cls[pot_at(G, x, y, z)] = c;
        }
    }
}

// x0 = V on fixed voxels, 0 on free ones; r = b; z = r / D; p = z; partials of r.z and b.b
__global__ void __launch_bounds__(256) k_pot_init(PotGrid G, double *xv, double *r, double *zv, double *p,
                                                 double *Dv, double *iDv, double *part)
{
    __shared__ double S[kCondLabels * kCondLabels];
    for (int k = threadIdx.x; k < kCondLabels * kCondLabels; k += blockDim.x) S[k] = G.S[k];
    __syncthreads();
    double rz = 0.0, bb = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < G.nvp; i += (size_t)gridDim.x * blockDim.x) {
        const uint8_t c = G.cls[i];
        double xi = c == CLS_ELECTRODE ? 1.0 : 0.0, ri = 0.0, zi = 0.0;
        if (c == CLS_FREE) {
            int x, y, z;
            pot_xyz(G, i, x, y, z);
            const int l = G.label[i];
            double D = 0.0, b = 0.0;
            for (int d = 0; d < 6; ++d) {
                size_t j;
                if (!pot_nb(G, i, x, y, z, d, j)) continue;
                const double sf = S[l * kCondLabels + G.label[j]];
                D += sf;
                if (G.cls[j] == CLS_ELECTRODE) b += sf;
            }
            ri = b;
            const double iD = D > 0.0 ? 1.0 / D : 0.0;
            zi = b * iD;
            rz += ri * zi;
            bb += b * b;
            Dv[i] = D;
            iDv[i] = iD;
        }
        xv[i] = xi;
        r[i] = ri;
        zv[i] = zi;
        p[i] = zi;
    }
    rz = pot_block_sum(rz);
    bb = pot_block_sum(bb);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = rz;
        part[2 * blockIdx.x + 1] = bb;
    }
}

// Ap = A p on the free voxels; partial sums of p.Ap
__global__ void __launch_bounds__(256) k_pot_spmv(PotGrid G, const double *Dv, const double *p, double *Ap,
                                                 double *part)
{
    __shared__ double S[kCondLabels * kCondLabels];
    for (int k = threadIdx.x; k < kCondLabels * kCondLabels; k += blockDim.x) S[k] = G.S[k];
    __syncthreads();
    double acc = 0.0;
    POT_ROWS(G)
    {
        const size_t i = pot_at(G, x, y, z);
        if (G.cls[i] != CLS_FREE) continue;
        const int l = G.label[i];
        const double pi = p[i];
        double v = Dv[i] * pi;
        for (int d = 0; d < 6; ++d) {
            size_t j;
            if (pot_nb(G, i, x, y, z, d, j) && G.cls[j] == CLS_FREE) v -= S[l * kCondLabels + G.label[j]] * p[j];
        }
        Ap[i] = v;
        acc += pi * v;
    }
    acc = pot_block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// the scalar steps from the summed partials a (and b): which = 0 -> alpha =
// rz / a; 1 -> beta = a / rz, rz = a, rr = b; 2 -> a start: rz = a, rr = b
// (and b.b), beta = 0; 3 -> rr = a; 4 -> beta = a / rz, rz = a; 5 -> a start
// from r.z alone: rz = a, beta = 0; 6 -> rr = b
enum { SCW_ALPHA = 0, SCW_BETA_RR, SCW_START, SCW_RR, SCW_BETA, SCW_START_RZ, SCW_RR_B };
__device__ void pot_scalars_apply(int which, double a, double b, double *sc)
{
    if (which == SCW_ALPHA) {
        sc[SC_ALPHA] = a != 0.0 ? sc[SC_RZ] / a : 0.0;
    } else if (which == SCW_BETA_RR) {
        sc[SC_BETA] = sc[SC_RZ] != 0.0 ? a / sc[SC_RZ] : 0.0;
        sc[SC_RZ] = a;
        sc[SC_RR] = b;
    } else if (which == SCW_START) {
        sc[SC_RZ] = a;
        sc[SC_BB] = b;
        sc[SC_RR] = b;
        sc[SC_BETA] = 0.0;
    } else if (which == SCW_RR) {
        sc[SC_RR] = a;
    } else if (which == SCW_BETA) {
        sc[SC_BETA] = sc[SC_RZ] != 0.0 ? a / sc[SC_RZ] : 0.0;
        sc[SC_RZ] = a;
    } else if (which == SCW_START_RZ) {
        sc[SC_RZ] = a;
        sc[SC_BETA] = 0.0;
    } else {
        sc[SC_RR] = b;
    }
}

// sum of the per-block partials (one or two per block) in a fixed order, on one block
__device__ void pot_sum_partials(const double *part, int nblk, bool pairs, double &a, double &b)
{
    a = 0.0;
    b = 0.0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) {
        if (!pairs) {
            a += __ldcg(part + k);
        } else {
            a += __ldcg(part + 2 * k);
            b += __ldcg(part + 2 * k + 1);
        }
    }
    a = pot_block_sum(a);
    b = pot_block_sum(b);
}

// scalar steps on one block (which as in pot_scalars_apply)
__global__ void k_pot_scalars(const double *part, int nblk, int which, double *sc)
{
    double a, b;
    pot_sum_partials(part, nblk, which == SCW_BETA_RR || which == SCW_START || which == SCW_RR_B, a, b);
    if (threadIdx.x == 0) pot_scalars_apply(which, a, b, sc);
}

// after every block has written its partials: true in the last block to finish
// (the classic fence-and-count hand-over); that block then applies the scalar
// step itself and re-arms the counter, which saves a launch per reduction
__device__ bool pot_last_block(unsigned *ctr)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ctr, 1u) == gridDim.x - 1;
    __syncthreads();
    return last;
}

// x += alpha p; r -= alpha Ap; z = r / D; partial sums of r.z and r.r
__global__ void __launch_bounds__(256) k_pot_update(PotGrid G, const double *sc, const double *iDv, double *xv,
                                                   double *r, double *zv, const double *p, const double *Ap,
                                                   double *part)
{
    const double alpha = sc[SC_ALPHA];
    double rz = 0.0, rr = 0.0;
    POT_ROWS(G)
    {
        const size_t i = pot_at(G, x, y, z);
        if (G.cls[i] != CLS_FREE) continue;
        xv[i] += alpha * p[i];
        const double ri = r[i] - alpha * Ap[i];
        const double zi = ri * iDv[i];
        r[i] = ri;
        zv[i] = zi;
        rz += ri * zi;
        rr += ri * ri;
    }
    rz = pot_block_sum(rz);
    rr = pot_block_sum(rr);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = rz;
        part[2 * blockIdx.x + 1] = rr;
    }
}

__global__ void __launch_bounds__(256) k_pot_direction(PotGrid G, const double *sc, const double *zv, double *p)
{
    const double beta = sc[SC_BETA];
    POT_ROWS(G)
    {
        const size_t i = pot_at(G, x, y, z);
        if (G.cls[i] == CLS_FREE) p[i] = zv[i] + beta * p[i];
    }
}

// ---- FP32 inner iterations and the FP64 correction

// the FP32 face-conductance table in shared memory
__device__ __forceinline__ void pot_table32(const PotGrid &G, float *S)
{
    for (int k = threadIdx.x; k < kCondLabels * kCondLabels; k += blockDim.x) S[k] = (float)G.S[k];
    __syncthreads();
}

// true residual r = b - A x = sum_nb sigma_f (x_nb - x_i) in FP64 on the free
// voxels (x holds 1 on the electrode and 0 on the ground); partials of r.r
__global__ void __launch_bounds__(256) k_pot_resid64(PotGrid G, const double *xv, double *r, double *part)
{
    __shared__ double S[kCondLabels * kCondLabels];
    for (int k = threadIdx.x; k < kCondLabels * kCondLabels; k += blockDim.x) S[k] = G.S[k];
    __syncthreads();
    double rr = 0.0;
    POT_ROWS(G)
    {
        const size_t i = pot_at(G, x, y, z);
        if (G.cls[i] != CLS_FREE) continue;
        const int l = G.label[i];
        const double xi = xv[i];
        double v = 0.0;
        for (int d = 0; d < 6; ++d) {
            size_t j;
            if (pot_nb(G, i, x, y, z, d, j)) v += S[l * kCondLabels + G.label[j]] * (xv[j] - xi);
        }
        r[i] = v;
        rr += v * v;
    }
    rr = pot_block_sum(rr);
    if (threadIdx.x == 0) part[blockIdx.x] = rr;
}

// The FP32 vectors keep an invariant: every entry off the free set (electrode,
// ground, row padding) is exactly 0.  Then the update and direction steps
// need no class test, and a non-free neighbour's term in A p is sigma_f * 0,
// an exact no-op, so the operator is that of the free unknowns.  Each lane
// takes a quad of 4 x voxels (16-byte vectors; rows are padded to 4).
#define POT_QUADS(G)                                                                                                \
    for (int row = blockIdx.x * 8 + (int)(threadIdx.x >> 5); row < (G).ny * (G).nz; row += gridDim.x * 8)         \
        for (int y = row % (G).ny, z = row / (G).ny, x0 = 4 * (int)(threadIdx.x & 31); x0 < (G).nx; x0 += 128)

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ uchar4 ldb4(const uint8_t *p) { return *reinterpret_cast<const uchar4 *>(p); }
__device__ __forceinline__ float f4at(const float4 &v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }
__device__ __forceinline__ int b4at(const uchar4 &v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }

// start of a cycle: r32 = r, e = 0, z = r32 / D on the free voxels, 0
// elsewhere; FP32 diagonal from the FP64 one; partials of r32.z and r32.r32
// (FP32 per thread, FP64 per block).  The previous direction is set to 0 at the
// first cycle (with beta = 0 the first direction is z) and kept at a residual
// replacement (beta = (r.z)_new / (r.z)_old continues the iteration).
__global__ void __launch_bounds__(256) k_pot_init32(PotGrid G, const double *r, const double *Dv, float *r32,
                                                   float *e32, float *z32, float *p32, float *D32, float *iD32,
                                                   int keep_direction, double *part)
{
    float rz = 0.f, rr = 0.f;
    POT_QUADS(G)
    {
        const size_t i = pot_at(G, x0, y, z);
        const uchar4 c4 = ldb4(G.cls + i);
        float D[4], iD[4], rv[4], zv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool fr = b4at(c4, q) == CLS_FREE;
            D[q] = fr ? (float)Dv[i + q] : 0.f;
            iD[q] = D[q] > 0.f ? 1.f / D[q] : 0.f;
            rv[q] = fr ? (float)r[i + q] : 0.f;
            zv[q] = rv[q] * iD[q];
            rz = fmaf(rv[q], zv[q], rz);
            rr = fmaf(rv[q], rv[q], rr);
        }
        st4(D32 + i, make_float4(D[0], D[1], D[2], D[3]));
        st4(iD32 + i, make_float4(iD[0], iD[1], iD[2], iD[3]));
        st4(r32 + i, make_float4(rv[0], rv[1], rv[2], rv[3]));
        st4(e32 + i, make_float4(0.f, 0.f, 0.f, 0.f));
        st4(z32 + i, make_float4(zv[0], zv[1], zv[2], zv[3]));
        if (!keep_direction) st4(p32 + i, make_float4(0.f, 0.f, 0.f, 0.f));
    }
    const double a = pot_block_sum((double)rz), b = pot_block_sum((double)rr);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// per quad, once per solve: 1 + the label when the quad and its six
// neighbour sets (x edges, y and z neighbour quads) share one label, else 0
__global__ void __launch_bounds__(256) k_pot_quni(PotGrid G, uint8_t *quni)
{
    POT_QUADS(G)
    {
        const size_t i = pot_at(G, x0, y, z);
        const uchar4 bz = make_uchar4(0, 0, 0, 0);
        const bool hasL = x0 > 0, hasR = x0 + 4 < G.pitch, hasYm = y > 0, hasYp = y + 1 < G.ny, hasZm = z > 0,
                   hasZp = z + 1 < G.nz;
        const size_t oy = G.pitch, oz = G.plane;
        const uchar4 l4 = ldb4(G.label + i);
        const int lL = hasL ? G.label[i - 1] : 0, lR = hasR ? G.label[i + 4] : 0;
        const uchar4 lym = hasYm ? ldb4(G.label + i - oy) : bz, lyp = hasYp ? ldb4(G.label + i + oy) : bz;
        const uchar4 lzm = hasZm ? ldb4(G.label + i - oz) : bz, lzp = hasZp ? ldb4(G.label + i + oz) : bz;
        const uint32_t l0 = l4.x, rep4 = l0 * 0x01010101u;
        auto w32 = [](const uchar4 &v) { return (uint32_t)v.x | (uint32_t)v.y << 8 | (uint32_t)v.z << 16 | (uint32_t)v.w << 24; };
        const bool uni = w32(l4) == rep4 && (uint32_t)lL == l0 && (uint32_t)lR == l0 && w32(lym) == rep4 &&
                         w32(lyp) == rep4 && w32(lzm) == rep4 && w32(lzp) == rep4;
        quni[i >> 2] = uni ? (uint8_t)(l0 + 1) : 0;
    }
}

// The search direction and the operator in one pass: p = z + beta p_prev on
// the quad and its six neighbour points (p_prev and p are separate buffers,
// swapped every iteration), p written for the quad, Ap = A p in FP32 (0 off
// the free set); partials of p.Ap, and alpha = rz / (p.Ap) by the last block.
// Neighbour terms in the order x-, x+, y-, y+, z-, z+; where the quad and all
// its neighbours share one label, one table entry serves every face.
__global__ void __launch_bounds__(256) k_pot_spmv32(PotGrid G, double *sc, const float *D32, const float *z32,
                                                   const float *pprev, float *p, float *Ap, double *part,
                                                   unsigned *ctr)
{
    __shared__ float S[kCondLabels * kCondLabels];
    pot_table32(G, S);
    const float beta = (float)sc[SC_BETA];
    auto dir = [&](float zv, float pv) { return fmaf(beta, pv, zv); };
    auto dir4 = [&](const float4 &zv, const float4 &pv) {
        return make_float4(dir(zv.x, pv.x), dir(zv.y, pv.y), dir(zv.z, pv.z), dir(zv.w, pv.w));
    };
    float acc = 0.f;
    POT_QUADS(G)
    {
        const size_t i = pot_at(G, x0, y, z);
        const uchar4 c4 = ldb4(G.cls + i);
        const int fl = G.quni[i >> 2];
        const float4 p4 = dir4(ld4(z32 + i), ld4(pprev + i)), D4 = ld4(D32 + i);
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        const uchar4 bz = make_uchar4(0, 0, 0, 0);
        const bool hasL = x0 > 0, hasR = x0 + 4 < G.pitch, hasYm = y > 0, hasYp = y + 1 < G.ny, hasZm = z > 0,
                   hasZp = z + 1 < G.nz;
        const float pL = hasL ? dir(z32[i - 1], pprev[i - 1]) : 0.f;
        const float pR = hasR ? dir(z32[i + 4], pprev[i + 4]) : 0.f;
        const size_t oy = G.pitch, oz = G.plane;
        const float4 pym = hasYm ? dir4(ld4(z32 + i - oy), ld4(pprev + i - oy)) : zero;
        const float4 pyp = hasYp ? dir4(ld4(z32 + i + oy), ld4(pprev + i + oy)) : zero;
        const float4 pzm = hasZm ? dir4(ld4(z32 + i - oz), ld4(pprev + i - oz)) : zero;
        const float4 pzp = hasZp ? dir4(ld4(z32 + i + oz), ld4(pprev + i + oz)) : zero;
        // labels only where the quad's neighbourhood is not of one label (the flag)
        uchar4 l4 = bz, lym = bz, lyp = bz, lzm = bz, lzp = bz;
        int lL = 0, lR = 0;
        if (fl == 0) {
            l4 = ldb4(G.label + i);
            lL = hasL ? G.label[i - 1] : 0;
            lR = hasR ? G.label[i + 4] : 0;
            if (hasYm) lym = ldb4(G.label + i - oy);
            if (hasYp) lyp = ldb4(G.label + i + oy);
            if (hasZm) lzm = ldb4(G.label + i - oz);
            if (hasZp) lzp = ldb4(G.label + i + oz);
        }
        const bool uni = fl != 0;
        const float su = uni ? S[(fl - 1) * (kCondLabels + 1)] : 0.f;
        float out[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float pq = f4at(p4, q);
            const float nb[6] = {q == 0 ? pL : f4at(p4, q - 1), q == 3 ? pR : f4at(p4, q + 1), f4at(pym, q),
                                 f4at(pyp, q), f4at(pzm, q), f4at(pzp, q)};
            float w[6];
            if (uni) {
#pragma unroll
                for (int d = 0; d < 6; ++d) w[d] = su;
            } else {
                const int l = b4at(l4, q);
                const int ln[6] = {q == 0 ? lL : b4at(l4, q - 1), q == 3 ? lR : b4at(l4, q + 1), b4at(lym, q),
                                   b4at(lyp, q), b4at(lzm, q), b4at(lzp, q)};
#pragma unroll
                for (int d = 0; d < 6; ++d) w[d] = S[l * kCondLabels + ln[d]];
            }
            float v = f4at(D4, q) * pq;
#pragma unroll
            for (int d = 0; d < 6; ++d) v = fmaf(-w[d], nb[d], v);
            v = b4at(c4, q) == CLS_FREE ? v : 0.f;
            out[q] = v;
            acc = fmaf(pq, v, acc);
        }
        st4(p + i, p4);
        st4(Ap + i, make_float4(out[0], out[1], out[2], out[3]));
    }
    const double a = pot_block_sum((double)acc);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
    if (pot_last_block(ctr)) {
        double s0, s1;
        pot_sum_partials(part, gridDim.x, false, s0, s1);
        if (threadIdx.x == 0) {
            pot_scalars_apply(0, s0, s1, sc);
            *ctr = 0u;
        }
    }
}

// e += alpha p; r32 -= alpha Ap; z = r32 / D; partials of r32.z and r32.r32
// (off the free set every operand is 0 and stays 0)
__global__ void __launch_bounds__(256) k_pot_update32(PotGrid G, double *sc, const float *iD32, float *e32,
                                                     float *r32, float *z32, const float *p, const float *Ap,
                                                     double *part, unsigned *ctr)
{
    const float alpha = (float)sc[SC_ALPHA];
    float rz = 0.f, rr = 0.f;
    POT_QUADS(G)
    {
        const size_t i = pot_at(G, x0, y, z);
        const float4 e = ld4(e32 + i), r0 = ld4(r32 + i), p4 = ld4(p + i), a4 = ld4(Ap + i), iD = ld4(iD32 + i);
        const float4 e1 = make_float4(fmaf(alpha, p4.x, e.x), fmaf(alpha, p4.y, e.y), fmaf(alpha, p4.z, e.z),
                                      fmaf(alpha, p4.w, e.w));
        const float4 r1 = make_float4(fmaf(-alpha, a4.x, r0.x), fmaf(-alpha, a4.y, r0.y), fmaf(-alpha, a4.z, r0.z),
                                      fmaf(-alpha, a4.w, r0.w));
        const float4 z1 = make_float4(r1.x * iD.x, r1.y * iD.y, r1.z * iD.z, r1.w * iD.w);
        st4(e32 + i, e1);
        st4(r32 + i, r1);
        st4(z32 + i, z1);
        rz = fmaf(r1.x, z1.x, fmaf(r1.y, z1.y, fmaf(r1.z, z1.z, fmaf(r1.w, z1.w, rz))));
        rr = fmaf(r1.x, r1.x, fmaf(r1.y, r1.y, fmaf(r1.z, r1.z, fmaf(r1.w, r1.w, rr))));
    }
    const double a = pot_block_sum((double)rz), b = pot_block_sum((double)rr);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
    if (pot_last_block(ctr)) {
        double s0, s1;
        pot_sum_partials(part, gridDim.x, true, s0, s1);
        if (threadIdx.x == 0) {
            pot_scalars_apply(1, s0, s1, sc);
            *ctr = 0u;
        }
    }
}

// end of a cycle: x += e (e is 0 off the free set, so x keeps its fixed values)
__global__ void __launch_bounds__(256) k_pot_correct(PotGrid G, const float *e32, double *xv)
{
    POT_QUADS(G)
    {
        const size_t i = pot_at(G, x0, y, z);
        const float4 e = ld4(e32 + i);
        double2 *xp = reinterpret_cast<double2 *>(xv + i);
        const double2 a = xp[0], b = xp[1];
        xp[0] = make_double2(a.x + (double)e.x, a.y + (double)e.y);
        xp[1] = make_double2(b.x + (double)e.z, b.y + (double)e.w);
    }
}

// ---- multigrid preconditioner (FP32)
//
// z = M r for the FP32 conjugate gradients: one symmetric V-cycle of
// unsmoothed aggregation.  Level l+1 has a cell per 2 x 2 x 2 cells of level l
// (a grid's odd last cell pairs with nothing); prolongation P copies a cell's
// value to its free children, restriction is P^T (the children's sum), and the
// coarse operator is the Galerkin product P^T A P, which for these aggregates
// is again a 7-point operator: the conductance between two cells is the sum
// of the fine face conductances between their free children, and the
// diagonal is that sum over the cell's six faces plus the couplings of its
// free children to fixed voxels (G, kept separately so every diagonal is a
// sum of positive terms).  Smoother: damped Jacobi, kMgNu sweeps before and
// after the coarse correction (the first from zero); the coarsest level
// (at most kMgCoarsest cells) applies its exact inverse, formed once per
// solve on the host by Cholesky in FP64.  Same sweeps before and after, a
// symmetric smoother and an exact coarsest solve make M symmetric positive
// definite, as conjugate gradients need.  Every vector stays 0 off the free
// set (the diagonal there is 0, so Jacobi and the prolongation leave it).
// The coarse correction is scaled by kMgGamma = 1.5 (piecewise-constant
// prolongation undershoots smooth errors; any positive scale keeps M symmetric
// positive definite).
constexpr int kMgCoarsest = 128;
constexpr float kMgOmega = 0.8f;
constexpr int kMgNu = 2;
constexpr float kMgGamma = 1.5f;

struct MgLevel {
    int nx, ny, nz, n;
    float *D, *iD, *Wx, *Wy, *Wz, *G;  // operator: diagonal, its inverse, +x/+y/+z conductances, fixed couplings
    float *b, *x, *t, *r;              // right side, two iterates, residual
};

// fine level: coarse right side bc = P^T r (sum of the up to 8 fine children)
__global__ void __launch_bounds__(256) k_mg0_restrict(PotGrid G, const float *r, MgLevel C, float *bc)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C.n; c += gridDim.x * blockDim.x) {
        const int X = c % C.nx, Y = (c / C.nx) % C.ny, Z = c / (C.nx * C.ny);
        float s = 0.f;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
                    if (x < G.nx && y < G.ny && z < G.nz) s += r[pot_at(G, x, y, z)];
                }
        bc[c] = s;
    }
}

// A v at cell c of a coarse level
__device__ __forceinline__ float mg_av(const MgLevel &L, const float *v, int c, int X, int Y, int Z)
{
    const int sy = L.nx, sz = L.nx * L.ny;
    float a = L.D[c] * v[c];
    if (X > 0) a = fmaf(-L.Wx[c - 1], v[c - 1], a);
    if (X + 1 < L.nx) a = fmaf(-L.Wx[c], v[c + 1], a);
    if (Y > 0) a = fmaf(-L.Wy[c - sy], v[c - sy], a);
    if (Y + 1 < L.ny) a = fmaf(-L.Wy[c], v[c + sy], a);
    if (Z > 0) a = fmaf(-L.Wz[c - sz], v[c - sz], a);
    if (Z + 1 < L.nz) a = fmaf(-L.Wz[c], v[c + sz], a);
    return a;
}

#define MG_CELLS(L)                                                                                           \
    for (int c = blockIdx.x * blockDim.x + threadIdx.x, X, Y, Z; c < (L).n; c += gridDim.x * blockDim.x)     \
        if ((X = c % (L).nx), (Y = (c / (L).nx) % (L).ny), (Z = c / ((L).nx * (L).ny)), true)

// fine level: x += gamma P xc on the free voxels (those with a nonzero diagonal)
__global__ void __launch_bounds__(256) k_mg0_prolong(PotGrid G, const float *iD32, MgLevel C, const float *xc,
                                                    float *x)
{
    POT_QUADS(G)
    {
        const size_t i = pot_at(G, x0, y, z);
        const float4 d4 = ld4(iD32 + i);
        float4 x4 = ld4(x + i);
        const size_t cb = ((size_t)(z >> 1) * C.ny + (y >> 1)) * C.nx;
        const int X0 = x0 >> 1;  // children x0, x0+1 of cell X0; x0+2, x0+3 of X0+1
        if (d4.x > 0.f) x4.x = fmaf(kMgGamma, xc[cb + X0], x4.x);
        if (d4.y > 0.f) x4.y = fmaf(kMgGamma, xc[cb + X0], x4.y);
        if (d4.z > 0.f) x4.z = fmaf(kMgGamma, xc[cb + X0 + 1], x4.z);
        if (d4.w > 0.f) x4.w = fmaf(kMgGamma, xc[cb + X0 + 1], x4.w);
        st4(x + i, x4);
    }
}

// Coarse-level passes, each over the cells c of a level that this thread takes
// in its grid (grid-stride): the per-level kernels below and the one-block tail
// of the V-cycle run the same code.
// coarse level: x = omega b / D
__device__ __forceinline__ void mg_first_cells(const MgLevel &L, const float *b, float *x)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < L.n; c += gridDim.x * blockDim.x)
        x[c] = kMgOmega * L.iD[c] * b[c];
}

// coarse level: out = in + omega (b - A in) / D (RESID: out = b - A in)
template <bool RESID>
__device__ __forceinline__ void mg_sweep_cells(const MgLevel &L, const float *b, const float *in, float *out)
{
    MG_CELLS(L)
    {
        const float r = b[c] - mg_av(L, in, c, X, Y, Z);
        out[c] = RESID ? r : fmaf(kMgOmega * L.iD[c], r, in[c]);
    }
}

// coarse level l -> l+1: bc = P^T r
__device__ __forceinline__ void mg_restrict_cells(const MgLevel &F, const float *r, const MgLevel &C, float *bc)
{
    MG_CELLS(C)
    {
        float s = 0.f;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
                    if (x < F.nx && y < F.ny && z < F.nz) s += r[(z * F.ny + y) * F.nx + x];
                }
        bc[c] = s;
    }
}

// coarse level l+1 -> l: x += gamma P xc on the cells with free children
__device__ __forceinline__ void mg_prolong_cells(const MgLevel &F, const MgLevel &C, const float *xc, float *x)
{
    MG_CELLS(F)
    {
        if (F.iD[c] > 0.f) x[c] = fmaf(kMgGamma, xc[((Z >> 1) * C.ny + (Y >> 1)) * C.nx + (X >> 1)], x[c]);
    }
}

// coarsest level: x = A^-1 b with the dense inverse (n <= kMgCoarsest, one block;
// sb: kMgCoarsest floats of shared memory)
__device__ __forceinline__ void mg_coarsest_cells(int n, const float *Ainv, const float *b, float *x, float *sb)
{
    for (int k = threadIdx.x; k < n; k += blockDim.x) sb[k] = b[k];
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        float s = 0.f;
        for (int k = 0; k < n; ++k) s = fmaf(Ainv[(size_t)k * n + t], sb[k], s);
        x[t] = s;
    }
}

__global__ void __launch_bounds__(256) k_mg_first(MgLevel L, const float *b, float *x) { mg_first_cells(L, b, x); }

// fine level: out = in + omega (b - A in) / D (RESID: out = b - A in), streaming
// z: a thread per quad of 4 x voxels of one row walks a chunk of planes with the
// quad's values of planes z-1, z, z+1 in registers; the x neighbours come from
// the adjacent lanes (a row's outer lanes load theirs).  Per voxel, A v = D v -
// sum over the faces x-, x+, y-, y+, z-, z+ (in that order) of the face
// conductance times the neighbour's v, 0 off the free set (v is 0 there; the
// labels are read only where the quad's neighbourhood has more than one).
// Blocks of 32 x 8 quads (plain_grid_dims).
// FIRST: the first sweep, from zero: the iterate v = omega b / D is formed where
// it is read (no pass stores it; in is not read).  Fusing the prolongation into
// the first post-sweep the same way was measured slower (every neighbour read
// then also loads 1/D and the coarse value): 143 us against 40 + 93 us at 256^3.
// the cache line holding p into L2 (no register is written): a thread streaming z
// asks for its fields two planes ahead, so their HBM latency overlaps the planes
// in between (the fine-grid sweeps: 4 % of the solve, the same iterates)
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <bool RESID, bool FIRST>
__global__ void __launch_bounds__(256) k_mg0_sweep_z(PotGrid G, const float *D32, const float *iD32, const float *b,
                                                    const float *in, float *out, int zchunk)
{
    __shared__ float S[kCondLabels * kCondLabels];
    for (int k = threadIdx.y * 32 + threadIdx.x; k < kCondLabels * kCondLabels; k += 256) S[k] = (float)G.S[k];
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    if (y >= G.ny) return;  // whole warp
    const int x0 = 4 * (blockIdx.x * 32 + lane);
    const bool inrow = x0 < G.nx;
    const int zb = blockIdx.z * zchunk, ze = min(G.nz, zb + zchunk);
    const size_t oy = G.pitch, oz = G.plane;
    const bool hasL = x0 > 0, hasR = x0 + 4 < G.pitch, hasYm = y > 0, hasYp = y + 1 < G.ny;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const uchar4 bz = make_uchar4(0, 0, 0, 0);
    // v of the voxel j and of the quad at j
    auto v1 = [&](size_t j) -> float { return FIRST ? kMgOmega * iD32[j] * b[j] : in[j]; };
    auto v4 = [&](size_t j) -> float4 {
        if (FIRST) {
            const float4 b4 = ld4(b + j), d4 = ld4(iD32 + j);
            return make_float4(kMgOmega * d4.x * b4.x, kMgOmega * d4.y * b4.y, kMgOmega * d4.z * b4.z,
                               kMgOmega * d4.w * b4.w);
        }
        return ld4(in + j);
    };
    size_t i = (size_t)zb * oz + (size_t)y * oy + x0;
    float4 vm = zero, vc = zero, vp = zero;
    if (inrow) {
        vc = v4(i);
        if (zb > 0) vm = v4(i - oz);
    }
    for (int z = zb; z < ze; ++z, i += oz) {
        const bool hasZm = z > 0, hasZp = z + 1 < G.nz;
        if (inrow && z + 2 < G.nz) {  // the streamed fields two planes ahead into L2
            const size_t iq = i + 2 * oz;
            prefetch_l2(b + iq);
            prefetch_l2(FIRST ? iD32 + iq : in + iq);
            prefetch_l2(D32 + iq);
            if (!RESID && !FIRST) prefetch_l2(iD32 + iq);
            prefetch_l2(G.cls + iq);
        }
        vp = inrow && hasZp ? v4(i + oz) : zero;
        // x neighbours: lanes hold consecutive quads of the row; a quad past nx
        // holds zeros, as the padding does
        float pL = __shfl_up_sync(FULL, vc.w, 1), pR = __shfl_down_sync(FULL, vc.x, 1);
        if (lane == 0) pL = inrow && hasL ? v1(i - 1) : 0.f;
        if (lane == 31) pR = inrow && hasR ? v1(i + 4) : 0.f;
        if (!inrow) continue;
        const uchar4 c4 = ldb4(G.cls + i);
        const int fl = G.quni[i >> 2];
        const float4 D4 = ld4(D32 + i);
        const float4 pym = hasYm ? v4(i - oy) : zero, pyp = hasYp ? v4(i + oy) : zero;
        uchar4 l4 = bz, lym = bz, lyp = bz, lzm = bz, lzp = bz;
        int lL = 0, lR = 0;
        if (fl == 0) {
            l4 = ldb4(G.label + i);
            lL = hasL ? G.label[i - 1] : 0;
            lR = hasR ? G.label[i + 4] : 0;
            if (hasYm) lym = ldb4(G.label + i - oy);
            if (hasYp) lyp = ldb4(G.label + i + oy);
            if (hasZm) lzm = ldb4(G.label + i - oz);
            if (hasZp) lzp = ldb4(G.label + i + oz);
        }
        const bool uni = fl != 0;
        const float su = uni ? S[(fl - 1) * (kCondLabels + 1)] : 0.f;
        float a4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float pq = f4at(vc, q);
            const float nb[6] = {q == 0 ? pL : f4at(vc, q - 1), q == 3 ? pR : f4at(vc, q + 1), f4at(pym, q),
                                 f4at(pyp, q), f4at(vm, q), f4at(vp, q)};
            float w[6];
            if (uni) {
#pragma unroll
                for (int d = 0; d < 6; ++d) w[d] = su;
            } else {
                const int l = b4at(l4, q);
                const int ln[6] = {q == 0 ? lL : b4at(l4, q - 1), q == 3 ? lR : b4at(l4, q + 1), b4at(lym, q),
                                   b4at(lyp, q), b4at(lzm, q), b4at(lzp, q)};
#pragma unroll
                for (int d = 0; d < 6; ++d) w[d] = S[l * kCondLabels + ln[d]];
            }
            float a = f4at(D4, q) * pq;
#pragma unroll
            for (int d = 0; d < 6; ++d) a = fmaf(-w[d], nb[d], a);
            a4[q] = b4at(c4, q) == CLS_FREE ? a : 0.f;
        }
        const float4 b4 = ld4(b + i);
        const float4 r4 = make_float4(b4.x - a4[0], b4.y - a4[1], b4.z - a4[2], b4.w - a4[3]);
        if (RESID) {
            st4(out + i, r4);
        } else {
            const float4 d4 = ld4(iD32 + i);
            st4(out + i, make_float4(fmaf(kMgOmega * d4.x, r4.x, vc.x), fmaf(kMgOmega * d4.y, r4.y, vc.y),
                                     fmaf(kMgOmega * d4.z, r4.z, vc.z), fmaf(kMgOmega * d4.w, r4.w, vc.w)));
        }
        vm = vc;
        vc = vp;
    }
}

template <bool RESID>
__global__ void __launch_bounds__(256) k_mg_sweep(MgLevel L, const float *b, const float *in, float *out)
{
    mg_sweep_cells<RESID>(L, b, in, out);
}

__global__ void __launch_bounds__(256) k_mg_restrict(MgLevel F, const float *r, MgLevel C, float *bc)
{
    mg_restrict_cells(F, r, C, bc);
}

__global__ void __launch_bounds__(256) k_mg_prolong(MgLevel F, MgLevel C, const float *xc, float *x)
{
    mg_prolong_cells(F, C, xc, x);
}

// The V-cycle on the smallest levels in one block: every level of at most
// kMgTailCells cells, the coarsest included, where a launch per pass would cost
// more than the pass.  Down: first sweep, kMgNu - 1 sweeps, residual and
// restriction per level; the coarsest level's dense inverse; up: prolongation
// and kMgNu sweeps per level; a block barrier after every pass (the next pass
// reads what other threads wrote).  The iterates alternate between x and t as
// in the per-level launches, so the same buffer ends up with the result.
constexpr int kMgTailCells = 4096;
constexpr int kMgTailMax = 8;
struct MgTail {
    MgLevel L[kMgTailMax];  // L[n - 1] is the coarsest level
    int n;
    const float *Ainv;
};
__global__ void __launch_bounds__(1024) k_mg_tail(const MgTail T)
{
    __shared__ float sb[kMgCoarsest];
    float *cur[kMgTailMax], *oth[kMgTailMax];
    for (int l = 0; l + 1 < T.n; ++l) {
        const MgLevel &L = T.L[l];
        cur[l] = L.x;
        oth[l] = L.t;
        mg_first_cells(L, L.b, cur[l]);
        __syncthreads();
        for (int s = 1; s < kMgNu; ++s) {
            mg_sweep_cells<false>(L, L.b, cur[l], oth[l]);
            __syncthreads();
            float *t = cur[l];
            cur[l] = oth[l];
            oth[l] = t;
        }
        mg_sweep_cells<true>(L, L.b, cur[l], L.r);
        __syncthreads();
        mg_restrict_cells(L, L.r, T.L[l + 1], T.L[l + 1].b);
        __syncthreads();
    }
    cur[T.n - 1] = T.L[T.n - 1].x;
    mg_coarsest_cells(T.L[T.n - 1].n, T.Ainv, T.L[T.n - 1].b, cur[T.n - 1], sb);
    __syncthreads();
    for (int l = T.n - 2; l >= 0; --l) {
        const MgLevel &L = T.L[l];
        mg_prolong_cells(L, T.L[l + 1], cur[l + 1], cur[l]);
        __syncthreads();
        for (int s = 0; s < kMgNu; ++s) {
            mg_sweep_cells<false>(L, L.b, cur[l], oth[l]);
            __syncthreads();
            float *t = cur[l];
            cur[l] = oth[l];
            oth[l] = t;
        }
    }
}

// level 1 from the fine grid: +x/+y/+z conductances between the free children of
// neighbouring cells, and G, the couplings of the free children to fixed voxels
__global__ void __launch_bounds__(256) k_mg0_build(PotGrid G, MgLevel C)
{
    __shared__ float S[kCondLabels * kCondLabels];
    pot_table32(G, S);
    MG_CELLS(C)
    {
        float wx = 0.f, wy = 0.f, wz = 0.f, gf = 0.f;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
                    if (x >= G.nx || y >= G.ny || z >= G.nz) continue;
                    const size_t i = pot_at(G, x, y, z);
                    if (G.cls[i] != CLS_FREE) continue;
                    const int l = G.label[i];
                    for (int d = 0; d < 6; ++d) {
                        size_t j;
                        if (!pot_nb(G, i, x, y, z, d, j)) continue;
                        const float sf = S[l * kCondLabels + G.label[j]];
                        if (G.cls[j] != CLS_FREE) {
                            gf += sf;
                        } else if (d == 1 && dx == 1) {
                            wx += sf;
                        } else if (d == 3 && dy == 1) {
                            wy += sf;
                        } else if (d == 5 && dz == 1) {
                            wz += sf;
                        }
                    }
                }
        C.Wx[c] = wx;
        C.Wy[c] = wy;
        C.Wz[c] = wz;
        C.G[c] = gf;
    }
}

// level l+1 from level l: sums over the children
__global__ void __launch_bounds__(256) k_mg_build(MgLevel F, MgLevel C)
{
    MG_CELLS(C)
    {
        float wx = 0.f, wy = 0.f, wz = 0.f, gf = 0.f;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
                    if (x >= F.nx || y >= F.ny || z >= F.nz) continue;
                    const int f = (z * F.ny + y) * F.nx + x;
                    gf += F.G[f];
                    if (dx == 1 && x + 1 < F.nx) wx += F.Wx[f];
                    if (dy == 1 && y + 1 < F.ny) wy += F.Wy[f];
                    if (dz == 1 && z + 1 < F.nz) wz += F.Wz[f];
                }
        C.Wx[c] = wx;
        C.Wy[c] = wy;
        C.Wz[c] = wz;
        C.G[c] = gf;
    }
}

// diagonal of a level: G plus the six face conductances; its inverse (0 where 0)
__global__ void __launch_bounds__(256) k_mg_diag(MgLevel L)
{
    MG_CELLS(L)
    {
        const int sy = L.nx, sz = L.nx * L.ny;
        float d = L.G[c] + L.Wx[c] + L.Wy[c] + L.Wz[c];
        if (X > 0) d += L.Wx[c - 1];
        if (Y > 0) d += L.Wy[c - sy];
        if (Z > 0) d += L.Wz[c - sz];
        L.D[c] = d;
        L.iD[c] = d > 0.f ? 1.f / d : 0.f;
    }
}

#undef MG_CELLS

// CG steps around the preconditioner: e += alpha p; r32 -= alpha Ap; partials of
// r32.r32, rr by the last block
__global__ void __launch_bounds__(256) k_pot_update32_mg(PotGrid G, double *sc, float *e32, float *r32,
                                                        const float *p, const float *Ap, double *part, unsigned *ctr)
{
    const float alpha = (float)sc[SC_ALPHA];
    float rr = 0.f;
    POT_QUADS(G)
    {
        const size_t i = pot_at(G, x0, y, z);
        const float4 e = ld4(e32 + i), r0 = ld4(r32 + i), p4 = ld4(p + i), a4 = ld4(Ap + i);
        st4(e32 + i, make_float4(fmaf(alpha, p4.x, e.x), fmaf(alpha, p4.y, e.y), fmaf(alpha, p4.z, e.z),
                                 fmaf(alpha, p4.w, e.w)));
        const float4 r1 = make_float4(fmaf(-alpha, a4.x, r0.x), fmaf(-alpha, a4.y, r0.y), fmaf(-alpha, a4.z, r0.z),
                                      fmaf(-alpha, a4.w, r0.w));
        st4(r32 + i, r1);
        rr = fmaf(r1.x, r1.x, fmaf(r1.y, r1.y, fmaf(r1.z, r1.z, fmaf(r1.w, r1.w, rr))));
    }
    const double a = pot_block_sum((double)rr);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
    if (pot_last_block(ctr)) {
        double s0, s1;
        pot_sum_partials(part, gridDim.x, false, s0, s1);
        if (threadIdx.x == 0) {
            pot_scalars_apply(SCW_RR, s0, s1, sc);
            *ctr = 0u;
        }
    }
}

// partials of r.z; the last block applies the scalar step `which` (SCW_BETA or SCW_START_RZ)
__global__ void __launch_bounds__(256) k_pot_dot32(PotGrid G, const float *r32, const float *zv, int which,
                                                  double *sc, double *part, unsigned *ctr)
{
    float rz = 0.f;
    POT_QUADS(G)
    {
        const size_t i = pot_at(G, x0, y, z);
        const float4 r4 = ld4(r32 + i), z4 = ld4(zv + i);
        rz = fmaf(r4.x, z4.x, fmaf(r4.y, z4.y, fmaf(r4.z, z4.z, fmaf(r4.w, z4.w, rz))));
    }
    const double a = pot_block_sum((double)rz);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
    if (pot_last_block(ctr)) {
        double s0, s1;
        pot_sum_partials(part, gridDim.x, false, s0, s1);
        if (threadIdx.x == 0) {
            pot_scalars_apply(which, s0, s1, sc);
            *ctr = 0u;
        }
    }
}

#undef POT_QUADS

// hand-over to FP64 conjugate gradients from the current x: z = r / D, p = z;
// partials of r.z and r.r
__global__ void __launch_bounds__(256) k_pot_restart64(PotGrid G, const double *r, const double *iDv, double *zv,
                                                      double *p, double *part)
{
    double rz = 0.0, rr = 0.0;
    POT_ROWS(G)
    {
        const size_t i = pot_at(G, x, y, z);
        if (G.cls[i] != CLS_FREE) continue;
        const double ri = r[i], zi = ri * iDv[i];
        zv[i] = zi;
        p[i] = zi;
        rz += ri * zi;
        rr += ri * ri;
    }
    rz = pot_block_sum(rz);
    rr = pot_block_sum(rr);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = rz;
        part[2 * blockIdx.x + 1] = rr;
    }
}

#undef POT_ROWS

// q = sum_nb sigma_f (V_nb - V_i)^2 / (2 h^2) into wbuf on the thermally free
// voxels (the 1/r^4 source's rule), per-block partial sums of q over them
__global__ void __launch_bounds__(256) k_pot_joule(PotGrid G, const double *V, const LabelCoef *tab, int face,
                                                  double h, double *wbuf, double *part)
{
    __shared__ double S[kCondLabels * kCondLabels];
    for (int k = threadIdx.x; k < kCondLabels * kCondLabels; k += blockDim.x) S[k] = G.S[k];
    __syncthreads();
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < G.nvp; i += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        pot_xyz(G, i, x, y, z);
        if (x >= G.nx) continue;
        const bool face_vox = x == 0 || y == 0 || z == 0 || x == G.nx - 1 || y == G.ny - 1 || z == G.nz - 1;
        const int l = G.label[i];
        if (tab[l].fixed || (face == RFA_FACE_DIRICHLET && face_vox)) continue;
        double q = 0.0;
        const double vi = V[i];
        for (int d = 0; d < 6; ++d) {
            size_t j;
            if (!pot_nb(G, i, x, y, z, d, j)) continue;
            const double dv = V[j] - vi;
            q += S[l * kCondLabels + G.label[j]] * dv * dv;
        }
        q /= 2.0 * h * h;
        wbuf[i] = q;
        acc += q;
    }
    acc = pot_block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// the multigrid hierarchy of the FP32 iterations: levels 1 .. nl (L[0] is the
// fine grid, unused here) and the dense inverse of the coarsest level
struct MgHost {
    std::vector<MgLevel> L;
    float *mem = nullptr, *Ainv = nullptr;
    ~MgHost()
    {
        if (mem) cudaFree(mem);
        if (Ainv) cudaFree(Ainv);
    }
};

inline unsigned mg_blocks(int n) { return (unsigned)std::min((n + 255) / 256, 148 * 8); }

// Builds the levels and the coarsest inverse.  ok = false (and RFA_OK) where the
// grid needs no coarse level or the coarsest matrix is not positive definite:
// the caller then uses the Jacobi preconditioner.
rfa_status mg_setup(rfa_grid *g, const PotGrid &G, MgHost &H, bool &ok)
{
    ok = false;
    int nx = g->nx, ny = g->ny, nz = g->nz;
    H.L.assign(1, MgLevel{});
    while ((long long)nx * ny * nz > kMgCoarsest) {
        nx = (nx + 1) / 2;
        ny = (ny + 1) / 2;
        nz = (nz + 1) / 2;
        MgLevel l{};
        l.nx = nx;
        l.ny = ny;
        l.nz = nz;
        l.n = nx * ny * nz;
        H.L.push_back(l);
    }
    const int nl = (int)H.L.size() - 1;
    if (nl == 0) return RFA_OK;
    size_t total = 0;
    for (int l = 1; l <= nl; ++l) total += 10 * (((size_t)H.L[l].n + 63) / 64 * 64);
    if (cudaMalloc(&H.mem, total * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&H.Ainv, (size_t)kMgCoarsest * kMgCoarsest * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        set_error("potential solve multigrid allocation failed");
        return RFA_E_OOM;
    }
    float *q = H.mem;
    for (int l = 1; l <= nl; ++l) {
        MgLevel &L = H.L[l];
        const size_t m = ((size_t)L.n + 63) / 64 * 64;
        float **arr[10] = {&L.D, &L.iD, &L.Wx, &L.Wy, &L.Wz, &L.G, &L.b, &L.x, &L.t, &L.r};
        for (float **a : arr) {
            *a = q;
            q += m;
        }
    }
    k_mg0_build<<<mg_blocks(H.L[1].n), 256, 0, g->stream>>>(G, H.L[1]);
    k_mg_diag<<<mg_blocks(H.L[1].n), 256, 0, g->stream>>>(H.L[1]);
    for (int l = 2; l <= nl; ++l) {
        k_mg_build<<<mg_blocks(H.L[l].n), 256, 0, g->stream>>>(H.L[l - 1], H.L[l]);
        k_mg_diag<<<mg_blocks(H.L[l].n), 256, 0, g->stream>>>(H.L[l]);
    }
    RFA_CUDA(cudaGetLastError());
    // the coarsest operator on the host: Cholesky in FP64 over its cells with a
    // nonzero diagonal, then the inverse (zero rows and columns elsewhere)
    const MgLevel &C = H.L[nl];
    const int n = C.n;
    std::vector<float> hD(n), hx(n), hy(n), hz(n);
    RFA_CUDA(cudaMemcpyAsync(hD.data(), C.D, n * sizeof(float), cudaMemcpyDeviceToHost, g->stream));
    RFA_CUDA(cudaMemcpyAsync(hx.data(), C.Wx, n * sizeof(float), cudaMemcpyDeviceToHost, g->stream));
    RFA_CUDA(cudaMemcpyAsync(hy.data(), C.Wy, n * sizeof(float), cudaMemcpyDeviceToHost, g->stream));
    RFA_CUDA(cudaMemcpyAsync(hz.data(), C.Wz, n * sizeof(float), cudaMemcpyDeviceToHost, g->stream));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    std::vector<int> cid(n, -1), cell;
    for (int c = 0; c < n; ++c)
        if (hD[c] > 0.f) {
            cid[c] = (int)cell.size();
            cell.push_back(c);
        }
    const int m = (int)cell.size();
    std::vector<double> A((size_t)m * m, 0.0);
    const int sy = C.nx, sz = C.nx * C.ny;
    for (int a = 0; a < m; ++a) {
        const int c = cell[a];
        const int X = c % C.nx, Y = (c / C.nx) % C.ny, Z = c / sz;
        A[(size_t)a * m + a] = hD[c];
        auto couple = [&](int o, float w) {
            if (cid[o] >= 0) {
                A[(size_t)a * m + cid[o]] -= w;
                A[(size_t)cid[o] * m + a] -= w;
            }
        };
        if (X + 1 < C.nx) couple(c + 1, hx[c]);
        if (Y + 1 < C.ny) couple(c + sy, hy[c]);
        if (Z + 1 < C.nz) couple(c + sz, hz[c]);
    }
    // A = L L^T in place (lower triangle)
    for (int j = 0; j < m; ++j) {
        double d = A[(size_t)j * m + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * m + k] * A[(size_t)j * m + k];
        if (!(d > 0.0)) return RFA_OK;  // not positive definite: Jacobi instead
        d = std::sqrt(d);
        A[(size_t)j * m + j] = d;
        for (int i = j + 1; i < m; ++i) {
            double v = A[(size_t)i * m + j];
            for (int k = 0; k < j; ++k) v -= A[(size_t)i * m + k] * A[(size_t)j * m + k];
            A[(size_t)i * m + j] = v / d;
        }
    }
    // columns of A^-1: L y = e_k, then L^T x = y
    std::vector<float> inv((size_t)n * n, 0.f);
    std::vector<double> y(m);
    for (int k = 0; k < m; ++k) {
        for (int i = 0; i < m; ++i) {
            double v = i == k ? 1.0 : 0.0;
            for (int j = 0; j < i; ++j) v -= A[(size_t)i * m + j] * y[j];
            y[i] = v / A[(size_t)i * m + i];
        }
        for (int i = m - 1; i >= 0; --i) {
            double v = y[i];
            for (int j = i + 1; j < m; ++j) v -= A[(size_t)j * m + i] * y[j];
            y[i] = v / A[(size_t)i * m + i];
        }
        for (int i = 0; i < m; ++i) inv[(size_t)cell[k] * n + cell[i]] = (float)y[i];
    }
    RFA_CUDA(cudaMemcpyAsync(H.Ainv, inv.data(), inv.size() * sizeof(float), cudaMemcpyHostToDevice, g->stream));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    ok = true;
    return RFA_OK;
}

}  // namespace

rfa_status potential_place(rfa_grid *g)
{
    const int L = g->n_labels;
    if (L > kCondLabels) {
        set_error("the potential-solve source supports at most 16 labels");
        return RFA_E_UNSUPPORTED;
    }
    if ((int)g->sigma.size() != L) {
        set_error("one electrical conductivity per label is needed");
        return RFA_E_INVALID;
    }
    std::vector<double> S(kCondLabels * kCondLabels, 0.0);
    for (int l = 0; l < L; ++l)
        for (int m = 0; m < L; ++m) {
            const double s = g->sigma[l] + g->sigma[m];
            if (s > 0.0) S[l * kCondLabels + m] = 2.0 * g->sigma[l] * g->sigma[m] / s;
        }
    const size_t nvp = g->nvp;
    struct Bufs {
        void *p[11] = {};
        ~Bufs()
        {
            for (void *q : p)
                if (q) cudaFree(q);
        }
    } B;
    for (int k = 0; k < 7; ++k)
        if (cudaMalloc(&B.p[k], nvp * 8) != cudaSuccess) {
            cudaGetLastError();
            set_error("potential solve workspace allocation failed");
            return RFA_E_OOM;
        }
    if (cudaMalloc(&B.p[7], nvp) != cudaSuccess ||
        cudaMalloc(&B.p[8], kCondLabels * kCondLabels * 8 + SC_N * 8 + 8) != cudaSuccess ||
        cudaMalloc(&B.p[9], 10 * nvp * sizeof(float)) != cudaSuccess || cudaMalloc(&B.p[10], nvp / 4 + 1) != cudaSuccess) {
        cudaGetLastError();
        set_error("potential solve workspace allocation failed");
        return RFA_E_OOM;
    }
    double *xv = (double *)B.p[0], *r = (double *)B.p[1], *zv = (double *)B.p[2], *p = (double *)B.p[3];
    double *Ap = (double *)B.p[4], *Dv = (double *)B.p[5], *iDv = (double *)B.p[6];
    uint8_t *cls = (uint8_t *)B.p[7];
    double *dS = (double *)B.p[8], *sc = dS + kCondLabels * kCondLabels;
    unsigned *ctr = (unsigned *)(sc + SC_N);  // last-block counter of the fused reductions
    double *part = (double *)g->red;  // 2 * kReduceBlocks doubles
    RFA_CUDA(cudaMemcpyAsync(dS, S.data(), S.size() * 8, cudaMemcpyHostToDevice, g->stream));
    RFA_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned), g->stream));
    uint8_t *quni = (uint8_t *)B.p[10];
    PotGrid G{cls, g->label, quni, dS, g->nx, g->ny, g->nz, g->pitch, g->plane, nvp};
    const unsigned nb = kReduceBlocks;
    k_pot_class<<<nb, 256, 0, g->stream>>>(g->geom, G, g->h, needle_margin(g), cls);
    k_pot_quni<<<nb, 256, 0, g->stream>>>(G, quni);
    k_pot_init<<<nb, 256, 0, g->stream>>>(G, xv, r, zv, p, Dv, iDv, part);
    k_pot_scalars<<<1, 1024, 0, g->stream>>>(part, nb, SCW_START, sc);
    RFA_CUDA(cudaGetLastError());
    double host_sc[SC_N];
    RFA_CUDA(cudaMemcpyAsync(host_sc, sc, sizeof host_sc, cudaMemcpyDeviceToHost, g->stream));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    const double bnorm = std::sqrt(host_sc[SC_BB]);
    double rel = bnorm > 0.0 ? 1.0 : 0.0;
    int it = 0;
    auto read_scalars = [&]() -> rfa_status {
        RFA_CUDA(cudaGetLastError());
        RFA_CUDA(cudaMemcpyAsync(host_sc, sc, sizeof host_sc, cudaMemcpyDeviceToHost, g->stream));
        RFA_CUDA(cudaStreamSynchronize(g->stream));
        return RFA_OK;
    };
    // FP32 cycles inside the FP64 defect correction (r = b at the start, x = the fixed values)
    float *r32 = (float *)B.p[9], *e32 = r32 + nvp, *z32 = e32 + nvp, *Ap32 = z32 + nvp;
    float *D32 = Ap32 + nvp, *iD32 = D32 + nvp, *pbuf[2] = {iD32 + nvp, iD32 + 2 * nvp};
    float *zB = pbuf[1] + nvp, *rt = zB + nvp;  // the V-cycle's second fine iterate and residual
    MgHost H;
    bool use_mg = false;
    if (g->pot_precond == RFA_PRECOND_MULTIGRID)
        if (rfa_status st = mg_setup(g, G, H, use_mg)) return st;
    const int nl = (int)H.L.size() - 1;
    // the levels of at most kMgTailCells cells (and the coarsest) run in one block
    int lt = nl;
    MgTail tail{};
    if (use_mg) {
        while (lt > 1 && H.L[lt - 1].n <= kMgTailCells && nl - lt + 2 <= kMgTailMax) --lt;
        tail.n = nl - lt + 1;
        tail.Ainv = H.Ainv;
        for (int l = lt; l <= nl; ++l) tail.L[l - lt] = H.L[l];
    }
    // z = M b: one V-cycle (the fine iterates alternate between z32 and zB)
    // the fine-level sweeps stream z in chunks (32 x 8 quads a block)
    const int zc0 = choose_zchunk(g, 3);
    const dim3 sblk(32, 8), sgrd = plain_grid_dims(g, zc0);
    static_assert(kMgNu >= 2, "the first pre-sweep is the fused pass from zero");
    auto vcycle = [&](const float *b0) -> float * {
        float *cur0 = z32, *oth0 = zB;
        // the first sweep from zero (v = omega b / D formed where it is read), written to zB
        k_mg0_sweep_z<false, true><<<sgrd, sblk, 0, g->stream>>>(G, D32, iD32, b0, nullptr, oth0, zc0);
        std::swap(cur0, oth0);
        for (int s = 2; s < kMgNu; ++s) {
            k_mg0_sweep_z<false, false><<<sgrd, sblk, 0, g->stream>>>(G, D32, iD32, b0, cur0, oth0, zc0);
            std::swap(cur0, oth0);
        }
        k_mg0_sweep_z<true, false><<<sgrd, sblk, 0, g->stream>>>(G, D32, iD32, b0, cur0, rt, zc0);
        k_mg0_restrict<<<mg_blocks(H.L[1].n), 256, 0, g->stream>>>(G, rt, H.L[1], H.L[1].b);
        std::vector<float *> cur(nl + 1), oth(nl + 1);
        for (int l = 1; l < lt; ++l) {
            const MgLevel &L = H.L[l];
            const unsigned bl = mg_blocks(L.n);
            cur[l] = L.x;
            oth[l] = L.t;
            k_mg_first<<<bl, 256, 0, g->stream>>>(L, L.b, cur[l]);
            for (int s = 1; s < kMgNu; ++s) {
                k_mg_sweep<false><<<bl, 256, 0, g->stream>>>(L, L.b, cur[l], oth[l]);
                std::swap(cur[l], oth[l]);
            }
            k_mg_sweep<true><<<bl, 256, 0, g->stream>>>(L, L.b, cur[l], L.r);
            k_mg_restrict<<<mg_blocks(H.L[l + 1].n), 256, 0, g->stream>>>(L, L.r, H.L[l + 1], H.L[l + 1].b);
        }
        // levels lt .. nl in one block; their iterates alternate as in k_mg_tail
        k_mg_tail<<<1, 1024, 0, g->stream>>>(tail);
        for (int l = lt; l < nl; ++l) {
            cur[l] = H.L[l].x;
            oth[l] = H.L[l].t;
            for (int s = 1; s < 2 * kMgNu; ++s) std::swap(cur[l], oth[l]);
        }
        cur[nl] = H.L[nl].x;
        for (int l = lt - 1; l >= 1; --l) {
            const MgLevel &L = H.L[l];
            const unsigned bl = mg_blocks(L.n);
            k_mg_prolong<<<bl, 256, 0, g->stream>>>(L, H.L[l + 1], cur[l + 1], cur[l]);
            for (int s = 0; s < kMgNu; ++s) {
                k_mg_sweep<false><<<bl, 256, 0, g->stream>>>(L, L.b, cur[l], oth[l]);
                std::swap(cur[l], oth[l]);
            }
        }
        k_mg0_prolong<<<nb, 256, 0, g->stream>>>(G, iD32, H.L[1], cur[1], cur0);
        for (int s = 0; s < kMgNu; ++s) {
            k_mg0_sweep_z<false, false><<<sgrd, sblk, 0, g->stream>>>(G, D32, iD32, b0, cur0, oth0, zc0);
            std::swap(cur0, oth0);
        }
        return cur0;
    };
    float *zfin = z32;  // the preconditioned residual of the current iteration
    bool fp64_cg = false;
    int pk = 0;     // pbuf[pk]: the previous direction (kept across replacements)
    int cycle = 0;  // 0: the first cycle starts from direction 0
    while (rel > g->pot_tol && it < g->pot_max_iters && !fp64_cg) {
        const double eta = std::max(kInnerEta, 0.25 * g->pot_tol / rel);
        // Jacobi keeps the search direction across a replacement; the multigrid
        // iteration restarts from direction 0 (with its strong preconditioner a
        // kept direction is no longer conjugate to the new residual's Krylov
        // space, and convergence stalls)
        k_pot_init32<<<nb, 256, 0, g->stream>>>(G, r, Dv, r32, e32, z32, pbuf[pk], D32, iD32, !use_mg && cycle > 0,
                                               part);
        if (use_mg) {
            k_pot_scalars<<<1, 1024, 0, g->stream>>>(part, nb, SCW_RR_B, sc);
            zfin = vcycle(r32);
            k_pot_dot32<<<nb, 256, 0, g->stream>>>(G, r32, zfin, SCW_START_RZ, sc, part, ctr);
        } else {
            k_pot_scalars<<<1, 1024, 0, g->stream>>>(part, nb, cycle > 0 ? SCW_BETA_RR : SCW_START, sc);
            zfin = z32;
        }
        ++cycle;
        if (rfa_status st = read_scalars()) return st;
        const double r0 = std::sqrt(std::fmax(host_sc[SC_RR], 0.0));
        double rin = r0, best = r0;
        int flat = 0;  // checks without a new minimum of the FP32 residual
        while (rin > eta * r0 && it < g->pot_max_iters && flat < kFlatChecks) {
            const int n = std::min(use_mg ? kCheckMg : kCheck, g->pot_max_iters - it);
            for (int k = 0; k < n; ++k) {
                k_pot_spmv32<<<nb, 256, 0, g->stream>>>(G, sc, D32, zfin, pbuf[pk], pbuf[pk ^ 1], Ap32, part, ctr);
                if (use_mg) {
                    k_pot_update32_mg<<<nb, 256, 0, g->stream>>>(G, sc, e32, r32, pbuf[pk ^ 1], Ap32, part, ctr);
                    zfin = vcycle(r32);
                    k_pot_dot32<<<nb, 256, 0, g->stream>>>(G, r32, zfin, SCW_BETA, sc, part, ctr);
                } else {
                    k_pot_update32<<<nb, 256, 0, g->stream>>>(G, sc, iD32, e32, r32, z32, pbuf[pk ^ 1], Ap32, part,
                                                              ctr);
                }
                pk ^= 1;
            }
            it += n;
            if (rfa_status st = read_scalars()) return st;
            rin = std::sqrt(std::fmax(host_sc[SC_RR], 0.0));
            if (!std::isfinite(rin)) {
                set_error("potential solve diverged");
                return RFA_E_NONFINITE;
            }
            if (rin < 0.99 * best) {
                best = rin;
                flat = 0;
            } else {
                ++flat;
            }
        }
        k_pot_correct<<<nb, 256, 0, g->stream>>>(G, e32, xv);
        k_pot_resid64<<<nb, 256, 0, g->stream>>>(G, xv, r, part);
        k_pot_scalars<<<1, 1024, 0, g->stream>>>(part, nb, SCW_RR, sc);
        if (rfa_status st = read_scalars()) return st;
        const double rel_new = std::sqrt(std::fmax(host_sc[SC_RR], 0.0)) / bnorm;
        if (!std::isfinite(rel_new)) {
            set_error("potential solve diverged");
            return RFA_E_NONFINITE;
        }
        fp64_cg = !(rel_new <= 0.5 * rel);  // FP32 stagnated: FP64 from here
        rel = rel_new;
    }
    // FP64 conjugate gradients from the current x (r already holds b - A x)
    if (rel > g->pot_tol && it < g->pot_max_iters) {
        k_pot_restart64<<<nb, 256, 0, g->stream>>>(G, r, iDv, zv, p, part);
        k_pot_scalars<<<1, 1024, 0, g->stream>>>(part, nb, SCW_START, sc);
    }
    while (rel > g->pot_tol && it < g->pot_max_iters) {
        const int n = std::min(kCheck, g->pot_max_iters - it);
        for (int k = 0; k < n; ++k) {
            k_pot_spmv<<<nb, 256, 0, g->stream>>>(G, Dv, p, Ap, part);
            k_pot_scalars<<<1, 1024, 0, g->stream>>>(part, nb, SCW_ALPHA, sc);
            k_pot_update<<<nb, 256, 0, g->stream>>>(G, sc, iDv, xv, r, zv, p, Ap, part);
            k_pot_scalars<<<1, 1024, 0, g->stream>>>(part, nb, SCW_BETA_RR, sc);
            k_pot_direction<<<nb, 256, 0, g->stream>>>(G, sc, zv, p);
        }
        it += n;
        if (rfa_status st = read_scalars()) return st;
        rel = std::sqrt(std::fmax(host_sc[SC_RR], 0.0)) / bnorm;
        if (!std::isfinite(rel)) {
            set_error("potential solve diverged");
            return RFA_E_NONFINITE;
        }
    }
    g->pot_iters = it;
    g->pot_res = rel;
    k_pot_joule<<<nb, 256, 0, g->stream>>>(G, xv, g->d_table, g->face, g->h, (double *)g->stage, part);
    RFA_CUDA(cudaGetLastError());
    RFA_CUDA(launch_source_write(g, part, (int)nb));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    return RFA_OK;
}

}  // namespace rfa
