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
// Solver: conjugate gradients with the Jacobi preconditioner, matrix-free, in
// FP64 (the source sets the heating of every later step; FP64 keeps the solve
// far below the FP32 state's resolution).  The diagonal and its inverse are
// stored once (B300's FP64 pipe is narrow: no per-iteration division).
// Scalars stay on the device; the host reads the residual every kCheck
// iterations.
//
// Heating: q_i = sum_nb sigma_f (V_nb - V_i)^2 / (2 h^2), each face's
// dissipation split between its two voxels, so that sum_i q_i h^3 equals the
// network's dissipated power; then q is scaled so that the free voxels receive
// the needle power P, exactly like the 1/r^4 weights (launch_source_write).
#include "rfa_internal.cuh"

#include <cmath>
#include <vector>

namespace rfa {

namespace {

constexpr int kCheck = 20;
enum { CLS_FREE = 0, CLS_ELECTRODE = 1, CLS_GROUND = 2, CLS_PAD = 3 };
// scalars: rz, alpha, beta, rr, bb
enum { SC_RZ = 0, SC_ALPHA, SC_BETA, SC_RR, SC_BB, SC_N };

struct PotGrid {
    const uint8_t *cls, *label;
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

__global__ void k_pot_class(NeedleGeom geom, PotGrid G, double h, uint8_t *cls)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < G.nvp; i += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        pot_xyz(G, i, x, y, z);
        uint8_t c = CLS_FREE;
        if (x >= G.nx) c = CLS_PAD;
        else if (x == 0 || y == 0 || z == 0 || x == G.nx - 1 || y == G.ny - 1 || z == G.nz - 1) c = CLS_GROUND;
        else if (needle_dist2(geom, x * h, y * h, z * h) <= geom.r0 * geom.r0) c = CLS_ELECTRODE;
        cls[i] = c;
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
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < G.nvp; i += (size_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        if (G.cls[i] == CLS_FREE) {
            int x, y, z;
            pot_xyz(G, i, x, y, z);
            const int l = G.label[i];
            const double pi = p[i];
            v = Dv[i] * pi;
            for (int d = 0; d < 6; ++d) {
                size_t j;
                if (pot_nb(G, i, x, y, z, d, j) && G.cls[j] == CLS_FREE) v -= S[l * kCondLabels + G.label[j]] * p[j];
            }
            acc += pi * v;
        }
        Ap[i] = v;
    }
    acc = pot_block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// scalar steps on one block: which = 0 -> alpha = rz / sum(part); 1 -> rz_new, beta, rr
__global__ void k_pot_scalars(const double *part, int nblk, int which, double *sc)
{
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) {
        if (which == 0) {
            a += part[k];
        } else {
            a += part[2 * k];
            b += part[2 * k + 1];
        }
    }
    a = pot_block_sum(a);
    b = pot_block_sum(b);
    if (threadIdx.x == 0) {
        if (which == 0) {
            sc[SC_ALPHA] = a != 0.0 ? sc[SC_RZ] / a : 0.0;
        } else if (which == 1) {
            sc[SC_BETA] = sc[SC_RZ] != 0.0 ? a / sc[SC_RZ] : 0.0;
            sc[SC_RZ] = a;
            sc[SC_RR] = b;
        } else {  // initial: rz and b.b
            sc[SC_RZ] = a;
            sc[SC_BB] = b;
            sc[SC_RR] = b;
        }
    }
}

// x += alpha p; r -= alpha Ap; z = r / D; partial sums of r.z and r.r
__global__ void __launch_bounds__(256) k_pot_update(PotGrid G, const double *sc, const double *iDv, double *xv,
                                                   double *r, double *zv, const double *p, const double *Ap,
                                                   double *part)
{
    const double alpha = sc[SC_ALPHA];
    double rz = 0.0, rr = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < G.nvp; i += (size_t)gridDim.x * blockDim.x) {
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

__global__ void k_pot_direction(PotGrid G, const double *sc, const double *zv, double *p)
{
    const double beta = sc[SC_BETA];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < G.nvp; i += (size_t)gridDim.x * blockDim.x)
        if (G.cls[i] == CLS_FREE) p[i] = zv[i] + beta * p[i];
}

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
        void *p[9] = {};
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
    if (cudaMalloc(&B.p[7], nvp) != cudaSuccess || cudaMalloc(&B.p[8], kCondLabels * kCondLabels * 8 + SC_N * 8) != cudaSuccess) {
        cudaGetLastError();
        set_error("potential solve workspace allocation failed");
        return RFA_E_OOM;
    }
    double *xv = (double *)B.p[0], *r = (double *)B.p[1], *zv = (double *)B.p[2], *p = (double *)B.p[3];
    double *Ap = (double *)B.p[4], *Dv = (double *)B.p[5], *iDv = (double *)B.p[6];
    uint8_t *cls = (uint8_t *)B.p[7];
    double *dS = (double *)B.p[8], *sc = dS + kCondLabels * kCondLabels;
    double *part = (double *)g->red;  // 2 * kReduceBlocks doubles
    RFA_CUDA(cudaMemcpyAsync(dS, S.data(), S.size() * 8, cudaMemcpyHostToDevice, g->stream));
    PotGrid G{cls, g->label, dS, g->nx, g->ny, g->nz, g->pitch, g->plane, nvp};
    const unsigned nb = kReduceBlocks;
    k_pot_class<<<nb, 256, 0, g->stream>>>(g->geom, G, g->h, cls);
    k_pot_init<<<nb, 256, 0, g->stream>>>(G, xv, r, zv, p, Dv, iDv, part);
    k_pot_scalars<<<1, 1024, 0, g->stream>>>(part, nb, 2, sc);
    RFA_CUDA(cudaGetLastError());
    double host_sc[SC_N];
    RFA_CUDA(cudaMemcpyAsync(host_sc, sc, sizeof host_sc, cudaMemcpyDeviceToHost, g->stream));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    const double bnorm = std::sqrt(host_sc[SC_BB]);
    double rel = bnorm > 0.0 ? 1.0 : 0.0;
    int it = 0;
    while (rel > g->pot_tol && it < g->pot_max_iters) {
        const int n = std::min(kCheck, g->pot_max_iters - it);
        for (int k = 0; k < n; ++k) {
            k_pot_spmv<<<nb, 256, 0, g->stream>>>(G, Dv, p, Ap, part);
            k_pot_scalars<<<1, 1024, 0, g->stream>>>(part, nb, 0, sc);
            k_pot_update<<<nb, 256, 0, g->stream>>>(G, sc, iDv, xv, r, zv, p, Ap, part);
            k_pot_scalars<<<1, 1024, 0, g->stream>>>(part, nb, 1, sc);
            k_pot_direction<<<nb, 256, 0, g->stream>>>(G, sc, zv, p);
        }
        it += n;
        RFA_CUDA(cudaGetLastError());
        RFA_CUDA(cudaMemcpyAsync(host_sc, sc, sizeof host_sc, cudaMemcpyDeviceToHost, g->stream));
        RFA_CUDA(cudaStreamSynchronize(g->stream));
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
