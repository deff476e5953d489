/*
 * oracle.c -- plain FP64 CPU reference of the RFA bioheat explicit scheme.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or constant with the CUDA path; both sides only read the same
 * seeded inputs (labels, tissue table, needle description).
 *
 * What it computes, in the paper's order:
 *   - or_setup:   labels -> per-voxel coefficients (Sec. "Implementation": the
 *                 label image becomes the start temperature image; vessels and
 *                 the tip are held at fixed temperature, Eq. 2675-eq6 / Alg. 1's
 *                 else-branch).
 *   - or_source:  RF heat source q_i placed by the needle geometry; the paper
 *                 gives only the resistive term sigma|grad V|^2 of Eq.
 *                 2675-eq1_Linte, whose point-electrode closed form decays as
 *                 1/r^4; q_i ~ max(d_i, r0)^-4 normalised to the needle power.
 *   - or_run:     forward Euler of Eq. 2675-eq2 discretised with the central
 *                 second difference (Eq. 2675-eq3) into Eq. CUDAbioheat3d,
 *                 a Jacobi (double-buffer) update as in Alg. 2; plus the 60 C
 *                 necrosis latch (Sec. "Introduction") and the Arrhenius damage
 *                 integral of Eq. eq-tissState, Kahan-summed.
 *   - or_adjoint: discrete reverse of or_run (transpose of the step matrix) for
 *                 gradients w.r.t. per-label conductivity and perfusion.
 *   - or_source_grad: contraction of the summed adjoint with dq/dP, dq/dtip.
 *
 * Readings of the paper (see the design notes of the repository):
 *   state theta = T - T_a; theta' = theta + a*sum_nb(theta_nb - theta)
 *   - b*theta + s + qm, with a = K dt/(rho c h^2), b = w_b rho_b c_b dt/(rho c),
 *   s = q dt/(rho c), qm = Q_m dt/(rho c); fixed voxels keep their value;
 *   a neighbour outside the grid contributes nothing (mirror ghost); Dirichlet
 *   faces are expressed by fixing the outer voxel layer at theta = 0.
 *
 * Every function here is pinned by CPU tests against closed forms, a dense
 * brute-force matrix, the paper's monotonicity property or finite differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(x, y, z) ((size_t)(z) * (size_t)ny * (size_t)nx + (size_t)(y) * (size_t)nx + (size_t)(x))

/* Tissue table row layout (9 doubles per label). */
enum { T_K = 0, T_RHO, T_C, T_WB, T_RHOB, T_CB, T_QM, T_FIXED, T_TFIX, T_NCOL };

/* Needle description layout (14 doubles). */
enum { N_KIND = 0, N_TIP0, N_TIP1, N_TIP2, N_AX0, N_AX1, N_AX2, N_ACTIVE, N_TINE, N_POLAR,
       N_NTINES, N_AXIAL, N_POWER, N_RCLAMP, N_NCOL };

/* ---------------------------------------------------------------- rounding */

/* Round to the nearest value with 8 significant bits (bfloat16), ties to even. */
double or_round_bf16(double x)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    double m = frexp(x, &e);              /* x = m * 2^e, 0.5 <= |m| < 1 */
    double r = nearbyint(ldexp(m, 8));    /* 8 significant bits, default mode = ties-to-even */
    return ldexp(r, e - 8);
}

static double round_param(double x, int mode)
{
    if (mode == 1) return (double)(float)x;  /* IEEE binary32, round to nearest even */
    if (mode == 2) return or_round_bf16(x);
    return x;
}

/* ---------------------------------------------------------------- setup */

/*
 * Per-voxel coefficients from labels.  param_mode: 0 exact FP64, 1 rounded to
 * FP32, 2 rounded to BF16 (the values the GPU path stores).  face_bc: 0 =
 * Dirichlet (outer layer fixed at T_a), 1 = insulated.
 */
int or_setup(int nx, int ny, int nz, double h, double dt, int face_bc, double T_a, int param_mode,
             const uint8_t *labels, int n_labels, const double *tab,
             double *a, double *b, double *qm, double *rhoc, uint8_t *isfixed, double *theta0)
{
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = IDX(x, y, z);
                int l = labels[i];
                if (l >= n_labels) return 1;
                const double *t = tab + (size_t)l * T_NCOL;
                double k = t[T_K], rho = t[T_RHO], c = t[T_C], w_b = t[T_WB];
                double rho_b = t[T_RHOB], c_b = t[T_CB], Q_m = t[T_QM];
                rhoc[i] = rho * c;
                int on_face = (x == 0 || y == 0 || z == 0 || x == nx - 1 || y == ny - 1 || z == nz - 1);
                if (t[T_FIXED] != 0.0) {
                    isfixed[i] = 1;
                    a[i] = b[i] = qm[i] = 0.0;
                    theta0[i] = t[T_TFIX] - T_a;
                } else if (face_bc == 0 && on_face) {
                    isfixed[i] = 1;
                    a[i] = b[i] = qm[i] = 0.0;
                    theta0[i] = 0.0;
                } else {
                    isfixed[i] = 0;
                    /* a = K dt / (rho c h^2), b = w_b rho_b c_b dt / (rho c): Eq. CUDAbioheat3d */
                    a[i] = round_param((k / (rho * c)) * dt / (h * h), param_mode);
                    b[i] = round_param((w_b * rho_b * c_b / (rho * c)) * dt, param_mode);
                    qm[i] = Q_m * dt / (rho * c);
                    theta0[i] = 0.0;
                }
            }
    return 0;
}

/* ---------------------------------------------------------------- source */

typedef struct { double p0[3], p1[3]; } segment;

static double dot3(const double *u, const double *v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; }

/* Active segments of the needle: straight = the last active_len behind the tip;
 * umbrella = n tines leaving the tip at a polar angle off the axis, evenly
 * spaced in azimuth, plus an optional axial tine.  Returns the count. */
static int needle_segments(const double *nd, segment *seg)
{
    int kind = (int)nd[N_KIND];
    double tip[3] = { nd[N_TIP0], nd[N_TIP1], nd[N_TIP2] };
    double ax[3] = { nd[N_AX0], nd[N_AX1], nd[N_AX2] };
    double n = sqrt(dot3(ax, ax));
    for (int d = 0; d < 3; ++d) ax[d] /= n;
    int ns = 0;
    if (kind == 0) {
        for (int d = 0; d < 3; ++d) {
            seg[0].p0[d] = tip[d] - nd[N_ACTIVE] * ax[d];
            seg[0].p1[d] = tip[d];
        }
        ns = 1;
    } else if (kind == 1) {
        /* basis (e1, e2) perpendicular to the axis; for axis +z it is (x, y) */
        double ref[3] = { 1.0, 0.0, 0.0 };
        if (fabs(ax[2]) < 0.9) { ref[0] = 0.0; ref[2] = 1.0; }
        double pr = dot3(ref, ax), e1[3], e2[3];
        for (int d = 0; d < 3; ++d) e1[d] = ref[d] - pr * ax[d];
        double n1 = sqrt(dot3(e1, e1));
        for (int d = 0; d < 3; ++d) e1[d] /= n1;
        e2[0] = ax[1] * e1[2] - ax[2] * e1[1];
        e2[1] = ax[2] * e1[0] - ax[0] * e1[2];
        e2[2] = ax[0] * e1[1] - ax[1] * e1[0];
        int nt = (int)nd[N_NTINES];
        double pol = nd[N_POLAR] * M_PI / 180.0, len = nd[N_TINE];
        for (int j = 0; j < nt; ++j) {
            double phi = 2.0 * M_PI * j / nt;
            for (int d = 0; d < 3; ++d) {
                double dir = cos(pol) * ax[d] + sin(pol) * (cos(phi) * e1[d] + sin(phi) * e2[d]);
                seg[ns].p0[d] = tip[d];
                seg[ns].p1[d] = tip[d] + len * dir;
            }
            ++ns;
        }
        if ((int)nd[N_AXIAL]) {
            for (int d = 0; d < 3; ++d) {
                seg[ns].p0[d] = tip[d];
                seg[ns].p1[d] = tip[d] + len * ax[d];
            }
            ++ns;
        }
    }
    return ns;
}

/* Euclidean distance from p to segment [p0, p1]; closest point in q. */
static double seg_dist(const double *p, const segment *s, double *q)
{
    double u[3], w[3];
    for (int d = 0; d < 3; ++d) { u[d] = s->p1[d] - s->p0[d]; w[d] = p[d] - s->p0[d]; }
    double uu = dot3(u, u), t = uu > 0.0 ? dot3(w, u) / uu : 0.0;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) { q[d] = s->p0[d] + t * u[d]; double e = p[d] - q[d]; r2 += e * e; }
    return sqrt(r2);
}

/* Minimum distance to all segments, and the closest point on the nearest one. */
static double needle_dist(const double *p, const segment *seg, int ns, double *qbest)
{
    double best = INFINITY, q[3];
    for (int k = 0; k < ns; ++k) {
        double d = seg_dist(p, &seg[k], q);
        if (d < best) { best = d; qbest[0] = q[0]; qbest[1] = q[1]; qbest[2] = q[2]; }
    }
    return best;
}

/*
 * s_i = q_i dt / (rho c)_i with q_i = P w_i / (h^3 sum_{free j} w_j),
 * w_i = max(d_i, r0)^-4; fixed voxels get s = 0.  dist (optional) receives d_i.
 */
int or_source(int nx, int ny, int nz, double h, double dt, const double *nd,
              const double *rhoc, const uint8_t *isfixed, double *s, double *dist, double *W_out)
{
    segment seg[64];
    int ns = needle_segments(nd, seg);
    double r0 = nd[N_RCLAMP], P = nd[N_POWER];
    size_t n = (size_t)nx * ny * nz;
    double *w = (double *)malloc(n * sizeof(double));
    if (!w) return 2;
    double W = 0.0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = IDX(x, y, z);
                double p[3] = { x * h, y * h, z * h }, q[3];
                double d = ns > 0 ? needle_dist(p, seg, ns, q) : INFINITY;
                if (dist) dist[i] = d;
                double r = d > r0 ? d : r0;
                w[i] = ns > 0 ? 1.0 / (r * r * r * r) : 0.0;
                if (!isfixed[i]) W += w[i];
            }
    for (size_t i = 0; i < n; ++i)
        s[i] = (isfixed[i] || W == 0.0) ? 0.0 : P * w[i] / (h * h * h * W) * dt / rhoc[i];
    if (W_out) *W_out = W;
    free(w);
    return 0;
}

/* ---------------------------------------------------------------- forward */

/*
 * nsteps explicit Euler steps of Eq. CUDAbioheat3d in theta = T - T_a.
 * latch_i |= (T_i >= T_thr) after every step; with damage != 0,
 * omega_i += dt * A * exp(-Ea / (R * T_K)) (Eq. eq-tissState's integrand,
 * right-rectangle rule on the new temperature), compensated by Kahan's method.
 */
/*
 * Conductive term of free voxel i.  Centre form (wf == NULL): the paper's
 * K * (sum of second differences) with K taken at the voxel, a_i * sum_nb
 * (theta_nb - theta_i).  Conservative form (wf != NULL): div(K grad T) with the
 * face conductance between two voxels the harmonic mean of their K,
 * sum_nb wf[d][i] (theta_nb - theta_i), wf[d][i] = dt/(rho c_i h^2) *
 * 2 K_i K_nb / (K_i + K_nb) for direction d = x-, x+, y-, y+, z-, z+ (0 outside
 * the grid).
 */
static double conduction(int nx, int ny, int nz, const double *a, const double *wf, const double *cur,
                         int x, int y, int z)
{
    const size_t n = (size_t)nx * ny * nz, i = IDX(x, y, z);
    const double t = cur[i];
    if (!wf) {
        double sum = 0.0;
        if (x > 0)      sum += cur[IDX(x - 1, y, z)] - t;
        if (x < nx - 1) sum += cur[IDX(x + 1, y, z)] - t;
        if (y > 0)      sum += cur[IDX(x, y - 1, z)] - t;
        if (y < ny - 1) sum += cur[IDX(x, y + 1, z)] - t;
        if (z > 0)      sum += cur[IDX(x, y, z - 1)] - t;
        if (z < nz - 1) sum += cur[IDX(x, y, z + 1)] - t;
        return a[i] * sum;
    }
    double f = 0.0;
    if (x > 0)      f += wf[0 * n + i] * (cur[IDX(x - 1, y, z)] - t);
    if (x < nx - 1) f += wf[1 * n + i] * (cur[IDX(x + 1, y, z)] - t);
    if (y > 0)      f += wf[2 * n + i] * (cur[IDX(x, y - 1, z)] - t);
    if (y < ny - 1) f += wf[3 * n + i] * (cur[IDX(x, y + 1, z)] - t);
    if (z > 0)      f += wf[4 * n + i] * (cur[IDX(x, y, z - 1)] - t);
    if (z < nz - 1) f += wf[5 * n + i] * (cur[IDX(x, y, z + 1)] - t);
    return f;
}

int or_run(int nx, int ny, int nz, int64_t nsteps,
           const double *a, const double *b, const double *s, const double *qm,
           const uint8_t *isfixed, double *theta, uint8_t *latch, double T_a, double T_thr,
           int damage, double dt, double A, double Ea, double R, double *omega, double *omega_c,
           int nthreads, const double *wf, int alpha_perf)
{
    size_t n = (size_t)nx * ny * nz;
    double *cur = theta;
    double *nxt = (double *)malloc(n * sizeof(double));
    if (!nxt) return 2;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int64_t step = 0; step < nsteps; ++step) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t i = IDX(x, y, z);
                    double t = cur[i], tn;
                    if (isfixed[i]) {
                        tn = t;   /* Alg. 1 else-branch: copy the input value */
                    } else {
                        /* central second differences in x, y, z (Eq. 2675-eq3); with the
                           tissue-state coupling the perfusion is weighted by
                           alpha = 1 / max(1, Omega) (Eq. eq-tissState, capped at 1) */
                        const double bi = alpha_perf ? b[i] / fmax(1.0, omega[i]) : b[i];
                        tn = t + conduction(nx, ny, nz, a, wf, cur, x, y, z) - bi * t + s[i] + qm[i];
                    }
                    nxt[i] = tn;
                    if (tn + T_a >= T_thr) latch[i] = 1;
                    if (damage) {
                        double TK = tn + T_a + 273.15;
                        double inc = dt * A * exp(-Ea / (R * TK));
                        double yk = inc - omega_c[i];
                        double tk = omega[i] + yk;
                        omega_c[i] = (tk - omega[i]) - yk;
                        omega[i] = tk;
                    }
                }
        double *tmp = cur; cur = nxt; nxt = tmp;
    }
    if (cur != theta) {
        memcpy(theta, cur, n * sizeof(double));
        free(cur);
    } else {
        free(nxt);
    }
    return 0;
}

/* ---------------------------------------------------------------- adjoint */

/* d theta'_j / d theta_i of one step (the step matrix entry A[j][i]). */
static double step_entry(int nx, int ny, int nz, const double *a, const double *b, const double *wf,
                         const uint8_t *isfixed, int xj, int yj, int zj, int xi, int yi, int zi)
{
    const size_t n = (size_t)nx * ny * nz, j = IDX(xj, yj, zj);
    if (isfixed[j]) return (xj == xi && yj == yi && zj == zi) ? 1.0 : 0.0;
    if (!wf) {
        if (xj == xi && yj == yi && zj == zi) {
            int deg = (xj > 0) + (xj < nx - 1) + (yj > 0) + (yj < ny - 1) + (zj > 0) + (zj < nz - 1);
            return 1.0 - a[j] * deg - b[j];
        }
        return a[j];  /* i is a grid neighbour of j */
    }
    if (xj == xi && yj == yi && zj == zi) {
        double w = 0.0;
        if (xj > 0)      w += wf[0 * n + j];
        if (xj < nx - 1) w += wf[1 * n + j];
        if (yj > 0)      w += wf[2 * n + j];
        if (yj < ny - 1) w += wf[3 * n + j];
        if (zj > 0)      w += wf[4 * n + j];
        if (zj < nz - 1) w += wf[5 * n + j];
        return 1.0 - w - b[j];
    }
    /* i is the neighbour of j in direction d */
    const int d = xi < xj ? 0 : xi > xj ? 1 : yi < yj ? 2 : yi > yj ? 3 : zi < zj ? 4 : 5;
    return wf[(size_t)d * n + j];
}

/* one forward step without latch/damage (used to recompute the trajectory) */
static void plain_step(int nx, int ny, int nz, const double *a, const double *b, const double *wf,
                       const double *s, const double *qm, const uint8_t *isfixed, const double *cur,
                       double *nxt)
{
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = IDX(x, y, z);
                double t = cur[i];
                if (isfixed[i]) { nxt[i] = t; continue; }
                nxt[i] = t + conduction(nx, ny, nz, a, wf, cur, x, y, z) - b[i] * t + s[i] + qm[i];
            }
}

/*
 * Discrete adjoint of nsteps forward steps from theta0.  lam (in: dL/dtheta_N,
 * out: dL/dtheta_0).  Lambda_i = sum_{n=1..N} lambda^n_i.  g_k[l] and g_wb[l]
 * receive dL/dK_l and dL/dw_b,l through a_i = K dt/(rho c h^2) and
 * b_i = w_b rho_b c_b dt/(rho c) of the free voxels carrying label l.
 * The trajectory is recomputed from checkpoints every ceil(sqrt(N)) steps.
 */
int or_adjoint(int nx, int ny, int nz, int64_t nsteps, double h, double dt,
               const double *a, const double *b, const double *s, const double *qm,
               const uint8_t *isfixed, const uint8_t *labels, int n_labels, const double *tab,
               const double *rhoc, const double *theta0, double *lam,
               double *Lambda, double *g_k, double *g_wb, int nthreads,
               const double *wf, const double *dwa, const double *dwb)
{
    size_t n = (size_t)nx * ny * nz;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int64_t seg = (int64_t)ceil(sqrt((double)(nsteps > 0 ? nsteps : 1)));
    int64_t nck = (nsteps + seg - 1) / seg;
    double *ck = (double *)malloc((size_t)(nck > 0 ? nck : 1) * n * sizeof(double));
    double *traj = (double *)malloc((size_t)(seg + 1) * n * sizeof(double));
    double *lnew = (double *)malloc(n * sizeof(double));
    double *pk = (double *)calloc((size_t)nz * n_labels, sizeof(double));
    double *pw = (double *)calloc((size_t)nz * n_labels, sizeof(double));
    if (!ck || !traj || !lnew || !pk || !pw) return 2;

    /* forward sweep storing checkpoints theta^{j*seg} */
    memcpy(traj, theta0, n * sizeof(double));
    for (int64_t st = 0; st < nsteps; ++st) {
        if (st % seg == 0) memcpy(ck + (size_t)(st / seg) * n, traj, n * sizeof(double));
        plain_step(nx, ny, nz, a, b, wf, s, qm, isfixed, traj, traj + n);
        memcpy(traj, traj + n, n * sizeof(double));
    }
    memset(Lambda, 0, n * sizeof(double));
    for (int l = 0; l < n_labels; ++l) { g_k[l] = 0.0; g_wb[l] = 0.0; }

    for (int64_t c = nck - 1; c >= 0; --c) {
        int64_t s0 = c * seg, s1 = s0 + seg < nsteps ? s0 + seg : nsteps;
        /* recompute theta^{s0} .. theta^{s1-1} */
        memcpy(traj, ck + (size_t)c * n, n * sizeof(double));
        for (int64_t st = s0; st + 1 < s1; ++st)
            plain_step(nx, ny, nz, a, b, wf, s, qm, isfixed, traj + (size_t)(st - s0) * n,
                       traj + (size_t)(st - s0 + 1) * n);
        for (int64_t st = s1 - 1; st >= s0; --st) {
            const double *th = traj + (size_t)(st - s0) * n;   /* theta^st; lam = lambda^{st+1} */
            memset(pk, 0, (size_t)nz * n_labels * sizeof(double));
            memset(pw, 0, (size_t)nz * n_labels * sizeof(double));
#pragma omp parallel for schedule(static)
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x) {
                        size_t i = IDX(x, y, z);
                        Lambda[i] += lam[i];
                        if (!isfixed[i]) {
                            int l = labels[i];
                            const double *t = tab + (size_t)l * T_NCOL;
                            double t0 = th[i];
                            if (!wf) {
                                double lap = 0.0;
                                if (x > 0)      lap += th[IDX(x - 1, y, z)] - t0;
                                if (x < nx - 1) lap += th[IDX(x + 1, y, z)] - t0;
                                if (y > 0)      lap += th[IDX(x, y - 1, z)] - t0;
                                if (y < ny - 1) lap += th[IDX(x, y + 1, z)] - t0;
                                if (z > 0)      lap += th[IDX(x, y, z - 1)] - t0;
                                if (z < nz - 1) lap += th[IDX(x, y, z + 1)] - t0;
                                double da_dk = (1.0 / rhoc[i]) * dt / (h * h);
                                pk[(size_t)z * n_labels + l] += lam[i] * da_dk * lap;
                            } else {
                                /* d wf[d][i] / dK of the voxel's label (dwa) and of the
                                   neighbour's label (dwb) */
                                const int nbx[6] = {x - 1, x + 1, x, x, x, x}, nby[6] = {y, y, y - 1, y + 1, y, y};
                                const int nbz[6] = {z, z, z, z, z - 1, z + 1};
                                for (int d = 0; d < 6; ++d) {
                                    if (nbx[d] < 0 || nbx[d] >= nx || nby[d] < 0 || nby[d] >= ny || nbz[d] < 0 ||
                                        nbz[d] >= nz)
                                        continue;
                                    const size_t j = IDX(nbx[d], nby[d], nbz[d]);
                                    const double v = lam[i] * (th[j] - t0);
                                    pk[(size_t)z * n_labels + l] += dwa[(size_t)d * n + i] * v;
                                    pk[(size_t)z * n_labels + labels[j]] += dwb[(size_t)d * n + i] * v;
                                }
                            }
                            double db_dw = (t[T_RHOB] * t[T_CB] / rhoc[i]) * dt;
                            pw[(size_t)z * n_labels + l] -= lam[i] * db_dw * t0;
                        }
                        /* (A^T lam)_i = sum_j A[j][i] lam_j over j = i and its neighbours */
                        double acc = step_entry(nx, ny, nz, a, b, wf, isfixed, x, y, z, x, y, z) * lam[i];
                        if (x > 0)      acc += step_entry(nx, ny, nz, a, b, wf, isfixed, x - 1, y, z, x, y, z) * lam[IDX(x - 1, y, z)];
                        if (x < nx - 1) acc += step_entry(nx, ny, nz, a, b, wf, isfixed, x + 1, y, z, x, y, z) * lam[IDX(x + 1, y, z)];
                        if (y > 0)      acc += step_entry(nx, ny, nz, a, b, wf, isfixed, x, y - 1, z, x, y, z) * lam[IDX(x, y - 1, z)];
                        if (y < ny - 1) acc += step_entry(nx, ny, nz, a, b, wf, isfixed, x, y + 1, z, x, y, z) * lam[IDX(x, y + 1, z)];
                        if (z > 0)      acc += step_entry(nx, ny, nz, a, b, wf, isfixed, x, y, z - 1, x, y, z) * lam[IDX(x, y, z - 1)];
                        if (z < nz - 1) acc += step_entry(nx, ny, nz, a, b, wf, isfixed, x, y, z + 1, x, y, z) * lam[IDX(x, y, z + 1)];
                        lnew[i] = acc;
                    }
            for (int z = 0; z < nz; ++z)
                for (int l = 0; l < n_labels; ++l) {
                    g_k[l] += pk[(size_t)z * n_labels + l];
                    g_wb[l] += pw[(size_t)z * n_labels + l];
                }
            memcpy(lam, lnew, n * sizeof(double));
        }
    }
    free(ck); free(traj); free(lnew); free(pk); free(pw);
    return 0;
}

/*
 * grad[0] = sum_i Lambda_i ds_i/dP, grad[1..3] = sum_i Lambda_i ds_i/dtip with
 * s_i = P dt w_i / (h^3 W rho c_i), W = sum_free w, w_i = max(d_i, r0)^-4.
 * Every segment moves rigidly with the tip, so for d_i > r0
 * dw_i/dtip = 4 d_i^-6 (x_i - p*_i) with p*_i the closest needle point;
 * inside the clamp radius w_i does not depend on the tip.
 */
int or_source_grad(int nx, int ny, int nz, double h, double dt, const double *nd,
                   const double *rhoc, const uint8_t *isfixed, const double *Lambda, double *grad)
{
    segment seg[64];
    int ns = needle_segments(nd, seg);
    double r0 = nd[N_RCLAMP], P = nd[N_POWER];
    size_t n = (size_t)nx * ny * nz;
    double *w = (double *)malloc(n * sizeof(double));
    double *dw = (double *)malloc(3 * n * sizeof(double));
    if (!w || !dw) return 2;
    double W = 0.0, dW[3] = { 0.0, 0.0, 0.0 };
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = IDX(x, y, z);
                double p[3] = { x * h, y * h, z * h }, q[3];
                double d = needle_dist(p, seg, ns, q);
                double r = d > r0 ? d : r0;
                w[i] = 1.0 / (r * r * r * r);
                for (int c = 0; c < 3; ++c)
                    dw[3 * i + c] = d > r0 ? 4.0 * (p[c] - q[c]) / (d * d * d * d * d * d) : 0.0;
                if (!isfixed[i]) {
                    W += w[i];
                    for (int c = 0; c < 3; ++c) dW[c] += dw[3 * i + c];
                }
            }
    double gP = 0.0, gt[3] = { 0.0, 0.0, 0.0 };
    for (size_t i = 0; i < n; ++i) {
        if (isfixed[i]) continue;
        double f = P * dt / (h * h * h * rhoc[i]);
        gP += Lambda[i] * (f / P) * w[i] / W;
        for (int c = 0; c < 3; ++c)
            gt[c] += Lambda[i] * f * (dw[3 * i + c] / W - w[i] * dW[c] / (W * W));
    }
    grad[0] = gP;
    grad[1] = gt[0]; grad[2] = gt[1]; grad[3] = gt[2];
    free(w); free(dw);
    return 0;
}
