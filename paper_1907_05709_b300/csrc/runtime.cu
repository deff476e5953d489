// runtime.cu -- the C ABI of include/rfa.h: grid objects, device memory,
// argument checks, status codes, stepping schedule and state (de)serialisation.
#include "rfa_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <new>

namespace rfa {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

rfa_status cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return RFA_E_CUDA;
}

static rfa_status fail(rfa_status st, const std::string &msg)
{
    set_error(msg);
    return st;
}

static void free_grid_memory(rfa_grid *g)
{
    void *ptrs[] = {g->th[0], g->th[1], g->lo[0], g->lo[1], g->ab, g->s, g->label, g->latch,
                    g->omega, g->omega_c, g->status, g->red, g->stage, g->d_table, g->d_wpair,
                    g->d_wadj};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (g->status_host) cudaFreeHost(g->status_host);
    g->th[0] = g->th[1] = g->lo[0] = g->lo[1] = nullptr;
}

// Host-side copy of the needle geometry definition: straight = the last
// active_len behind the tip; umbrella = tines from the tip at a polar angle off
// the axis, evenly spaced in azimuth from e1, optional axial tine.
static rfa_status build_geometry(const rfa_needle &nd, NeedleGeom &g)
{
    double ax[3] = {nd.axis[0], nd.axis[1], nd.axis[2]};
    double n = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
    if (!(n > 0.0) || !std::isfinite(n)) return fail(RFA_E_INVALID, "needle axis must be non-zero");
    for (double &v : ax) v /= n;
    g.nseg = 0;
    const double *tip = nd.tip_m;
    if (nd.kind == RFA_NEEDLE_FIXED_TIP) {
        // no RF source: the tip is a voxel hemisphere held at T_tip_C (painted after
        // the source is written)
        int nonzero = 0;
        for (double v : ax) nonzero += v != 0.0;
        if (nonzero != 1) return fail(RFA_E_INVALID, "a FIXED_TIP needle needs a coordinate axis (+-x, +-y or +-z)");
        if (!std::isfinite(nd.T_tip_C)) return fail(RFA_E_INVALID, "T_tip_C must be finite");
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(tip[d])) return fail(RFA_E_INVALID, "tip_m must be finite");
        g.r0 = 1.0;
        g.P = 0.0;
        return RFA_OK;
    }
    if (!(nd.r_clamp_m > 0.0)) return fail(RFA_E_INVALID, "needle r_clamp_m must be > 0");
    if (nd.power_W < 0.0) return fail(RFA_E_INVALID, "needle power_W must be >= 0");
    g.r0 = nd.r_clamp_m;
    g.P = nd.power_W;
    if (nd.kind == RFA_NEEDLE_STRAIGHT) {
        if (nd.active_len_m < 0.0) return fail(RFA_E_INVALID, "active_len_m must be >= 0");
        for (int d = 0; d < 3; ++d) {
            g.seg[0].p0[d] = tip[d] - nd.active_len_m * ax[d];
            g.seg[0].p1[d] = tip[d];
        }
        g.nseg = 1;
    } else if (nd.kind == RFA_NEEDLE_UMBRELLA) {
        if (nd.n_tines < 0 || nd.n_tines > kMaxSegments - 1 || nd.tine_len_m < 0.0 ||
            (nd.tine_axial != 0 && nd.tine_axial != 1) || nd.n_tines + nd.tine_axial < 1)
            return fail(RFA_E_INVALID, "umbrella needs 1..16 tines and tine_len_m >= 0");
        double ref[3] = {1.0, 0.0, 0.0};
        if (std::fabs(ax[2]) < 0.9) { ref[0] = 0.0; ref[2] = 1.0; }
        double pr = ref[0] * ax[0] + ref[1] * ax[1] + ref[2] * ax[2];
        double e1[3], e2[3];
        for (int d = 0; d < 3; ++d) e1[d] = ref[d] - pr * ax[d];
        double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        for (double &v : e1) v /= n1;
        e2[0] = ax[1] * e1[2] - ax[2] * e1[1];
        e2[1] = ax[2] * e1[0] - ax[0] * e1[2];
        e2[2] = ax[0] * e1[1] - ax[1] * e1[0];
        double pol = nd.tine_polar_deg * M_PI / 180.0;
        for (int j = 0; j < nd.n_tines; ++j) {
            double phi = 2.0 * M_PI * j / nd.n_tines;
            for (int d = 0; d < 3; ++d) {
                double dir = std::cos(pol) * ax[d] + std::sin(pol) * (std::cos(phi) * e1[d] + std::sin(phi) * e2[d]);
                g.seg[g.nseg].p0[d] = tip[d];
                g.seg[g.nseg].p1[d] = tip[d] + nd.tine_len_m * dir;
            }
            ++g.nseg;
        }
        if (nd.tine_axial) {
            for (int d = 0; d < 3; ++d) {
                g.seg[g.nseg].p0[d] = tip[d];
                g.seg[g.nseg].p1[d] = tip[d] + nd.tine_len_m * ax[d];
            }
            ++g.nseg;
        }
    } else {
        return fail(RFA_E_INVALID, "unknown needle kind");
    }
    for (int k = 0; k < g.nseg; ++k) {
        double uu = 0.0;
        for (int d = 0; d < 3; ++d) uu += (g.seg[k].p1[d] - g.seg[k].p0[d]) * (g.seg[k].p1[d] - g.seg[k].p0[d]);
        g.seg[k].inv_uu = uu > 0.0 ? 1.0 / uu : 0.0;
    }
    return RFA_OK;
}

// Give the voxels of a painted FIXED_TIP hemisphere back what their labels define.
static cudaError_t remove_tip(rfa_grid *g)
{
    if (!g->tip_on) return cudaSuccess;
    g->tip_on = false;
    return launch_tip(g, false, 0.0);
}

// Write the source of g->needle (g->geom built from it) and, for a FIXED_TIP
// needle, paint its hemisphere: the voxel nearest the tip, the axis and its sign.
static cudaError_t place_source(rfa_grid *g)
{
    cudaError_t e = remove_tip(g);
    if (e != cudaSuccess) return e;
    if ((e = launch_source(g)) != cudaSuccess) return e;
    if (g->needle.kind != RFA_NEEDLE_FIXED_TIP) return cudaSuccess;
    for (int d = 0; d < 3; ++d) {
        const double c = std::nearbyint(g->needle.tip_m[d] / g->h);
        g->tip_c[d] = (int)std::max(-1e6, std::min(1e6, c));  // far outside the grid: nothing is painted
        if (g->needle.axis[d] != 0.0) {
            g->tip_ax = d;
            g->tip_sgn = g->needle.axis[d] > 0.0 ? 1 : -1;
        }
    }
    g->tip_on = true;
    return launch_tip(g, true, g->needle.T_tip_C);
}

rfa_status read_status(rfa_grid *g)
{
    RFA_CUDA(cudaMemcpyAsync(g->status_host, g->status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                             g->stream));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    unsigned st = *g->status_host;
    if (st & kStatusNonfinite) return fail(RFA_E_NONFINITE, "a step produced a non-finite temperature");
    if (st & kStatusBadIndex)
        return fail(RFA_E_INTERNAL, "an index check of the checked build failed (an access outside its array)");
    if (st & kStatusGridTimeout) return fail(RFA_E_TIMEOUT, "a grid barrier wait of a batched launch exceeded its limit");
    if (st & kStatusTimeout) return fail(RFA_E_TIMEOUT, "a TMA (mbarrier) wait exceeded its limit");
    return RFA_OK;
}

rfa_status advance(rfa_grid *g, int64_t nsteps, bool damage, bool latch)
{
    int64_t left = nsteps;
    while (left > 0) {
        int m = g->sched.tb_depth;
        cudaError_t e;
        const bool use_tb = m > 1 && left >= m && latch && tb_supported(g, m, g->sched.tile_variant);
        const int n = use_tb ? m : 1;
        // fold the FP32 damage carry once it holds kCarrySteps steps
        const bool fold = damage && g->carry_steps + n >= kCarrySteps;
        if (use_tb) {
            e = launch_step_tb(g, m, g->sched.tile_variant, g->th[g->cur], g->lo[g->cur],
                               g->th[g->cur ^ 1], g->lo[g->cur ^ 1], damage, fold);
        } else if (g->cond == RFA_COND_HARMONIC || g->alpha_perf) {
            e = launch_step_model(g, g->th[g->cur], g->lo[g->cur], g->th[g->cur ^ 1], g->lo[g->cur ^ 1], damage,
                                  latch, fold);
        } else {
            e = launch_step_plain(g, g->th[g->cur], g->lo[g->cur], g->th[g->cur ^ 1],
                                  g->lo[g->cur ^ 1], damage, latch, fold);
        }
        left -= n;
        if (damage) g->carry_steps = fold ? 0 : g->carry_steps + n;
        if (e != cudaSuccess) return cuda_fail(e, "step launch");
        g->cur ^= 1;
    }
    return RFA_OK;
}

}  // namespace rfa

using namespace rfa;

extern "C" {

const char *rfa_last_error(void) { return g_err.c_str(); }

rfa_status rfa_create_grid(int nx, int ny, int nz, double h_m, double dt_s, int state_prec,
                           int param_prec, int face_bc, double T_a_C, void *cuda_stream,
                           rfa_grid **out)
{
    if (!out) return fail(RFA_E_INVALID, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || nx > (1 << 16) || ny > (1 << 16) || nz > (1 << 16))
        return fail(RFA_E_INVALID, "grid extents must be in 1..65536");
    if (!(h_m > 0.0) || !(dt_s > 0.0) || !std::isfinite(h_m) || !std::isfinite(dt_s))
        return fail(RFA_E_INVALID, "h and dt must be positive and finite");
    if (state_prec < 0 || state_prec > 2 || param_prec < 0 || param_prec > 2 || face_bc < 0 ||
        face_bc > 1)
        return fail(RFA_E_INVALID, "bad precision or face enum");
    rfa_grid *g = new (std::nothrow) rfa_grid();
    if (!g) return fail(RFA_E_OOM, "host allocation failed");
    g->nx = nx; g->ny = ny; g->nz = nz;
    g->pitch = (nx + 3) & ~3;
    g->plane = (size_t)g->pitch * ny;
    g->nvp = g->plane * nz;
    g->h = h_m; g->dt = dt_s; g->T_a = T_a_C;
    g->sp = state_prec; g->pp = param_prec; g->face = face_bc;
    g->stream = (cudaStream_t)cuda_stream;
    size_t nvp = g->nvp;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc(&g->th[0], nvp * g->state_elem());
    alloc(&g->th[1], nvp * g->state_elem());
    if (state_prec == RFA_STATE_F32C) {
        alloc(&g->lo[0], nvp * 4);
        alloc(&g->lo[1], nvp * 4);
    }
    alloc(&g->ab, nvp * g->ab_elem());
    alloc(&g->s, nvp * g->state_elem());
    alloc((void **)&g->label, nvp);
    alloc((void **)&g->latch, nvp);
    alloc((void **)&g->omega, nvp * 8);
    alloc((void **)&g->omega_c, nvp * 4);
    alloc((void **)&g->status, 256);
    alloc(&g->red, kReduceBlocks * 32 + 256);
    alloc((void **)&g->d_table, 256 * sizeof(LabelCoef));
    alloc(&g->d_wpair, kCondLabels * kCondLabels * 8);
    alloc((void **)&g->d_wadj, 3 * kCondLabels * kCondLabels * 4);
    alloc(&g->stage, nvp * 8);  // labels in, source weights, host copies
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->status_host, 256);
    if (e != cudaSuccess) {
        rfa_status st = (e == cudaErrorMemoryAllocation) ? fail(RFA_E_OOM, "device allocation failed")
                                                          : cuda_fail(e, "cudaMalloc");
        cudaGetLastError();
        free_grid_memory(g);
        delete g;
        return st;
    }
    cudaStream_t s = g->stream;
    void *zero_ptrs[] = {g->th[0], g->th[1], g->lo[0], g->lo[1], g->ab, g->s, g->label,
                         g->latch, g->omega, g->omega_c, g->status};
    size_t zero_sizes[] = {nvp * g->state_elem(), nvp * g->state_elem(), nvp * 4, nvp * 4,
                           nvp * g->ab_elem(), nvp * g->state_elem(), nvp, nvp, nvp * 8, nvp * 4, 256};
    for (int k = 0; k < 11; ++k)
        if (zero_ptrs[k] && e == cudaSuccess) e = cudaMemsetAsync(zero_ptrs[k], 0, zero_sizes[k], s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        rfa_status st = cuda_fail(e, "grid initialisation");
        free_grid_memory(g);
        delete g;
        return st;
    }
    *out = g;
    return RFA_OK;
}

rfa_status rfa_destroy_grid(rfa_grid *g)
{
    if (!g) return RFA_OK;
    cudaStreamSynchronize(g->stream);
    record_free(g);
    tb_forget_maps(g);
    free_grid_memory(g);
    delete g;
    return RFA_OK;
}

rfa_status rfa_set_tissue(rfa_grid *g, const uint8_t *labels, const rfa_tissue *table, int n_labels)
{
    if (!g || !labels || !table) return fail(RFA_E_INVALID, "null argument");
    if (n_labels < 1 || n_labels > 256) return fail(RFA_E_INVALID, "n_labels must be in 1..256");
    size_t n = g->nvox();
    cudaPointerAttributes pa{};
    bool dev_labels = cudaPointerGetAttributes(&pa, labels) == cudaSuccess &&
                      (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    std::vector<LabelCoef> tab(256);
    for (int l = 0; l < n_labels; ++l) {
        const rfa_tissue &t = table[l];
        if (!(t.rho > 0.0) || !(t.c > 0.0) || t.k < 0.0 || t.w_b < 0.0 || t.rho_b < 0.0 ||
            t.c_b < 0.0 || !std::isfinite(t.Q_m) || !std::isfinite(t.T_fixed_C))
            return fail(RFA_E_INVALID, "tissue parameters must be finite, rho and c > 0, others >= 0");
        LabelCoef &c = tab[l];
        c.k = t.k; c.rho = t.rho; c.c = t.c; c.w_b = t.w_b; c.rho_b = t.rho_b; c.c_b = t.c_b;
        c.Q_m = t.Q_m; c.T_fixed = t.T_fixed_C; c.fixed = t.fixed ? 1 : 0;
        if (!c.fixed) {
            // positivity of the explicit scheme: 1 - deg*a - b >= 0 with the stored
            // coefficients, deg = the largest neighbour count (2 per axis of extent > 1)
            double a = round_coef(coef_a(c, g->dt, g->h), g->pp);
            double b = round_coef(coef_b(c, g->dt), g->pp);
            double deg = 2.0 * ((g->nx > 1) + (g->ny > 1) + (g->nz > 1));
            if (1.0 - deg * a - b < 0.0) {
                char buf[192];
                std::snprintf(buf, sizeof buf, "label %d: 1 - %g a - b = %.6g < 0 (a = %.6g, b = %.6g); reduce dt", l, deg, 1.0 - deg * a - b, a, b);
                return fail(RFA_E_UNSTABLE, buf);
            }
        }
    }
    if (g->cond == RFA_COND_HARMONIC) {
        const rfa_status st = cond_build_tables(g, table, n_labels);
        if (st != RFA_OK) return st;
    }
    RFA_CUDA(cudaMemcpyAsync(g->d_table, tab.data(), 256 * sizeof(LabelCoef), cudaMemcpyHostToDevice, g->stream));
    RFA_CUDA(cudaMemcpyAsync(g->stage, labels, n, dev_labels ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream));
    RFA_CUDA(cudaMemsetAsync(g->status, 0, 256, g->stream));
    RFA_CUDA(launch_setup(g, (const uint8_t *)g->stage, n_labels));
    g->tip_on = false;  // the set-up rewrote every voxel
    g->table.assign(table, table + n_labels);
    g->n_labels = n_labels;
    g->cur = 0;
    g->steps = 0;
    g->carry_steps = 0;
    g->have_tissue = true;
    record_reset(g);
    RFA_CUDA(cudaMemcpyAsync(g->status_host, g->status, sizeof(unsigned), cudaMemcpyDeviceToHost, g->stream));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    if (*g->status_host & kStatusBadLabel) {
        g->have_tissue = false;
        return fail(RFA_E_INVALID, "label value >= n_labels");
    }
    if (g->have_needle) {
        if (g->src_mode == 1) {
            if ((int)g->sigma.size() != n_labels) {
                g->have_needle = false;
                return fail(RFA_E_STATE, "the potential-solve source needs one sigma per label: place the needle again");
            }
            const rfa_status st = potential_place(g);
            if (st != RFA_OK) return st;
        } else {
            RFA_CUDA(place_source(g));
            RFA_CUDA(cudaStreamSynchronize(g->stream));
        }
    }
    return RFA_OK;
}

rfa_status rfa_place_needle(rfa_grid *g, const rfa_needle *needle)
{
    if (!g || !needle) return fail(RFA_E_INVALID, "null argument");
    if (!g->have_tissue) return fail(RFA_E_STATE, "rfa_set_tissue must come first");
    if (needle->kind == RFA_NEEDLE_FIXED_TIP && g->cond != RFA_COND_CENTRE)
        return fail(RFA_E_UNSUPPORTED, "a FIXED_TIP needle runs with the centre conduction form only");
    NeedleGeom geom{};
    rfa_status st = build_geometry(*needle, geom);
    if (st != RFA_OK) return st;
    g->geom = geom;
    g->needle = *needle;
    g->src_mode = 0;
    RFA_CUDA(place_source(g));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    g->have_needle = true;
    if (g->steps > 0) g->rec.valid = false;  // the recorded trajectory used another source
    return RFA_OK;
}

rfa_status rfa_place_needle_potential(rfa_grid *g, const rfa_needle *needle, const double *sigma_S_per_m,
                                      int n_sigma, int max_iters, double tol, int *iters_out,
                                      double *rel_residual_out)
{
    if (!g || !needle || !sigma_S_per_m) return fail(RFA_E_INVALID, "null argument");
    if (!g->have_tissue) return fail(RFA_E_STATE, "rfa_set_tissue must come first");
    if (n_sigma != g->n_labels) return fail(RFA_E_INVALID, "n_sigma must equal the number of labels");
    if (max_iters < 1 || !(tol > 0.0)) return fail(RFA_E_INVALID, "max_iters >= 1 and tol > 0 are needed");
    for (int l = 0; l < n_sigma; ++l)
        if (!(sigma_S_per_m[l] >= 0.0) || !std::isfinite(sigma_S_per_m[l]))
            return fail(RFA_E_INVALID, "sigma must be finite and >= 0");
    if (needle->kind == RFA_NEEDLE_FIXED_TIP)
        return fail(RFA_E_INVALID, "the potential-solve source needs a straight or umbrella needle");
    NeedleGeom geom{};
    rfa_status st = build_geometry(*needle, geom);
    if (st != RFA_OK) return st;
    RFA_CUDA(remove_tip(g));
    g->geom = geom;
    g->needle = *needle;
    g->sigma.assign(sigma_S_per_m, sigma_S_per_m + n_sigma);
    g->pot_max_iters = max_iters;
    g->pot_tol = tol;
    g->src_mode = 1;
    st = potential_place(g);
    if (st != RFA_OK) return st;
    g->have_needle = true;
    if (g->steps > 0) g->rec.valid = false;
    if (iters_out) *iters_out = g->pot_iters;
    if (rel_residual_out) *rel_residual_out = g->pot_res;
    return RFA_OK;
}

rfa_status rfa_set_potential_preconditioner(rfa_grid *g, int mode)
{
    if (!g) return fail(RFA_E_INVALID, "null grid");
    if (mode != RFA_PRECOND_MULTIGRID && mode != RFA_PRECOND_JACOBI)
        return fail(RFA_E_INVALID, "unknown preconditioner");
    g->pot_precond = mode;
    return RFA_OK;
}

rfa_status rfa_set_damage(rfa_grid *g, int enable, double A, double Ea, double R, double T_thr_C)
{
    if (!g) return fail(RFA_E_INVALID, "null grid");
    if (enable && (!(A > 0.0) || !(Ea >= 0.0) || !(R > 0.0)))
        return fail(RFA_E_INVALID, "Arrhenius constants must be positive");
    if (!std::isfinite(T_thr_C)) return fail(RFA_E_INVALID, "threshold must be finite");
    g->dmg = enable ? 1 : 0;
    if (enable) { g->A = A; g->Ea = Ea; g->R = R; }
    g->T_thr = T_thr_C;
    return RFA_OK;
}

rfa_status rfa_step(rfa_grid *g, int64_t nsteps, int record_for_backward)
{
    if (!g) return fail(RFA_E_INVALID, "null grid");
    if (nsteps < 0) return fail(RFA_E_INVALID, "nsteps must be >= 0");
    if (!g->have_tissue) return fail(RFA_E_STATE, "rfa_set_tissue must come first");
    if (nsteps == 0) return RFA_OK;
    bool dmg = g->dmg != 0;
    if (record_for_backward) {
        if (g->steps == 0) {
            rfa_status st = record_begin(g, nsteps);
            if (st != RFA_OK) return st;
        }
        if (!g->rec.valid) {
            rfa_status st = advance(g, nsteps, dmg, true);
            g->steps += nsteps;
            return st;
        }
        int64_t left = nsteps;
        while (left > 0) {
            int64_t k = g->steps;
            if (k % g->rec.seg == 0) {
                rfa_status st = record_checkpoint(g, k);
                if (st != RFA_OK) return st;
            }
            int64_t chunk = g->rec.seg - k % g->rec.seg;
            if (chunk > left) chunk = left;
            rfa_status st = advance(g, chunk, dmg, true);
            if (st != RFA_OK) return st;
            g->steps += chunk;
            g->rec.nsteps += chunk;
            left -= chunk;
        }
        return RFA_OK;
    }
    g->rec.valid = false;
    rfa_status st = advance(g, nsteps, dmg, true);
    g->steps += nsteps;
    return st;
}

rfa_status rfa_synchronize(rfa_grid *g)
{
    if (!g) return fail(RFA_E_INVALID, "null grid");
    RFA_CUDA(cudaGetLastError());
    return read_status(g);
}

int64_t rfa_steps_done(const rfa_grid *g) { return g ? g->steps : -1; }

rfa_status rfa_get_temperature(rfa_grid *g, void *dst, int dst_is_device, int as_f64)
{
    if (!g || !dst) return fail(RFA_E_INVALID, "null argument");
    if (dst_is_device) {
        RFA_CUDA(launch_to_temperature(g, dst, as_f64));
        return RFA_OK;
    }
    if (!g->stage && cudaMalloc(&g->stage, g->nvox() * 8) != cudaSuccess) {
        cudaGetLastError();
        return fail(RFA_E_OOM, "staging allocation failed");
    }
    RFA_CUDA(launch_to_temperature(g, g->stage, as_f64));
    RFA_CUDA(cudaMemcpyAsync(dst, g->stage, g->nvox() * (as_f64 ? 8 : 4), cudaMemcpyDeviceToHost, g->stream));
    return read_status(g);
}

rfa_status rfa_get_field(rfa_grid *g, int field, double *dst_host)
{
    if (!g || !dst_host) return fail(RFA_E_INVALID, "null argument");
    if (field < 0 || field > RFA_FIELD_THETA_LO) return fail(RFA_E_INVALID, "unknown field");
    if (!g->stage && cudaMalloc(&g->stage, g->nvox() * 8) != cudaSuccess) {
        cudaGetLastError();
        return fail(RFA_E_OOM, "staging allocation failed");
    }
    RFA_CUDA(launch_get_field(g, field, (double *)g->stage));
    RFA_CUDA(cudaMemcpyAsync(dst_host, g->stage, g->nvox() * 8, cudaMemcpyDeviceToHost, g->stream));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    return RFA_OK;
}

rfa_status rfa_necrosis_mask(rfa_grid *g, uint8_t *mask_or_null, int64_t *counts,
                             double *volumes_m3, double *smooth_volume_m3, double smooth_width_K)
{
    if (!g) return fail(RFA_E_INVALID, "null grid");
    if (!(smooth_width_K > 0.0)) return fail(RFA_E_INVALID, "smooth_width_K must be > 0");
    if (!g->stage && cudaMalloc(&g->stage, g->nvox() * 8) != cudaSuccess) {
        cudaGetLastError();
        return fail(RFA_E_OOM, "staging allocation failed");
    }
    void *result = (char *)g->red + kReduceBlocks * 32;
    RFA_CUDA(launch_necrosis(g, mask_or_null ? (uint8_t *)g->stage : nullptr, smooth_width_K, result));
    struct { unsigned long long c0, c1; double sm, pad; } r;
    RFA_CUDA(cudaMemcpyAsync(g->status_host + 16, result, sizeof r, cudaMemcpyDeviceToHost, g->stream));
    if (mask_or_null)
        RFA_CUDA(cudaMemcpyAsync(mask_or_null, g->stage, g->nvox(), cudaMemcpyDeviceToHost, g->stream));
    rfa_status st = read_status(g);
    std::memcpy(&r, g->status_host + 16, sizeof r);
    double h3 = g->h * g->h * g->h;
    if (counts) { counts[0] = (int64_t)r.c0; counts[1] = (int64_t)r.c1; }
    if (volumes_m3) { volumes_m3[0] = h3 * (double)r.c0; volumes_m3[1] = h3 * (double)r.c1; }
    if (smooth_volume_m3) *smooth_volume_m3 = h3 * r.sm;
    return st;
}

// blob: header | theta | lo | latch | omega | omega_c.  The header keeps the
// steps since the damage carry was last folded, so a resumed run folds at the
// same steps as an uninterrupted one and ends in the same bits.
struct StateHeader {
    uint64_t magic;
    int32_t nx, ny, nz, sp;
    int64_t steps;
    int64_t carry_steps;
};
static const uint64_t kStateMagic = 0x3230353730394646ull;  // format 2 (with carry_steps)

rfa_status rfa_get_state(rfa_grid *g, void *blob, size_t *n)
{
    if (!g || !n) return fail(RFA_E_INVALID, "null argument");
    size_t nvp = g->nvp;
    size_t need = sizeof(StateHeader) + nvp * g->state_elem() +
                  (g->sp == RFA_STATE_F32C ? nvp * 4 : 0) + nvp + nvp * 8 + nvp * 4;
    if (!blob) { *n = need; return RFA_OK; }
    if (*n < need) return fail(RFA_E_INVALID, "blob too small");
    StateHeader hd{kStateMagic, g->nx, g->ny, g->nz, g->sp, g->steps, (int64_t)g->carry_steps};
    char *p = (char *)blob;
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    RFA_CUDA(cudaMemcpyAsync(p, g->th[g->cur], nvp * g->state_elem(), cudaMemcpyDeviceToHost, g->stream));
    p += nvp * g->state_elem();
    if (g->sp == RFA_STATE_F32C) {
        RFA_CUDA(cudaMemcpyAsync(p, g->lo[g->cur], nvp * 4, cudaMemcpyDeviceToHost, g->stream));
        p += nvp * 4;
    }
    RFA_CUDA(cudaMemcpyAsync(p, g->latch, nvp, cudaMemcpyDeviceToHost, g->stream));
    p += nvp;
    RFA_CUDA(cudaMemcpyAsync(p, g->omega, nvp * 8, cudaMemcpyDeviceToHost, g->stream));
    p += nvp * 8;
    RFA_CUDA(cudaMemcpyAsync(p, g->omega_c, nvp * 4, cudaMemcpyDeviceToHost, g->stream));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    *n = need;
    return RFA_OK;
}

rfa_status rfa_set_state(rfa_grid *g, const void *blob, size_t n)
{
    if (!g || !blob) return fail(RFA_E_INVALID, "null argument");
    if (!g->have_tissue) return fail(RFA_E_STATE, "rfa_set_tissue must come first");
    size_t nvp = g->nvp;
    size_t need = sizeof(StateHeader) + nvp * g->state_elem() +
                  (g->sp == RFA_STATE_F32C ? nvp * 4 : 0) + nvp + nvp * 8 + nvp * 4;
    StateHeader hd;
    if (n < need) return fail(RFA_E_INVALID, "blob too small");
    std::memcpy(&hd, blob, sizeof hd);
    if (hd.magic != kStateMagic || hd.nx != g->nx || hd.ny != g->ny || hd.nz != g->nz || hd.sp != g->sp)
        return fail(RFA_E_INVALID, "blob does not match this grid");
    // a corrupt counter would delay the FP64 fold of the FP32 damage carry indefinitely
    if (hd.steps < 0 || hd.carry_steps < 0 || hd.carry_steps >= kCarrySteps || hd.carry_steps > hd.steps)
        return fail(RFA_E_INVALID, "blob step counters out of range");
    const char *p = (const char *)blob + sizeof hd;
    RFA_CUDA(cudaMemcpyAsync(g->th[g->cur], p, nvp * g->state_elem(), cudaMemcpyHostToDevice, g->stream));
    p += nvp * g->state_elem();
    if (g->sp == RFA_STATE_F32C) {
        RFA_CUDA(cudaMemcpyAsync(g->lo[g->cur], p, nvp * 4, cudaMemcpyHostToDevice, g->stream));
        p += nvp * 4;
    }
    RFA_CUDA(cudaMemcpyAsync(g->latch, p, nvp, cudaMemcpyHostToDevice, g->stream));
    p += nvp;
    RFA_CUDA(cudaMemcpyAsync(g->omega, p, nvp * 8, cudaMemcpyHostToDevice, g->stream));
    p += nvp * 8;
    RFA_CUDA(cudaMemcpyAsync(g->omega_c, p, nvp * 4, cudaMemcpyHostToDevice, g->stream));
    RFA_CUDA(cudaStreamSynchronize(g->stream));
    g->steps = hd.steps;
    g->carry_steps = hd.carry_steps;
    record_reset(g);  // a restored state has no recorded history
    return RFA_OK;
}

rfa_status rfa_set_schedule(rfa_grid *g, int tb_depth, int tile_variant)
{
    if (!g) return fail(RFA_E_INVALID, "null grid");
    if (tb_depth < 1 || tb_depth > 8) return fail(RFA_E_INVALID, "tb_depth must be in 1..8");
    if (tb_depth > 1 && !tb_supported(g, tb_depth, tile_variant))
        return fail(RFA_E_UNSUPPORTED, "no blocked kernel for this grid/precision/depth/tile");
    g->sched.tb_depth = tb_depth;
    g->sched.tile_variant = tile_variant;
    return RFA_OK;
}

rfa_status rfa_get_schedule(rfa_grid *g, int *tb_depth, int *tile_variant)
{
    if (!g) return fail(RFA_E_INVALID, "null grid");
    if (tb_depth) *tb_depth = g->sched.tb_depth;
    if (tile_variant) *tile_variant = g->sched.tile_variant;
    return RFA_OK;
}

}  // extern "C"
