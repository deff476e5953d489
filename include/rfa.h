/*
 * rfa.h -- C ABI of the B300 (sm_103a) radio-frequency-ablation bioheat library.
 *
 * The library advances the simplified bioheat equation of Kath, Handels and
 * Mastmeyer (arXiv 1907.05709, Eq. 2675-eq1_Kath, discretised as Eq.
 * CUDAbioheat3d) on a 3D voxel grid by explicit Euler steps, with
 *   - a 7-point central-difference diffusion stencil (Eq. 2675-eq3),
 *   - the blood-perfusion sink toward arterial temperature T_a,
 *   - an RF heat source placed by the needle geometry (straight or umbrella),
 *   - voxels held at a fixed temperature (vessels, Eq. 2675-eq6 and the
 *     else-branch of Alg. 1),
 *   - a 60 C necrosis latch (Sec. "Introduction") and the Arrhenius damage
 *     integral of Eq. eq-tissState (FP32 increments summed in an FP32 carry
 *     that is folded into an FP64 integral every 256 steps; FP64 throughout
 *     for the FP64 state),
 *   - a hand-written discrete adjoint for gradients (the paper has none).
 *
 * Conventions shared by every call:
 *   - Units are SI (metres, seconds, watts, W/m/K, kg/m^3, J/kg/K) and
 *     temperatures at the ABI are degrees Celsius.
 *   - Voxel (i, j, k) has its centre at (i*h, j*h, k*h) metres; host volumes
 *     are dense [nz][ny][nx] arrays with x fastest.
 *   - The library owns all device memory of a grid.  Host pointers are borrowed
 *     for the duration of the call only; device pointers passed in stay owned
 *     by the caller.
 *   - Work is enqueued on the CUDA stream given at creation and runs
 *     asynchronously; a fault in asynchronous work is reported by the next call
 *     that synchronises (rfa_synchronize, rfa_get_*, rfa_necrosis_mask,
 *     rfa_backward).
 *   - No call throws across the ABI.  On failure a call returns a non-zero
 *     rfa_status and rfa_last_error() gives a message (thread-local).
 *   - A grid is not thread-safe; distinct grids may be used from distinct threads.
 */
#ifndef RFA_H
#define RFA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rfa_grid rfa_grid;    /* opaque, library-owned */
typedef struct rfa_batch rfa_batch;  /* opaque, library-owned */

typedef enum {
    RFA_OK = 0,
    RFA_E_INVALID = 1,      /* bad argument (null pointer, size, enum value) */
    RFA_E_OOM = 2,          /* device or host allocation failed */
    RFA_E_CUDA = 3,         /* a CUDA runtime/driver call failed */
    RFA_E_UNSTABLE = 4,     /* 1 - deg*a - b < 0 for some free voxel (scheme not positive) */
    RFA_E_STATE = 5,        /* call out of order (e.g. step before set_tissue) */
    RFA_E_NONFINITE = 6,    /* a step produced a non-finite temperature */
    RFA_E_TIMEOUT = 7,      /* a bounded device-side wait gave up */
    RFA_E_UNSUPPORTED = 8,  /* a valid request the library does not serve on this path */
    RFA_E_INTERNAL = 9      /* an internal consistency check failed (index checks of the
                               checked build, librfa_check.so) */
} rfa_status;

/* State precision: FP32, FP32 hi + FP32 lo compensated pair, FP64. */
enum { RFA_STATE_F32 = 0, RFA_STATE_F32C = 1, RFA_STATE_F64 = 2 };
/* Storage of the static per-voxel coefficients a = K dt/(rho c h^2) and
 * b = w_b rho_b c_b dt/(rho c): BF16 (rounded to nearest even), FP32, FP64. */
enum { RFA_PARAM_BF16 = 0, RFA_PARAM_F32 = 1, RFA_PARAM_F64 = 2 };
/* Outer faces: Dirichlet = the outer voxel layer is held at T_a; insulated =
 * zero flux (a neighbour outside the grid contributes nothing). */
enum { RFA_FACE_DIRICHLET = 0, RFA_FACE_INSULATED = 1 };
enum { RFA_NEEDLE_STRAIGHT = 0, RFA_NEEDLE_UMBRELLA = 1, RFA_NEEDLE_FIXED_TIP = 2 };
/* Field ids for rfa_get_field. */
enum { RFA_FIELD_THETA = 0, RFA_FIELD_A = 1, RFA_FIELD_B = 2, RFA_FIELD_S = 3,
       RFA_FIELD_LATCH = 4, RFA_FIELD_OMEGA = 5, RFA_FIELD_THETA_LO = 6 };

/* Per-label tissue parameters (Eq. 2675-eq1_Kath symbols), SI units.
 * Perfusion enters as beta = w_b * rho_b * c_b [W/m^3/K]; the paper's
 * per-volume blood flow (kg/m^3/s) corresponds to rho_b = 1.
 * fixed != 0 holds every voxel of the label at T_fixed_C (vessels). */
typedef struct {
    double k, rho, c, w_b, rho_b, c_b, Q_m;
    int fixed;
    double T_fixed_C;
} rfa_tissue;

/* Needle.  STRAIGHT: the active segment is [tip - active_len*axis, tip].
 * UMBRELLA: n_tines tines of length tine_len leave the tip at tine_polar_deg
 * off the axis, at azimuths 2*pi*j/n_tines measured from e1, where
 * (e1, e2, axis) is right-handed and e1 is the unit projection onto the plane
 * normal to the axis of +x if |axis_z| >= 0.9, else of +z (for axis +z:
 * e1 = +x, e2 = +y); tine_axial adds one tine along
 * the axis.  Source: q_i = P w_i / (h^3 sum_free w), w_i = max(d_i, r_clamp)^-4
 * with d_i the distance from the voxel centre to the nearest active segment
 * (the 1/r^4 fall-off of the resistive term sigma|grad V|^2 of Eq.
 * 2675-eq1_Linte around a point electrode).
 * FIXED_TIP: the paper's own set-up (Sec. "Evaluation Methods"): no RF source;
 * the needle tip is a voxel hemisphere held at T_tip_C (the paper uses 90 and
 * 60 C).  With (i, j, k) the voxel nearest tip_m and axis one of +-x, +-y, +-z,
 * the hemisphere is the voxels at offsets u, v in -2..2 across the axis and
 * w = 0, 1, 2 along it with 36 u^2 + 36 v^2 + 25 w^2 <= 225, i.e.
 * (u/2.5)^2 + (v/2.5)^2 + (w/3)^2 <= 1: 5 x 5 voxels across, 3 deep, the flat
 * face through tip_m and the dome toward +axis.  Its voxels get a = b = s = 0
 * and the temperature T_tip_C (those outside the grid are skipped); placing
 * another needle, or rfa_set_tissue, gives them back what their labels define
 * (free voxels keep their current temperature).  power_W, the lengths, the
 * tine fields and r_clamp_m are ignored; Q_m still heats the free voxels.
 * Runs with the centre conduction form only; rfa_backward returns
 * RFA_E_UNSUPPORTED while such a needle is placed.  T_tip_C is read for
 * FIXED_TIP only. */
typedef struct {
    int kind;
    double tip_m[3];
    double axis[3];
    double active_len_m;
    double tine_len_m;
    double tine_polar_deg;
    int n_tines;
    int tine_axial;
    double power_W;
    double r_clamp_m;
    double T_tip_C;
} rfa_needle;

/*
 * Create a grid of nx*ny*nz voxels of edge h_m, time step dt_s, ambient
 * (arterial) temperature T_a_C.  state_prec / param_prec / face_bc take the
 * enum values above.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream) on which all work of this grid is enqueued.  Allocates the device
 * fields; the state starts at T_a everywhere until rfa_set_tissue.
 * Errors: RFA_E_INVALID (size < 1, h or dt <= 0, bad enum), RFA_E_OOM, RFA_E_CUDA.
 */
rfa_status rfa_create_grid(int nx, int ny, int nz, double h_m, double dt_s, int state_prec,
                           int param_prec, int face_bc, double T_a_C, void *cuda_stream,
                           rfa_grid **out);

/* Free every device and host resource of the grid (synchronises its stream). */
rfa_status rfa_destroy_grid(rfa_grid *g);

/*
 * Tissue set-up (Sec. "Implementation": the label image becomes the start
 * temperature image).  labels: nx*ny*nz uint8, x fastest, every value
 * < n_labels, in host or device memory (the library detects which; a device
 * array stays owned by the caller).  table: host, n_labels entries
 * (1 <= n_labels <= 256).  Synchronous.
 * Builds the per-voxel coefficients on the device, resets the state to T_a
 * (T_fixed for fixed voxels), the latch and the damage integral to zero, the
 * step counter to zero and clears any recording for rfa_backward.
 * A needle placed earlier is placed again (the source depends on rho c).
 * Errors: RFA_E_INVALID (also a label >= n_labels, detected on the device),
 * RFA_E_UNSTABLE (1 - deg*a - b < 0 for a free label, deg = 2 per axis of
 * extent > 1, i.e. 6 for a 3D grid).
 */
rfa_status rfa_set_tissue(rfa_grid *g, const uint8_t *labels, const rfa_tissue *table,
                          int n_labels);

/*
 * Place the needle: builds the per-voxel source term
 * s_i = (q_i + Q_m,i) dt / (rho c)_i on the device (FP64 geometry and
 * normalisation sum, stored in the state precision).  Fixed voxels get no
 * source.  Does not reset the state (a FIXED_TIP needle sets its tip voxels'
 * temperature).  Errors: RFA_E_STATE (no tissue yet), RFA_E_INVALID (zero
 * axis, n_tines outside 0..16, negative lengths, r_clamp_m <= 0; FIXED_TIP: an
 * axis that is not a coordinate axis, a non-finite T_tip_C),
 * RFA_E_UNSUPPORTED (FIXED_TIP with the conservative conduction form).
 */
rfa_status rfa_place_needle(rfa_grid *g, const rfa_needle *needle);

/*
 * Damage model.  enable != 0 accumulates, after every step,
 * Omega_i += dt * A * exp(-Ea / (R * T_K)) with T_K = T + 273.15 (Eq.
 * eq-tissState's integral, right-rectangle rule).  FP32 and compensated FP32
 * states evaluate the increment in FP32 and add it to an FP32 carry, which is
 * folded into the FP64 integral with an error-free sum every 256 steps (the
 * carry keeps the fold's rounding error; at most 256 increments, about
 * 1.5e-5 relative, sit in FP32); the FP64 state adds every increment to the
 * FP64 integral with an error-free sum whose rounding error joins the carry.  T_thr_C is the necrosis-latch threshold used whether or not
 * the integral is enabled (default 60 C).  Defaults: disabled, A = 7.39e39,
 * Ea = 2.577e5, R = 8.31 (the paper's printed gas constant).
 */
rfa_status rfa_set_damage(rfa_grid *g, int enable, double A, double Ea, double R,
                          double T_thr_C);

/*
 * Advance nsteps explicit steps (Eq. CUDAbioheat3d, Jacobi double buffer as
 * in Alg. 2), updating the 60 C latch and, if enabled, the damage integral
 * after every step.  Asynchronous on the grid's stream.
 * record_for_backward != 0 stores sqrt(N) checkpoints so that rfa_backward can
 * differentiate the state after this call; recording is only valid when
 * every step since rfa_set_tissue was recorded.  Checkpoint buffers come from
 * a pool owned by the grid: a recording reuses the buffers of earlier ones and
 * allocates only when it needs more (they are freed with the grid).
 * Errors: RFA_E_STATE (no tissue or needle), RFA_E_INVALID (nsteps < 0),
 * RFA_E_OOM (a checkpoint buffer could not be allocated).
 */
rfa_status rfa_step(rfa_grid *g, int64_t nsteps, int record_for_backward);

/*
 * Copy the temperature T = theta + T_a in Celsius to dst (nx*ny*nz, x fastest)
 * as float (as_f64 = 0) or double (as_f64 = 1).  dst_is_device selects a
 * device (stream-ordered, asynchronous) or host (synchronous) destination;
 * dst is caller-owned.  Reports RFA_E_NONFINITE if a previous step produced a
 * non-finite value.  Errors: RFA_E_INVALID (null argument), RFA_E_OOM (host
 * staging), RFA_E_NONFINITE, RFA_E_TIMEOUT (a device wait that ran out).
 */
rfa_status rfa_get_temperature(rfa_grid *g, void *dst, int dst_is_device, int as_f64);

/* Diagnostic copy of one field (RFA_FIELD_*) to host doubles, nx*ny*nz (x
 * fastest, caller-owned), synchronous.  THETA is theta = T - T_a (hi + lo for
 * the compensated state); OMEGA is the FP64 integral plus its FP32 carry.
 * Errors: RFA_E_INVALID (null argument, unknown field), RFA_E_OOM. */
rfa_status rfa_get_field(rfa_grid *g, int field, double *dst_host);

/*
 * Necrosis: mask bit0 = thermal latch (T ever >= T_thr), bit1 = Arrhenius
 * (Omega >= 1).  mask_or_null: host nx*ny*nz bytes or NULL.  counts[2] and
 * volumes_m3[2] (h^3 * count) for the two criteria; smooth_volume_m3 =
 * h^3 * sum_i sigmoid((T_i - T_thr) / smooth_width_K) on the current state.
 * Any output pointer may be NULL (host, caller-owned).  Deterministic two-pass
 * reduction on device; synchronous.  Errors: RFA_E_INVALID (null grid,
 * smooth_width_K <= 0), RFA_E_OOM, RFA_E_NONFINITE, RFA_E_TIMEOUT.
 */
rfa_status rfa_necrosis_mask(rfa_grid *g, uint8_t *mask_or_null, int64_t *counts,
                             double *volumes_m3, double *smooth_volume_m3,
                             double smooth_width_K);

/*
 * Necrosis counts and smoothed volume without allocating memory.  The paper has
 * no counterpart; this exists for callers that may not allocate device memory
 * once running (a per-frame real-time loop where an allocation would stall the
 * device, or an application that pre-reserves its whole memory budget).
 * result_dev: caller-owned device buffer of 32 bytes, 8-byte aligned, receiving
 * {int64 count_thermal, int64 count_arrhenius, double smooth_volume_m3, 0.0},
 * the same quantities rfa_necrosis_mask reports.  Asynchronous on the grid's
 * stream; calls no allocator and does not synchronise.  Scratch is one fixed
 * 512 KiB device array inside the library (16384 records, one per 16384 padded
 * voxels), so grids above 268,435,456 padded voxels are rejected with
 * RFA_E_INVALID.  The first call with a device current looks up that array's
 * address; if the CUDA runtime loads device code lazily (the default), that
 * look-up loads the library's code on the device and may allocate and block
 * then, so make the first call during set-up, before any stream capture.
 * Calls share the array: each call rewrites every record it reads, but calls
 * that overlap on the GPU race.
 * Errors: RFA_E_INVALID (null grid or result_dev, result_dev not 8-byte
 * aligned, smooth_width_K <= 0, grid too large), RFA_E_CUDA (launch).
 */
rfa_status rfa_necrosis_reduce_noalloc(rfa_grid *g, double smooth_width_K, void *result_dev);

/*
 * Discrete adjoint of every recorded step (the paper has no adjoint).
 * dLdT_final_dev: device float array nx*ny*nz (x fastest), dL/dT of the final
 * state.  grads (host, 4 + 2*n_labels doubles) receives
 *   [dL/dP, dL/dtip_x, dL/dtip_y, dL/dtip_z, dL/dk[0..L-1], dL/dw_b[0..L-1]].
 * Recomputes the trajectory from the sqrt(N) checkpoints.  Synchronous.
 * Differentiates the centre and the conservative (RFA_COND_HARMONIC) forms.
 * Errors: RFA_E_INVALID (null argument), RFA_E_STATE (nothing recorded, or
 * unrecorded steps since set-up), RFA_E_UNSUPPORTED (FP64 state, the
 * potential-solve source, the tissue-state perfusion coupling, a FIXED_TIP
 * needle, more than 8 labels), RFA_E_OOM (workspace).
 */
rfa_status rfa_backward(rfa_grid *g, const float *dLdT_final_dev, double *grads);

/*
 * Serialise the evolving state (theta, lo, latch, Omega and its compensation,
 * step counter, steps since the last fold of the damage carry) to blob, so
 * that a resumed run ends in the same bits as an uninterrupted one.  With
 * blob == NULL, *n receives the required size.
 * rfa_set_state restores a blob made by a grid of the same shape/precision
 * (it needs rfa_set_tissue first; the restored state has no recorded history).
 * blob is host memory owned by the caller.  Errors: RFA_E_INVALID (null
 * argument, blob too small or from another grid), RFA_E_STATE (no tissue).
 */
rfa_status rfa_get_state(rfa_grid *g, void *blob, size_t *n);
rfa_status rfa_set_state(rfa_grid *g, const void *blob, size_t n);

/*
 * Temporal blocking: advance tb_depth steps per launch (1 = one step per
 * launch); tile_variant selects the xy tile of the blocked kernel (0: 64 x 12
 * output voxels per plane at depth 2, 64 x 10 at depth 3; 1: 64 x 28 at depth
 * 2).  All variants give bit-identical states.  The blocked kernel needs
 * compensated FP32 state, BF16 coefficients and Dirichlet faces; otherwise
 * rfa_set_schedule returns RFA_E_UNSUPPORTED and the autotuner keeps one step
 * per launch.
 * rfa_autotune times the candidates on a scratch copy of the grid's state and
 * keeps the fastest; cache_path (may be NULL) is a JSON file read and updated.
 * Errors: RFA_E_INVALID (null grid, tb_depth outside 1..8), RFA_E_UNSUPPORTED.
 */
rfa_status rfa_set_schedule(rfa_grid *g, int tb_depth, int tile_variant);
rfa_status rfa_get_schedule(rfa_grid *g, int *tb_depth, int *tile_variant);
rfa_status rfa_autotune(rfa_grid *g, const char *cache_path);

/*
 * Batched stepping of several grids in one persistent launch per call
 * (independent needle configurations on grids of uneven size; the paper runs
 * one configuration at a time).  Members must be F32C grids with BF16
 * coefficients, Dirichlet faces and tissue set, all on the same stream and with the same damage
 * setting; they stay owned by the caller and must outlive the batch.
 * rfa_batch_step advances every member by nsteps: whole blocks of tb_depth steps
 * in one cooperative persistent launch (replayed from a CUDA graph captured per
 * block count), the remainder as one-step launches.  States are bit-identical
 * to stepping each member alone.  Device-side faults of the batched launch are
 * reported by rfa_synchronize on the first member.
 * Errors: RFA_E_INVALID (null or repeated members, mixed streams or damage
 * settings, nsteps < 0), RFA_E_STATE (a member without tissue),
 * RFA_E_UNSUPPORTED (a member the blocked kernel cannot step), RFA_E_OOM,
 * RFA_E_CUDA (tensor maps, graph).
 */
rfa_status rfa_batch_create(rfa_grid *const *members, int n, rfa_batch **out);
rfa_status rfa_batch_step(rfa_batch *b, int64_t nsteps);
rfa_status rfa_batch_destroy(rfa_batch *b);
/* Pick the batch's steps-per-block depth and tile variant by timing every
 * candidate on snapshots of all members' states (restored afterwards);
 * cache_path (may be NULL) is a text file of cached choices. */
rfa_status rfa_batch_autotune(rfa_batch *b, const char *cache_path);
/* Current batch schedule; uses_graph = 1 if launches replay a CUDA graph
 * (when 0, rfa_last_error() gives the reason capture was not used). */
rfa_status rfa_batch_get_schedule(rfa_batch *b, int *tb_depth, int *tile_variant, int *uses_graph);

/*
 * Perfusion coupled to the tissue state (Linte's alpha(t) of Eq. 2675-eq1_Linte
 * and Eq. eq-tissState): with RFA_PERF_TISSUE_STATE the perfusion term of a
 * voxel is multiplied by alpha = 1 / max(1, Omega), Omega its Arrhenius
 * integral at the start of the step (the inverse integral, capped at 1 below
 * the damage threshold where it would be singular).  Needs the damage integral
 * on (rfa_set_damage), else Omega = 0 and alpha = 1.  Runs one step per launch
 * (no blocked or batched stepping); rfa_backward returns RFA_E_UNSUPPORTED
 * while it is on.  Errors: RFA_E_INVALID (unknown mode).
 */
enum { RFA_PERF_CONSTANT = 0, RFA_PERF_TISSUE_STATE = 1 };
rfa_status rfa_set_perfusion_coupling(rfa_grid *g, int mode);

/*
 * RF source from the electric potential (Linte's resistive term sigma |grad V|^2
 * of Eq. 2675-eq1_Linte) instead of the max(d, r0)^-4 weights of
 * rfa_place_needle: div(sigma grad V) = 0 with the electrode -- the voxels within
 * r_clamp_m of the needle's active segments -- at V = 1 and the outer faces at
 * V = 0 (ground), face conductances the harmonic mean of the voxels' sigma.
 * The heating q_i = sum_nb sigma_f (V_nb - V_i)^2 / (2 h^2) (each face's
 * dissipation split between its voxels) is scaled so that the free voxels
 * receive power_W, and written to the source field like rfa_place_needle.
 *   sigma_S_per_m : host, n_sigma = number of labels, electrical conductivity.
 *   max_iters, tol: preconditioned conjugate gradients (the preconditioner is
 *                   chosen by rfa_set_potential_preconditioner) stop when the
 *                   FP64 residual ||b - A x|| <= tol ||b|| or after max_iters
 *                   iterations.  The iterations run in FP32 with residual
 *                   replacement: whenever the FP32 residual has fallen 100x
 *                   (or stagnates), x and b - A x are formed in FP64 and the
 *                   iteration goes on (Jacobi: from its kept direction;
 *                   multigrid: restarted); if a cycle gains less than 2x,
 *                   Jacobi-preconditioned FP64 conjugate gradients continue
 *                   from the current x.
 *   iters_out, rel_residual_out (may be NULL): iterations used (FP32 and FP64
 *                   together), final FP64 ||b - A x||/||b|| (check it against
 *                   tol: reaching max_iters is not an error).
 * Synchronous.  rfa_set_tissue re-solves with the same settings.  rfa_backward
 * returns RFA_E_UNSUPPORTED while this source is in use.  A FIXED_TIP needle
 * is not accepted here; one placed earlier is removed first.
 * Errors: RFA_E_STATE (no tissue), RFA_E_INVALID (needle, sigma, n_sigma,
 * max_iters, tol), RFA_E_UNSUPPORTED (more than 16 labels), RFA_E_OOM,
 * RFA_E_NONFINITE (the iteration diverged).
 */
rfa_status rfa_place_needle_potential(rfa_grid *g, const rfa_needle *needle, const double *sigma_S_per_m,
                                      int n_sigma, int max_iters, double tol, int *iters_out,
                                      double *rel_residual_out);

/*
 * Preconditioner of the potential solve's FP32 iterations (the FP64 hand-over
 * always uses Jacobi).  Linear solves of this kind are the standard numerical
 * step behind the resistive source of Eq. 2675-eq1_Linte; the paper names no
 * solver.
 *   RFA_PRECOND_MULTIGRID (default): one symmetric V-cycle per iteration --
 *     coarse levels of 2x2x2 aggregated cells with Galerkin operators (7-point:
 *     summed face conductances), two damped-Jacobi sweeps (weight 0.8) before
 *     and after each coarse correction, and the exact inverse of the coarsest
 *     level (at most 128 cells, FP64 Cholesky on the host once per solve).
 *     Grids of at most 128 voxels, or a coarsest matrix that is not positive
 *     definite, fall back to Jacobi.  Device workspace: about 10/7 FP32 values
 *     per voxel for the levels plus two FP32 fine vectors.
 *   RFA_PRECOND_JACOBI: the inverse diagonal.
 * Takes effect at the next potential solve (rfa_place_needle_potential, or
 * rfa_set_tissue with that source in use).  Errors: RFA_E_INVALID (null grid,
 * unknown mode).
 */
enum { RFA_PRECOND_MULTIGRID = 0, RFA_PRECOND_JACOBI = 1 };
rfa_status rfa_set_potential_preconditioner(rfa_grid *g, int mode);

/*
 * Conduction form.  RFA_COND_CENTRE (default): K taken at the voxel,
 * K_i * sum of second differences -- the paper's Eq. 2675-eq2 with scalar K,
 * applied voxel-wise.  RFA_COND_HARMONIC: the conservative div(K grad T) of Eq.
 * 2675-eq1_Kath with the face conductance of two voxels the harmonic mean of
 * their K: theta'_i = theta_i + sum_nb w(l_i, l_nb) (theta_nb - theta_i) - ...,
 * w(l, m) = dt / (rho_l c_l h^2) * 2 K_l K_m / (K_l + K_m) (FP32 label-pair
 * table; FP64 with FP64 coefficients).  The two agree where K is uniform.  The
 * harmonic form runs one step per launch (no blocked or batched stepping), at
 * most 16 labels; rfa_backward differentiates it (dL/dK through both labels of
 * every face).  May be set before or after rfa_set_tissue; changing it after
 * recorded steps invalidates the recording.
 * Errors: RFA_E_INVALID (unknown mode), RFA_E_UNSUPPORTED (more than 16
 * labels, or the harmonic form while a FIXED_TIP needle is placed),
 * RFA_E_UNSTABLE (1 - deg * max_m w(l, m) - b_l < 0 for a free label).
 */
enum { RFA_COND_CENTRE = 0, RFA_COND_HARMONIC = 1 };
rfa_status rfa_set_conduction(rfa_grid *g, int mode);

/*
 * Breathing motion (Sec. "Consideration of Breathing Motion", Eq. breathing):
 * the simulation runs in the reference space; the temperature in the moving
 * space at one instant is T(x) = T_ref(x + u_inv(x)), with u_inv the inverse
 * motion vector field of that instant.  T_ref is sampled by trilinear
 * interpolation of the current state; sample positions outside the grid take
 * the nearest face value (a non-finite displacement samples the low face).
 *   u_inv_dev : device float, 3 dense planes [3][nz][ny][nx] (x, y, z
 *               components, metres), caller-owned, read only.
 *   dst_dev   : device, nx*ny*nz values in degrees C, x fastest; float, or
 *               double when as_f64 != 0.  Caller-owned.
 * FP64 states interpolate in FP64; FP32 states in FP32.  A compensated state
 * interpolates hi and lo separately and sums them with the ambient
 * temperature in FP64 for a double output; a float output interpolates hi
 * alone (|lo| <= ulp(hi)/2, below its resolution) and sums in FP32.
 * Asynchronous on the grid's stream; the state is not changed.
 * Errors: RFA_E_INVALID (null pointer), RFA_E_STATE (no tissue yet).
 */
rfa_status rfa_warp_temperature(rfa_grid *g, const float *u_inv_dev, void *dst_dev, int as_f64);

/* Diagnostic (the paper has no counterpart): launch a kernel that waits on a
 * device flag nothing sets, with the same bounded-spin pattern as the
 * library's real waits, and report how it ended.  Returns RFA_E_TIMEOUT when the
 * wait gave up after spin_limit_cycles (1..2^32) SM clocks; the context stays
 * usable.  Uses the current device and the legacy default stream; synchronous. */
rfa_status rfa_selftest_wait_timeout(long long spin_limit_cycles);

/* Diagnostic (the paper has no counterpart): spin limits, in SM clock cycles,
 * of the library's real device-side waits -- the TMA (mbarrier) waits of the
 * blocked and batched step kernels, and the batch's grid barrier between time
 * blocks -- for kernels launched afterwards on the current device, by any grid
 * of this process.  Defaults 2^32 each (about 2 s at 2 GHz).  A wait that runs
 * out records a timeout; the next synchronising call of the grid (of the
 * batch's first member) returns RFA_E_TIMEOUT and names the wait; the kernel's
 * outputs are then undefined until rfa_set_tissue or rfa_set_state.  A CTA that
 * gives up first waits, with the full limit, for its own copies in flight, so
 * short limits never leave a copy landing in released shared memory.  Limits
 * below 2^20 cycles poll without suspending the waiting thread.  Synchronous.
 * Errors: RFA_E_INVALID (a limit outside 1..2^32), RFA_E_CUDA. */
rfa_status rfa_set_wait_limits(long long mbarrier_cycles, long long grid_barrier_cycles);

/* Wait for the grid's stream and report deferred device errors. */
rfa_status rfa_synchronize(rfa_grid *g);

/* Number of steps taken since the last rfa_set_tissue. */
int64_t rfa_steps_done(const rfa_grid *g);

/* Message of the last failure on this thread ("" if none). */
const char *rfa_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RFA_H */
