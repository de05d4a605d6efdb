/*
 * cdi.h -- C ABI of the GB300 (sm_103a) conservative diffuse interface
 * (CDI) phase-field library.
 *
 * The library advances the phase field phi of Eq. 1 of Mirjalili, Ivey &
 * Mani, "A conservative diffuse interface method for two-phase flows with
 * provable boundedness properties" (arXiv 1803.01262):
 *
 *     d phi/dt + div(u phi) = div[ gamma ( eps grad phi - phi (1-phi) grad phi/|grad phi| ) ]
 *
 * discretised as in Section 2.2 on a periodic, uniform, isotropic staggered
 * grid: phi at cell centres, velocity components on faces, second-order
 * central differences, explicit Euler in time (Eq. 11 in 1D, Eq. 18-22 in
 * coefficient form).  Per face between cells L and R along axis d:
 *
 *     F = (vs * u_f) (phi_L + phi_R)/2 - gamma eps (phi_R - phi_L)/dx
 *         + gamma (s_L + s_R)/2,     s = phi (1 - phi) n_d,
 *     n = g/|g|, g_d = phi_{c+e_d} - phi_{c-e_d}   (n = 0 where g = 0),
 *     phi'_c = phi_c - (dt/dx) sum_d (F_{c+1/2 e_d} - F_{c-1/2 e_d}),
 *
 * where vs is the caller's velocity scale (the time factor of a
 * time-periodic field, e.g. cos(pi t/T) in Eq. 33).  The kernels evaluate
 * the normal as g * rsqrt(|g|^2 + tau), tau the smallest normal number of
 * the dtype (FLT_MIN, DBL_MIN): finite at g = 0, where s = 0 exactly, and
 * the unit normal wherever |g|^2 is far above tau (the paper divides by
 * |grad phi| and is silent where it vanishes).
 *
 * Conventions shared by every call:
 *  - Arrays are dense [nz][ny][nx] (x fastest), element type float
 *    (CDI_F32) or double (CDI_F64) as fixed at grid creation.
 *  - u[k][j][i] is the x-velocity on the face (i+1/2, j, k) (right face of
 *    cell i); v on (i, j+1/2, k); w on (i, j, k+1/2).  All axes periodic.
 *  - Device pointers are owned by the caller and borrowed for the duration
 *    of the work enqueued by the call.  They must be aligned to 16 bytes.
 *  - The library owns only small device scratch (per-block reduction
 *    partials, a statistics record) allocated in cdi_create_grid.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every kernel is enqueued on it; nothing synchronises unless
 *    the call says so.
 *  - A grid (with its scratch) must be used by one stream at a time.
 *  - Every call returns CDI_OK (0) or a negative CDI_ERR_* code and records
 *    a message readable with cdi_last_error_string() (thread-local).  No
 *    call aborts or throws.
 */
#ifndef CDI_H
#define CDI_H

#ifdef __cplusplus
extern "C" {
#endif

#define CDI_VERSION 1

#if defined(__GNUC__)
#define CDI_API __attribute__((visibility("default")))
#else
#define CDI_API
#endif

enum {
    CDI_OK = 0,
    CDI_ERR_ARG = -1,        /* bad pointer, size, or parameter value      */
    CDI_ERR_DIM = -2,        /* grid extent out of range                   */
    CDI_ERR_CUDA = -3,       /* a CUDA runtime call failed                 */
    CDI_ERR_CONDITION = -4,  /* Eq. 17/24 or A <= 1/(2 D_f) not satisfied */
    CDI_ERR_NAN = -5,        /* non-finite value detected in a reduction   */
    CDI_ERR_TIMEOUT = -6,    /* a bounded device-side wait gave up         */
    CDI_ERR_STATE = -7,      /* call out of order (e.g. no velocity set)   */
    CDI_ERR_BOUNDS = -8      /* checked build: a kernel index was out of range */
};

enum { CDI_F32 = 0, CDI_F64 = 1 };

/* Time schemes for cdi_max_dt (Eq. 25-28). */
enum { CDI_EULER = 0, CDI_RK2 = 1, CDI_RK3 = 2, CDI_RK4 = 3 };

/* Flags of cdi_step / cdi_run. */
#define CDI_CHECK_CONDITION 1  /* refuse (CDI_ERR_CONDITION) unless Eq. 24 and A <= 1/(2 D_f) hold */

typedef struct cdi_grid cdi_grid;

/*
 * Mass and bounds of a phase field (conservation, Section 2.2.1 and
 * Fig. 5c; boundedness criterion of Section 3.2).
 *   mass      = dV * sum(phi), dV = dx^D_f, D_f = number of axes with extent > 1
 *   n_strict  = #(phi < 0 or phi > 1)
 *   n_tol     = #(phi < -tol or phi > 1 + tol), tol = machine epsilon of the dtype
 * The *_run fields accumulate over every fused step since the last
 * cdi_reset_run_stats (min/max over steps, summed violation counts).
 * Sums are accumulated in double on the device in a fixed order, so a
 * result is reproducible run to run.
 */
typedef struct cdi_stats {
    double mass;
    double sum;
    double min;
    double max;
    long long n_strict;
    long long n_tol;
    double min_run;
    double max_run;
    long long n_strict_run;
    long long n_tol_run;
    long long steps_run;
} cdi_stats;

/* Create a periodic nx x ny x nz grid of spacing dx (> 0) holding phi of
 * type dtype.  ny = nz = 1 (nz = 1) gives the 1D (2D) scheme exactly.
 * Extents must be >= 1 with nx*ny < 2^31 and nx*ny*nz < 2^36.  Allocates the
 * reduction scratch (device memory) on the current device. */
CDI_API int cdi_create_grid(cdi_grid **g, int nx, int ny, int nz, double dx, int dtype);

/* Free a grid and its scratch (NULL is a no-op).  Does not synchronise
 * beyond what cudaFree implies. */
CDI_API int cdi_destroy_grid(cdi_grid *g);

/* Query extents, spacing and dtype. */
CDI_API int cdi_grid_info(const cdi_grid *g, int *nx, int *ny, int *nz, double *dx, int *dtype);

/* Borrow face velocities (device, dtype of the grid).  w may be NULL only
 * when nz == 1 (w is then inert: the z-faces coincide, Eq. 18 in 2D); v
 * likewise when ny == 1 and nz == 1.  umax >= 0 sets U, the largest face
 * |component| used by the condition check (Eq. 24); umax < 0 computes U on
 * the device (synchronises the stream). */
CDI_API int cdi_set_velocity(cdi_grid *g, const void *u, const void *v, const void *w,
                     double umax, void *stream);

/* U as set or computed by cdi_set_velocity. */
CDI_API int cdi_get_umax(const cdi_grid *g, double *U);

/* One explicit Euler step phi_out = phi_in + dt * RHS(phi_in) (Eq. 11 / 18),
 * with face velocity vel_scale * (u, v, w).  phi_in and phi_out are device
 * arrays of nx*ny*nz elements and must not overlap.  The fused reduction
 * (cdi_stats of phi_out) is written to the grid's device record; read it
 * with cdi_step_stats.  With CDI_CHECK_CONDITION the call first checks
 * eps/dx >= (g + 1)/(2 g), g = gamma/(|vel_scale| U) (Eq. 24), and
 * A = dt gamma eps/dx^2 <= 1/(2 D_f) (Eq. 25) and returns
 * CDI_ERR_CONDITION without launching if either fails.  The check allows a
 * relative slack of 1e-12 (CDI_F64) or 4 FLT_EPSILON (CDI_F32, where U is
 * measured on the float-rounded velocity) so that configurations placed
 * exactly on the crossover line pass. */
CDI_API int cdi_step(cdi_grid *g, const void *phi_in, void *phi_out, double dt, double eps,
             double gamma, double vel_scale, int flags, void *stream);

/* nsteps Euler steps starting at time t0, ping-ponging between buf_a (holds
 * phi at t0 on entry) and buf_b; vel_scale = cos(pi t / period) at each
 * step's start time t (period <= 0: vel_scale = 1).  The launch loop runs
 * in native code.  On return *final_in_b tells which buffer holds the
 * result.  Stats of the last step are in the device record. */
CDI_API int cdi_run(cdi_grid *g, void *buf_a, void *buf_b, int nsteps, double t0, double dt,
            double eps, double gamma, double period, int flags, int *final_in_b,
            void *stream);

/* The Euler step of cdi_step restricted to the planes z_lo <= k < z_hi
 * (0 <= z_lo < z_hi <= nz): those planes of phi_out are written, the others
 * are left as they are; the stencil reads planes z_lo-2 .. z_hi+1 of phi_in
 * (periodic in nz) and the w faces below each plane.  The statistics record
 * covers the updated planes only (mass = dV * their sum) and counts as one
 * step of the run accumulators.  This is the kernel of a z-slab domain
 * decomposition: a rank holds its slab with two halo planes on each side
 * (nz = slab planes + 4), fills the halos from its neighbours, and steps
 * planes [2, nz - 2), where no periodic wrap is taken.  Centre-product
 * sharpening only (CDI_ERR_ARG otherwise). */
CDI_API int cdi_step_planes(cdi_grid *g, const void *phi_in, void *phi_out, int z_lo, int z_hi,
                            double dt, double eps, double gamma, double vel_scale, int flags,
                            void *stream);

/* One step of a Runge-Kutta scheme of Section 2.3 from phi_in (left unchanged)
 * to phi_out, with velocity cos(pi t_s/period) (u, v, w) at each stage time
 * t_s (period <= 0: 1).  scheme: CDI_EULER (= cdi_step), CDI_RK2 (explicit
 * midpoint), CDI_RK3 (Wray's low-storage scheme: stage weights 8/15, 5/12,
 * 3/4 and -17/60, -5/12), CDI_RK4 (classic).  Each stage is one fused launch
 * that evaluates the right-hand side and combines the stage in its
 * epilogue.  work1 and work2 are caller-owned device arrays of the grid's
 * size (unused for CDI_EULER); none of phi_in, phi_out, work1, work2 may
 * overlap.  With CDI_CHECK_CONDITION the diffusive limit is the scheme's
 * (Eq. 26-28: A <= 1/(2 D_f), 2.51/(4 D_f), 2.79/(4 D_f)).  The statistics
 * record holds the step's result; the run accumulators count steps. */
CDI_API int cdi_step_rk(cdi_grid *g, const void *phi_in, void *phi_out, void *work1, void *work2,
                        double dt, double eps, double gamma, double t, double period, int scheme,
                        int flags, void *stream);

/* nsteps steps of cdi_step_rk ping-ponging buf_a (phi at t0) and buf_b;
 * *final_in_b tells which buffer holds the result. */
CDI_API int cdi_run_rk(cdi_grid *g, void *buf_a, void *buf_b, void *work1, void *work2, int nsteps,
                       double t0, double dt, double eps, double gamma, double period, int scheme,
                       int flags, int *final_in_b, void *stream);

/* Copy the device statistics record of the last fused step to *out;
 * synchronises the stream.  Returns CDI_ERR_NAN if the sum is not finite. */
CDI_API int cdi_step_stats(cdi_grid *g, cdi_stats *out, void *stream);

/* Reset the run accumulators (*_run, steps_run) of the device record. */
CDI_API int cdi_reset_run_stats(cdi_grid *g, void *stream);

/* Reduce an arbitrary phi (device) into *out (host); synchronises. */
CDI_API int cdi_mass_and_bounds(cdi_grid *g, const void *phi, cdi_stats *out, void *stream);

/* Host-buffer step: copies phi_in (host, ideally pinned) to the device,
 * performs cdi_step with the velocity set by cdi_set_velocity, copies
 * phi_out and the statistics back to host memory and synchronises.  Uses
 * two device staging buffers owned by the grid (allocated on first use).
 * For nz >= 16 the step runs as a pipeline of 8 z slabs on two copy streams
 * of the grid and the given stream: the two seam planes and then the slabs
 * are copied in, a slab is stepped as soon as the piece holding its halo
 * planes has landed and copied out while later slabs are still arriving, so
 * both copy directions and the kernel overlap.
 * The slabs run the vector kernel where nx allows (else the one-cell-per-
 * thread kernel), so the result equals cdi_step's up to that kernel's
 * rounding (bit for bit when the grid's forward tile is the same). */
CDI_API int cdi_step_host(cdi_grid *g, const void *phi_in_host, void *phi_out_host, double dt,
                  double eps, double gamma, double vel_scale, int flags,
                  cdi_stats *stats_out, void *stream);

/*
 * Discrete adjoint of one Euler step (reverse mode through the five steps
 * of Section 2.2).  With J = d phi^{k+1}/d phi^k at phi_k:
 *     lam_k = J^T lam_next
 * and, if gu/gv/gw are non-NULL, (d phi^{k+1}/d u_f)^T lam_next is ADDED to
 * them (accumulated over steps by the caller).  phi_k is the forward input
 * of the step (recomputed by the caller from a checkpoint).  lam_k must not
 * overlap lam_next or phi_k.  Same dt/eps/gamma/vel_scale as the forward.
 *
 * J is taken with the interface normal n = g / sqrt(|g|^2 + delta^2)
 * (g the central difference of phi; n = 0 where g = 0), delta = 8 machine
 * epsilons of the working precision (2^-20 in FP32, 2^-49 in FP64, i.e.
 * 16 units in the last place of values just below 1).  Where |g| is far
 * above delta -- every interface cell -- this is the derivative of the
 * forward step.  Where |g| falls to the rounding level of phi (the flat
 * bulk next to phi = 1 or 0, where neighbours differ by a unit or two in the
 * last place) the unit normal is rounding noise and its derivative
 * phi (1 - phi)/|g| is unbounded; the floor caps it, which keeps the
 * backward recursion of long rollouts from amplifying that noise.
 */
CDI_API int cdi_step_adjoint(cdi_grid *g, const void *phi_k, const void *lam_next, void *lam_k,
                     void *gu, void *gv, void *gw, double dt, double eps, double gamma,
                     double vel_scale, void *stream);

/* Boundedness condition (Eq. 17/24 with U the face maximum) and the Euler
 * diffusive limit A <= 1/(2 D_f) (Eq. 25).  Returns 1 if both hold, 0 if
 * not, CDI_ERR_ARG on bad input.  gamma_over_U = +inf is allowed.  A
 * relative slack of 1e-12 admits values placed exactly on the line. */
CDI_API int cdi_check_condition(double eps_over_dx, double gamma_over_U, double A, int Df);

/* Largest stable, bounded time step for a scheme above the crossover line:
 * Euler and RK2 dx^2/(2 D_f gamma eps) (Eq. 25, 26), RK3 2.51 dx^2/(4 D_f
 * gamma eps) (Eq. 27), RK4 2.79 dx^2/(4 D_f gamma eps) (Eq. 28). */
CDI_API int cdi_max_dt(double dx, double eps, double gamma, int Df, int scheme, double *dt);

/* Time step for points that may lie below the crossover line: the smaller of
 * the scheme's diffusive limit (cdi_max_dt) and a mixed advective-diffusive
 * limit c dx / (sum_d umax[d] + D_f gamma), umax[d] (d < Df) the largest face
 * |velocity component| along each non-degenerate axis.  CDI_RK4: c = 2.83, the
 * mixed criterion of Eq. 32 (2D: dx 2.83/(max u + max v + 2 gamma)), so the
 * result is min(Eq. 31, Eq. 32) in 2D.  CDI_EULER: c = 1, the 1D step of
 * Eq. 10 at the crossover line, dx/(u + gamma), summed over the axes
 * (2D: dx/(max u + max v + 2 gamma)).  The paper gives no mixed criterion for
 * RK2 and RK3: CDI_ERR_ARG.  Host arithmetic only. */
CDI_API int cdi_max_dt_mixed(double dx, double eps, double gamma, const double *umax, int Df,
                             int scheme, double *dt);

/*
 * Batched boxes.  Many independent periodic boxes of uneven sizes, each with
 * its own spacing, eps, gamma, dt and face velocities, advance together: one
 * kernel launch per step covers every box (a persistent grid taking work
 * units -- a tile of one box and a chunk of its planes -- from one list), and
 * cdi_batch_run replays a captured CUDA graph of nsteps such launches.  Each
 * box evolves exactly as with cdi_step on its own grid.  Arrays follow the
 * conventions above and are borrowed for the batch's lifetime.  Like a grid,
 * a batch (its counters, epochs and statistics scratch) must be used by one
 * stream at a time.
 */
typedef struct cdi_box_desc {
    int nx, ny, nz;
    double dx, dt, eps, gamma;
    const void *u, *v, *w;  /* face velocities (v, w NULL as for cdi_set_velocity) */
    void *phi_a, *phi_b;    /* ping-pong phase fields; the state starts in phi_a */
} cdi_box_desc;

typedef struct cdi_batch cdi_batch;

/* Build the device box table and work list (allocates). */
CDI_API int cdi_batch_create(cdi_batch **b, const cdi_box_desc *boxes, int nbox, int dtype);
CDI_API int cdi_batch_destroy(cdi_batch *b);

/* Which buffer holds the current state (*parity: 0 = phi_a, 1 = phi_b), the
 * number of work units and blocks per launch, and the total cell count. */
CDI_API int cdi_batch_info(const cdi_batch *b, int *parity, int *total_units, int *nblocks,
                           long long *cells);

/* One step of every box with face velocity vel_scale * (u, v, w); flips the
 * parity.  Per-box statistics of the result are written to the device. */
CDI_API int cdi_batch_step(cdi_batch *b, double vel_scale, void *stream);

/* nsteps steps (vel_scale = 1) as one CUDA graph launch; the graph is
 * captured on first use for each (nsteps, parity) and replayed after.  The
 * launches of a run overlap: launch i + 1 starts on the SMs that launch i
 * leaves, and each of its work units waits (on the device, for at most one
 * second plus 2 ns per cell of the batch) only until its own box has completed
 * step i.  The results are those
 * of nsteps cdi_batch_step calls, bit for bit.  A wait that runs out is
 * recorded in the status words (the units after it are skipped) and reported
 * by the next cdi_batch_stats as CDI_ERR_TIMEOUT; the next run starts afresh.
 * Allocates one pair of 32-bit counters per step on the first run of a new
 * largest nsteps. */
CDI_API int cdi_batch_run(cdi_batch *b, int nsteps, void *stream);

/* Copy the nbox statistics records (last step + run accumulators) to out[];
 * synchronises.  CDI_ERR_NAN if a box's sum is not finite; CDI_ERR_TIMEOUT if
 * a run's device-side wait gave up since the last call (the status words are
 * then cleared); CDI_ERR_BOUNDS from checked builds. */
CDI_API int cdi_batch_stats(cdi_batch *b, cdi_stats *out, void *stream);
CDI_API int cdi_batch_reset_run_stats(cdi_batch *b, void *stream);

/* Test of the run's bounded wait: one launch whose work units wait for a step
 * their boxes never reach, the first wait for limit_s seconds (0 < limit_s <=
 * 2), the others giving up when they see it has.  No unit is stepped: fields,
 * statistics and parity are unchanged.  Returns CDI_ERR_TIMEOUT (the expected
 * result; the status words are cleared) or CDI_OK if no wait ran out (the
 * time-out path is broken).  Synchronises. */
CDI_API int cdi_batch_probe_box_wait(cdi_batch *b, double limit_s, void *stream);

/* Sharpening form of every box of the batch (see cdi_set_sharpening):
 * CDI_SHARPEN_CENTRE (Section 2.2, the default) or CDI_SHARPEN_FACE, the
 * face-product form, which runs on batch tiles 0 and 4 only (setting it
 * selects tile 0; cdi_batch_set_launch refuses other tiles and the autotuner
 * skips them while it is set).  Rebuilds the work list. */
CDI_API int cdi_batch_set_sharpening(cdi_batch *b, int mode);
CDI_API int cdi_batch_get_sharpening(const cdi_batch *b, int *mode);

/* Launch configuration of the batch (a performance control, not part of the
 * paper): tile 0..3 = 32x8, 32x16, 64x8, 32x4 cells per work unit (one cell
 * per thread), zdepth = about that many planes per unit (0: whole box depth).
 * Tile 4 = one work unit per box, for batches of 2D boxes only (every nz = 1)
 * whose largest plane fits in one block's shared memory as 3 nx ny values
 * (about 9600 cells in FP64, 19000 in FP32): the whole plane is staged once
 * and each cell's sharpening evaluated once; the results are those of tiles
 * 0..3 bit for bit (the statistics' sums to rounding).  CDI_ERR_ARG, with the
 * launch unchanged, where it does not apply; zdepth is ignored for it.
 * Tile 5 = bands of whole rows (up to 1024 cells per band, 256 threads, several
 * cells per thread), for batches that hold a 3D box and whose rows are at most
 * 1024 cells wide: each plane's band and halo rows are one contiguous run of
 * the array, staged by 16-byte copies whatever the row alignment; the fields
 * are those of tiles 0..3 bit for bit.  CDI_ERR_ARG where it does not apply.
 * Tile 6 = bands of whole rows of the batch's own padded copy of every box
 * (rows padded to 16-byte multiples with periodic ghost cells at both ends,
 * allocated on first use: 5 arrays of the padded box size): 16-byte copies and
 * 16-byte shared loads of four (FP32) or two (FP64) cells per thread whatever
 * nx is.  Each step or run call first copies the caller's current state into
 * the padded copy and its last step also writes the caller's array, so the
 * caller's buffers behave as for the other tiles; rows of at most 400 (FP32)
 * or 200 (FP64) cells.  Centre-form sharpening only; the fields
 * are those of tiles 0..3 bit for bit.
 * tile = -1 / zdepth = -1 restore the defaults (32x8, CDI_BATCH_DEFAULT_ZDEPTH).
 * Rebuilds the work list (synchronises the device; drops captured graphs). */
#define CDI_BATCH_DEFAULT_ZDEPTH 32
CDI_API int cdi_batch_set_launch(cdi_batch *b, int tile, int zdepth);
CDI_API int cdi_batch_get_launch(const cdi_batch *b, int *tile, int *zdepth, int *nblocks,
                                 int *total_units);

/* Time every tile x zdepth in {8, 16, 32, 64, whole} (a batch of 2D boxes: every
 * tile once, tile 4 where it applies; tile 5 where it applies) with reps launches each
 * (after one warm-up) and keep the fastest; *best_ms (nullable) gets its time
 * per launch.  The trial launches read the current state and write the other
 * buffer only, and the statistics records are restored, so the batch's state
 * and records are as before the call.  Synchronises. */
CDI_API int cdi_batch_autotune(cdi_batch *b, int reps, float *best_ms, void *stream);

/* Sharpening form of the forward step.  CDI_SHARPEN_CENTRE (the default) is
 * Section 2.2's: s = phi (1 - phi) n at cell centres, averaged onto the faces,
 * the form Eq. 13 and Eq. 19 and the boundedness proof hold for.
 * CDI_SHARPEN_FACE is the product of face values instead, the sharpening flux
 * gamma phi_f (1 - phi_f) n_f with phi_f = (phi_L + phi_R)/2 and n_f =
 * (n_L + n_R)/2 (the cell-centre unit normals interpolated to the face): not
 * covered by the proof, and not stationary on the scheme's discrete
 * equilibrium.  It runs on forward tile 0 with explicit Euler steps only;
 * cdi_step_rk, cdi_run_rk and cdi_step_adjoint return CDI_ERR_ARG while it is
 * set (batches choose their own form: cdi_batch_set_sharpening).  Setting a
 * mode resets the forward launch configuration to the mode's default. */
enum { CDI_SHARPEN_CENTRE = 0, CDI_SHARPEN_FACE = 1 };
CDI_API int cdi_set_sharpening(cdi_grid *g, int mode);
CDI_API int cdi_get_sharpening(const cdi_grid *g, int *mode);

/* Diagnostic of the failure path: launches one block that waits, with the
 * library's bounded device wait, on an mbarrier that nothing completes.  The
 * wait must run out after limit_s seconds (0 < limit_s <= 2), record the time-
 * out in the grid's status word and let the kernel end; the call then reads
 * and clears that word and returns CDI_ERR_TIMEOUT -- the expected result.
 * CDI_OK would mean a time-out went unreported.  Synchronises the stream. */
CDI_API int cdi_probe_bounded_wait(cdi_grid *g, double limit_s, void *stream);

/* Checked builds.  A library compiled with -DCDI_CHECKED (build.py
 * --checked, _lib/libcdi_checked.so) tests every index its kernels derive for a
 * global access -- in-plane offsets of staged tiles, plane indices, output
 * offsets -- against the array extent before use; an index out of range is
 * replaced by 0 (the access stays inside the array) and recorded in the
 * grid's device status words, and the next statistics read-back
 * (cdi_step_stats, cdi_mass_and_bounds, cdi_step_host) returns CDI_ERR_BOUNDS
 * with the count and the last bad index in the message.  A debugging aid, not
 * part of the paper; the regular build has no checks. */
CDI_API int cdi_is_checked_build(void);

/* Diagnostic of the checked build: one kernel thread tests an index one past
 * its limit.  Returns CDI_ERR_BOUNDS (the expected result: the check recorded
 * it), CDI_OK if nothing was recorded, CDI_ERR_STATE in a regular build.
 * Synchronises the stream. */
CDI_API int cdi_probe_bounds_check(cdi_grid *g, void *stream);

/* Measured FP64 fused multiply-add rate of the current device (FMA
 * instructions per second, each 2 flops): a kernel of independent FMA chains
 * on every SM, best of three timed launches after a warm-up.  The roof of the
 * FP64 step, which is bound by the FP64 pipe rather than by memory (not part
 * of the paper).  Synchronises the stream. */
CDI_API int cdi_probe_fp64_rate(double *fma_per_s, void *stream);

/* The slab plan cdi_step_host uses for nz >= 16 planes (host arithmetic only,
 * no CUDA call): bounds[0..8] the 8 slabs [bounds[j], bounds[j+1]); after the
 * two seam planes nz-2, nz-1, copy-in piece j is planes [copy_lo[j],
 * copy_hi[j]) (8 entries each), which ends with the two halo planes above slab
 * j, so slab j is stepped once piece j has landed.  CDI_ERR_DIM for nz < 16,
 * CDI_ERR_ARG for a NULL array. */
CDI_API int cdi_host_slab_plan(int nz, int *bounds, int *copy_lo, int *copy_hi);

/* Kernels with a tunable launch configuration. */
enum { CDI_KERNEL_FORWARD = 0, CDI_KERNEL_ADJOINT = 1 };

/* Forward work split of cdi_set_launch: equal contiguous shares per block;
 * near-equal shares, a share that starts a second tile column being 4 planes
 * shorter to pay for that column's prologue, with each tile's column visited
 * rotated so that the blocks on neighbouring tiles work on the same planes at
 * the same time (their shared halo rows then come from L2 rather than memory).
 * The rotated split needs tiles * (nz + 4) < 2^31 (else CDI_ERR_DIM). */
#define CDI_NCHUNKS_BALANCED (-1)
#define CDI_NCHUNKS_ROTATED (-2)

/* Choose the launch configuration of a kernel of this grid (not part of the
 * paper: a performance control).  Forward tiles: 0..3 one cell per thread
 * (32x8, 32x16, 64x8, 32x4 cells), 4 and 5 sixteen-byte vectors per thread
 * (16x16 and 16x8 threads; need nx % (16/sizeof(element)) == 0); tile < 0
 * restores the default.  blocks_per_sm <= 0 fills the GPU.  Forward work
 * split: nchunks >= 1 cuts every tile column into that many z chunks, taken
 * round-robin by the persistent blocks; CDI_NCHUNKS_BALANCED gives every block
 * an equal contiguous share of the tile-planes (tile-major, cut at column
 * ends), CDI_NCHUNKS_ROTATED the same shares with rotated columns; 0 picks
 * chunks or CDI_NCHUNKS_ROTATED from a cost model.  Adjoint
 * tiles: 0..2 (32x8, 32x16, 32x4 cells) and 3 (vector), nchunks sets the z
 * chunking (CDI_NCHUNKS_BALANCED / CDI_NCHUNKS_ROTATED: balanced shares, tile 3
 * only; the vector adjoint's default takes the rotated shares where the cost
 * model favours balanced ones).  Every forward configuration (and the batch
 * and two-steps-per-pass paths) computes the same field bit for bit; the
 * statistics' sum may differ in its last bits with the order of the block
 * partials. */
CDI_API int cdi_set_launch(cdi_grid *g, int which, int tile, int blocks_per_sm, int nchunks);

/* Current launch configuration (any pointer may be NULL). */
CDI_API int cdi_get_launch(const cdi_grid *g, int which, int *tile, int *nblocks, int *nchunks);

/* Steps per pass of cdi_run (not part of the paper: temporal blocking, a
 * performance control).  depth 1: one launch per step.  depth 2: two Euler
 * steps per launch -- each block evaluates the first step on its tile grown
 * by the second step's two-cell halo, keeps those phi values in shared
 * memory, and evaluates the second step from them, so phi is read and written
 * and the face velocities read once per two steps; each step's statistics are
 * still reduced, the record holds the last step's and the run accumulators
 * count both.  The results are those of depth 1 on forward tile 4 bit for
 * bit.  Needs nx % (16/sizeof(element)) == 0 and the centre-product
 * sharpening (CDI_ERR_ARG otherwise); an odd step count ends with one single
 * step.  nchunks: the work split as in cdi_set_launch. */
CDI_API int cdi_set_run_depth(cdi_grid *g, int depth, int nchunks);
CDI_API int cdi_get_run_depth(const cdi_grid *g, int *depth, int *nblocks, int *nchunks);

/* Time every forward launch configuration on phi_a/phi_b (device, contents
 * overwritten) with CUDA events on the stream (one warm-up + reps launches
 * each) and keep the fastest for cdi_step; then time the two-steps-per-pass
 * kernel (where it applies) and set the run depth of cdi_run to 2 if it is
 * faster per step than that, else to 1.  *best_ms (may be NULL) gets the time
 * per step of what cdi_run will use.  Synchronises the stream. */
CDI_API int cdi_autotune(cdi_grid *g, void *phi_a, void *phi_b, double dt, double eps,
                         double gamma, int reps, double *best_ms, void *stream);

/*
 * One forward step that allocates nothing (the paper has no counterpart: this
 * is an interface for callers that may not allocate device memory).
 *
 * Some callers cannot call cudaMalloc: code running inside a stream callback
 * or an allocator hook, a framework that fixes its memory pool up front, or a
 * latency-critical loop that must never enter the driver's allocator.  The
 * grid API allocates its reduction scratch in cdi_create_grid; this call
 * takes no grid.  Its scratch is a fixed device array inside the library
 * (CDI_NOALLOC_MAX_BLOCKS partials of 40 bytes plus a counter, about 320 KB),
 * held by every GPU that loads the library until the process exits.
 *
 * Arguments are those of cdi_create_grid + cdi_set_velocity + cdi_step:
 * extents, spacing, dtype, device phi_in / phi_out (not overlapping), face
 * velocities (v may be NULL only when ny == nz == 1, w only when nz == 1),
 * dt, eps, gamma, vel_scale.  stats_dev is a caller-owned DEVICE buffer of
 * sizeof(cdi_stats) bytes; the step writes mass, sum, min, max, n_strict and
 * n_tol of phi_out into it (the *_run fields are left untouched).  No
 * condition check is made.  Returns CDI_ERR_DIM if the launch would need more
 * blocks than the fixed scratch holds (not reachable on a 152-SM GB300).
 *
 * The first call on a device, made with that device current, looks up the
 * scratch's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  The address is kept per device together with
 * the id of the context it was found in; a call in a new context of the
 * device (after cudaDeviceReset) looks it up again, and that call too should
 * come before any stream capture.  Every call shares the one scratch array,
 * which keeps the last call's contents: calls that overlap on the GPU race on
 * it.  Each call clears the block counter on its stream before its launch.
 * phi_out and stats_dev may overlap none of the other arrays (CDI_ERR_ARG).
 */
#define CDI_NOALLOC_MAX_BLOCKS 8192
CDI_API int cdi_step_noalloc(int nx, int ny, int nz, double dx, int dtype, const void *phi_in,
                             void *phi_out, const void *u, const void *v, const void *w,
                             double dt, double eps, double gamma, double vel_scale,
                             void *stats_dev, void *stream);

/* Message of the last failed call on this thread ("" if none). */
CDI_API const char *cdi_last_error_string(void);

/* CDI_VERSION of the loaded library. */
CDI_API int cdi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CDI_H */
