/*
 * gbib.h -- C ABI of the GB300-native multidirect-forcing immersed-boundary
 * library (Zeng et al., "IAMReX", arXiv 2408.14140).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Grid (ib_grid): n[0] x n[1] x n[2] cells of uniform spacing h, first
 *    cell centre at origin + h/2 on every axis, periodic with period n[a]*h.
 *    This is the cell-centred "finest level" of Sec. 3.1 (semi-staggered grid:
 *    velocity, force and PVF at cell centres, level set at nodes).
 *    Each n[a] must be >= 12; prec is IB_F64 or IB_F32 and fixes the element
 *    type of every Eulerian field argument (u, f).
 *  * Eulerian fields are structure-of-arrays u[3][n2][n1][n0] (x fastest),
 *    contiguous, 16-byte aligned.
 *  * Lagrangian vectors are [count][3] row-major FP64, 8-byte aligned.
 *  * Every pointer passed to a compute call is a DEVICE pointer on the
 *    context's device, owned by the caller; the library never frees or keeps
 *    it after the work queued on `stream` completes.  `stream` is a
 *    cudaStream_t (NULL = legacy default stream).
 *  * Calls are asynchronous on `stream`.  Their return value reports argument
 *    and launch errors synchronously; errors found on the device (non-finite
 *    input, a wait that gave up, a bin overflow) are latched in the context
 *    and returned by ib_ctx_status().
 *  * Work scratch lives in the context's workspace, allocated by
 *    ib_ctx_create()/ib_ctx_reserve(); calls never allocate.  A call whose
 *    scratch does not fit returns IB_ERR_OOM and ib_last_error() states the
 *    bytes needed.  Calls on one context must not overlap on the GPU (they
 *    share its workspace): use one context per concurrent stream.
 *  * Results are deterministic: the same inputs give bitwise identical
 *    outputs run to run (fixed summation orders, no floating-point atomics),
 *    unless a context selects the atomic spreading form
 *    (ib_ctx_set_spread_mode).
 */
#ifndef GBIB_H
#define GBIB_H

#include <stddef.h>
#include <stdint.h>

#if defined(GBIB_BUILD) && defined(__GNUC__)
#define GBIB_API __attribute__((visibility("default")))
#else
#define GBIB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define IB_OK 0
#define IB_ERR_INVALID (-1)      /* bad argument (null pointer, size, value)  */
#define IB_ERR_OOM (-2)          /* workspace too small / allocation failed   */
#define IB_ERR_CUDA (-3)         /* a CUDA runtime call failed                */
#define IB_ERR_TIMEOUT (-4)      /* a bounded device-side wait gave up        */
#define IB_ERR_NONFINITE (-5)    /* NaN/Inf in a particle or marker input     */
#define IB_ERR_UNSUPPORTED (-6)  /* valid but beyond the library's limits      */

/* ---- enumerations ------------------------------------------------------ */
typedef enum { IB_F64 = 0, IB_F32 = 1 } ib_prec;
/* Regularised delta kernels (Sec. 3.1 Step 2: "three-point or four-point").
 * ROMA3: Roma, Peskin & Berger (1999); PESKIN4: Peskin (2002).            */
typedef enum { IB_DELTA_ROMA3 = 0, IB_DELTA_PESKIN4 = 1 } ib_delta;
/* Particle order of Algorithm 1 (Sec. 3.1: "each particle goes into 1 to
 * Ns loop sequentially").  SEQUENTIAL: particle p starts from the field left
 * by particles 0..p-1.  SIMULTANEOUS: one Ns loop over all markers.        */
typedef enum { IB_ORDER_SEQUENTIAL = 0, IB_ORDER_SIMULTANEOUS = 1 } ib_order;

/* ---- problem description ----------------------------------------------- */
typedef struct {
    int n[3];          /* cells per axis (each >= 12)                       */
    double h;          /* cell size (> 0)                                   */
    double origin[3];  /* corner of cell (0,0,0)                            */
    int prec;          /* ib_prec of every Eulerian field argument          */
} ib_grid;

/* P rigid spheres (Sec. 3.2).  Xr, Ur, Wr are [P][3]; radius, rho_p are [P];
 * marker_offset is [P+1] (CSR: markers of particle p are
 * marker_offset[p] .. marker_offset[p+1]-1, increasing, marker_offset[0]=0). */
typedef struct {
    int P;
    double *Xr;        /* centroid X_r                                      */
    double *Ur;        /* centroid velocity U_r                             */
    double *Wr;        /* angular velocity W_r                              */
    const double *radius;
    const double *rho_p;
    const int *marker_offset;
} ib_particles;

/* Surface markers (Sec. 3.1 Step 2, markers on the surface only).
 * R[M][3] = X_l - X_r, the marker's offset from its particle's centroid
 * (Eq. pr1); dV[M] = the marker's volume weight Delta V_l (Algorithm 1).    */
typedef struct {
    int M;
    const double *R;
    const double *dV;
} ib_markers;

/* Physical constants of Eqs. (particle1), (particle2), (DKT_model). */
typedef struct {
    double rho_f;      /* fluid density                                     */
    double g[3];       /* gravitational acceleration                        */
    double g_coll;     /* ||g|| of Eq. (DKT_model)                          */
    double eps_c;      /* stiffness parameter epsilon_c (paper: 1e-4)       */
    double d_c;        /* collision range d_c (paper: finest grid spacing)  */
} ib_phys;

typedef struct ib_ctx ib_ctx;

/* ---- context ----------------------------------------------------------- */
/* Create a context on the current CUDA device with a device workspace of
 * `workspace_bytes` (0 selects 64 MiB).  Returns IB_OK, IB_ERR_INVALID
 * (ctx NULL) or IB_ERR_OOM / IB_ERR_CUDA.                                 */
GBIB_API int ib_ctx_create(ib_ctx **ctx, size_t workspace_bytes);
/* Grow the workspace to at least `bytes` (synchronises the device).       */
GBIB_API int ib_ctx_reserve(ib_ctx *ctx, size_t bytes);
/* Free the context and its workspace (synchronises the device).           */
GBIB_API int ib_ctx_destroy(ib_ctx *ctx);
/* Synchronise `stream`, then return and clear the first device-side error
 * latched by work queued since the last call (IB_OK when none).           */
GBIB_API int ib_ctx_status(ib_ctx *ctx, void *stream);
/* Human-readable message of the last failing call on this host thread.    */
GBIB_API const char *ib_last_error(void);
/* Workspace bytes the last call that returned IB_ERR_OOM on this host
 * thread needed (0 if none); pass it to ib_ctx_reserve() and retry.       */
GBIB_API size_t ib_workspace_needed(void);
/* Number of streaming multiprocessors of the context's device.            */
GBIB_API int ib_ctx_sm_count(const ib_ctx *ctx);

/* ---- optional device timing of the library's own kernels ---------------
 * When enabled, every call records a CUDA event pair on its stream around
 * each phase below.  ib_ctx_read_timing() waits for the recorded events,
 * returns the summed device time (ms) and the number of launches of one
 * phase since the last read, and resets that phase.  Timing adds two event
 * records per phase and must stay off while a stream is being captured.  */
#define IB_PHASE_MDF_PREP 0    /* marker preparation, levels, tile binning  */
#define IB_PHASE_MDF_PASSES 1  /* all Ns passes (resident or wavefront form) */
#define IB_PHASE_SPREAD 2      /* ib_spread (binning + gather)              */
#define IB_PHASE_INTERP 3      /* ib_interpolate                            */
#define IB_PHASE_VOLUME 4      /* particle_volume_integrals                 */
#define IB_PHASE_FORCE 5       /* particle_force_torque                     */
#define IB_PHASE_COLLIDE 6     /* particle_collide_update                   */
#define IB_PHASE_MDF_INTERP 7  /* each wavefront-pass interpolation kernel  */
#define IB_PHASE_MDF_GATHER 8  /* each wavefront-pass gather kernel         */
#define IB_PHASE_FLUID_PREDICTOR 9   /* fluid_predictor                   */
#define IB_PHASE_FLUID_PROJECTION 10 /* level_projection                  */
#define IB_PHASE_COUNT 11
GBIB_API int ib_ctx_set_timing(ib_ctx *ctx, int enable);
GBIB_API int ib_ctx_read_timing(ib_ctx *ctx, int phase, double *ms_total,
                                int *launches);

/* ---- kernels of the sequential-order passes ----------------------------
 * Every form computes bitwise the same result (same summation orders).
 * WAVEFRONT (the default, AUTO): per wavefront of non-conflicting particles
 *   and per pass, an interpolation kernel and a gather kernel through global
 *   memory (a persistent cooperative kernel takes the wavefronts beyond the
 *   count the previous call on the context saw).
 * RESIDENT: one thread-block cluster per particle keeps the particle's band
 *   tiles in shared memory for all Ns passes; particles start as soon as the
 *   earlier particles they conflict with are stored.
 * GROUPS: a persistent cooperative kernel split into groups of CTAs; a group
 *   runs all Ns passes of one particle (barriers over the group's CTAs only),
 *   and particles start as soon as the earlier particles they conflict with
 *   are done.
 * The simultaneous order always runs the wavefront form (one wavefront),
 * and so do FP64 fields, whose pass sums run in double-float arithmetic on
 * the FP32 pipes (RESIDENT and GROUPS serve FP32 fields).
 * Returns IB_ERR_INVALID for any other value.                             */
#define IB_PASSES_AUTO 0
#define IB_PASSES_WAVEFRONT 1
#define IB_PASSES_RESIDENT 2
#define IB_PASSES_GROUPS 3
GBIB_API int ib_ctx_set_pass_kernels(ib_ctx *ctx, int which);

/* ---- spreading form (Eq. f, Eq. fs; Algorithm 1's spreading step) ------
 * GATHER (the default): every cell sums the contributions of the markers
 *   whose stencils cover it in a fixed order, from per-tile marker lists
 *   built once per call: bitwise reproducible.
 * ATOMIC: every marker adds its KW^3 contributions to the cells with atomic
 *   additions, combined first across the lanes of a warp that target the
 *   same cell (one addition per distinct cell and warp).  No tile lists are
 *   built, so a forcing call's preparation is shorter.  The sums agree with
 *   the gather to rounding, but the order of the additions varies, so
 *   results are not bitwise reproducible run to run.
 * Applies to ib_spread and to every multidirect-forcing call on the context
 * (in the sequential order with the wavefront form; the resident and group
 * forms always gather).  IB_ERR_INVALID for any other value.                */
#define IB_SPREAD_GATHER 0
#define IB_SPREAD_ATOMIC 1
GBIB_API int ib_ctx_set_spread_mode(ib_ctx *ctx, int mode);

/* ---- CTAs per particle of the volume integrals (tuning knob) -----------
 * Each particle's box is cut into this many slabs of cell planes, one CTA
 * each (1 <= n <= 32), or 0 (the default): as many as fill one resident wave
 * of the device for the call's particle count (at least 1, at most 32).
 * Results do not depend on it beyond the rounding of the partial sums'
 * grouping.  The automatic choice depends on the call's particle count, so
 * a case's integrals computed inside a batch agree with the same case alone
 * only to rounding; a fixed split makes them bitwise equal.
 * IB_ERR_INVALID outside [0, 32].                                          */
GBIB_API int ib_ctx_set_volume_split(ib_ctx *ctx, int ctas_per_particle);

/* ---- wavefront gather layout (tuning knobs) ------------------------------
 * ctas_per_sm: resident gather CTAs per SM (0, the default: as many as fit;
 * 1..32 caps it).  stage: the candidates of a tile that a gather CTA stages
 * in shared memory (0, the default: the largest capacity, 256 for FP32 and
 * 192 for FP64 fields; else a multiple of 32 in [32, 256], capped at the
 * largest); a tile with more candidates reads them from memory, and a smaller
 * capacity lets more CTAs share an SM.  Neither changes a result: every cell
 * adds the same values in the same order.  IB_ERR_INVALID otherwise.       */
GBIB_API int ib_ctx_set_gather(ib_ctx *ctx, int ctas_per_sm, int stage);

/* ---- overlap: a dependency before the field is written ------------------
 * `event` is a cudaEvent_t (or NULL, the default, for none).  Every
 * multidirect-forcing call on this context (single or batched) makes its
 * stream wait for the event after its preparation kernels -- which read only
 * the particles and markers -- and before the first kernel that reads or
 * writes the field.  A caller can so run work that reads the same field (for
 * example the volume integrals of the same time step, on another stream and
 * another context) concurrently with the preparation: record the event after
 * that work and before the forcing call.  The event is waited on as recorded
 * when the forcing call is enqueued (also inside CUDA-graph capture, where the
 * wait becomes a graph dependency).  The context does not own the event.    */
GBIB_API int ib_ctx_set_field_wait(ib_ctx *ctx, void *event);

/* ---- self-test of the failure path (no paper counterpart) ----------------
 * Enqueues on `stream` a one-thread kernel that waits on a device word that
 * nothing ever sets and gives up after `cycles` SM clock cycles, raising
 * IB_ERR_TIMEOUT in the context's device status the way every bounded wait
 * of the library does.  The next ib_ctx_status(ctx, stream) returns
 * IB_ERR_TIMEOUT and clears the status; the context stays usable.  Nothing
 * faults and nothing hangs: the wait ends after `cycles` (1e6 cycles is about
 * half a millisecond at 2 GHz).  IB_ERR_INVALID for a NULL ctx or `cycles`
 * outside [1, 4e9]; IB_ERR_CUDA if the launch fails.                        */
GBIB_API int ib_selftest_wait_timeout(ib_ctx *ctx, long long cycles, void *stream);

/* ---- velocity interpolation J: Eq. (u), Eq. (vi), Algorithm 1 -----------
 * U[l] = sum_ijk u(x_ijk) delta_h(x_ijk - X[l]) h^3 for l < M, where
 * delta_h(x) = h^-3 prod_a phi(x_a / h) (Sec. 2).  X[M][3] are absolute
 * positions (any value; the grid is periodic).  u is [3][n2][n1][n0] in the
 * grid precision; U[M][3] is FP64 and overwritten.  M = 0 is a no-op.      */
GBIB_API int ib_interpolate(ib_ctx *ctx, const ib_grid *grid, const void *u, int M,
                   const double *X, int delta, double *U, void *stream);

/* ---- force spreading S: Eq. (f), Eq. (fs), Algorithm 1 ------------------
 * f(x_ijk) += sum_l F[l] delta_h(x_ijk - X[l]) dV[l] for every cell.  f is
 * ACCUMULATED (zero it first for a plain spread), grid precision.  The sum
 * per cell is a deterministic gather over markers binned by cell tile.     */
GBIB_API int ib_spread(ib_ctx *ctx, const ib_grid *grid, int M, const double *X,
              const double *F, const double *dV, int delta, void *f,
              void *stream);

/* ---- Algorithm 1, multidirect forcing over all particles ---------------
 * u (in/out, grid precision) holds u~*,n+1 on entry and u*,n+1 on exit.
 * Marker positions X_l = X_r + R_l and desired velocities
 * U^d_l = U_r + W_r x R_l (Eq. pr1) are formed from `parts` and `marks`.
 * Starting from F^0 = 0, each of the Ns passes interpolates U^{m-1}, sets
 * F^m = F^{m-1} + (U^d - U^{m-1})/dt, spreads it and corrects
 * u(m) = u(0) + dt f^m (Algorithm 1).  F_out[M][3] (FP64) receives F^Ns of
 * every marker; f_out (nullable, grid precision) is ACCUMULATED with the
 * Eulerian force dt^-1 (u_exit - u_entry) contributed by every particle.
 * Sphere markers must lie within a box smaller than the grid.  Ns >= 1,
 * dt > 0 finite.                                                          */
GBIB_API int ib_multidirect_forcing(ib_ctx *ctx, const ib_grid *grid, void *u,
                           const ib_particles *parts, const ib_markers *marks,
                           int Ns, double dt, int delta, int order,
                           double *F_out, void *f_out, void *stream);

/* ---- particle volume integrals through the PVF (Sec. 4.1, Eq. level-set
 * function, Eq. Heaviside; the flow-unsteadiness terms of Eqs. particle1/2):
 *   Iu[p]   = sum_c alpha_c u_c h^3
 *   Irxu[p] = sum_c alpha_c (x_c - X_r) x u_c h^3
 *   vol[p]  = sum_c alpha_c h^3
 * alpha_c = sum_m -phi_m H(-phi_m) / sum_m |phi_m| over the 8 cell corners,
 * phi = |x - X_r| / radius - 1 (nearest periodic image).  Outputs FP64,
 * overwritten; any of Iu, Irxu, vol may be NULL.                          */
GBIB_API int particle_volume_integrals(ib_ctx *ctx, const ib_grid *grid, const void *u,
                              const ib_particles *parts, double *Iu,
                              double *Irxu, double *vol, void *stream);

/* ---- volume integrals twice at the same particle positions --------------
 * The step integrates the PVF of each particle over the field before and
 * after the forcing (Eqs. particle1/particle2, Sec. 3.2.2) with the particles
 * where they are: the cells and their volume fractions alpha are the same.
 * particle_volume_integrals_keep computes what particle_volume_integrals
 * computes (bitwise) and keeps in `plan` the cells each CTA visited, plane by
 * plane, with the boundary cells' alpha; particle_volume_integrals_plan then
 * integrates another field u (same grid, same particles) over the kept cells
 * with the kept alpha and the same per-cell arithmetic, without evaluating a
 * level set: each particle's kept cells are one list spread evenly over the
 * context's split of CTAs per particle (ib_ctx_set_volume_split; automatic:
 * one resident wave), so its sums agree with particle_volume_integrals on
 * that field to rounding (another summation order; deterministic for a given
 * split).  A plan holds up to P particles
 * whose stencil boxes have at most max_box_cells cells (at most 40 cells per
 * axis); a larger box raises IB_ERR_UNSUPPORTED in the context status.  The
 * plan call checks the grid (IB_ERR_INVALID) and, on the device, that every
 * particle's X_r and radius equal the kept ones (IB_ERR_INVALID in the status;
 * that particle's integrals are then 0).  The plan is device memory owned by
 * the caller: create it once (not under stream capture), destroy it after its
 * last call has run.                                                       */
typedef struct ib_pvf_plan ib_pvf_plan;
GBIB_API int ib_pvf_plan_create(ib_ctx *ctx, int P, int max_box_cells, ib_pvf_plan **plan);
GBIB_API int ib_pvf_plan_destroy(ib_pvf_plan *plan);
GBIB_API int particle_volume_integrals_keep(ib_ctx *ctx, const ib_grid *grid, const void *u,
                                            const ib_particles *parts, ib_pvf_plan *plan, double *Iu,
                                            double *Irxu, double *vol, void *stream);
GBIB_API int particle_volume_integrals_plan(ib_ctx *ctx, const ib_grid *grid, const void *u,
                                            const ib_particles *parts, const ib_pvf_plan *plan,
                                            double *Iu, double *Irxu, double *vol, void *stream);

/* ---- PVF volume integrals of ellipsoids: Sec. 4.1, Eq. (level-set
 * function of spheroidal geometries) -----------------------------------
 * As particle_volume_integrals, for P axis-aligned ellipsoids centred at
 * Xr[P][3] with semi-axes axes[P][3] = (a, b, c): phi = sqrt((x/a)^2 +
 * (y/b)^2 + (z/c)^2) - 1 at the nodes, alpha from the eight corners of each
 * cell.  A sphere is a = b = c = R.  Outputs Iu[P][3], Irxu[P][3], vol[P]
 * (FP64, overwritten).  IB_ERR_NONFINITE for a non-finite centre or a
 * non-positive axis; IB_ERR_UNSUPPORTED when an ellipsoid's box exceeds the
 * grid.                                                                     */
GBIB_API int particle_volume_integrals_ellipsoid(ib_ctx *ctx, const ib_grid *grid, const void *u,
                                                 int P, const double *Xr, const double *axes,
                                                 double *Iu, double *Irxu, double *vol,
                                                 void *stream);

/* ---- drag diagnostic: Sec. 4.3 (flow past a fixed sphere), Eq. (FD) -------
 * F_D[P][3] = -rho_f sum_l F_l dV_l + rho_f d/dt int_Vp u dV, with the first
 * term given as F_ib (particle_force_torque) and the time derivative as
 * (Iu_new - Iu_old) / dt of the PVF integrals.  FP64, overwritten.          */
GBIB_API int particle_drag_force(ib_ctx *ctx, int P, const double *F_ib, const double *Iu_new,
                                 const double *Iu_old, double rho_f, double dt, double *F_D,
                                 void *stream);

/* ---- batches of independent cases (continuous batching, serving) -------
 * A batch runs many independent periodic cases -- each with its own grid
 * size, field and particles -- through the same kernel launches.  The
 * particles of all cases sit in one flat ib_particles (marker_offset global
 * over the flat marker arrays); case c owns particles p_begin .. p_end-1 and
 * their markers.  Cases must partition [0, P) in order: cases[0].p_begin = 0,
 * cases[c+1].p_begin = cases[c].p_end, cases[n-1].p_end = P (a case may have
 * no particles).  Every case's grid must have the same prec.  Particles of
 * different cases never interact.  Each batch entry point computes, for every
 * case, exactly what the single-case entry point of the same name computes
 * (bitwise: the same kernels and summation orders).
 * The case table is copied to the workspace through a small ring of pinned
 * host buffers owned by the context (asynchronous on `stream`; a buffer is
 * reused once the copy that read it has run), so batch calls must not be
 * captured into a CUDA graph (single-case calls can).  Errors as for the single-case entry points, plus
 * IB_ERR_INVALID for ranges that do not partition [0, P) or mixed precisions
 * (the message names the case).                                            */
typedef struct {
    ib_grid grid;   /* the case's grid                                      */
    void *u;        /* the case's field [3][n2][n1][n0] (in/out where written) */
    void *f_out;    /* nullable: the case's accumulated Eulerian force        */
    int p_begin;    /* first particle of the case                           */
    int p_end;      /* one past its last particle                           */
} ib_case;

/* Algorithm 1 over every case (see ib_multidirect_forcing). */
GBIB_API int ib_batch_multidirect_forcing(ib_ctx *ctx, int ncases, const ib_case *cases,
                                          const ib_particles *parts,
                                          const ib_markers *marks, int Ns, double dt,
                                          int delta, int order, double *F_out,
                                          void *stream);
/* PVF volume integrals of every particle in its case's field. */
GBIB_API int ib_batch_volume_integrals(ib_ctx *ctx, int ncases, const ib_case *cases,
                                       const ib_particles *parts, double *Iu,
                                       double *Irxu, double *vol, void *stream);
/* Collision (pairs within a case, the case's periodic box) + Newton-Euler.
 * phys[ncases]: the physical parameters of each case (the contact distance
 * d_c is usually the case's own h).                                       */
GBIB_API int ib_batch_collide_update(ib_ctx *ctx, int ncases, const ib_case *cases,
                                     ib_particles *parts, const ib_phys *phys,
                                     double dt, const double *F_ib,
                                     const double *T_ib, const double *Iu_new,
                                     const double *Iu_old, const double *Irxu_new,
                                     const double *Irxu_old, double *Fc_out,
                                     void *stream);
/* (particle_force_torque works on any flat particle set, batched or not.) */

/* ---- prepared batches: the case table uploaded once --------------------
 * ib_batch_table_create validates `cases` as the ib_batch_* calls do (and
 * phys, when given: eps_c, d_c > 0 per case) and copies the case table into
 * device memory that the returned table owns.  It allocates (cudaMalloc) and
 * waits for its copies (made on a private non-blocking stream, so they wait
 * for no work the caller has queued), so create tables before any stream
 * capture.  The
 * table keeps the cases' field pointers: it serves calls on exactly those
 * fields and particle ranges (P particles) until ib_batch_table_destroy.
 * The ib_batch_table_* calls compute what the ib_batch_* calls of the same
 * name compute (same kernels: bitwise equal) but upload nothing and never
 * wait on the host, so they can be captured into a CUDA graph, provided the
 * context's workspace already fits the call (make one call outside capture
 * first; a capture that meets IB_ERR_OOM cannot grow it).  phys may be NULL
 * when the table is not used for ib_batch_table_collide_update (which then
 * returns IB_ERR_INVALID).  Errors: IB_ERR_INVALID for bad cases, a NULL
 * table, a table of another device or a call whose P differs; IB_ERR_OOM /
 * IB_ERR_CUDA when the device copy cannot be made.  Destroy frees the device
 * memory once the work already queued on the device has finished.            */
typedef struct ib_batch_table ib_batch_table;
GBIB_API int ib_batch_table_create(ib_ctx *ctx, int ncases, const ib_case *cases, int P,
                                   const ib_phys *phys, ib_batch_table **table);
GBIB_API int ib_batch_table_destroy(ib_batch_table *table);
/* Re-points a table at another batch (validated as at creation): the new
 * case table is uploaded asynchronously on `stream` from a pinned copy the
 * table owns, so calls enqueued on `stream` afterwards see it and calls
 * before it see the old one; only when the new batch outgrows the table's
 * memory does it reallocate (waiting for the device).  Not capturable.  A
 * CUDA graph captured with the table keeps reading its memory, so replay
 * such a graph only while the table still describes the batch it captured. */
GBIB_API int ib_batch_table_update(ib_batch_table *table, int ncases, const ib_case *cases, int P,
                                   const ib_phys *phys, void *stream);
GBIB_API int ib_batch_table_multidirect_forcing(ib_ctx *ctx, const ib_batch_table *table,
                                                const ib_particles *parts, const ib_markers *marks,
                                                int Ns, double dt, int delta, int order,
                                                double *F_out, void *stream);
GBIB_API int ib_batch_table_volume_integrals(ib_ctx *ctx, const ib_batch_table *table,
                                             const ib_particles *parts, double *Iu, double *Irxu,
                                             double *vol, void *stream);
GBIB_API int ib_batch_table_collide_update(ib_ctx *ctx, const ib_batch_table *table,
                                           ib_particles *parts, double dt, const double *F_ib,
                                           const double *T_ib, const double *Iu_new,
                                           const double *Iu_old, const double *Irxu_new,
                                           const double *Irxu_old, double *Fc_out, void *stream);

/* ---- allocation-free volume integrals ----------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: code that runs while a CUDA stream is
 * being captured (where cudaMalloc is not allowed), latency-critical loops
 * that must not take cudaMalloc's implicit device synchronisation, and hosts
 * whose device memory is all owned by another allocator.  It computes the
 * same Iu, Irxu, vol as particle_volume_integrals with the same kernel, its
 * slab split fixed at 8 CTAs per particle: the sums agree with a context call
 * to rounding, and bitwise with one whose ib_ctx_set_volume_split is 8.  It
 * takes no context: its per-particle partial sums live
 * in a fixed array inside the library, sized for IB_STATIC_VOLUME_MAX_P
 * particles (896 KiB of device memory, held on every device that loads the
 * library until the process exits).
 *  * P > IB_STATIC_VOLUME_MAX_P returns IB_ERR_INVALID (nothing is queued).
 *  * The first call on a device looks up the array's device address (one
 *    cudaGetSymbolAddress per device); make that first call before any
 *    stream capture begins.  No call allocates or frees memory.
 *  * Every call shares the one array and overwrites the part it uses, so
 *    calls that overlap on the GPU (different streams, no ordering between
 *    them) race and give wrong sums: order them on one stream or by events.
 *  * Device-side input checks are not reported (there is no context to
 *    latch them); non-finite inputs give non-finite sums.                  */
#define IB_STATIC_VOLUME_MAX_P 2048
GBIB_API int particle_volume_integrals_static(const ib_grid *grid, const void *u,
                                              const ib_particles *parts,
                                              double *Iu, double *Irxu,
                                              double *vol, void *stream);

/* ---- the fluid step around the forcing, one periodic level --------------
 * Sec. 3.1 on a uniform periodic grid: velocity at cell centres
 * ([3][n2][n1][n0], grid precision), pressure at nodes ([n2][n1][n0], grid
 * precision; node (i, j, k) is the lower corner of cell (i, j, k)).  The
 * gradient of a nodal field at a cell centre averages the four node
 * differences across the cell; the divergence of a cell field at a node is
 * its negative adjoint.  The implicit solves are exact in Fourier space, so
 * every n[a] must be a power of two in [16, 1024] (else IB_ERR_UNSUPPORTED).
 * Workspace: two complex grid fields (predictor), one (projection).
 *
 * fluid_predictor -- Step 1, Eq. (31): writes u_star = u~*,n+1 from
 *   (I - nu dt/2 L) u~* = u^n + dt (-div(u u)^{n+1/2} - grad p^{n-1/2} / rho_f
 *                                   + (nu/2) L u^n + g),   nu = mu / rho_f,
 *   L the 7-point cell Laplacian, div(u u)^{n+1/2} a second-order Godunov edge
 *   extrapolation (monotonized-central limited slopes, upwinded by the Burgers
 *   Riemann solution of the normal states).  u (u^n), p (p^{n-1/2}) are read;
 *   g[3] is a host array.  u_star must not alias u.
 * level_projection -- Step 3, Eqs. (ns_lp1)-(ns_lp3): with V = u / dt +
 *   grad p / rho_f, solves div((1/rho_f) grad p') = div V (exactly, the
 *   divergence-free part's null modes set to 0) and writes
 *   u = dt (V - grad p' / rho_f) (divergence-free to rounding) and p = p'
 *   (p^{n+1/2}), both in place.
 * IB_ERR_INVALID for NULL arrays or rho_f <= 0, mu < 0, dt <= 0, non-finite g. */
GBIB_API int fluid_predictor(ib_ctx *ctx, const ib_grid *grid, const void *u, const void *p,
                             double rho_f, double mu, const double *g, double dt, void *u_star,
                             void *stream);
GBIB_API int level_projection(ib_ctx *ctx, const ib_grid *grid, void *u, void *p, double rho_f,
                              double dt, void *stream);

/* ---- marker force and torque (Eqs. particle1, particle2, first terms) ---
 * F_ib[p] = -rho_f sum_l F[l] dV[l],  T_ib[p] = -rho_f sum_l R[l] x F[l] dV[l]
 * over the markers of particle p; FP64, overwritten.  Each particle's
 * markers are summed in a fixed number of contiguous ranges whose sums are
 * added in order, so the result is deterministic and does not depend on the
 * other particles of the call.  Scratch comes from the context workspace
 * (IB_ERR_OOM when it is short).                                           */
GBIB_API int particle_force_torque(ib_ctx *ctx, const ib_particles *parts,
                          const ib_markers *marks, const double *F,
                          double rho_f, double *F_ib, double *T_ib,
                          void *stream);

/* ---- collision + Newton-Euler + centroid update ------------------------
 * F_c,i = sum_j F_c,ij of Eq. (DKT_model) with delta_ij = X_j - X_i (nearest
 * image), D_c = R_i + R_j + d_c, mass (m_i + m_j)/2, evaluated at X^n; then
 *   U^{n+1} = U^n + dt/(rho_p V_p) [F_ib + rho_f (Iu_new - Iu_old)/dt
 *                                   + (rho_p - rho_f) V_p g + F_c]
 *   W^{n+1} = W^n + dt/I_p [T_ib + rho_f (Irxu_new - Irxu_old)/dt]
 *   X^{n+1} = X^n + dt/2 (U^{n+1} + U^n)                        (Eq. pr2)
 * V_p = 4/3 pi R^3, I_p = 2/5 rho_p V_p R^2.  Ur, Wr, Xr of `parts` are
 * updated in place; Fc_out[P][3] (nullable) receives F_c.                  */
GBIB_API int particle_collide_update(ib_ctx *ctx, ib_particles *parts,
                            const ib_grid *grid, const ib_phys *phys,
                            double dt, const double *F_ib, const double *T_ib,
                            const double *Iu_new, const double *Iu_old,
                            const double *Irxu_new, const double *Irxu_old,
                            double *Fc_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GBIB_H */
