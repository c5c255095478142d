/*
 * schur.h - C ABI of the GB300 Pressure Schur Complement Stokes solver.
 *
 * The method (Pimanov, Iliev, Oseledets, Muravleva, "On the efficient preconditioning
 * of the Stokes equations in tight geometries"):
 *   - a binary voxel image (Section 2.1, eqs. cube_domain, domains_partition) defines
 *     the fluid region; the no-slip wall is the fluid/solid interface (eq.
 *     interior_boundary, eq. stokes_bc_noslip); the exterior box is periodic along
 *     the flagged axes (Section 2.2) and solid along the others;
 *   - the MAC discretisation gives the block system of eq. coupled_matrix with the
 *     no-slip vector Laplacian A and the negative divergence B;
 *   - the pressure solves S p = g with S = B A^-1 B^T, g = B A^-1 f (eqs. schur_system,
 *     schur_rhs) by the preconditioned CG of Algorithm 1, preconditioned by Uzawa
 *     (S-hat = I) or diffusive SIMPLE (S-hat = B diag(A)^-1 B^T), eq. schur_uzawa_prec;
 *   - the velocity follows from A u = f - B^T p (eq. velocity_schur) and the
 *     permeability from Darcy's law (eq. darcy_law) as the box average of u.
 *
 * Conventions shared by every entry point
 *   mask      uint8, C order [z][y][x] (x fastest), 1 = fluid, 0 = solid.
 *   dims      dims[0] = n_x, dims[1] = n_y, dims[2] = n_z (ignored when ndim == 2);
 *             every used extent must be >= 2.
 *   h         voxel size 1 / n_x (unit box length along x, Section 2.3).
 *   faces     face (a, c) is the lower face of cell c along axis a (between cells
 *             c - e_a and c).  Face-space device buffers are laid out [a][stride]
 *             with element (a, c) at a * stride + c; stride is reported by
 *             schur_geometry_info (the cell count rounded up to 64).  Cell-space
 *             buffers hold n_x * n_y * n_z elements in C order.
 *   flags     one byte per face: bit 0 = unknown (both cells fluid), bits 1..3 =
 *             number of solid-solid tangential neighbour faces (ghost walls); 0 on
 *             faces that are not unknowns.
 *   streams   every call runs on the stream given at creation and is stream-ordered;
 *             calls that return values to the host synchronise that stream.
 *   errors    every int-returning call returns 0 (SCHUR_OK) or a SCHUR_E* code and
 *             leaves a message for schur_last_error() (thread-local).  A handle whose
 *             call failed with SCHUR_ECUDA should be destroyed.
 *   threads   one handle must not be used by two host threads at once.
 */
#ifndef SCHUR_H
#define SCHUR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCHUR_OK          0
#define SCHUR_EINVAL      1   /* bad argument (dims, ndim, mask values, axis, null pointer) */
#define SCHUR_ENOMEM      2   /* device allocation failed */
#define SCHUR_ENOTCONV    3   /* an iteration cap was hit; the last iterate is kept */
#define SCHUR_EBREAKDOWN  4   /* CG breakdown: d^T q <= 0 or not finite */
#define SCHUR_ECUDA       5   /* a CUDA runtime call failed */
#define SCHUR_ESTATE      6   /* call out of order (e.g. recover before solve) */

enum { SCHUR_UZAWA = 0, SCHUR_SIMPLE = 1 };
/* Choose per geometry: SIMPLE when its fluid fraction is below SCHUR_AUTO_SIMPLE_BELOW
 * (tight geometries, where Uzawa stagnates: Section 4), Uzawa otherwise.  Accepted by every
 * call that takes schur_opts. */
enum { SCHUR_PRECOND_AUTO = 2 };
#define SCHUR_AUTO_SIMPLE_BELOW 0.25
enum { SCHUR_STOP_UNPRECOND = 0, SCHUR_STOP_PRECOND = 1 };
enum { SCHUR_FP64 = 0, SCHUR_MIXED = 1 };
enum { SCHUR_LOOP_GRAPH = 0, SCHUR_LOOP_HOST = 1 };
/* Preconditioner of the inner A and S-hat solves: Jacobi (the diagonal), or an aggregation
 * multigrid V-cycle (2 x 2 x 2 voxel aggregates, Galerkin coarse operators down to a single
 * cell solved exactly, one weighted-Jacobi sweep before and after the coarse correction);
 * the paper uses BoomerAMG there (Section 3.2). */
enum { SCHUR_INNER_JACOBI = 0, SCHUR_INNER_MG = 1 };
enum { SCHUR_FIELD_P = 0, SCHUR_FIELD_U = 1, SCHUR_FIELD_FLAGS = 2, SCHUR_FIELD_MASK = 3,
       SCHUR_FIELD_G = 4 };
enum { SCHUR_DTYPE_U8 = 0, SCHUR_DTYPE_F32 = 1, SCHUR_DTYPE_F64 = 2 };

typedef struct schur_geom* schur_geom_t;
typedef struct schur_batch* schur_batch_t;
typedef struct schur_server* schur_server_t;

/* Solver options.  Defaults (schur_opts_default): SIMPLE, unpreconditioned stop,
 * FP64, graph loop, tol 1e-8, tol_inner_A = tol_inner_S = 1e-12, max_outer 2000,
 * max_inner 20000; mixed precision: tol_inner_f32 1e-4, refine_factor 1e-3,
 * max_refine 30, step_max 1000; Jacobi inner preconditioner. */
typedef struct {
    int precond;        /* SCHUR_UZAWA | SCHUR_SIMPLE (eq. schur_uzawa_prec) | _PRECOND_AUTO  */
    int stop_norm;      /* SCHUR_STOP_UNPRECOND: ||r_k||/||r_0|| < tol (Section 4.2.2);
                           SCHUR_STOP_PRECOND: ||z_k||/||z_0|| < tol (Algorithm 1)          */
    int precision;      /* SCHUR_FP64: everything in FP64 (Algorithm 1 as in the paper);
                           SCHUR_MIXED: FP32 inner A and SIMPLE solves inside an FP64
                           flexible outer CG (Notay FCG(1)) wrapped in FP64 defect
                           correction; the stop is on the FP64 true residual            */
    int loop_mode;      /* SCHUR_LOOP_GRAPH: one CUDA graph with device-side while loops;
                           SCHUR_LOOP_HOST: the host drives every loop (debugging)         */
    int max_outer;      /* cap on outer iterations (S applications)                         */
    int max_inner;      /* cap on iterations of each inner solve                            */
    double tol;         /* outer relative tolerance eps_S                                   */
    double tol_inner_A; /* inner tolerance eps_A: ||M^-1 r||/||M^-1 r_0|| (Section 3.2)     */
    double tol_inner_S; /* inner tolerance eps_S-hat for the SIMPLE solve (Section 3.2)     */
    double tol_inner_f32;  /* MIXED: tolerance of the FP32 inner solves (default 1e-4)      */
    double refine_factor;  /* MIXED: residual reduction of one refinement step (1e-3)       */
    int max_refine;        /* MIXED: cap on refinement steps (true residuals) (30)          */
    int step_max;          /* MIXED: cap on FCG iterations in one step (1000)               */
    int inner_precond;     /* SCHUR_INNER_JACOBI (default) | SCHUR_INNER_MG: preconditioner of
                              every inner solve of the call (and of the recovery that follows);
                              multigrid inner solves always run as persistent loop kernels   */
} schur_opts;

typedef struct {
    int status;                  /* SCHUR_OK, SCHUR_ENOTCONV, SCHUR_EBREAKDOWN, or
                                    SCHUR_ECUDA when an inner-solve grid barrier wait ran
                                    past its limit (the results are then meaningless)      */
    int outer_iters;             /* S applications in Algorithm 1                          */
    int zero_rhs;                /* 1 when g vanished to rounding and p = 0 was returned   */
    int inner_status;            /* worst status of the inner solves                       */
    long long inner_iters_A;     /* all inner A iterations of the call                     */
    long long inner_iters_S;     /* all inner SIMPLE iterations of the call                */
    double rel_res;              /* ||r_k|| / ||r_0|| at exit                              */
    double rel_res_precond;      /* ||z_k|| / ||z_0|| at exit (NaN when not formed)        */
    double g_norm;               /* ||g||_2                                                */
    long long kernel_launches;   /* kernels this call ran on the GPU                       */
    long long inner_iters_A_f32; /* MIXED: FP32 inner A iterations (inner_iters_A: FP64)   */
    long long inner_iters_S_f32; /* MIXED: FP32 inner SIMPLE iterations                    */
    int refinements;             /* MIXED: refinement steps (FP64 true residuals formed)   */
} schur_stats;

typedef struct {
    int ndim;
    int64_t dims[3];
    int periodic[3];
    int64_t n_cells;             /* n_x n_y n_z                                            */
    int64_t face_stride;         /* stride of face-space buffers (elements)                */
    int64_t n_unknown[3];        /* unknown faces per axis                                 */
    int64_t n_fluid;             /* fluid cells                                            */
    double h;                    /* voxel size 1/n_x                                       */
    int64_t device_bytes;        /* device memory held by the handle                       */
} schur_geom_info;

/* Fill *o with the defaults listed above. */
void schur_opts_default(schur_opts* o);

/* Build a geometry: copies the mask (host or device pointer, detected), builds the face
 * flags on the GPU and allocates all solver state.  ndim is 2 or 3; periodic[a] != 0
 * makes axis a periodic (Section 2.2), otherwise the exterior is solid.  stream is a
 * cudaStream_t (NULL = legacy default stream).  Errors: SCHUR_EINVAL (ndim, dims < 2,
 * mask value not 0/1), SCHUR_ENOMEM, SCHUR_ECUDA.  The handle owns its device memory. */
int schur_create_geometry(const uint8_t* mask, int ndim, const int64_t dims[3],
                          const int periodic[3], void* stream, schur_geom_t* out);

/* Uniform body force f (f[2] ignored in 2D).  Section 2.3: a pressure drop dp over the
 * unit box along axis a is the force f = dp e_a; the default is f = e_x. */
int schur_set_force(schur_geom_t g, const double f[3]);

/* Solve S p = g (eqs. schur_system, schur_rhs) by Algorithm 1 from p_0 = 0.  The
 * residual sign follows standard PCG (r = g - S p).  A right-hand side that vanishes to
 * rounding (||g|| <= 1e-12 || |B| |A^-1 f| ||) returns p = 0 after 0 iterations.
 * stats may be NULL.  Returns SCHUR_OK, SCHUR_ENOTCONV, SCHUR_EBREAKDOWN (the iterate
 * is kept), or SCHUR_EINVAL / SCHUR_ECUDA. */
int schur_solve(schur_geom_t g, const schur_opts* opts, schur_stats* stats);

/* Asynchronous solve + velocity recovery + permeability (graph mode only): one graph
 * launch on the handle's stream, returns at once.  schur_query tells whether it ended;
 * schur_finish waits, fills the stats of the solve and of the recovery (either may be
 * NULL) and returns the solve's status (or the recovery's when the solve succeeded).
 * Other calls on the handle return SCHUR_ESTATE while the solve is in flight. */
int schur_solve_async(schur_geom_t g, const schur_opts* opts);
int schur_query(schur_geom_t g, int* done);
int schur_finish(schur_geom_t g, schur_stats* solve_stats, schur_stats* recover_stats);

/* Velocity recovery A u = f - B^T p (eq. velocity_schur) with the options of the last
 * schur_solve.  SCHUR_ESTATE before any solve. */
int schur_recover_velocity(schur_geom_t g, schur_stats* stats);

/* Darcy permeability along axis a (eq. darcy_law, mu = 1, L = 1): the sum of the
 * recovered u_a over the unknown faces divided by the number of voxels, accumulated in
 * FP64.  Synchronises the stream.  SCHUR_ESTATE before any recovery. */
int schur_permeability(schur_geom_t g, int axis, double* k_out);

/* Diagonal of the permeability tensor (Section 2.3): for each axis a < ndim, a unit body
 * force along a, schur_solve with *opts (NULL: defaults) and schur_recover_velocity on the
 * same handle (flags, components, tables and graphs are shared), then k_out[a] = k_aa;
 * k_out[a] = 0 for a >= ndim.  stats (may be NULL) receives ndim solve stats.  The force
 * is left at the last axis.  Returns the worst status (k_out still written for the axes
 * that converged).  Synchronises. */
int schur_permeability_diag(schur_geom_t g, const schur_opts* opts, double k_out[3],
                            schur_stats* stats);

/* Per-iteration record of the last solve's outer loop (Algorithm 1; in mixed precision
 * the flexible CG steps of all refinements): for outer iteration k < min(*n, cap) the
 * step length alpha_k, the direction coefficient beta_k (NaN when the loop stopped
 * before forming it), ||r_(k+1)|| / ||r_0|| (the recursive residual) and ||z_(k+1)|| /
 * ||z_0|| (NaN when z was not formed).  *n = number of recorded iterations (at most
 * min(max_outer, 131072)).  Any output array may be NULL.  Synchronises.
 * SCHUR_ESTATE before any solve. */
int schur_history(schur_geom_t g, int cap, double* alpha, double* beta, double* rel,
                  double* relz, int* n);

/* Condition-number estimate of the preconditioned Schur operator (S for Uzawa, S-hat^-1 S
 * for SIMPLE) from the outer CG coefficients of the last FP64 solve, as in Section 4.2:
 * the extreme eigenvalues of the Lanczos tridiagonal matrix T[j][j] = 1/alpha_j +
 * beta_(j-1)/alpha_(j-1), T[j][j+1] = sqrt(beta_j)/alpha_j (Saad, Section 6.7.3), by
 * Sturm-sequence bisection on the host.  The Ritz values lie inside the spectrum, so
 * *cond <= the effective condition number; it converges to it as the iteration proceeds.
 * SCHUR_ESTATE after a mixed-precision solve (flexible CG defines no Lanczos matrix) or a
 * solve without outer iterations. */
int schur_cond_estimate(schur_geom_t g, double* lambda_min, double* lambda_max, double* cond);

/* The host computation behind schur_cond_estimate for any CG run: the smallest and
 * largest eigenvalue of the m x m Lanczos tridiagonal built from the step lengths
 * alpha[0..m) (> 0) and direction coefficients beta[0..m-1) (>= 0).  No device work.
 * SCHUR_EINVAL on null pointers, m < 1 or coefficients outside those ranges. */
int schur_lanczos_extremes(const double* alpha, const double* beta, int m, double* lambda_min,
                           double* lambda_max);

/* Borrowed device pointer to a field (valid until the next solve/recover or destroy):
 * P (f64, cells), U (f64, faces), FLAGS (u8, faces), MASK (u8, cells), G (f64, cells). */
int schur_get_field(schur_geom_t g, int which, void** dev_ptr, int64_t* elems, int* dtype);

int schur_geometry_info(schur_geom_t g, schur_geom_info* info);

/* ---- single operators on caller-owned device buffers (FP64) --------------------------
 * Inputs are read only on unknown faces / fluid cells (other entries are ignored);
 * outputs are written everywhere (0 off the unknowns / fluid cells).  Buffers must not
 * overlap.  These run on the handle's stream and do not synchronise. */

/* y = A x: the no-slip vector Laplacian, h^-2 ((2d + g_f) x_f - sum of unknown
 * neighbours) on unknown faces (eq. coupled_matrix, MAC scheme of Section 2.1). */
int schur_apply_A(schur_geom_t g, const double* x, double* y);
/* p = B u = -div_h u on fluid cells. */
int schur_apply_B(schur_geom_t g, const double* u, double* p);
/* u = B^T p = grad_h p on unknown faces. */
int schur_apply_BT(schur_geom_t g, const double* p, double* u);
/* q = S-hat_simple p = B diag(A)^-1 B^T p (eq. schur_uzawa_prec) on fluid cells. */
int schur_apply_simple(schur_geom_t g, const double* p, double* q);
/* x = A^-1 b by Jacobi PCG from 0 with the relative preconditioned residual stop of
 * Section 3.2; *iters (may be NULL) gets the iteration count.  Synchronises. */
int schur_solve_A(schur_geom_t g, const double* b, double* x, double tol, int max_iter,
                  int* iters);

/* Profiling hook: one launch of a hot solver kernel on the handle's stream, bracketed by
 * two CUDA events; *ms receives the elapsed time.  kernel: 0 inner-A direction update,
 * 1 inner-A stencil A p (with p.q), 2 inner-A x/r update (with r.z, z.z), 3-5 the same
 * three for the SIMPLE operator, 6-11 the FP32 versions of 0-5 (after a mixed solve);
 * 12 the persistent inner-A CG kernel that the solver launches (one cooperative launch
 * running SCHUR_TIMED_LOOP_ITERS iterations of all three phases on a fixed right-hand
 * side), 13 the same for the SIMPLE operator, 14-15 their FP32 versions; 16-19 the
 * multigrid-preconditioned CG kernels (A, SIMPLE, A FP32, SIMPLE FP32; after a solve with
 * SCHUR_INNER_MG, which builds the hierarchies: SCHUR_ESTATE otherwise), one launch
 * running SCHUR_TIMED_LOOP_ITERS iterations.  Ids 0-11 time the phases one launch each (the
 * solver itself runs them inside 12-15).  The kernel works on the solver's own buffers
 * (their contents after the last call); results of later calls are unaffected.
 * Synchronises. */
#define SCHUR_TIMED_LOOP_ITERS 20
int schur_time_kernel(schur_geom_t g, int kernel, float* ms);

/* Sizes of the multigrid hierarchy of the inner A operator (simple = 0) or of S-hat
 * (simple = 1), built by the first solve with SCHUR_INNER_MG: *nlev receives the number of
 * levels (0 when not built), sizes[l] (l < min(nlev, max_levels)) the entries of level l
 * (level 0: unknown faces or fluid cells), *tail the first level that the loop kernel runs
 * in one block.  sizes may be NULL. */
int schur_mg_levels(schur_geom_t g, int simple, int64_t* sizes, int max_levels, int* nlev,
                    int* tail);

/* Measured FP64 pipe throughput of the current device (no counterpart in the paper: the
 * roofline denominator of the FP64 kernels).  One launch of a kernel in which every thread
 * of a grid of (SMs x 8) blocks of 256 threads runs 8 independent chains of `iters`
 * dependent DFMAs, timed with CUDA events on `stream` after one warm-up launch;
 * *lane_ops_per_s receives DFMA lane-operations per second (one DFMA = 2 FLOP).  iters in
 * [1, 1 << 20].  Synchronises `stream`. */
int schur_fp64_peak(void* stream, int iters, double* lane_ops_per_s);

/* Launch shape of a geometry's kernels: grids are capped at blocks_per_sm (1..32) x SMs
 * (and at the kernel's resident blocks) and give every thread at least
 * entries_per_thread (1..4096) entries; persistent_inner = 1 runs every inner solve as one
 * cooperative loop kernel, 0 as one graph node per CG phase inside a conditional while
 * node.  Default (8, 1, 1): one wave over the whole GPU, the fastest single solve.
 * Results depend on the shape only through the order of the floating-point reductions;
 * equal shapes give bitwise-equal results.  Drops the recorded graphs (they are rebuilt
 * on the next call).  Errors: SCHUR_EINVAL (range), SCHUR_ESTATE (an asynchronous solve
 * is in flight). */
int schur_set_launch(schur_geom_t g, int blocks_per_sm, int entries_per_thread,
                     int persistent_inner);

/* Bound of the grid-barrier waits inside the persistent inner-solve kernels of this
 * geometry (no counterpart in the paper: the failure path of the cooperative launches).
 * A wait polls the arrival counter at most `polls` times (0: the default, about ten
 * seconds); when it runs out, the kernel sets a sticky flag, every block leaves its loop
 * at its next barrier, the outer loops stop, and the call returns SCHUR_ECUDA with
 * schur_last_error() naming the barrier.  skip_block >= 0 makes that block of every loop
 * kernel leave out its barrier arrivals, so that the other blocks' waits run out: a test
 * hook for the failure path (it faults nothing and every wait still ends); -1 turns it
 * off.  Both settings stay on the handle until changed; the next solve starts with the
 * flag cleared.  Errors: SCHUR_EINVAL (skip_block out of range), SCHUR_ESTATE (an
 * asynchronous solve is in flight). */
int schur_set_barrier_limit(schur_geom_t g, unsigned int polls, int skip_block);

/* Allocation-free Darcy permeability of a caller-owned velocity field (no counterpart in
 * the paper: an entry point for callers that may not allocate device memory, e.g. code
 * running inside a memory pool it does not own or inside an already-captured graph).
 * u and flags are device buffers in the face layout [ndim][face_stride] (FP64 velocity,
 * flag bytes with bit 0 = unknown); dims are n_x, n_y, n_z as for
 * schur_create_geometry.  k_dev is a device array of 3 doubles that receives, for each
 * axis a < ndim, the sum of u_a over the unknown faces divided by the cell count (0 for
 * the other entries).  Runs on `stream` (a cudaStream_t) without synchronising.
 * It calls no cudaMalloc or cudaFree: its scratch is a static device array of 96 KiB
 * held by every device that loads the library until exit, so ndim * face_stride may not
 * exceed 8388608 faces (SCHUR_EINVAL otherwise).  The first call on a device looks up
 * the array's device address (and so does the first call after a device reset, which
 * replaces the context); make that first call before any stream capture.  All calls
 * share the array: calls that overlap on the GPU race and must be serialised. */
int schur_permeability_noalloc(const double* u, const uint8_t* flags, int ndim,
                               const int64_t dims[3], int64_t face_stride, void* stream,
                               double* k_dev);

/* ---- batched execution -------------------------------------------------------------
 * The solve + recovery of n geometries recorded as n parallel branches of ONE CUDA graph
 * (one cudaGraphLaunch runs all of them; the GPU overlaps the branches).  The handles
 * must stay alive and are used on `stream`.  blocks_per_sm in 1..32 gives every geometry
 * the launch shape (blocks_per_sm, 16 entries per thread, persistent inner loops) (see
 * schur_set_launch): small geometries then take a few SMs and the branches overlap;
 * blocks_per_sm = 0 keeps each geometry's current shape.  schur_batch_run launches the
 * graph, waits, and fills n solve / recovery stats and 3n permeabilities (each output may
 * be NULL); it returns the worst status.  schur_batch_autotune times the batch for a few
 * launch shapes (per-phase graph nodes and persistent loops, several grid sizes), leaves
 * the geometries on the fastest and writes it to best_shape = {blocks_per_sm,
 * entries_per_thread, persistent_inner}; create the batch with blocks_per_sm = 0 to run
 * it. */
int schur_batch_create(schur_geom_t* geoms, int n, const schur_opts* opts, int blocks_per_sm,
                       void* stream, schur_batch_t* out);
int schur_batch_run(schur_batch_t b, schur_stats* solve_stats, schur_stats* recover_stats,
                    double* k_out);
int schur_batch_autotune(schur_geom_t* geoms, int n, const schur_opts* opts, void* stream,
                         int best_shape[3], double* best_ms);
void schur_batch_destroy(schur_batch_t b);

/* ---- serving --------------------------------------------------------------------------
 * A request loop driven by the caller: schur_server_submit queues a permeability job
 * (host mask copied; unit force along `axis`); schur_server_progress admits queued jobs in
 * arrival order while their estimated device footprint (schur_footprint_bytes) fits the
 * budget and fewer than max_active run, launches each on its own stream (geometry +
 * asynchronous solve + recovery, launch shape (8, 1, 0) of schur_set_launch: per-phase
 * graph nodes, so that the jobs in flight interleave), and collects finished ones without
 * blocking; schur_server_take returns finished results.  opts->precond may be
 * SCHUR_PRECOND_AUTO (a per-job choice from the host mask's fluid fraction).  With
 * opts->inner_precond = SCHUR_INNER_MG a job's footprint also counts its multigrid
 * hierarchies (16 bytes per fine entry plus coarse levels of at most a seventh of them) and
 * its inner solves run as persistent loop kernels.  Times are seconds since creation. */
typedef struct {
    int64_t id;
    int status;
    int outer_iters;
    int64_t inner_iters;
    double k;                    /* permeability along the job's axis */
    double t_submit, t_start, t_done;
    int64_t bytes;               /* footprint charged to the budget */
    int precond;                 /* preconditioner the job ran with */
    int pad;
} schur_job_result;

/* Upper bound of the device memory of one geometry and its solve (Jacobi inner solves;
 * the server adds the multigrid hierarchies when its solves use them). */
int64_t schur_footprint_bytes(int ndim, const int64_t dims[3], int precision);
int schur_server_create(const schur_opts* opts, int64_t mem_budget_bytes, int max_active,
                        schur_server_t* out);
int schur_server_submit(schur_server_t s, const uint8_t* host_mask, int ndim,
                        const int64_t dims[3], const int periodic[3], int axis,
                        int64_t* job_id);
int schur_server_progress(schur_server_t s, int* n_active, int* n_pending);
int schur_server_take(schur_server_t s, schur_job_result* out, int max, int* n_out);
int schur_server_info(schur_server_t s, int64_t* peak_bytes, int* peak_active);
void schur_server_destroy(schur_server_t s);

/* Release the handle and all its device memory (NULL is ignored). */
void schur_destroy(schur_geom_t g);

/* Message of the last failing call on this thread ("" if none). */
const char* schur_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SCHUR_H */
