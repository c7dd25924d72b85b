/*
 * ppe.h -- C ABI of libppe: the split pressure-gradient projection step of
 * Poblador-Ibanez & Sirignano, "A Volume-of-Fluid method for variable-density,
 * two-phase flows at supercritical pressure" (arXiv 2103.01874), Sec. 5.4,
 * running on one NVIDIA GB300 (sm_103a).
 *
 * The paper states the problem as: given the predicted velocity u* (called u^p
 * in Eq. (29)), the new density rho^{n+1}, the divergence constraint
 * S = div u^{n+1} (Eq. (31)), the pressures p^n, p^{n-1} and dt, find p^{n+1}
 * and u^{n+1}.  With p_hat = 2 p^n - p^{n-1} and rho_0 = min(rho) (Eq. (32)):
 *
 *   L p^{n+1} = D[(1 - rho_0/rho_f) G p_hat] + (rho_0/dt)(D u* - S)     Eq. (34)
 *   u^{n+1}   = u* - dt [G p^{n+1}/rho_0 + (1/rho_f - 1/rho_0) G p_hat]  Eq. (33)
 *
 * G is the cell-to-face difference, D the face-to-cell divergence and L = D G
 * the 7-point Laplacian of the uniform staggered (MAC) mesh (Sec. 5); rho_f is
 * the face density (arithmetic mean of the two cells by default).  Eq. (34) has
 * constant coefficients and is solved directly, without iteration, by a fast
 * Poisson solver (the paragraph after Eq. (34)): real DFT in x, complex DFT in
 * z (both periodic), and a tridiagonal solve per (kx, kz) wavenumber in y
 * (homogeneous Neumann walls).  p^{n+1} is returned with zero mean (the zero
 * mode is dropped, which also removes any mean of the right-hand side).
 *
 * Array layout (every field argument): C order with x fastest,
 *   cell fields (S, rho, p^n, p^{n-1}, p, f) and u, w:  index (k*ny + j)*nx + i,
 *   v (y faces, walls at j = 0 and j = ny):              index (k*(ny+1) + j)*nx + i.
 * u[k][j][i] is the x face between cells i-1 and i (periodic), w[k][j][i] the z
 * face between cells k-1 and k (periodic).  All values are IEEE FP64.
 *
 * Ownership: every field pointer is DEVICE memory owned by the caller, unless
 * the function name ends in _host.  The plan owns its workspace (spectrum,
 * twiddle and tridiagonal tables, reduction scalars) and frees it in
 * ppe_destroy.  Calls are asynchronous on the plan's stream; errors found on
 * the host are returned at once, device-side results (sweeps, residual, rho_0)
 * are read with ppe_get_info, which synchronises the stream.
 *
 * Aliasing: inputs may not alias outputs, except u_out == u, v_out == v,
 * w_out == w (in-place correction) in ppe_correct and ppe_project.
 *
 * Error behaviour: a NULL plan or pointer, dt <= 0, or lengths <= 0 give
 * PPE_ERR_INVALID_ARG; a dimension that is not 2^a 3^b, below 8, above 1024,
 * or an odd nx, gives PPE_ERR_UNSUPPORTED_SIZE; allocation failure gives
 * PPE_ERR_OUT_OF_MEMORY; a CUDA launch error gives PPE_ERR_CUDA.  No call
 * falls back to the host: without a usable GPU every compute call fails.
 */
#ifndef PPE_H
#define PPE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ppe_plan_s* ppe_plan_t;

typedef enum {
    PPE_OK = 0,
    PPE_ERR_INVALID_ARG = 1,
    PPE_ERR_UNSUPPORTED_SIZE = 2,
    PPE_ERR_INCOMPATIBLE_RHS = 3,
    PPE_ERR_OUT_OF_MEMORY = 4,
    PPE_ERR_NOT_CONVERGED = 5,
    PPE_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out (see ppe_get_info) */
    PPE_ERR_CUDA = 7
} ppe_status;

/* Arithmetic of the projection.  Every field crosses the boundary as IEEE
 * FP64.  The stencils -- the Eq. (34) right-hand side, the refinement residual
 * r = f - L p, the p update and the Eq. (33) correction -- run in both forms
 * in double-float pairs (two FP32 numbers carrying about 48 significant bits,
 * relative rounding ~2^-48 = 3.6e-15 per operation), because FP64 issues at
 * about 1/64 of the FP32 rate on this GPU.
 * PPE_FP64: with walls and every dimension <= 512, the transforms and the
 * y solve (a cosine transform) in the same pairs, on the FP32 pipe; otherwise
 * (an outflow top, or 1024-point lines, where pair rounding would exceed 1e-12
 * of the result) the transforms and a tridiagonal y solve in native FP64.
 * PPE_FP32_REFINE: the transforms and the y solve in FP32 inside an iterative
 * refinement whose residual and update are formed in the pairs above. */
typedef enum { PPE_FP64 = 0, PPE_FP32_REFINE = 1 } ppe_precision;

/* Face density rho_f: arithmetic mean (default) or harmonic mean of the two
 * adjacent cells.  The paper's face-average rule, Eq. (35), is stated for
 * interface quantities only; the density rule is a reading of it. */
typedef enum { PPE_FACE_ARITHMETIC = 0, PPE_FACE_HARMONIC = 1 } ppe_face_rule;

/* Top boundary in y (y = ly); the bottom (y = 0) is always a wall.
 * PPE_BC_WALL: no penetration, homogeneous Neumann for p (the default).
 * PPE_BC_OUTFLOW: an open boundary as in the paper's jet cases (Sec. 6): p = 0
 * on the top face, imposed through the ghost value p_ny = -p_{ny-1}; the top
 * face's v is corrected like an interior face (face density: the top cell's),
 * there is no zero mode and no compatibility condition on S, and the y solve
 * is tridiagonal in both precisions.  Not supported by ppe_project_unsplit. */
typedef enum { PPE_BC_WALL = 0, PPE_BC_OUTFLOW = 1 } ppe_bc;

/* Uniform grid, nx x ny x nz cells in a box lx x ly x lz; periodic in x and z,
 * a wall (no penetration, homogeneous Neumann for p) at y = 0 and, by
 * default, at y = ly (see ppe_bc). */
typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;
} ppe_grid;

typedef struct {
    ppe_precision precision;
    ppe_face_rule face_rule;
    double refine_tol;  /* FP32_REFINE: stop once ||f - L p||_inf <= tol ||f||_inf (e.g. 1e-10) */
    int max_sweeps;     /* FP32_REFINE: refinement sweeps after the first FP32 solve (<= 16) */
    double compat_tol;  /* compatibility of the right-hand side with the walls.  The
                         * Neumann problem L p = f is solvable only if mean(f) = 0, i.e.
                         * mean(S) equals the mean wall flux (see ppe_info).  The solve
                         * always drops the mean of f (reported in
                         * ppe_info.f_mean_removed); with compat_tol > 0, ppe_get_info
                         * and ppe_project_host also return PPE_ERR_INCOMPATIBLE_RHS
                         * when |mean(f)| > compat_tol * ||f||_inf.  0: no check.  The
                         * paper has no such check; it follows from the divergence
                         * theorem on the periodic/wall box of Sec. 5. */
    ppe_bc bc_top;      /* top boundary in y (PPE_BC_WALL when opt is NULL) */
} ppe_options;

/* Read back by ppe_get_info after a solve or projection. */
typedef struct {
    int sweeps;           /* refinement sweeps run (0 for PPE_FP64) */
    double rel_residual;  /* FP32_REFINE: last ||f - L p||_inf / ||f||_inf measured; -1 for FP64 */
    double f_max;         /* ||f||_inf of the last right-hand side (-1 if not computed) */
    double rho0;          /* rho_0 used by the last ppe_rhs / ppe_project */
    /* Compatibility of the last assembled right-hand side (NaN if no ppe_rhs /
     * ppe_project ran since the plan was made).  f_mean_removed and s_mean need
     * the sum of f, which the solve forms: after ppe_rhs alone they are NaN. */
    double s_mean;          /* (walls only; NaN with an open top) mean of S over the cells, from the divergence theorem:
                             * sum over cells of D u* keeps only the wall faces and
                             * sum D(beta G p_hat) = 0, so by Eq. (34)
                             * mean(S) = wall_flux_mean - (dt/rho_0) mean(f) */
    double s_absmax;        /* max |S| (float precision) */
    double wall_flux_mean;  /* sum over (i, k) of (v*(ny) - v*(0)) / dy, divided by nx ny nz */
    double wall_vmax;       /* max |v*| on the wall faces (float precision) */
    double f_mean_removed;  /* mean of f (summed in pairs), which the solve drops; the
                             * refinement residual of PPE_FP32_REFINE leaves it out too
                             * unless it is below 2^-40 ||f||_inf (rounding noise) */
} ppe_info;

/* All inputs and outputs of one projection (Eqs. (32)-(34)); device pointers. */
typedef struct {
    const double *u, *v, *w;     /* predicted velocity u* on the faces */
    const double *S;             /* divergence constraint div u^{n+1}, Eq. (31); mean ~ 0 */
    const double *rho;           /* rho^{n+1} at cell centres, > 0 */
    const double *p_n, *p_nm1;   /* p^n, p^{n-1} */
    double rho0;                 /* <= 0: rho_0 = min(rho), computed on the device */
    double dt;                   /* > 0 */
    double *p;                   /* out: p^{n+1}, zero mean */
    double *u_out, *v_out, *w_out; /* out: u^{n+1} (may equal u, v, w) */
    double *f;                   /* optional out: the Eq. (34) right-hand side, or NULL */
} ppe_fields;

/* Create a plan: validate sizes, allocate the workspace with cudaMalloc, build
 * twiddle tables (host FP64, octant-reduced cos/sin) and the tridiagonal
 * elimination tables for every (kx, kz).  `stream` is a cudaStream_t (NULL =
 * legacy default stream).  opt may be NULL (FP64, arithmetic faces, compat_tol
 * 1e-12). */
ppe_status ppe_plan(ppe_plan_t* out, const ppe_grid* g, const ppe_options* opt, void* stream);

/* Re-bind the plan to another stream (for graph capture or serving slots). */
ppe_status ppe_set_stream(ppe_plan_t plan, void* stream);

/* Bytes of device workspace a plan of this grid and options allocates. */
size_t ppe_workspace_bytes(const ppe_grid* g, const ppe_options* opt);

/* Eq. (34) right-hand side f (device, nx*ny*nz).  rho0 <= 0 selects min(rho). */
ppe_status ppe_rhs(ppe_plan_t plan, const double* u, const double* v, const double* w,
                   const double* S, const double* rho, const double* p_n, const double* p_nm1,
                   double rho0, double dt, double* f);

/* Solve L p = f - mean(f) with mean(p) = 0 (device, nx*ny*nz each).  In
 * PPE_FP32_REFINE mode this runs the refinement loop on the device. */
ppe_status ppe_solve(ppe_plan_t plan, const double* f, double* p);

/* Eq. (33) velocity correction.  rho0 <= 0 uses the rho_0 that the last
 * ppe_rhs or ppe_project on this plan computed on the device. */
ppe_status ppe_correct(ppe_plan_t plan, const double* u, const double* v, const double* w,
                       const double* rho, const double* p, const double* p_n, const double* p_nm1,
                       double rho0, double dt, double* u_out, double* v_out, double* w_out);

/* The whole projection: rho_0, Eq. (34) assembly fused with the forward x
 * transform, the solve, and Eq. (33).  Same result as rhs + solve + correct. */
ppe_status ppe_project(ppe_plan_t plan, const ppe_fields* fields);

/* ppe_project with HOST input and output arrays (pinned memory recommended):
 * copies the inputs to plan-owned device buffers (allocated on first use),
 * projects, and copies p, u, v, w (and f if non-NULL) back.  Synchronises the
 * plan's stream before returning, and returns the device-side status as
 * ppe_get_info does. */
ppe_status ppe_project_host(ppe_plan_t plan, const ppe_fields* host_fields);

/* Pipelined form of ppe_project_host for a sequence of projections with host
 * buffers: enqueues the input copies, the projection and the output copies
 * and returns without waiting.  The plan keeps two sets of device staging
 * buffers used in turn, with the input copies on one stream, the projection
 * on the plan's stream and the output copies on a third, so that one call's
 * input copies run while the previous call computes and its outputs travel
 * back.  A call whose staging set is still in use first waits for the call
 * that used it (two calls in flight at most).  The host buffers of a call
 * (pinned memory, for the copies to be asynchronous) must stay untouched and
 * its outputs unread until ppe_host_wait returns.  Returns PPE_ERR_INVALID_ARG
 * on missing arguments or while the plan's stream is capturing, a CUDA or
 * allocation error if enqueueing fails, else PPE_OK; the device-side status of
 * the projections is reported by ppe_host_wait.  Staging: 9 arrays of the grid
 * per set, allocated on first use.  No counterpart in the paper: it is the
 * host-memory interface of the projection step. */
ppe_status ppe_project_host_async(ppe_plan_t plan, const ppe_fields* host_fields);

/* Waits for every ppe_project_host_async call of the plan and returns the
 * first status other than PPE_OK among the calls retired since the previous
 * ppe_host_wait (PPE_ERR_NOT_CONVERGED or PPE_ERR_INCOMPATIBLE_RHS as
 * ppe_get_info reports it for that call; a CUDA error if a wait fails), else
 * PPE_OK.  ppe_get_info afterwards describes the last projection. */
ppe_status ppe_host_wait(ppe_plan_t plan);

/* Eq. (31): the divergence constraint S = div u^{n+1} from the phase-wise
 * quantities (all device arrays of nx*ny*nz cells, cell layout):
 *   S = -(1 - C) comp_g - C comp_l + mdot (1/rho_g - 1/rho_l)
 * with C the liquid volume fraction in [0, 1], comp_f = (1/rho_f) D rho_f/Dt
 * the phase compressibilities, mdot the volumetric phase-change rate (> 0 for
 * liquid turning into gas) and rho_g, rho_l > 0 the phase densities.  Where
 * under_resolved[c] != 0 and 0 < C < 1 (an under-resolved interface cell) S is
 * 0, the paper's treatment of under-resolved regions; under_resolved may be
 * NULL.  When rho is non-NULL it receives the one-fluid density
 * rho_g (1 - C) + rho_l C.  Evaluated in float pairs (relative error < 5e-14), on the
 * plan's stream.  The result is an input of ppe_project (S) and, for the
 * density, of ppe_project and ppe_project_unsplit (rho). */
ppe_status ppe_divergence_constraint(ppe_plan_t plan, const double* C, const double* comp_g, const double* comp_l,
                                     const double* mdot, const double* rho_g, const double* rho_l,
                                     const unsigned char* under_resolved, double* S, double* rho);

/* The unsplit projection, Eqs. (29)-(30) -- the iterative baseline that the
 * split method replaces.  The variable-coefficient equation
 *   D[(1/rho_f) G p] = (D u* - S) / dt
 * (rho_f by the plan's face rule, walls as in ppe_project) is solved by
 * conjugate gradients preconditioned with this plan's constant-coefficient FFT
 * solve (FP32 or FP64 by the plan's precision; the Polak-Ribiere update keeps
 * CG convergent with the FP32 preconditioner), starting from p = 0 and
 * stopping when max|r - mean r| <= tol max|g| (g the right side) or after
 * max_iter iterations; then u^{n+1} = u* - dt G p / rho_f (Eq. (29)).
 * Uses fields->u, v, w, S, rho, dt and writes p (zero mean), u_out, v_out,
 * w_out; p_n, p_nm1, rho0 and f are ignored.  Vectors and the operator are
 * evaluated in float pairs (~48 bits).  The plan allocates 64 bytes per cell
 * on the first call.  Asynchronous on the plan's stream; not capturable
 * (PPE_ERR_INVALID_ARG if the stream is capturing).  tol >= 0,
 * 0 <= max_iter <= 100000. */
ppe_status ppe_project_unsplit(ppe_plan_t plan, const ppe_fields* fields, double tol, int max_iter);
/* Synchronise and read the last unsplit projection's iteration count and
 * relative residual; PPE_ERR_NOT_CONVERGED if it stopped above its tolerance. */
ppe_status ppe_unsplit_info(ppe_plan_t plan, int* iterations, double* rel_residual);

/* Batched projections (many grids of any sizes in one launch).  Each plan
 * (distinct; a plan may appear once per batch) is paired with its fields.
 * ppe_batch_create captures the projections once into a CUDA graph whose
 * independent branches (up to 16, the projections balanced over them by
 * cells, largest first) run concurrently; every ppe_batch_launch then replays
 * the whole batch with one graph launch on `stream`.  The field pointers are
 * baked into the graph: launch again only with the same buffers (their
 * contents may change).  Per-plan results (ppe_get_info) are valid after the
 * caller has synchronised `stream`.  PPE_ERR_INVALID_ARG for n < 1, NULL
 * arrays, a repeated plan or invalid fields; PPE_ERR_CUDA if capture fails. */
typedef struct ppe_batch_s* ppe_batch_t;
ppe_status ppe_batch_create(ppe_batch_t* out, int n, const ppe_plan_t* plans, const ppe_fields* fields,
                            void* stream);
ppe_status ppe_batch_launch(ppe_batch_t batch);
void ppe_batch_destroy(ppe_batch_t batch);
/* One-shot form: create, launch, synchronise `stream`, destroy. */
ppe_status ppe_project_batched(int n, const ppe_plan_t* plans, const ppe_fields* fields, void* stream);

/* Persistent form of the batch: one kernel launch (after a small reset kernel,
 * both in the batch's graph) runs every projection of the batch.  The host
 * lists the (grid, stage, tile) items of all grids in a queue order; resident
 * CTAs take items in that order, and a stage of a grid starts once every tile
 * of the grid's previous stage has counted itself done on the device.  The
 * stages of one grid are those of ppe_project's FP32_REFINE form: rho_0, the
 * constants, the right-hand side of Eq. (34), the x, z, y, z, x passes of the
 * direct solve, then one refinement sweep: the residual and the same five
 * passes, Eq. (33) fused with the new residual, and the loop test.  When a
 * loop test asks for another sweep, the graph's WHILE loop launches the same
 * kernel again over the sweep stages (grids whose test stopped them skip
 * their items), until no grid asks for one; each grid stops as its own
 * refinement would (tolerance reached or max_sweeps applied).  Every plan must
 * be PPE_FP32_REFINE with walls (no outflow top), the LEGACY spectral
 * schedule, 1 <= max_sweeps, and each dimension in {32, 48, 64, 96, 128, 192,
 * 256}; otherwise form PERSISTENT is refused (PPE_ERR_INVALID_ARG).
 *   form          PPE_BATCH_GRAPH (the graph branches of ppe_batch_create),
 *                 PPE_BATCH_PERSISTENT, or PPE_BATCH_AUTO (the library's
 *                 choice: the graph form, the faster on every batch measured).
 *   window,       queue order: grids in windows of `window` (0: all grids in one
 *   stagger       window), stage-major within a window, each window entering
 *                 `stagger` stages after the one before (-1: the default, 2).
 *   ctas_per_sm   resident CTAs per SM (0: as many as fit, at most 3).
 *   wait_seconds  limit of one wait for a stage (0: 2 s).  A wait that runs out
 *                 stops the launch: every CTA stops taking items, the batch's
 *                 status and every plan's ppe_get_info report PPE_ERR_TIMEOUT.
 *   test_unset_wait  non-zero: grid 0's second stage waits on a counter that
 *                 nothing increments, so that the wait runs out (a test of the
 *                 bounded wait; the batch's results are then incomplete).
 *   grain         elements (cells, faces or spectrum values) per queue item: an
 *                 item is a run of up to 255 consecutive tiles of one stage of
 *                 one grid, about `grain` elements in all (0: 65536). */
typedef enum { PPE_BATCH_AUTO = 0, PPE_BATCH_GRAPH = 1, PPE_BATCH_PERSISTENT = 2 } ppe_batch_form;
typedef struct {
  int form;
  int window;
  int stagger;
  int ctas_per_sm;
  double wait_seconds;
  int test_unset_wait;
  int grain;
} ppe_batch_options;
/* ppe_batch_create with options (NULL: the defaults, form AUTO). */
ppe_status ppe_batch_create_ex(ppe_batch_t* out, int n, const ppe_plan_t* plans, const ppe_fields* fields,
                               void* stream, const ppe_batch_options* opt);
/* Synchronise the batch's stream and read the status of its last launch:
 * PPE_ERR_TIMEOUT if a stage wait of the persistent form ran out (then
 * *err_grid and *err_stage name it), else PPE_OK.  *form receives the form the
 * batch took (PPE_BATCH_GRAPH or PPE_BATCH_PERSISTENT), *items the number of
 * items of its first queue (0 for the graph form), *ctas the persistent
 * kernel's CTAs and *launches how many times the last run launched it (1 +
 * the further sweeps); any output pointer may be NULL. */
ppe_status ppe_batch_status(ppe_batch_t batch, int* form, long long* items, int* ctas, int* launches,
                            int* err_grid, int* err_stage);
/* Host-side queue of the persistent form, without device work (a planning
 * and test aid): grids of dims[3 g .. 3 g + 2] = (nx, ny, nz), rho_0 given
 * (rho_given[g] != 0) or reduced; window, stagger and grain as in
 * ppe_batch_options; first = 0 (the whole projection: the first launch) or 8
 * (the sweep stages: a further sweep).  Returns the number of items (-1 if a
 * grid does not qualify or an argument is out of range), and writes
 * min(cap, items) of them to out as (grid, stage, first tile, tiles)
 * quadruples in queue order; need and tiles (either may be NULL) receive, for
 * all 15 stages of every grid (grid after grid), the stage's items and tiles. */
long long ppe_batch_schedule(int n, const int* dims, const int* rho_given, int window, int stagger, int grain,
                             int first, int* out, long long cap, int* need, int* tiles);

/* Synchronise the plan's stream and read the device-side results.  Returns
 * PPE_ERR_NOT_CONVERGED if the refinement stopped above its tolerance, else
 * PPE_ERR_INCOMPATIBLE_RHS if the compatibility test of ppe_options.compat_tol
 * failed for the last solve's f (info is filled in both cases), else PPE_OK. */
ppe_status ppe_get_info(ppe_plan_t plan, ppe_info* info);

/* Wait for the plan's streams (its own and, if ppe_project_host_async was used,
 * its copy streams; pending host-buffer calls complete but their status is
 * dropped), then free the workspace and the staging buffers.  NULL is ignored. */
void ppe_destroy(ppe_plan_t plan);

/* Schedule and launch-shape tuning of a plan (what an autotuner sweeps).
 *   rhs_lines   y-lines per CTA of the right-hand-side kernel: 1, 2, 4 or 8
 *   rhs_planes  z-planes each of its CTAs marches through: 1 .. nz
 *   x_lines     x-lines per CTA of the x transforms: power of two in 1 .. 64
 *   z_cols      kx columns per CTA of the z transforms: 1, 2, 4, 8 or 16
 *   y_cols      kx columns per CTA of the y pass (FP32_REFINE): 1 .. 32, power of two
 *   spectral    schedule of the z and y steps of the solve (PPE_SPECTRAL_*):
 *               LEGACY  three passes (z, y, inverse z) on the spectrum stored
 *                       [kz][j][kx], kx fastest; every plan supports it;
 *               FUSED   one pass per kx plane: a thread-block cluster whose
 *                       shared memory holds the plane (tiles moved by bulk
 *                       tensor copies, y lines read across the cluster's CTAs);
 *               PENCIL  three persistent passes on the spectrum stored
 *                       [kx][kz][j], each tile (32 KB) moved in and out by bulk
 *                       copies (a tensor map for the z tiles) while the previous
 *                       one is transformed.
 *               FUSED and PENCIL serve PPE_FP32_REFINE plans with walls, ny and
 *               nz in {32, 64, 128, 256} and nx/2 a power of two in [16, 512].
 *               LEGACY is the default of every plan; ppe_get_tuning reports
 *               the schedule in use.
 *   y_solve     method of the LEGACY schedule's y step in a PPE_FP32_REFINE plan
 *               with walls (PPE_Y_*): COSINE, the DCT-II, eigenvalue divide and
 *               DCT-III through FFTs; TRIDIAGONAL, the Thomas elimination of the
 *               Neumann system with tabulated multipliers, written as two affine
 *               scans over 16-element segments of each line (ny <= 512), the
 *               singular line kx = kz = 0 solved in FP64.  COSINE is the
 *               default; other plans report and accept COSINE only.
 * The first five are tile sizes and change no result bit.  The schedules run
 * the same arithmetic, but the compiler may contract the FP32 products of the
 * y pass differently, and the two y methods round differently, so their FP32
 * solves can differ in the last bits; the refined results then agree to the
 * refinement's tolerance.
 * ppe_set_tuning returns PPE_ERR_INVALID_ARG (and changes nothing) if a value
 * is outside its range, a schedule is not available for the plan, or a pass
 * would need more than 227 KB of shared memory per CTA.  Synchronises the
 * plan's stream (captured refinement graphs are rebuilt with the new
 * schedule). */
enum { PPE_SPECTRAL_LEGACY = 0, PPE_SPECTRAL_FUSED = 1, PPE_SPECTRAL_PENCIL = 2 };
enum { PPE_Y_COSINE = 0, PPE_Y_TRIDIAGONAL = 1 };
typedef struct {
    int rhs_lines, rhs_planes, x_lines, z_cols, y_cols, spectral, y_solve;
} ppe_tuning;
ppe_status ppe_get_tuning(ppe_plan_t plan, ppe_tuning* out);
ppe_status ppe_set_tuning(ppe_plan_t plan, const ppe_tuning* tuning);

/* Per-kernel timing.  While enabled, every kernel the plan launches is
 * bracketed by two CUDA events on the plan's stream.  ppe_profile_read
 * synchronises the stream, aggregates the records by kernel into `out`
 * (at most max_entries), clears them and returns the number of entries
 * written, or -1 on error.  Adds two event records per launch; meant for
 * measurement runs, off by default. */
typedef struct {
    char name[32];     /* kernel name, e.g. "k_zfft_fwd" */
    int launches;      /* launches recorded */
    double total_ms;   /* summed event-to-event time */
} ppe_kernel_time;
ppe_status ppe_profile(ppe_plan_t plan, int enable);
int ppe_profile_read(ppe_plan_t plan, ppe_kernel_time* out, int max_entries);

/* rho_0 = min(rho) without allocating device memory.  The paper has no
 * counterpart of this entry point: it serves callers that cannot call
 * cudaMalloc -- code whose device memory belongs to another owner's budget (a
 * framework's caching allocator, a serving loop's admission control), where an
 * extra allocation can fail or overrun the budget, and latency-critical code
 * for which cudaMalloc may synchronise the device.  It computes the same value
 * as the reduction ppe_rhs / ppe_project run when rho0 <= 0.
 *   rho       device, n doubles, all > 0 (densities), not NaN;
 *   n         1 <= n <= 67,108,864 (16384 blocks of 4096 cells); larger n
 *             returns PPE_ERR_UNSUPPORTED_SIZE before anything is launched,
 *             n == 0 or a NULL pointer returns PPE_ERR_INVALID_ARG;
 *   rho0_out  device pointer to one double, written asynchronously on `stream`
 *             (a cudaStream_t, NULL = legacy default stream).
 * Scratch: a static __device__ array of about 128 KiB inside libppe (one copy
 * on every GPU that loads the library, held until the process exits).  Every
 * call shares it, so calls that overlap on the GPU race and must be serialised
 * by the caller; each call clears the part that must start at zero.  The first
 * call on each device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.
 * No call allocates: no cudaMalloc, cudaFree or allocating library routine. */
ppe_status ppe_rho0_noalloc(const double* rho, size_t n, double* rho0_out, void* stream);

/* Static text for a status code. */
const char* ppe_strerror(ppe_status status);

/* Returns 1 if nx, ny, nz are supported by ppe_plan, else 0 (host only). */
int ppe_size_supported(int nx, int ny, int nz);

#ifdef __cplusplus
}
#endif

#endif /* PPE_H */
