/*
 * fld.h -- C ABI of the GB300 flux-limited diffusion (FLD) solver.
 *
 * The library solves the discretised flux-limited diffusion equation of
 * Koerner et al., "Flux-Limited Diffusion for Multiple Scattering in
 * Participating Media" (CGF 33(2), 2014), Sec. 5:
 *
 *   [sum_s D_ps phi_s - phi_p sum_s D_ps] / dl^2 = (1 - albedo_p) sigma_p phi_p - j_p   (Eq. 31)
 *
 * over the unknown voxels p of a uniform grid, with the six face neighbours
 * s, D_ps = (D_p + D_s)/2, and the flux-limited coefficient
 * D_p = F(R_p) / max(sigma_p, sigma_eps) (Eq. 33) evaluated from the floored
 * Knudsen number of Eq. 35 and a limiter of Table 2.  The solve is the
 * red-black Gauss-Seidel relaxation with over-relaxation of Algorithm 1.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid      nx x ny x nz unknown voxels of edge h (the paper's dl), voxel
 *           (i, j, k) centred at ((i+1/2)h, (j+1/2)h, (k+1/2)h).  A one-voxel
 *           ghost layer outside the unknowns holds the Dirichlet boundary
 *           values of phi and D; it is never updated by a sweep.
 * Layout    Unpadded fields: nx*ny*nz values, x fastest
 *           (index (k*ny + j)*nx + i).  Padded fields (phi, D incl. ghosts):
 *           (nx+2)*(ny+2)*(nz+2) values, x fastest, unknown (i,j,k) at
 *           ((k+1)*(ny+2) + j+1)*(nx+2) + i+1.
 * Memory    `where` selects FLD_MEM_HOST (ordinary host memory) or
 *           FLD_MEM_DEVICE (memory of the grid's GPU).  Input pointers are
 *           borrowed for the duration of the call only: the library copies
 *           or converts what it needs.  Output pointers must hold the stated
 *           number of values.
 * Ownership A grid owns all device memory it allocates; fld_destroy frees it.
 * Streams   All device work of a grid is ordered on the stream given at
 *           creation (a cudaStream_t passed as void*; NULL = a stream the
 *           library creates and owns).  Calls that return host results
 *           (fld_solve, fld_residual, fld_get_* to host memory) synchronise
 *           that stream; the others only enqueue work.
 * Errors    Every call returns an fld_status; nothing is thrown across the
 *           ABI.  fld_last_error() gives a thread-local text for the last
 *           failure on the calling thread.  A CUDA error is reported as
 *           FLD_ERR_CUDA and leaves the grid usable only for fld_destroy.
 * Threads   A grid must not be used from two threads at once.
 */
#ifndef FLD_H
#define FLD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fld_grid_s *fld_grid;

typedef enum {
    FLD_OK = 0,
    FLD_ERR_INVALID_ARG = 1,   /* bad size, pointer, parameter or input value   */
    FLD_ERR_OOM = 2,           /* device or host allocation failed              */
    FLD_ERR_CUDA = 3,          /* a CUDA call failed                            */
    FLD_ERR_STATE = 4,         /* call order: e.g. solve before set_medium      */
    FLD_ERR_NOT_CONVERGED = 5, /* max_iters reached; result still filled        */
    FLD_ERR_DIVERGED = 6,      /* residual became NaN or infinite               */
    FLD_ERR_NO_DEVICE = 7,     /* no CUDA device / extension unusable           */
    FLD_ERR_TIMEOUT = 8        /* a bounded wait inside a kernel gave up (a TMA
                                  copy that never completed); the state is not
                                  trusted, the grid stays usable                 */
} fld_status;

/* Flux limiters F(R), Table 2 of the paper, plus the CDA constant 1/3. */
typedef enum {
    FLD_LIM_CDA = 0,      /* F = 1/3 (classical diffusion)            */
    FLD_LIM_SUM = 1,      /* F = 1/(3 + R)                            */
    FLD_LIM_MAX = 2,      /* F = 1/max(3, R)                          */
    FLD_LIM_KERSHAW = 3,  /* F = 2/(3 + sqrt(9 + 4 R^2))              */
    FLD_LIM_LARSEN = 4,   /* F = (3^n + R^n)^(-1/n)                   */
    FLD_LIM_LP = 5        /* F = (coth R - 1/R)/R  Levermore-Pomraning */
} fld_limiter;

typedef enum { FLD_MEM_HOST = 0, FLD_MEM_DEVICE = 1 } fld_mem;

/* Arithmetic of the sweeps.
 * FP64  : phi, D and the medium in double precision throughout.
 * FP32  : phi, D and the medium in single precision; the residual check is
 *         evaluated with a double-single (float-float) sum so it is not
 *         limited by cancellation.
 * MIXED : single-precision sweeps until the residual stalls or falls below
 *         fp32_switch; then sweeps that keep phi as a hi/lo float pair
 *         (about 44 significant bits) with FP32-summed updates, until they
 *         stall or reach 3 * tol; then correction sweeps that form each
 *         update from a float-float sum with correctly rounded D.  Reaches
 *         residuals far below the single-precision floor (Sec. 6.2 notes
 *         1e-4 as the practical single-precision limit). */
/* PAIR  : only the middle stage of MIXED -- phi kept as a hi/lo float pair,
 *         updates summed in FP32 with the approximate D of the bulk sweeps. */
typedef enum { FLD_PREC_FP64 = 0, FLD_PREC_FP32 = 1, FLD_PREC_MIXED = 2, FLD_PREC_PAIR = 3 } fld_precision;

/* Iteration scheme.  RED_BLACK: Algorithm 1, the red unknowns (i+j+k even)
 * then the black ones, each update using the newest neighbours and D
 * (Gauss-Seidel order), over-relaxed by omega (Eq. 36).  JACOBI: every
 * unknown from the previous iterate only -- D^k = F(R(phi^k))/sigma' at all
 * unknowns (Eq. 33-35), then phi^{k+1} from phi^k and D^k (Eq. 32) into a
 * second buffer, damped by omega <= 1.  Both have the same fixed point (Eq.
 * 31); Jacobi needs many more iterations and runs in FP32 or FP64 only. */
typedef enum { FLD_SCHEME_RED_BLACK = 0, FLD_SCHEME_JACOBI = 1 } fld_scheme;

typedef struct {
    int limiter;          /* fld_limiter                                             */
    double larsen_n;      /* n of Larsen-n, > 0 (default 2)                          */
    double omega;         /* SOR factor of Eq. 36, 0 < omega < 2; <= 0 selects
                             2/(1 + sin(pi/(n+1))) clamped to [1, 1.98], n the
                             largest extent.  fld_solve keeps the state with the
                             best residual and, if the residual turns non-finite
                             or grows 1000-fold (against the best and the initial
                             residual), returns to it with omega - 1 reduced by
                             3 % (at most 8 times)                                   */
    int local_iters;      /* rounds of Knudsen -> D_p -> phi' per point before the
                             SOR blend, >= 1.  1 is Algorithm 1 as printed; 2 makes
                             each point's update self-consistent in its own D_p,
                             which keeps over-relaxation stable next to vacuum.  The
                             fixed point is the same.                                */
    double tol;           /* stop when Rbar / jbar <= tol (Algorithm 1: 1e-6)        */
    int max_iters;        /* iteration cap (one iteration = red + black pass)        */
    int check_every;      /* iterations between residual evaluations, >= 1; 0: the
                             autotuner's choice (the smallest power of two from
                             32 to 1024 at which one check costs at most 2 % of
                             the iterations between two checks)                */
    double sigma_eps;     /* extinction floor; <= 0 selects 1e-3 / L, L the largest
                             grid extent (Sec. 5)                                    */
    double eps;           /* epsilon of Eq. 35; <= 0 selects 1e-20                   */
    int precision;        /* fld_precision                                           */
    double fp32_switch;   /* MIXED only: residual at which correction sweeps begin;
                             <= 0 selects 2e-5                                       */
    int residual_margin;  /* residual RMS taken over unknowns at least this many
                             voxels from the faces (Sec. 5); default 0              */
    int warm_start;       /* 1: keep the grid's current phi and D (from a previous
                             solve or fld_set_state); 0: initialise them            */
    double phi0, D0;      /* initial phi and D of the unknowns; < 0 selects the
                             paper's eps*jbar*h and eps*h (Algorithm 1)             */
    double phi_b, D_b;    /* Dirichlet ghost values; < 0 selects eps*jbar*h and
                             eps*h                                                   */
    int warmup_iters;     /* iterations run with omega = 1 before over-relaxation
                             starts: over-relaxing the near-zero initial state
                             diverges for omega above ~1.9 on grids of 192^3 and
                             more, the same omega is stable after a short warm-up.
                             -1 (default): 4 x the largest extent on a cold start,
                             0 with warm_start; 0: none; > 0: that many           */
    int medium_bf16;      /* 1: store sigma' and sigma_a' in bfloat16 (8 significant
                             bits) for the single-precision and hi/lo sweeps, which
                             then read 24 instead of 28 bytes per update.  Both are
                             formed in single precision and rounded to nearest
                             (ties to even); every kernel of the solve, including
                             the FP64 residual and the float-float and FP64
                             sweeps, uses the rounded values, so the fixed point
                             is that of the rounded medium.  The rounding moves
                             the medium by at most 2^-8 relative.  0 (default):
                             the single-precision medium.  Not in the paper.  */
    int scheme;           /* fld_scheme (default RED_BLACK).  JACOBI: precision
                             FP32 or FP64, 0 < omega <= 1 (<= 0 selects 1), no
                             warm-up; local_iters does not apply               */
    int nested;           /* cold fld_solve only: start from the solution of
                             `nested` successively 2x coarser problems (medium
                             and source box-averaged as in fld_downsample; the
                             coarsest solved cold to 1e-4, each finer one from
                             its coarser neighbour's phi, blended trilinearly,
                             with D recomputed).  The fixed point is the same;
                             the start removes the smooth error SOR is slowest
                             on.  Coarse edges stay >= 8.  0 (default): the
                             paper's initial state.  Not in the paper.        */
    int anderson;         /* fld_solve, fld_solve_batch and fld_server (per
                             grid): Anderson mixing over the last
                             `anderson` blocks (at most 16; 1 mixes nothing) of
                             check_every sweeps.
                             Each block of red-black sweeps (Algorithm 1) is a
                             map G(phi) with the solution of Eq. 31 as its fixed
                             point; after a block, the next one starts from
                             sum_i a_i G(x_i), sum a_i = 1, with the weights that
                             minimise |sum_i a_i (G(x_i) - x_i)| (Gram matrix
                             reduced on the device, solved on the host; images
                             and mix in float-float).
                             The fixed point is the same; SOR's slow smooth
                             error is removed much faster.  The history restarts
                             after the warm-up, at precision switches and when
                             the safeguard returns to its best state.  If the
                             mixed iteration stalls above tol, the solve returns
                             to its best state and continues with plain sweeps
                             (fld_solve, batch and server alike).  Costs
                             12 bytes per voxel per slot plus 8.  Red-black
                             scheme only (mixed Jacobi sweeps, whose error
                             modes near -1 the mix amplifies, diverged on the
                             oracle).  0 (default): plain red-black SOR.  Not
                             in the paper.                                     */
    int fp64_verify;      /* MIXED only.  1 (default): once the single-precision
                             sweeps (FP32, hi/lo or float-float) bring the
                             residual (D evaluated in single precision) to tol,
                             the state is converted to FP64 and the stop
                             test of Algorithm 1 is taken on the residual of
                             Eq. 37 evaluated entirely in FP64 (D recomputed from
                             phi in double).  If that residual is still above tol
                             -- the single-precision rounding of D leaves a floor
                             of a few 1e-7 on large grids -- FP64 red-black sweeps
                             follow, checked every min(check_every, 16)
                             iterations, until it is at or below tol; the solve
                             then ends in FP64.  0: stop on the single-precision-D
                             residual.                                          */
    int temporal_depth;   /* single-precision and hi/lo red-black sweeps:
                             -1: one launch per colour pass (two unknowns per
                             thread); 1, 2 or 4: temporally blocked launches of
                             T iterations each (TMA-staged 3-D tiles in shared
                             memory with a 2T-cell halo, a z-wavefront of the 2T
                             colour passes; bit-identical to the launched passes,
                             reading each field once per T iterations; costs a
                             second copy of phi, D and the low word of phi);
                             0 (default): chosen per grid shape, sweep family,
                             limiter and medium by the library's autotuner,
                             which times the launched passes (2 and 4 unknowns
                             per thread) and every blocked configuration on the
                             grid itself the first time that combination is
                             solved, keeps the fastest for the process and
                             appends it to a cache file (FLD_TUNE_CACHE, else
                             fld_tune_cache.txt beside the library).  The
                             choice changes the time only, not the result.
                             Not in the paper.                                 */
    int tile_y;           /* rows of the blocked tile: 0 (default) or the one
                             tile of the depth (T = 1: 56 x 32 unknowns, T = 2:
                             56 x 24, T = 4: 48 x 8)                           */
    int cells_per_thread; /* launched passes (temporal_depth -1): 2 unknowns
                             per thread (64-bit loads) or 4 (128-bit loads of
                             every own field and neighbour row; same bits);
                             0 (default): 2, or the autotuner's choice when
                             temporal_depth is 0                               */
    int batch_launch;     /* fld_solve_batch and fld_server.  0 (default): each
                             grid replays its own block graph (the one fld_solve
                             uses) on a stream of a pool of 16, so independent
                             grids run concurrently.  1: in each step the grids
                             in single-precision or hi/lo red-black sweeps whose
                             blocks have the same length run as multi-grid
                             launches: each colour pass is one launch of a
                             persistent kernel whose CTAs walk the work items of
                             every grid in a device table (up to 128 grids a
                             table, up to 8 tables on their own streams), and a
                             block of k iterations is one CUDA graph of 2k such
                             launches, captured once per table and k and replayed
                             whatever grids the table holds.  The same bits
                             either way; on GB300 the per-grid graphs measured
                             faster.  Not in the paper.                        */
} fld_solve_params;

typedef struct {
    int status;            /* fld_status of the solve                               */
    int iterations;        /* total iterations                                      */
    int iterations_fp32;   /* of which single-precision sweeps (FP32 / MIXED)       */
    int iterations_corr;   /* of which float-float correction sweeps (MIXED)        */
    int checks;            /* residual evaluations                                  */
    double rel_residual;   /* last Rbar / jbar                                      */
    double jbar;           /* RMS emission over the unknowns                        */
    double omega;          /* SOR factor used                                       */
    double ms;             /* device time of the solve, CUDA events                 */
    double ms_sweep_fp32;  /* device time inside blocks of single-precision sweeps  */
    double ms_sweep_corr;  /* device time inside blocks of float-float / FP64 sweeps */
    long long kernels;     /* kernel launches the solve issued (incl. graph nodes)  */
    int omega_backoffs;    /* times the solve returned to its best state and
                              reduced omega after the residual diverged         */
    int iterations_mid;    /* MIXED: sweeps with phi as a hi/lo pair and
                              FP32-summed updates (between the two above)       */
    double ms_sweep_mid;   /* device time inside those sweeps                     */
    int iterations_coarse; /* nested: iterations on the coarser grids (summed)    */
    double ms_coarse;      /* nested: their device time (included in ms)          */
    long long updates_coarse; /* nested: their voxel updates                      */
    int anderson_steps;    /* anderson: blocks whose successor started from a mix */
    int anderson_resets;   /* anderson: history restarts (ill-conditioned weights),
                              plus 1 if the mixed iteration stalled above tol and
                              the solve went on without mixing                */
    int iterations_fp64;   /* MIXED with fp64_verify: FP64 sweeps after the
                              float-float phase (counted in iterations too)   */
    double ms_sweep_fp64;  /* device time inside those sweeps                 */
    double rel_residual_single; /* MIXED with fp64_verify: the single-precision-D
                              residual at which the FP64 check was first taken
                              (rel_residual then holds the FP64 value)          */
} fld_solve_result;

/* Fill *p with the defaults: LP limiter, Larsen n = 2, omega auto,
 * local_iters 2, tol 1e-6, max_iters 1000000, check_every 64, paper sigma_eps
 * and eps, MIXED precision, margin 0, cold start, paper initial/ghost values,
 * automatic warm-up, single-precision medium. */
void fld_default_params(fld_solve_params *p);

/* Create a grid of nx*ny*nz unknowns (each >= 1) of edge h > 0 on the
 * current CUDA device.  stream: cudaStream_t or NULL.  *out receives the
 * handle.  Allocates the solver fields on the device (about 40 bytes per
 * voxel; the FP64 fields are added on first FP64 use and the solve's
 * snapshot of its best state on the first fld_solve). */
fld_status fld_create_grid(int nx, int ny, int nz, double h, void *stream, fld_grid *out);

/* Medium: extinction sigma_t >= 0 and albedo in [0, 1] (unpadded, float).
 * Values are validated (NaN, negative sigma, albedo outside [0,1] ->
 * FLD_ERR_INVALID_ARG).  The floor sigma' = max(sigma_t, sigma_eps) and
 * sigma_a' = (1 - albedo) sigma' of Algorithm 1 are formed at solve time. */
fld_status fld_set_medium(fld_grid g, const float *sigma_t, const float *albedo, int where);

/* Emission j >= 0 (unpadded, float): the j_p of Sec. 5, into which the
 * single-scatter source is absorbed.  Replaces the grid's source field. */
fld_status fld_set_source(fld_grid g, const float *j, int where);

/* Copy the grid's source field (after any bake) to j (unpadded, float). */
fld_status fld_get_source(fld_grid g, float *j, int where);

/* Single-scatter source of a directional light (Sec. 3, after Eq. 6):
 * q_ri = L sigma_s T with sigma_s = albedo * sigma_t and T the transmittance
 * towards the light (Eq. 3) marched from each voxel centre with step `step`
 * (<= 0 selects h/2).  dir is the direction the light travels (need not be
 * unit length, not zero).  Light along -z takes an exact column-scan path.
 * accumulate = 0 replaces the source field with q_ri, 1 adds q_ri to it.
 * Needs fld_set_medium. */
fld_status fld_bake_directional(fld_grid g, const double dir[3], double radiance, double step,
                                int accumulate);

/* Single-scatter source of an isotropic point light of power P at pos (world
 * units, may lie outside the grid): q_ri = P sigma_s T / (4 pi max(r, h/2)^2),
 * T marched from the voxel centre towards the light up to the grid boundary. */
fld_status fld_bake_point(fld_grid g, const double pos[3], double power, double step,
                          int accumulate);

/* Set phi and/or D (padded, double; either may be NULL) including the ghost
 * layer, e.g. analytic Dirichlet values or a warm start.  Allocates the FP64
 * fields on first use so that an FP64 continuation keeps the values exactly. */
fld_status fld_set_state(fld_grid g, const double *phi, const double *D, int where);

/* Read phi and/or D (padded, double; either may be NULL) of the current state. */
fld_status fld_get_state(fld_grid g, double *phi, double *D, int where);

/* Run `iterations` red-black iterations (Algorithm 1) with the given
 * parameters and no residual checks.  Initialises phi and D first unless
 * p->warm_start.  Enqueues only. */
fld_status fld_iterate(fld_grid g, const fld_solve_params *p, int iterations);

/* Solve until Rbar/jbar <= p->tol or p->max_iters (Algorithm 1), checking the
 * residual every p->check_every iterations.  r (may be NULL) receives the
 * outcome.  Returns FLD_OK, FLD_ERR_NOT_CONVERGED or FLD_ERR_DIVERGED (r
 * filled in every case), or an error. */
fld_status fld_solve(fld_grid g, const fld_solve_params *p, fld_solve_result *r);

/* Solve `count` independent grids together (not a paper item; the batched
 * form of fld_solve, built on the server below).  Grids are taken in order of
 * size and packed into groups whose per-iteration working set (24 bytes per
 * voxel) fits in 3/4 of the GPU's L2; groups run one after another.  Within a
 * group all grids step together: their iteration blocks run concurrently and
 * their residuals are reduced in one batched pass per check; grids leave as
 * they converge.  Each grid follows
 * exactly the decisions fld_solve would take for it alone (same omega, check
 * schedule, precision switch and safeguard), so its result equals its solo
 * solve.  Precision FP32, MIXED or PAIR (FP64: FLD_ERR_INVALID_ARG).  All grids must
 * live on one device and be distinct; the batch runs on grids[0]'s stream after
 * every grid's prior work finished.  results (may be NULL) receives count
 * entries; there `ms` is the time from the start of the batch to the check at
 * which that grid finished and `kernels` counts the launches of the whole
 * batch.  Returns FLD_OK if every grid converged, else FLD_ERR_DIVERGED if one
 * diverged, else FLD_ERR_NOT_CONVERGED. */
fld_status fld_solve_batch(fld_grid *grids, int count, const fld_solve_params *p, fld_solve_result *results);

/* ---------------------------------------------------------------------------
 * Server: continuous batching of independent solves (not a paper item).
 * A server holds a changing set of grids being solved with one set of
 * parameters (FP32, MIXED or PAIR).  fld_server_add admits a grid (medium
 * and source already set): it is initialised, its first residual evaluated,
 * and it joins the next step.  Each fld_server_step runs one block of
 * p->check_every iterations (the grid's tuned interval when it is 0) for every
 * active grid -- each grid replays its own block graph on a stream of a pool
 * of 16, so grids run concurrently, or with p->batch_launch = 1 grids in the
 * same single-precision family and block length share multi-grid launches --
 * then evaluates the
 * residuals of all active grids in one batched reduction and applies each
 * grid's own decisions (tolerance, precision switch, safeguard), exactly as
 * fld_solve would for that grid alone; finished grids leave the set and are
 * reported (tag + fld_solve_result, `ms` = time from admission to finish).
 * While in the server a grid's work is ordered on the server's stream; it
 * returns to its own stream when it finishes.  A grid must not be used
 * elsewhere while it is in a server.
 * ------------------------------------------------------------------------- */
typedef struct fld_server_s *fld_server;

/* Create a server for the given parameters (copied).  stream: cudaStream_t
 * or NULL (the server creates one). */
fld_status fld_server_create(const fld_solve_params *p, void *stream, fld_server *out);

/* Admit grid g under a caller-chosen tag.  Synchronises g's stream. */
fld_status fld_server_add(fld_server s, fld_grid g, long long tag);

/* One step (see above).  Up to `capacity` finished grids are reported in
 * tags[] / results[] and counted in *nfinished; more are kept for the next
 * call.  With no active grid, only pending reports are returned. */
fld_status fld_server_step(fld_server s, long long *tags, fld_solve_result *results, int capacity,
                           int *nfinished);

/* Number of grids still iterating. */
fld_status fld_server_active(fld_server s, int *count);

/* Voxel updates (one phi_p update each; one red-black iteration of an
 * nx*ny*nz grid is nx*ny*nz of them) the server's steps have performed so far,
 * over all grids, finished or not: the work a loaded server gets done, which
 * its finished results alone understate. */
fld_status fld_server_updates(fld_server s, long long *updates);

/* Destroy the server (grids still inside return to their own streams, their
 * state as left by the last step). */
void fld_server_destroy(fld_server s);

/* Relative residual Rbar/jbar of the current phi (Eq. 37 with D recomputed
 * from phi, RMS over the unknowns beyond p->residual_margin), evaluated in
 * the arithmetic of p->precision with an accurate sum.  Synchronises. */
fld_status fld_residual(fld_grid g, const fld_solve_params *p, double *rel);

/* Allocation-free residual.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need the
 * residual -- e.g. a renderer that runs the solver inside its frame loop,
 * where cudaMalloc/cudaFree are banned after start-up because they
 * synchronise the device, or a host application that owns all device memory
 * through its own pool and only lends the library its buffers.
 *
 * Computes the same quantity as fld_residual with FLD_PREC_FP64 (Rbar/jbar of
 * Eq. 37, D recomputed from phi, RMS over the unknowns beyond
 * p->residual_margin; p->limiter, larsen_n, sigma_eps, eps also apply) from
 * caller-owned DEVICE buffers: sigma_t, albedo, j unpadded floats; phi and D
 * padded doubles (only the ghost layer of D is read).  *rel is a host
 * double.  All work is enqueued on `stream` (a cudaStream_t, NULL = legacy
 * default stream), which the call then synchronises.
 *
 * Scratch: a fixed array of 2*FLD_NOALLOC_MAX_BLOCKS + 8 doubles (1 MiB + 64
 * bytes) in the library's device memory image, present on every GPU that
 * loads the library until the process exits.  The call launches one block
 * per 32x8 tile of an x-y plane, so grids with
 * ceil(nx/32)*ceil(ny/8)*nz > FLD_NOALLOC_MAX_BLOCKS (and nz > 65535) are
 * rejected with FLD_ERR_INVALID_ARG; 256^3 fits exactly.  No cudaMalloc,
 * cudaFree or other allocating routine is called.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array: calls whose work
 * overlaps on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  Each call writes every slot it reads, so no
 * state carries over between calls. */
#define FLD_NOALLOC_MAX_BLOCKS 65536
fld_status fld_residual_noalloc(int nx, int ny, int nz, double h, const fld_solve_params *p,
                                const float *sigma_t, const float *albedo, const float *j,
                                const double *phi, const double *D, double *rel, void *stream);

/* Primary ray march of the rendered image (Sec. 3): each pixel's radiance is
 * the background attenuated over the ray's chord through the grid's box
 * [0, nx h] x [0, ny h] x [0, nz h] plus, over march segments of length
 * `step`, the transmittance between the segment and the camera times
 * Q x step, with 4 pi Q = q + sigma_s phi (Sec. 3: q = the grid's source
 * field, i.e. q_ri + j after a bake; sigma_s = albedo sigma_t, raw; phi =
 * the grid's current fluence).  Fields are blended trilinearly between voxel
 * centres (clamped to the outermost centres) at each segment's midpoint; the
 * last segment ends at the exit; the transmittance to a segment covers the
 * segments before it.  The march stops where the transmittance falls below
 * t_min.  The camera is a pinhole at `eye` looking at `target`; `up` fixes
 * the roll; rows run top to bottom.  Not fixed by the paper: the camera
 * model, the trilinear sampling and the segment placement. */
typedef struct {
    double eye[3], target[3], up[3];
    double fov_deg;        /* vertical field of view, in (0, 180) degrees        */
    int width, height;     /* pixels, 1 .. 16384 each                            */
    double step;           /* segment length; <= 0 selects h / 2                 */
    double background;     /* radiance entering the far end of every ray, >= 0   */
    double t_min;          /* stop below this transmittance; < 0 selects 1e-6    */
} fld_camera;

/* Render the grid (needs a medium, a source and a state, e.g. after
 * fld_solve).  phi_grid: NULL to take phi from g itself, or a coarser grid
 * covering g's box whose solved phi is blended trilinearly (between its
 * voxel centres) to g's voxel centres before the march -- the
 * quarter-resolution solve of Sec. 6.2 (see fld_downsample).  radiance:
 * width*height floats, row-major, or NULL; codes:
 * width*height bytes of round(255 min(1, (exposure L)^(1/gamma))), the gamma
 * compression of Sec. 6.2, or NULL (one of the two must be given).  `where`
 * (fld_mem) applies to both outputs; with host outputs the call returns when
 * they are written.  Keeps a 16-byte-per-voxel sampling volume with the
 * grid, and for host outputs a device staging image of 5 bytes per pixel,
 * grown only for a larger image (a render loop allocates nothing after its
 * first frame).  Errors: FLD_ERR_INVALID_ARG for a bad camera, exposure <= 0 or
 * gamma <= 0; FLD_ERR_STATE without a medium or a state. */
fld_status fld_render(fld_grid g, fld_grid phi_grid, const fld_camera *cam, float *radiance, unsigned char *codes,
                      double exposure, double gamma, int where);

/* Quarter-resolution solve (Sec. 6.2: phi is solved on a grid with a quarter
 * of the data's resolution per axis, the multiply scattered light being much
 * smoother than the medium): set the coarse grid's medium and source from
 * the fine grid's by box averages over factor^3 blocks -- sigma_t and the
 * source averaged, the albedo as mean(albedo sigma_t) / mean(sigma_t) (0 in
 * vacuum); partial blocks at the far faces average the voxels that exist.
 * coarse must have ceil(n / factor) voxels per axis and spacing factor * h.
 * The paper gives no averaging rule: the box average is this library's.
 * Errors: FLD_ERR_INVALID_ARG for mismatched grids, FLD_ERR_STATE without a
 * fine medium. */
fld_status fld_downsample(fld_grid fine, fld_grid coarse, int factor);

/* Free the grid and everything it owns (NULL is ignored). */
void fld_destroy(fld_grid g);

/* Static text for a status code. */
const char *fld_status_string(fld_status s);

/* Thread-local description of the last failure on this thread ("" if none). */
const char *fld_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FLD_H */
