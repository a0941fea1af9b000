/*
 * ohm.h -- C ABI of libohm, a single-GPU (GB300, sm_103a) solver for one implicit step of
 * ohmic dissipation, dB/dt = -curl(eta curl B), on a block-structured AMR hierarchy of
 * 8^3-cell blocks (T. Matsumoto 2011, "An Implicit Scheme for Ohmic Dissipation with
 * Adaptive Mesh Refinement", Sec. 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named *_dev are CUDA device pointers; everything else is host memory.
 * - Vector fields are contiguous float64 arrays [nblocks][3][8][8][8] in the order of the
 *   descriptor's block list, innermost index along x ([comp][k][j][i]); eta is
 *   [nblocks][8][8][8].  The caller owns these buffers; the library never frees them.
 * - The hierarchy owns every scratch buffer.  It allocates them once, in
 *   ohm_create_hierarchy; no other call allocates device memory.
 * - Work is issued on the stream given in the descriptor (NULL = the legacy default
 *   stream).  Calls that return norms or convergence data synchronise that stream.
 * - Every entry point returns OHM_OK (0) or a negative status and never throws.  Arguments
 *   are validated before any work is issued: on OHM_ERR_INVALID nothing was modified.
 * - Periodic boundaries on all sides (every test of Sec. 3 is periodic).
 */
#ifndef OHM_H
#define OHM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OHM_OK                 0
#define OHM_ERR_INVALID       -1  /* bad descriptor, nesting, size, dt <= 0, NULL pointer   */
#define OHM_ERR_NOT_CONVERGED -2  /* max_outer cycles ran; B holds the last iterate       */
#define OHM_ERR_NONFINITE     -3  /* a residual norm became NaN or Inf                      */
#define OHM_ERR_OOM           -4  /* device allocation failed in ohm_create_hierarchy      */
#define OHM_ERR_CUDA          -5  /* a CUDA call or kernel launch failed                    */

#define OHM_FP64  0  /* every kernel in float64                                             */
#define OHM_MIXED 1  /* multigrid in float32 inside float64 defect correction: the residual
                        R = S - L B, the update B += e, refluxed fluxes and norms stay float64 */
#define OHM_MIXED_FF 2 /* as OHM_MIXED, but the outer residual R = S - L B is evaluated in
                        float-float arithmetic (pairs of float32, about 48 significant bits,
                        on the float32 pipe, which GB300 issues 58x faster than float64) and
                        its norms are accumulated in float32.  B and the update stay float64.
                        The relative residual it can certify is about
                        2^-48 (1 + 12 lambda dt eta_max / dx^2) (2e-13 for dt = 100x the
                        explicit limit).  B, eta and R must lie within the float32 range (|values| <
                        2^64 keeps the squared norms finite); values below 2^-126 count as
                        zero, NaN and values beyond 2^128 end the step with
                        OHM_ERR_NONFINITE.  Refluxed fluxes stay float64.                    */
#define OHM_MIXED_FF_CHECKED 3 /* as OHM_MIXED, but an intermediate outer residual (one that the
                        preceding correction is not expected to bring below tol: it only sets
                        the next inner solve's right-hand side) is evaluated in float-float as
                        under OHM_MIXED_FF; the source, the first residual and every residual
                        that ends a step stay float64, and a float-float residual that meets tol
                        is re-evaluated in float64 before the step ends (the range limits of
                        OHM_MIXED_FF apply to the intermediate residuals).  Batched hierarchies
                        (n_instances >= 1) evaluate every outer residual in float64, as
                        OHM_MIXED                                                            */

typedef struct ohm_hier ohm_hier;

/* The problem statement of Sec. 2.1 (Eqs. 7, 12-14): unknown B^{n+1} given b = B^n, eta,
 * dt and the theta parameter lambda, on a hierarchy of cubic cells. */
typedef struct {
    int32_t base_cells[3];      /* level-0 cells along x, y, z; each a positive multiple of 8  */
    double dx0;                 /* level-0 cell width; level l has dx0 / 2^l                   */
    int32_t nlevels;            /* 1 + number of refinement levels (ratio 2), at most 8        */
    int64_t nblocks;            /* blocks over all levels                                      */
    const int32_t *block_lijk;  /* host, 4 int32 per block: level, bi, bj, bk.  Sorted by
                                   level (level 0 first).  Level 0 must tile the base grid; a
                                   refined block has all 8 children; the 26 neighbours of a
                                   refined block's parent exist (proper nesting).  Copied.     */
    double lambda;              /* theta parameter of Eq. 7: 0.5 Crank-Nicolson, 1 backward
                                   Euler; any value in (0, 1]                                  */
    int32_t precision;          /* OHM_FP64, OHM_MIXED, OHM_MIXED_FF or OHM_MIXED_FF_CHECKED   */
    int32_t nu_pre, nu_post;    /* red-black sweeps before / after coarse correction (>= 0):
                                   on every grid, or on level 0 and the refined levels when
                                   nu_coarse_pre / nu_coarse_post are set                      */
    int32_t n_coarse;           /* red-black sweeps on the coarsest grid (>= 1)               */
    int32_t max_outer;          /* V-cycles allowed per step (>= 1)                           */
    int32_t krylov;             /* 0 = the paper's defect correction with the V-cycle (Eqs.
                                   16-18: the float32 inner solve of mixed precision, or one
                                   float64 V-cycle per outer iteration); m in 1..11 = FGMRES(m)
                                   right-preconditioned by the same V-cycle (not in the paper;
                                   same converged solution, fewer cycles): the float32 inner
                                   solve of mixed precision, or under OHM_FP64 one float64
                                   FGMRES solve to the step's tolerance per outer iteration
                                   (batched hierarchies: mixed precision only).                 */
    double inner_tol;           /* OHM_MIXED(_FF): each float32 inner solve reduces its residual by
                                   max(inner_tol, 0.3 tol / current ||R||/||S||); 0 selects
                                   1e-5.  Values below ~1e-6 ask more than float32 can give: the
                                   inner solve then stops when it stagnates.                   */
    int32_t n_instances;        /* 0: one problem, stepped by ohm_cn_step.  K >= 1: a batch of K
                                   independent problems with the block structure above (each
                                   its own eta, dt and convergence), stepped together by
                                   ohm_cn_step_batch; every kernel launch covers all K.  Field
                                   arrays then hold, level by level, the K instances' blocks
                                   of that level one instance after another (for one-level
                                   hierarchies: instance after instance).  With krylov = m
                                   each instance runs its own FGMRES(m) recurrence.             */
    int32_t use_graphs;         /* batches only: 1 = the defect-correction inner iteration
                                   (V-cycle, update and residual) and, with krylov > 0, every
                                   FGMRES restart cycle are captured once into a CUDA graph and
                                   replayed.  Needs a non-NULL stream; ignored otherwise.      */
    void *stream;               /* cudaStream_t used for all work, NULL = legacy default      */
    double omega;               /* relaxation factor of the red-black sweeps: each colour update
                                   becomes e + omega (e_GS - e) (red-black SOR).  0 selects 1,
                                   the paper's Gauss-Seidel (Eq. 19); allowed in (0, 2).  Not in
                                   the paper: it changes the iterates, not the converged
                                   solution (1.2 saves 2 of 15 V-cycles per step of the 256^3
                                   resistive bump; 1.5 and above slow convergence down).       */
    int32_t nu_coarse_pre, nu_coarse_post; /* red-black sweeps before / after the coarse
                                   correction on the grids coarser than level 0 (the base grid's
                                   coarsenings and the coarsest-grid solver's grids); both 0 =
                                   nu_pre / nu_post on every grid, the paper's single schedule.
                                   Not in the paper (V(3,2) on level 0 with V(1,1) below takes
                                   the 256^3 step 5% faster with the same V-cycle count).       */
} ohm_hier_desc;

typedef struct {
    int32_t cycles;             /* V-cycles applied (Eqs. 16-18 iterations)                   */
    int32_t converged;          /* 1 when ||R||/||S|| <= tol was reached                       */
    double rel_l2_initial;      /* ||S - L b||_2 / ||S||_2 before the first cycle             */
    double rel_l2;              /* final ||R||_2 / ||S||_2 (leaf cells, volume weighted)       */
    double max_abs;             /* final max over leaf cells and components of |R| (Sec. 3.1) */
} ohm_step_stats;

/* Builds the block tables, the multigrid grids below level 0 (coarsened by 2 while every
 * dimension is even and >= 4) and allocates all device scratch.  *out receives the handle
 * (NULL on failure).  Any base grid of multiples of 8 is accepted: the coarse grids below the
 * last one made of 8^3 blocks (under OHM_MIXED* also power-of-two grids of at most 16^3
 * cells) are stepped by grid-wide launches while they have more than 16384 cells and by a
 * one-thread-block solver below that (in shared memory where the grids fit). */
int ohm_create_hierarchy(const ohm_hier_desc *d, ohm_hier **out);

/* Copies eta (> 0 and finite, [nblocks][8][8][8], every block including covered ones) into
 * the hierarchy and derives the coarse-fine eta ghosts and the multigrid eta (mean of the 8
 * children, Sec. 2.2).  When eta is already set and the new values are bit-identical, only the
 * comparison runs (one pass over eta and a wait for its result) and the derived data are kept.
 * Returns OHM_ERR_INVALID for a NULL pointer. */
int ohm_set_eta(ohm_hier *h, const double *eta_dev);

/* One theta-scheme step, Sec. 2.1-2.3: S = b - (1-lambda) dt div f(b) (Eq. 14), then
 * R = S - L B and B += MG(0, R) (Eqs. 16-18) from B = b until ||R||/||S|| <= tol or
 * max_outer cycles.  B_dev is in/out: b on entry, B^{n+1} on return, with covered cells set
 * to the mean of their children.  eta_dev may be NULL to keep the current eta; otherwise it
 * is set first as by ohm_set_eta.  tol < 0 runs exactly max_outer cycles (fixed schedule).
 * stats may be NULL.  Returns OHM_OK, OHM_ERR_NOT_CONVERGED (B = last iterate),
 * OHM_ERR_NONFINITE, OHM_ERR_INVALID (dt <= 0, no eta set, NULL B) or OHM_ERR_CUDA. */
int ohm_cn_step(ohm_hier *h, double *B_dev, const double *eta_dev, double dt, double tol,
                ohm_step_stats *stats);

/* R = S - L B (Eq. 20) for the S and dt of the most recent ohm_cn_step: *rel_l2 receives
 * ||R||_2/||S||_2 over leaf cells (volume weighted), *max_abs the largest |R| component.
 * B_dev is read only (its covered cells are not used).  OHM_ERR_INVALID before any step. */
int ohm_residual_norm(ohm_hier *h, const double *B_dev, double *rel_l2, double *max_abs);

/* Batched step (n_instances = K >= 1; not in the paper, which solves one hierarchy): the step
 * of ohm_cn_step for every instance q with active[q] != 0 (active NULL = all), instance q
 * with its own dt[q] (host array of K) on the same tol.  Each instance is iterated and
 * stopped on its own residual norms (volume weighted over its own leaf cells), and its
 * result does not depend on which other instances are in the batch or active: the work of
 * every launch is per block and every reduction is per instance in a fixed order, so an
 * instance gives the same bits alone (K = 1) as in any batch.  Inactive instances are left
 * untouched.  stats (host array of K, may be NULL) receives each instance's statistics
 * (inactive ones zeroed).  Returns OHM_OK when every active instance converged (or tol < 0),
 * OHM_ERR_NOT_CONVERGED / OHM_ERR_NONFINITE when one did not, OHM_ERR_INVALID for a bad
 * argument, a hierarchy that is not a batch or no eta set. */
int ohm_cn_step_batch(ohm_hier *h, double *B_dev, const double *dt, double tol, const uint8_t *active,
                      ohm_step_stats *stats);

/* Device bytes that ohm_create_hierarchy would allocate for d (tables and scratch; the
 * caller's B and eta not included), without allocating.  OHM_ERR_INVALID as for create. */
int ohm_hierarchy_bytes(const ohm_hier_desc *d, int64_t *bytes);

/* ---------------------------------------------------------------------------------------
 * Autotuner (not in the paper): picks the multigrid schedule of a hierarchy by timing real
 * steps.  Candidates: (nu_pre, nu_post) in {(1,1), (2,1), (2,2), (3,2), (3,3), (4,4)} (the paper's
 * Table 1 uses 2/2 on the base grid and 4/4 on AMR levels) x n_coarse in {4, 16} x smoother
 * in {fused red+black sweep, two colour passes} (the fused sweep stages a 12^3 tile, the
 * two-pass smoother a 10^3 tile).  Each candidate runs one step of ohm_cn_step (batches:
 * ohm_cn_step_batch with dt) from B_dev on a private copy (B_dev is not modified), timed
 * with CUDA events; candidates that do not converge are discarded.  The best schedule is
 * then timed with V(1,1) and V(1,0) on the grids coarser than level 0, then with the relaxation
 * factors omega in {1, 1.15, 1.3, 1.45} besides the hierarchy's own.
 * The fastest is kept in the hierarchy and reported.  Allocates one copy of B for the duration of the call.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int32_t nu_pre, nu_post, n_coarse;
    int32_t smoother;           /* 0 = fused red+black sweep, 1 = two colour passes            */
    double ms;                  /* time of the chosen candidate's step                         */
    int32_t candidates;         /* candidates timed                                            */
    double omega;               /* chosen relaxation factor                                    */
    int32_t nu_coarse_pre, nu_coarse_post; /* chosen coarse-grid sweeps (0, 0 = as nu_pre/post)  */
} ohm_tune_result;
int ohm_autotune(ohm_hier *h, const double *B_dev, const double *dt, double tol, ohm_tune_result *res);

void ohm_destroy(ohm_hier *h);
const char *ohm_status_string(int status);

/* ---------------------------------------------------------------------------------------
 * Row-level entry points: each runs one step of the hot path on caller buffers, so every
 * step can be compared with an independent implementation.  Same layouts and status codes
 * as above; all are stream ordered and synchronise only where they return host scalars.
 * ------------------------------------------------------------------------------------- */

/* Composite flux divergence (Eqs. 4-11 and 8) on leaf cells: covered cells are first set to
 * the mean of their children in a private copy, coarse-fine ghosts are interpolated from
 * the parent level, and coarse faces at coarse-fine interfaces take the mean of the four
 * fine fluxes (refluxing, Sec. 4).  out_dev receives 0 on covered blocks. */
int ohm_op_div_flux(ohm_hier *h, const double *B_dev, double *out_dev);

/* S = b - (1 - lambda) dt div f(b) on leaf cells (Eq. 14), same rules as ohm_op_div_flux. */
int ohm_op_source(ohm_hier *h, const double *b_dev, double dt, double *S_dev);

/* R = S - B - lambda dt div F(B) on leaf cells (Eqs. 13, 20); norms (host, may be NULL)
 * receives {||R||/||S||, max|R|, ||R||, ||S||} over leaf cells. */
int ohm_op_residual(ohm_hier *h, const double *B_dev, const double *S_dev, double dt,
                    double *R_dev, double *norms);

/* Covered cells := mean of their 8 children, finest level first, in place. */
int ohm_op_sync_down(ohm_hier *h, double *B_dev);

/* One multigrid V-cycle from a zero guess for the composite residual R_dev (leaf cells):
 * e_dev receives the correction on leaf cells and 0 on covered blocks.  OHM_FP64 only. */
int ohm_op_vcycle(ohm_hier *h, const double *R_dev, double dt, double *e_dev);

/* Shape of base multigrid grid m (0 = level 0): dims[3] cells, *nblocks its 8^3 blocks
 * (0 when the grid lives in lexicographic [comp][z][y][x] layout inside the coarsest-grid
 * solver: not a multiple of 8, or under OHM_MIXED* a power-of-two grid of at most 16^3 cells); when ijk is not NULL it receives 3 int32 per
 * block (bi, bj, bk) in the grid's storage order (the caller's order for m = 0). */
int ohm_mg_grid_info(ohm_hier *h, int m, int32_t dims[3], int64_t *nblocks, int32_t *ijk);

/* Single-grid steps on blocked base multigrid grid m (OHM_FP64; arrays in that grid's
 * block layout; eta_dev [nblocks][8][8][8]):
 *   smooth:  one red-black colour pass (Eq. 19 with alpha from Eqs. 21-23) in place on e,
 *            relaxed by the hierarchy's omega: e + omega (e_GS - e);
 *   residual: t = r - (e + lambda dt div F(e));
 *   restrict: coarse grid m+1 (blocked) = mean of 8 children of fine grid m, ncomp comps;
 *   prolong_add: fine grid m += trilinear interpolation of coarse grid m+1 (blocked). */
int ohm_op_grid_smooth(ohm_hier *h, int m, double *e_dev, const double *r_dev,
                       const double *eta_dev, double dt, int colour);
int ohm_op_grid_residual(ohm_hier *h, int m, const double *e_dev, const double *r_dev,
                         const double *eta_dev, double dt, double *t_dev);
int ohm_op_grid_restrict(ohm_hier *h, int m, const double *fine_dev, double *coarse_dev, int ncomp);
int ohm_op_grid_prolong_add(ohm_hier *h, int m, const double *coarse_dev, double *fine_dev);

/* Float32 single-grid steps of the mixed-precision inner solve (OHM_MIXED / OHM_MIXED_FF
 * hierarchies; the same grids, layouts and rules as above, every array float32), each run by
 * the kernel the V-cycle launches on that grid:
 *   sweep_f32: one full red-black sweep (Eq. 19 with alpha from Eqs. 21-23; the red colour pass
 *              from the pre-sweep state, then the black pass from the post-red state, each
 *              update relaxed by the hierarchy's omega) from e_in (NULL = from e = 0, the first
 *              pre-smoothing sweep of a level) into e_out; variant 0 = the fused red+black sweep
 *              (block pairs where the grid's blocks pair up along x, else single blocks),
 *              variant 1 = two colour passes;
 *   resid_restrict_f32: t = r - (e + lambda dt div F(e)) (Eq. 20 on the grid) into t_dev and its
 *              restriction (mean of the 8 children, Sec. 2.2) into coarse_dev, either may be
 *              NULL; coarse_dev has grid m+1's layout: blocked, or lexicographic
 *              [3][nz][ny][nx] when grid m+1 is below the last blocked grid;
 *   prolong_add_f32: fine grid m += trilinear interpolation of grid m+1 (Sec. 2.2; grid m+1
 *              blocked or lexicographic as above). */
int ohm_op_grid_sweep_f32(ohm_hier *h, int m, const float *e_in_dev, float *e_out_dev, const float *r_dev,
                          const float *eta_dev, double dt, int variant);
int ohm_op_grid_resid_restrict_f32(ohm_hier *h, int m, const float *e_dev, const float *r_dev, const float *eta_dev,
                                   double dt, float *t_dev, float *coarse_dev);
int ohm_op_grid_prolong_add_f32(ohm_hier *h, int m, const float *coarse_dev, float *fine_dev);

/* The coarsest-grid solve of the float32 inner solve (Secs. 2.2-2.3): the V-cycle over the
 * lexicographic grids below the last blocked one, from e = 0, for the right-hand side r_dev on
 * the first of them, with the hierarchy's sweep counts for the grids coarser than level 0
 * (nu_coarse_pre / nu_coarse_post when set, else nu_pre / nu_post), n_coarse sweeps on the
 * coarsest grid and omega.  r_dev and e_dev are float32 [3][nz][ny][nx] and eta_dev float32
 * [nz][ny][nx] on that grid (the coarser grids take the mean of the 8 children, Sec. 2.2); the
 * launches are those of a V-cycle there (the shared-memory solver where the grids fit).  The
 * hierarchy's own eta-derived data are rebuilt by the next ohm_set_eta.  OHM_MIXED* hierarchies
 * of one instance. */
int ohm_op_coarsest_f32(ohm_hier *h, const float *r_dev, const float *eta_dev, double dt, float *e_dev);

/* out = L X = X + lambda dt div F(X) (Eq. 13) on leaf blocks, in float32: the operator the
 * float32 inner solve applies (covered cells of a private copy of X set to the mean of their
 * children, coarse-fine ghosts interpolated from the parent level, refluxing through float64
 * flux registers, Sec. 4).  X_dev, out_dev float32 [nblocks][3][8][8][8]; out_dev is 0 on covered
 * blocks.  OHM_MIXED(_FF) hierarchies after ohm_set_eta. */
int ohm_op_apply_L_f32(ohm_hier *h, const float *X_dev, double dt, float *out_dev);

/* ---------------------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper): launch counting and CUDA-event timing of
 * one kernel kind, used by the benchmark to measure a kernel inside a running step.
 * ------------------------------------------------------------------------------------- */
#define OHM_K_COMPOSITE      0  /* composite source / residual / flux divergence, float64    */
#define OHM_K_SMOOTH         1  /* red-black colour pass                                      */
#define OHM_K_RESID_RESTRICT 2  /* multigrid residual + restriction                           */
#define OHM_K_PROLONG        3  /* prolongation + correction                                  */
#define OHM_K_GHOST          4  /* coarse-fine ghost fill                                     */
#define OHM_K_SYNC_DOWN      5  /* covered cells from their children                          */
#define OHM_K_UPDATE         6  /* B += e                                                     */
#define OHM_K_BOTTOM         7  /* coarsest-grid V-cycle (one thread block)                   */
#define OHM_K_NORM           8  /* norm reduction                                             */
#define OHM_K_KRYLOV         9  /* FGMRES vector kernels (multi-dot, multi-axpy)              */

/* From now on, bracket every launch of `kernel` that covers at least min_blocks blocks with
 * a pair of CUDA events on the hierarchy's stream, up to max_launches launches (events are
 * created here; kernel < 0 disables and releases them).  Adds one event record before and
 * after each timed launch and nothing else. */
int ohm_prof_enable(ohm_hier *h, int kernel, int min_blocks, int max_launches);

/* Synchronises the stream, returns the summed event time of the timed launches since the
 * last read, their count and the cells they covered, then resets the counters.  In a batch,
 * cells count only the instances the launch iterated (blocks of stopped instances return at
 * once and are not counted). */
int ohm_prof_read(ohm_hier *h, double *total_ms, int64_t *launches, int64_t *cells);

/* Kernel launches this hierarchy has issued since creation (all kinds). */
int64_t ohm_launch_count(const ohm_hier *h);

/* Measured float64 FMA issue rate of the current device (no hierarchy needed): a kernel of
 * independent DFMA chains on every SM, timed with CUDA events on `stream` (a cudaStream_t, NULL
 * = legacy default; the call synchronises it), best of three launches after one warm-up.
 * *dfma_per_s receives FMA instructions per second (2 flops each); the float64 stencil kernels
 * are bound by this rate.  Changes no device setting. */
int ohm_fp64_fma_rate(double *dfma_per_s, void *stream);

/* ---------------------------------------------------------------------------------------
 * Allocation-free residual (the paper has no counterpart: this is a deployment interface).
 *
 * For callers that cannot allocate device memory: hosts that own every device allocation
 * through their own pool (a library-side cudaMalloc would escape their accounting and limits)
 * and real-time loops that must not enter the CUDA allocator (unbounded latency, possible
 * device synchronisation).  ohm_create_hierarchy allocates, so those callers use this entry
 * point, which needs no hierarchy and allocates nothing: its scratch (block index, neighbour
 * table, norm partials and reduction scratch, about 0.6 MB) is one fixed array that every
 * device loading the library holds until the process exits.
 *
 * Computes R = S - B - lambda dt div F(B) (Eqs. 13, 20) on ONE uniform periodic grid of
 * base_cells (multiples of 8) with cell width dx, the same arithmetic as ohm_op_residual.
 * block_ijk (host) lists every 8^3 block of the grid exactly once as (bi, bj, bk); B_dev, S_dev,
 * R_dev are [nblocks][3][8][8][8] and eta_dev [nblocks][8][8][8] in that order (caller owned).
 * norms (host, may be NULL) receives {||R||/||S||, max|R|, ||R||, ||S||}.  Work is issued on
 * `stream` (a cudaStream_t, NULL = legacy default); the call copies block_ijk to the device,
 * reads the norms back and synchronises the stream before returning.
 * Limits and errors: at most 4096 blocks (2,097,152 cells, e.g. 128^3); more, a list with a
 * coordinate out of range or a block twice (checked on the host), or a bad argument return
 * OHM_ERR_INVALID before any work is enqueued.
 * The first call on a device looks up the scratch array's address and keeps it for the life of
 * the process; do not call after a cudaDeviceReset of that device (the kept address is then
 * stale).  All calls share the scratch
 * array (it keeps the last call's contents; what must start at zero is cleared by each call),
 * so calls whose work overlaps on the GPU race with each other and must be serialised by the
 * caller. */
int ohm_residual_static(const int32_t base_cells[3], double dx, double lambda, double dt, int64_t nblocks,
                        const int32_t *block_ijk, const double *B_dev, const double *S_dev,
                        const double *eta_dev, double *R_dev, double *norms, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* OHM_H */
