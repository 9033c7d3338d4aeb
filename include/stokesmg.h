/*
 * stokesmg.h -- C ABI of the GB300 (sm_103a) symmetric multigrid-preconditioned SQMR solver for
 * the 3D staggered-grid (MAC) Stokes system of Tao & Sifakis, arXiv 2312.10615.
 *
 * Problem (Sec. 2, Eq. 2):  L x = b,  L = [[A, B^T], [B, 0]],  A = -eta Lap_h (7-point, per face
 * velocity component), B^T = grad_h (face = difference of the two adjacent cell pressures / h),
 * B = -div_h.  Domain: an nx x ny x nz box of interior cells with one Dirichlet ghost shell
 * (Sec. 5: faces between two interior cells and all cell pressures are the unknowns; faces of
 * Dirichlet cells carry Dirichlet data).  With all-Dirichlet walls constant pressure lies in ker L;
 * solutions are returned with zero pressure mean.
 *
 * VECTOR LAYOUT ("packed", FP64, x index fastest):
 *   [ u: (nx+1)*ny*nz | v: nx*(ny+1)*nz | w: nx*ny*(nz+1) | p: nx*ny*nz ]
 *   u(i,j,k) at face x = i*h between cells i-1 and i, index i + (nx+1)*(j + ny*k); v, w analogous;
 *   p(i,j,k) at the cell centre, index i + nx*(j + ny*k).  Entries that are not unknowns (the
 *   wall-normal faces i = 0, nx of u, etc.) are ignored on input and written as 0 on output.
 * DIRICHLET LAYOUT ("ghost-extended", FP64): [u: (nx+1)(ny+2)(nz+2) | v: (nx+2)(ny+1)(nz+2) |
 *   w: (nx+2)(ny+2)(nz+1)], each tangential index running -1..n (stored at offset +1), the normal
 *   index 0..n.  Only entries on faces of ghost cells are read.
 *
 * POINTERS: every vector argument may be a device pointer (CUDA device or managed memory of the
 * handle's device) or a host pointer (pageable or pinned); host data is staged through
 * handle-owned device buffers inside the call.  The caller owns all vectors; the handle owns
 * every internal buffer (hierarchy, smoother tables, coarse inverse, CUDA graphs, scratch).
 * STREAMS: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 * stream-ordered and asynchronous with respect to the host except where stated.
 * ERRORS: every call returns STOKES_OK (0) or a negative code below; no call aborts the process.
 * A handle is not thread-safe: one host thread (or external synchronisation) per handle.
 */
#ifndef STOKESMG_H
#define STOKESMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STOKES_OK 0
#define STOKES_ERR_INVALID_ARG -1   /* bad size, NULL where required, unsupported combination */
#define STOKES_ERR_OOM -2           /* device or host allocation failed */
#define STOKES_ERR_CUDA -3          /* a CUDA runtime call failed (context is left usable) */
#define STOKES_ERR_BREAKDOWN -4     /* SQMR: sigma = q^T L q = 0 or rho = s^T t = 0 (Alg. 4 divides by both) */
#define STOKES_ERR_NOT_CONVERGED -5 /* SQMR: max_iter reached before the tolerance */
#define STOKES_ERR_NAN -6           /* a NaN/Inf appeared in the SQMR scalars */
#define STOKES_ERR_TIMEOUT -7       /* a device-side grid barrier ran out of its iteration limit */
#define STOKES_ERR_UNSUPPORTED -8   /* valid request the library does not implement */

/* precision of the V-cycle (the SQMR recurrences, the true-residual check and the coarsest
 * solve always run in FP64) */
#define STOKES_PREC_FP64 0
#define STOKES_PREC_FP32 1
/* FP32 V-cycle whose two finest levels (never the coarsest) store their right-hand side b, residual
 * r and the pressure-sweep residual parts as BF16 (8 significant bits), read into FP32 arithmetic.
 * The preconditioner is then symmetric only up to BF16 rounding; SQMR, the true-residual check and
 * the tolerance are unchanged (FP64). */
#define STOKES_PREC_MIXED_BF16 2

typedef struct stokes_s *stokes_t;

typedef struct {
    int nx, ny, nz;   /* interior cells per axis (2 <= nx, ny <= 2047, 2 <= nz <= 1023) */
    double h;         /* cell size (> 0); <= 0 selects 1/nx (unit-width box) */
    int levels;       /* multigrid levels; 0 = automatic: halve while every dimension is even and
                         one exceeds coarsest_max (Alg. 1; 128^3 -> 5 levels) */
    int coarsest_max; /* 0 = 8 */
} stokes_grid_t;

typedef struct {
    /* cell labels on the ghost-extended cell grid (nx+2)(ny+2)(nz+2), x fastest, index
     * (i+1) + (nx+2)((j+1) + (ny+2)(k+1)) for cell (i,j,k), i = -1..nx: 0 interior, 1 Dirichlet,
     * 2 exterior (Sec. 5).  The ghost shell must be Dirichlet; a value above 2 or a non-Dirichlet
     * ghost cell gives STOKES_ERR_INVALID_ARG.  Faces of Dirichlet cells carry Dirichlet data (the
     * ghost-extended Dirichlet layout covers every face).  The unknowns are the pressures of interior
     * cells and the faces with an interior cell on at least one side and no Dirichlet cell: faces
     * between two interior cells, and Neumann faces between an interior and an exterior cell, whose
     * rows carry the homogeneous Neumann (do-nothing outflow) condition -- the exterior pressure is 0
     * and viscous terms that cross an exterior cell along the face normal, or reach a face between two
     * exterior cells, drop out (L stays symmetric; g is not read across an exterior cell).  Faces
     * between two exterior cells are inactive.  With a Neumann face the pressure has no null space and
     * sqmr_solve does not shift it to zero mean.  V1 holds the unknowns of interior cells with a
     * Dirichlet cell among their 26 neighbours or an exterior cell within two cells (Table 1 counts).
     * Coarse labels: Dirichlet if any child is, else interior if any child is, else exterior.  NULL =
     * the box (all interior, one Dirichlet ghost shell).  The array is copied; the caller keeps
     * ownership. */
    const uint8_t *cell_labels;
} stokes_bc_t;

typedef struct {
    double gamma;  /* penalty of L~ = [[A, B^T], [B, -gamma I]] used only inside the V-cycle (Sec. 4); default 1e-3 */
    int kb_vanka;  /* symmetric Vanka sweeps before and after the symmetric DGS in Alg. 3; default 1 */
    int precision; /* STOKES_PREC_FP64 (default) or STOKES_PREC_FP32 V-cycle */
    int use_graphs;/* capture the V-cycle / SQMR iteration in CUDA graphs (default 1) */
    int vanka_persistent; /* 0 (default): two launches per Vanka colour; 1: one cooperative launch per
                             symmetric sweep on every level (grid barrier with a bounded spin; expiry ->
                             STOKES_ERR_TIMEOUT) */
    int autotune;  /* 1 (default): at creation, time the Vanka schedule candidates of every smoothed
                      level (per-colour launches; one cooperative sweep with up to 5 grid sizes; one
                      cluster of 4, 8 or 16 CTAs; one block on a shared-memory copy of a small
                      level) and keep the fastest; all candidates give bit-identical results.
                      0: per-colour launches. */
    int vanka_additive; /* 0 (default): symmetric multiplicative Vanka (App. C); 1: the additive Vanka of
                           Eq. (av) in its place, damped by 1/2 (a face lies in two patches; the
                           undamped sum over-corrects) -- symmetric as well (Sec. 3.2 variant) */
    int cycle;     /* coarse-grid visits per level: 1 (default) V-cycle (Alg. 1), 2 W-cycle (Sec. 8.2) */
    int distributive_jacobi; /* 0 (default): symmetric DGS on V2 (Alg. 2 + Eq. ldist); 1: symmetric
                                distributive weighted Jacobi (Sec. 3.1), one Jacobi step per block of
                                L~M in the DGS block order and its reverse, weight 6/7 */
} stokes_opts_t;

typedef struct {
    int iterations;        /* SQMR iterations performed (Alg. 4 loop index j) */
    double rel_residual;   /* true ||b - L x||_2 / ||b||_2 of the returned x, explicit FP64: the residual
                            * that confirmed convergence (removing the pressure mean afterwards changes
                            * L x only by rounding, a constant pressure lies in ker L), else recomputed
                            * at exit */
    int status;            /* same value as the call's return code */
    int vcycles;           /* preconditioner applications (iterations + 1) */
} sqmr_info_t;

/* Fill *opts with the defaults listed above. */
void stokes_opts_default(stokes_opts_t *opts);

/* Build the multigrid hierarchy on the current CUDA device (Sec. 5 labels and DOF classes,
 * Alg. 1 re-discretised coarse levels, Alg. 2 diagonals, Sec. 6 pre-factorised Vanka local
 * problems, the exact coarsest solve as a symmetrised dense FP64 inverse).  `bc` and `opts` may
 * be NULL (box, defaults).  viscosity = eta > 0.  On success *out owns all device memory. */
int stokes_create(const stokes_grid_t *grid, const stokes_bc_t *bc, double viscosity, const stokes_opts_t *opts,
                  stokes_t *out);

/* Free everything the handle owns (after synchronising its work).  NULL is accepted. */
int stokes_destroy(stokes_t h);

/* Packed vector length of level `level` (0 = finest); 0 if out of range. */
long long stokes_vector_length(stokes_t h, int level);
/* Ghost-extended Dirichlet array length of the finest level. */
long long stokes_ghost_length(stokes_t h);
/* Number of multigrid levels. */
int stokes_num_levels(stokes_t h);

/* b = f on the unknowns with the Dirichlet data moved to the right-hand side (Sec. 5):
 * velocity rows add eta/h^2 * (Dirichlet neighbour values), pressure rows add
 * (g_high - g_low)/h over Dirichlet faces.  f: packed (the p block is the continuity source);
 * g: ghost-extended, NULL = homogeneous.  b: packed, written completely. */
int stokes_rhs(stokes_t h, const double *f, const double *g, double *b, void *stream);

/* y = L x on the unknowns (Eq. 2); other entries of y are set to 0.  FP64. */
int stokes_apply(stokes_t h, const double *x, double *y, void *stream);

/* t = V-cycle(L~, s, 0, n) (Alg. 1 with the Alg. 3 smoother, zero initial guess, Sec. 3), the
 * symmetric preconditioner W^dagger s of Alg. 4.  Linear and symmetric in s.  s, t packed FP64;
 * in FP32 precision the cycle runs on FP32 copies.  s and t may not alias. */
int mg_precondition(stokes_t h, const double *s, double *t, void *stream);

/* Alg. 4: MG-preconditioned SQMR on L.  rhs: packed b; x: x0 on entry, the solution on exit
 * (pressure mean removed).  Stops when the true relative residual ||b - Lx||/||b|| < tol
 * (tracked by the exact recursion r_j = (1 - c_j^2) r_{j-1} + c_j^2 s_j and confirmed by an
 * explicit FP64 b - Lx).  With graphs on (the default) the iterations run as one CUDA graph: a
 * while node around the iteration, whose stopping test (recursive residual below tol, breakdown,
 * non-finite value, max_iter) runs on the device, so the stream is synchronised only when that test
 * stops the loop (to confirm convergence by the explicit residual, then go on if it does not); if the
 * driver refuses such a graph, or with graphs off, the host synchronises once per iteration.  Fills
 * *info (may be NULL).  Returns STOKES_ERR_NOT_CONVERGED / BREAKDOWN / NAN with x holding
 * the last iterate. */
int sqmr_solve(stokes_t h, const double *rhs, double *x, double tol, int max_iter, sqmr_info_t *info, void *stream);

/* Alg. 4 with the identity in place of the preconditioner (t = s): the plain SQMR the paper compares
 * against (Sec. 6, Sec. 7).  Arguments, outputs and errors as sqmr_solve; info->vcycles = 0.  With
 * STOKES_PREC_FP64 every step is FP64; otherwise t is s rounded to FP32. */
int sqmr_solve_unpreconditioned(stokes_t h, const double *rhs, double *x, double tol, int max_iter,
                                sqmr_info_t *info, void *stream);

/* Alg. 1 used outright as the solver (Sec. 3), on the penalised system L~ x = b as in the paper's
 * pure-multigrid comparisons (Sec. 6): x_{k+1} = x_k + V-cycle(L~, b - L~ x_k, 0, n), the same iterate
 * as the cycle started at x_k.  Stops when ||b - L~ x_k||/||b|| < tol (FP64 residual, one stream
 * synchronisation per cycle).  The limit of the iteration is L~^{-1} b, which differs from the Stokes
 * solution by O(gamma); the pressure mean is not removed.  x: x0 on entry, the last iterate on exit.
 * info->iterations = info->vcycles = cycles run, info->rel_residual = the L~ residual.  Returns
 * STOKES_ERR_NOT_CONVERGED after max_iter cycles, STOKES_ERR_NAN on a non-finite residual. */
int mg_solve(stokes_t h, const double *rhs, double *x, double tol, int max_iter, sqmr_info_t *info, void *stream);

/* Batch of independent problems (the handles may have different grid sizes, all on one device):
 * solves problem i = sqmr_solve(handles[i], rhs[i], x[i], tol, max_iter, &infos[i]) for all i, with
 * nstreams host threads (1..64), each owning its own CUDA stream and pulling the next unsolved
 * problem, so solves of different problems overlap on the GPU (each replays its handle's CUDA
 * graphs).  done_ms[i] (may be NULL): milliseconds from the call's start to problem i's completion.
 * Returns STOKES_OK or the first non-OK status; infos (may be NULL) carries every problem's result.
 * A handle must not appear twice in one batch. */
int sqmr_solve_batch(int nprob, const stokes_t *handles, const double *const *rhs, double *const *x, double tol,
                     int max_iter, sqmr_info_t *infos, double *done_ms, int nstreams);

/* Batched handle: nprob (2..4096) independent problems on ONE grid (same grid, bc, viscosity and
 * options; nprob * 4 (nz + 1) <= 65535), created with stokes_create's arguments.  Every per-problem
 * buffer of a multigrid level lies in one device allocation (problem p's copy at a fixed stride), so
 * each step of the V-cycle (Alg. 1, Alg. 3) and of the SQMR iteration (Alg. 4) is ONE kernel launch
 * for all problems, and the iteration is one captured CUDA graph.  The schedule is fixed (per-colour
 * Vanka launches, in-place DGS; no autotuning, no distributive Jacobi, graphs on); results are
 * bit-identical to solving each problem with stokes_create + sqmr_solve.  stokes_rhs works as for a
 * single handle (it reads only the grid); the other single-problem calls return
 * STOKES_ERR_INVALID_ARG on a batched handle.  Free with stokes_destroy. */
int stokes_create_batch(int nprob, const stokes_grid_t *grid, const stokes_bc_t *bc, double viscosity,
                        const stokes_opts_t *opts, stokes_t *out);
/* problems in a handle (1 for stokes_create's handles, 0 for NULL) */
int stokes_batch_size(stokes_t h);
/* how this handle's SQMR loop runs (known after its first sqmr_solve): 0 host-driven (one iteration
 * graph per launch, a synchronisation per iteration), 1 one device-side graph with the kernels'
 * programmatic launch edges, 2 one device-side graph without them (the driver refused them there) */
int stokes_device_loop(stokes_t h);
/* enable = 1 (default) lets sqmr_solve run its loop as one device-side graph; 0 keeps the host loop */
int stokes_set_device_loop(stokes_t h, int enable);
/* Alg. 4 for every problem of a batched handle: rhs[p], x[p] (x0 in, solution out) as sqmr_solve's
 * (host or device).  Per-problem convergence: a problem stops (its state frozen on the device) at the
 * iteration its own explicit FP64 residual confirms tol, as in sqmr_solve; the call returns when every
 * problem has stopped.  infos (may be NULL) receives nprob results; returns STOKES_OK or the first
 * problem's non-OK status. */
int sqmr_solve_batched(stokes_t h, const double *const *rhs, double *const *x, double tol, int max_iter,
                       sqmr_info_t *infos, void *stream);

/* the Vanka schedule of a smoothed level (chosen by the autotuner): *mode 0 = two launches per
 * colour, 1 = one cooperative launch per symmetric sweep with *blocks thread blocks (grid barrier),
 * 2 = one launch per symmetric sweep in a single thread-block cluster of *blocks CTAs (hardware
 * cluster barriers), 3 = one launch per symmetric sweep in one thread block working on a
 * shared-memory copy of the level (small levels only; *blocks = 1), 4 = one launch per colour step on
 * two copies of the level's Vanka state (each step reads one and writes the other; *blocks = 0);
 * *ms = the autotuner's time per symmetric sweep (0 if not measured).  Any output pointer may be
 * NULL. */
int stokes_level_schedule(stokes_t h, int level, int *mode, int *blocks, float *ms);
/* override the schedule of one level (mode and blocks as above; blocks <= the co-resident limit for
 * mode 1, <= 16 for mode 2; mode 3 returns STOKES_ERR_UNSUPPORTED if the level does not fit in
 * shared memory, mode 4 if the handle has no second state copy: additive Vanka, vanka_persistent, or
 * a level of 2^31 entries or more); the handle's captured graphs are re-captured on next use.  All
 * schedules compute the same bits. */
int stokes_set_level_schedule(stokes_t h, int level, int mode, int blocks);

/* tiles of the transfers between `level` and level + 1 (0 <= level < levels-1): tiles[0..2] = block x,
 * block y and coarse z-planes per thread of the restriction R from this level, tiles[3..5] the same for
 * the prolongation P into it; *ms (optional, 2 floats) = the autotuner's time per launch of each (0 if
 * not measured).  With opts.autotune the handle times 8 candidate tiles per transfer and level at
 * creation and keeps the fastest; every tile computes the same bits (each entry is produced by one
 * thread with the same arithmetic). */
int stokes_level_tiles(stokes_t h, int level, int *tiles, float *ms);
/* override them (block x * block y a multiple of 32 and at most 1024, 1 <= z-planes <= 64); the
 * handle's captured graphs are re-captured on next use */
int stokes_set_level_tiles(stokes_t h, int level, const int *tiles);

/* how the symmetric DGS of a smoothed level runs its velocity blocks (Alg. 2 / Eq. ldist): *fused = 0,
 * two in-place launches per direction (one per parity of i+j+k); 1, one out-of-place pass per direction
 * that relaxes both parities (the second a plane behind the first, overlapped tiles) into the handle's
 * second state buffer and back.  *ms (optional, 2 floats) = the autotuner's time per symmetric DGS for
 * 0 and 1 (0 if not measured).  With opts.autotune the faster is kept per level; both compute the same
 * bits. */
int stokes_level_dgs(stokes_t h, int level, int *fused, float *ms);
/* override it (fused = 1 returns STOKES_ERR_UNSUPPORTED with the distributive weighted Jacobi or
 * without a second state buffer); the handle's captured graphs are re-captured on next use */
int stokes_set_level_dgs(stokes_t h, int level, int fused);

/* *out = ||b - L x||_2 (FP64, deterministic reduction); synchronises the stream.  Uses the
 * handle's reduction scratch. */
int stokes_residual_norm(stokes_t h, const double *b, const double *x, double *out, void *stream);

/* ---- diagnostics: single pieces of the V-cycle on one level (FP64 packed vectors of that level) ----
 * which: 0 Alg. 3 smoother, 1 symmetric DGS, 2 one symmetric Vanka sweep (colours 0..7, 7..0),
 *        3 forward DGS (Alg. 2), 4 backward DGS (Eq. ldist), 10+c one Vanka colour c (0..7).
 * x is updated in place with right-hand side b; level must be smoothed (< levels-1). */
int stokes_smooth(stokes_t h, int level, int which, double *x, const double *b, void *stream);
/* b_coarse = R r_fine (R = P^T/8, Sec. 2), level -> level+1 */
int stokes_restrict(stokes_t h, int level, const double *r_fine, double *b_coarse, void *stream);
/* x_fine += P e_coarse, level+1 -> level */
int stokes_prolong_add(stokes_t h, int level, const double *e_coarse, double *x_fine, void *stream);
/* x = L~^{-1} b on the coarsest level (Alg. 1 exact solve) */
int stokes_coarse_solve(stokes_t h, const double *b, double *x, void *stream);

/* ---- diagnostics: per-kernel timing ----
 * Runs one SQMR iteration (Alg. 4 loop body, V-cycle included) eagerly on `stream` with a CUDA
 * event pair around every kernel launch and returns, per kernel kind k (STOKES_K_*), the summed
 * duration in ms and the launch count, over all levels and over level 0 only.  Arrays have nkinds
 * >= STOKES_K_COUNT entries.  Meant to follow a sqmr_solve on the same handle (it advances the
 * handle's SQMR state); synchronises the stream. */
#define STOKES_K_APPLY_DOT 0
#define STOKES_K_UPDATE_S 1
#define STOKES_K_DOT2 2
#define STOKES_K_UPDATE_X 3
#define STOKES_K_SCALARS 4
#define STOKES_K_MEMSET 5
#define STOKES_K_VANKA_COMPUTE 6
#define STOKES_K_VANKA_APPLY 7
#define STOKES_K_DGS_U 8
#define STOKES_K_DGS_P_FWD 9
#define STOKES_K_DGS_P_GATHER 10
#define STOKES_K_DGS_P_BWD 11
#define STOKES_K_RESIDUAL 12
#define STOKES_K_RESTRICT 13
#define STOKES_K_PROLONG 14
#define STOKES_K_COARSE 15
#define STOKES_K_DGS_P_BWD_PREP 16
#define STOKES_K_COUNT 17
int stokes_profile_iteration(stokes_t h, int nkinds, double *ms_all, int *launches_all, double *ms_level0,
                             int *launches_level0, void *stream);

/* ---- diagnostics: the bounded device wait ----
 * Runs one cooperative symmetric Vanka sweep on `level` (0 <= level < levels-1) whose grid barrier
 * waits for `missing_blocks` more thread blocks than the launch has, giving up after `spin_limit`
 * polls per wait (1 .. 2^22; the solver's own sweeps use 2^22): with missing_blocks > 0 no wait can
 * complete, every block gives up, and the call returns STOKES_ERR_TIMEOUT with the GPU context intact;
 * with missing_blocks = 0 the sweep runs normally and the call returns STOKES_OK.  Exercises the
 * failure path of the persistent Vanka schedule without faulting or hanging the GPU.  Overwrites the
 * level's work vectors (they are zeroed before and after); synchronises `stream`.  Returns
 * STOKES_ERR_UNSUPPORTED if the device has no cooperative launch.  No counterpart in the paper. */
int stokes_test_grid_barrier(stokes_t h, int level, int missing_blocks, int spin_limit, void *stream);

/* ---- diagnostics: host-side classification of a labelled domain (no GPU needed) ----
 * flags[q] for every packed entry q of level `level` (n = that level's packed length; the labels are
 * coarsened per Sec. 5): bit 0 unknown, bit 1 V2 entry (an unknown that is not in the Vanka set V1),
 * bit 2 face of a Dirichlet cell, bits 3-5 the number of viscous terms of a face row that drop out next
 * to exterior cells, bit 6 / bit 7 the low / high neighbour along the face normal is one of them.
 * These are the flags the kernels read.  Labels and grid as in stokes_create; returns
 * STOKES_ERR_INVALID_ARG for invalid labels, a level the grid cannot coarsen to, or a wrong n. */
int stokes_label_flags(const stokes_grid_t *grid, const stokes_bc_t *bc, int level, uint8_t *flags, long long n);

/* ---- diagnostics: measured FMA rate of the CUDA cores ----
 * *flops_per_s = the fused multiply-add rate (2 flops per FMA) this GPU sustains in FP64 (fp64 != 0)
 * or FP32, measured on the current device with a grid of independent FMA chains (best of 5 timed
 * launches on `stream`, which is synchronised).  The FP64 figure is the roof of the FP64 kernels of
 * the path (operator apply and SQMR recurrences of Alg. 4), which are bound by the FP64 pipe, not
 * by memory.  A measurement aid with no counterpart in the paper; allocates and frees one small
 * device buffer.  Returns STOKES_ERR_INVALID_ARG for a NULL output, STOKES_ERR_CUDA / _OOM on a
 * CUDA failure. */
int stokes_measure_fma_peak(int fp64, double *flops_per_s, void *stream);

/* ---- allocation-free residual norm ----
 * *out = ||b - L x||_2 on an nx x ny x nz box (cell size h, <= 0 selects 1/nx; viscosity eta),
 * the same number stokes_residual_norm returns, computed without any handle and without allocating
 * anything.  The paper has no counterpart; this exists for callers that cannot allocate device
 * memory where they need the check (a fixed-budget memory pool, a host callback, an allocator-free
 * hook): creating a handle allocates the whole hierarchy.
 * b, x: packed FP64 vectors in device memory of the CURRENT device, read in place (entries of x
 * off the unknowns are ignored).  out: one double in device memory of the current device, written
 * asynchronously on `stream`, which must belong to the current device (NULL: the legacy default
 * stream).  Pointers to host memory or to another GPU's memory, a stream of another device, a
 * non-finite h or viscosity, or viscosity <= 0 return STOKES_ERR_INVALID_ARG.
 * Scratch: a fixed device array of 16384 doubles (128 KiB) inside the library, present on every
 * GPU that loads it until exit; grids needing more partial sums than that (more than 16384 blocks
 * of 32 x 8 x 16 cell positions, about 380^3) return STOKES_ERR_INVALID_ARG, as do host pointers.
 * The first call on a device looks up the array's address with that device current; make it
 * before any stream capture.  All calls share the array: calls that overlap on the GPU race, so
 * serialise them.  Calls no cudaMalloc / cudaFree. */
int stokes_residual_norm_noalloc(int nx, int ny, int nz, double h, double viscosity, const double *b,
                                 const double *x, double *out, void *stream);

/* Human-readable message for a status code (static storage). */
const char *stokes_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* STOKESMG_H */
