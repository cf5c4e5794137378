/*
 * libmg: GB300 (sm_103a) FAS multigrid solver for the DGP brane-bending mode.
 *
 * The equation (arXiv:1303.0008, Eq. code_eqn in code units, box length 1, mean
 * density 1) is written here as
 *
 *     lap(phi) + alpha [ (lap phi)^2 - (grad_i grad_j phi)^2 ] = kappa * delta
 *
 * so alpha = R_c^2 / (3 beta a^4) (the paper's own alpha is 1/alpha) and
 * kappa = Omega_m a / beta.  It is discretised as in Sec. III.B (7-point
 * Laplacian, four-point cross differences: a 19-point stencil), split with
 * w = 1/3 and solved for the root of Eq. two_branch; the smoother takes one
 * Newton step per cell (Sec. III.B) in a four-colour Gauss-Seidel order, inside
 * FAS V-cycles (Sec. III.C): residual, full-weighting restriction, the coarse
 * equation L^H(phi^H) = L^H(R phi^h) - R d^h, trilinear prolongation of the
 * correction.  Refinement levels take Dirichlet values interpolated from the
 * level below (Sec. III.C, first paragraph; Sec. IV.D).
 *
 * Conventions of every call:
 *   - A status code is returned; nothing throws across this boundary.
 *     mg_last_error() gives a message for the calling thread.
 *   - Arrays are float64, x fastest: a[i + n*(j + n*k)].  A patch array is
 *     [count][8][8][8] in the same order within each patch.
 *   - on_device = 1: the pointer is device memory of the current device and the
 *     copy is ordered on the handle's stream; on_device = 0: host memory, and the
 *     call returns when the copy is complete.
 *   - Inputs are copied, never retained.  Outputs go to caller-owned buffers.
 *   - The handle owns all of its device memory; calls on one handle are not
 *     thread-safe.
 *   - Periodic grids solve the bordered system L^h phi = lambda with
 *     mean(phi) = 0: the discrete nonlinear term does not sum to zero over a
 *     periodic box, and the constant lambda (reported in the statistics) takes up
 *     the difference.  The residual reported and tested against `tol` is
 *     max |d - lambda|, d = L^h phi.
 *   - Where the discriminant of Eq. two_branch could turn negative, mg_guard
 *     (below) selects the reading: by default the source is held at the bound
 *     that keeps every root real; the cells concerned are counted in guard_hits.
 */
#ifndef MG_H
#define MG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_grid mg_grid;

typedef enum {
  MG_OK = 0,
  MG_EINVAL = 1,   /* bad argument (size, level, patch index, branch, pointer) */
  MG_ENOMEM = 2,   /* device or host allocation failed */
  MG_ECUDA = 3,    /* a CUDA call failed; see mg_last_error() */
  MG_ENOCONV = 4,  /* max_cycles reached, residual grew 1e3-fold, or stalled */
  MG_ENAN = 5,     /* a residual was not finite */
  MG_ETIMEOUT = 6, /* a kernel waited longer than barrier_timeout_s for its data */
  MG_ESTATE = 7    /* call out of order (e.g. solve before set_density) */
} mg_status;

typedef enum {
  MG_FP64 = 0,  /* every step in FP64 */
  MG_MIXED = 1  /* FP32 correction V-cycles inside an FP64 defect-correction loop */
} mg_precision;

/*
 * What to do where the square root of Eq. two_branch would be imaginary.  The
 * operator splitting of Sec. III.A keeps the discriminant non-negative for any
 * field as long as 1 + 4(1-w) alpha kappa delta >= 0 in every cell; beyond that
 * (alpha*kappa > 3/8 in voids) the equation has no real local root.
 *   MG_GUARD_FLOOR (default): the source is held at that bound,
 *     kappa*delta -> the value with 1 + 4(1-w) alpha kappa delta = 0, so no root is
 *     ever imaginary; guard_hits counts the floored cells of the finest level.
 *   MG_GUARD_ROOT: the square root is taken of max(q, 0) (the real part of the
 *     complex root); guard_hits counts the cells where q < 0.  Far beyond the
 *     bound the Newton-Gauss-Seidel iteration can cycle instead of converging.
 * Both are the same system when every cell satisfies the bound.
 */
typedef enum {
  MG_GUARD_FLOOR = 0,
  MG_GUARD_ROOT = 1
} mg_guard;

typedef struct {
  mg_precision prec;
  int nu_pre;        /* pre-smoothing sweeps per level (default 2) */
  int nu_post;       /* post-smoothing sweeps per level (default 2) */
  int coarsest;      /* stop coarsening at this many cells per side or fewer (default 4) */
  int max_cycles;    /* V-cycles (FP64) or outer corrections (mixed); default 100 */
  int inner_cycles;  /* mixed: FP32 V-cycles per FP64 correction (default 3) */
  int use_graphs;    /* capture each V-cycle in a CUDA graph (default 1) */
  int coarse_sweeps; /* cap on coarsest-level sweeps (default 4: the 4^3 coarsest problem
                        converges slowly per sweep, and more sweeps leave the V-cycle
                        count of the 128^3 lognormal solves unchanged) */
  double coarse_drop;/* coarsest solve stops when its residual fell by this (default
                        1e-2: a tighter coarsest solve leaves the V-cycle count of the
                        128^3 lognormal solves unchanged and only costs time) */
  int time_kernels;  /* 1: time every launch of the finest-level smoother with CUDA
                        events on the handle's stream (stats.kernel_ms); 2: time the
                        first colour stage of each smoothing call only (an event
                        between two launches removes their programmatic overlap, so
                        this disturbs the solve less); default 0.  With MG_MIXED the
                        timed launches are the finest level's FP32 colour stages (a half
                        sweep with half32; a whole sweep of slab launches with slab32;
                        not timed with sweep32 or pair32). */
  mg_guard guard;    /* default MG_GUARD_FLOOR */
  int patch_coarse_sweeps; /* sweeps on the coarsest (2^3 per patch) level of a
                              refinement union per V-cycle (default 8) */
  int fuse_coarse;   /* 1: run the levels with <= 16 cells per side, down to the
                        coarsest, as one launch of a thread-block cluster (default 1) */
  double omega;      /* relaxation of the FP64 Newton step on the periodic grid:
                        phi += omega (phi_newton - phi); default 1 (the plain step) */
  double omega_patch;/* the same on refinement levels (default 1) */
  int patch_mg_levels;/* multigrid levels of a refinement union: 1 (smoothing only),
                        2 (8^3 and 4^3 per patch) or 3 (down to 2^3; default) */
  double patch_cgc;  /* scale of the coarse-grid correction on refinement unions
                        (1 = the full FAS correction; default 1) */
  int sweep32;       /* mixed precision: 1 runs each pair of FP32 correction sweeps on
                        levels with n >= 32, n % 4 == 0 as two one-launch four-colour
                        sweeps (same arithmetic, same bits as the per-colour launches);
                        0 keeps four launches per sweep (default). */
  int pair32;        /* mixed precision: 1 updates two cells of a row per thread in the
                        per-colour FP32 stages of levels with n % 4 == 0 (same bits as one
                        cell per thread); 0 one cell per thread (default: the paired loads
                        touch each sector twice and the stage is load-bound, so pairs
                        measured 5-9 % slower per solve). */
  double tau_stop;   /* FP64 domain solves: > 0 also stops once max|d - lambda| <=
                        tau_stop * max|tau - mean tau|, tau = L^H(R phi) - R L^h(phi) the
                        truncation-error estimate of Sec. III.C (the paper's criterion
                        |d^h| <~ alpha |tau^h| with alpha <= 1/3); 0 (default) uses tol only */
  double w;          /* operator-splitting constant of Sigma (Sec. III.A; the paper takes
                        1/3, the default).  Another value in [0, 1) makes Sigma depend on
                        the cell's own value and each smoothing update a full Newton step
                        with the Jacobian diagonal of Sec. III.B; FP64 domain solves only
                        (MG_EINVAL with MG_MIXED, refinement levels or batches). */
  int patch_galerkin;/* coarse-grid correction of refinement unions: 1 (default) solves
                        the linear correction equation with Galerkin coarse operators
                        R J P of the union's Jacobian J at the current iterate (FP32,
                        eight-colour Gauss-Seidel on the 27-point coarse operators);
                        0 uses the FAS coarse equations with the rediscretised operator.
                        The converged solution is the same; with alpha*kappa*delta >> 1
                        in dense regions only the Galerkin correction converges. */
  int half32;        /* mixed precision, levels with n = 256 or 512: 1 runs each FP32
                        correction sweep as two launches of two colours each, streaming
                        planes of whole rows through shared memory with bulk asynchronous
                        copies (same arithmetic, same bits as the per-colour launches);
                        0 keeps four launches per sweep. */
  double barrier_timeout_s; /* longest wait of a kernel for its asynchronous copies
                        (default 1 s); a kernel that waits longer records the failure
                        and returns, and the solve returns MG_ETIMEOUT */
  int slab32;        /* mixed precision, levels with n >= 256 (a power of two) and
                        n % slab32 == 0: > 0 runs each FP32 correction sweep slab by slab,
                        slab32 z planes per launch and colour, each colour a few planes
                        behind the one before it, so that a colour stage finds the planes
                        it reads in L2 (same arithmetic, same bits as whole colour
                        stages); one of 0 (whole colour stages, default), 8, 16, 32, 64,
                        128, 256. */
  int tile32;        /* mixed precision, levels with n >= 64 (a power of two): the cells a
                        256-thread CTA of an FP32 colour stage updates, a tile of 32 cells
                        in x by 8 / tile32 rows of the colour by tile32 planes (1, 2, 4 or
                        8; default 4), so that the rows around its cells overlap in L1; 0
                        takes 256 consecutive cells.  From n = 256 on, where each thread
                        updates two cells on planes k and k + 2, the tile counts such pairs
                        of planes.  Same bits whatever the shape. */
} mg_options;

typedef struct {
  int cycles;          /* V-cycles (FP64) or total inner V-cycles (mixed) */
  int outer;           /* FP64 residual evaluations (mixed) */
  int status;          /* the mg_status of the solve */
  int levels;          /* multigrid levels used */
  double res0;         /* residual at the first check */
  double res;          /* final max |d - lambda| */
  double lambda;       /* compatibility constant (periodic) */
  double wall_s;       /* device time of the solve */
  long long guard_hits;/* finest-level cells floored (MG_GUARD_FLOOR) or with a negative
                          discriminant at the last check (MG_GUARD_ROOT) */
  int hist_len;
  double res_hist[128];/* residual at each check */
  long long launches;  /* kernels launched by the solve (graph nodes included) */
  long long kernel_launches; /* finest-level smoother launches timed (time_kernels) */
  double kernel_ms;    /* their summed device time in milliseconds */
  double kernel_cells; /* cell updates those launches performed */
  double tau;          /* with tau_stop > 0: max |tau - mean tau| of the truncation-error
                          estimate at the last check (FP64 domain solves), else 0 */
} mg_solve_stats;

/* Fill `opt` with the defaults listed above. */
void mg_default_options(mg_options* opt);

/*
 * Create a periodic n^3 domain grid (n even, 4 <= n <= 1024).  `opt` may be NULL
 * (defaults).  Allocates the level hierarchy n, n/2, ... down to `coarsest`
 * (halving while the half is even and at least 4) on the current device.
 * Errors: MG_EINVAL for a bad n or options, MG_ENOMEM, MG_ECUDA.
 */
mg_status mg_create_grid(mg_grid** out, int n, const mg_options* opt);

/* Order the handle's work on `stream` (a cudaStream_t; NULL = the handle's own
 * non-blocking stream, the default).  The stream must outlive its use. */
mg_status mg_set_stream(mg_grid* g, void* stream);

/*
 * Add `count` 8^3 refinement patches to level `level` (1 or 2; level 1 needs the
 * domain, level 2 needs level 1 in place).  origin[3*p..3*p+2] = (x, y, z) of
 * patch p in level cells (cell size 1/(n 2^level)), each a multiple of 8 and in
 * [0, n 2^level).  Patches of one level must not overlap; the level's parent
 * cells dilated by one cell must lie in level-1 patches (proper nesting, checked
 * when level 2 is solved).  Replaces any patches the level had.
 * Errors: MG_EINVAL (alignment, range, duplicates), MG_ENOMEM, MG_ECUDA.
 */
mg_status mg_add_patches(mg_grid* g, int level, int count, const int32_t* origin);

/*
 * Set the density contrast delta = rho - 1 (Eq. code_eqn).  level 0 with patch = -1:
 * the n^3 domain array (restricted to every coarse level here).  level >= 1 with
 * patch = -1: all patches of the level, [count][8][8][8]; patch >= 0: one patch.
 * For a batch handle (mg_create_batch) `level` must be 0 and `patch` selects
 * the solve.  Errors: MG_EINVAL, MG_ECUDA.
 */
mg_status mg_set_density(mg_grid* g, int level, int patch, const double* delta, int on_device);

/* Set the field phi (initial guess, or a saved state to resume from); same
 * addressing as mg_set_density.  The domain field starts at zero otherwise.  A
 * refinement level that has no initial guess (never set, or reset by passing
 * phi = NULL with patch = -1) starts its next solve from the cell-centred
 * trilinear interpolation of the level below, as a new refinement inherits the
 * coarse solution; after a solve its last iterate is the next initial guess. */
mg_status mg_set_field(mg_grid* g, int level, int patch, const double* phi, int on_device);

/*
 * Solve every level of the grid: the domain by FAS V-cycles until
 * max|d - lambda| < tol, then each refinement level in turn with its Dirichlet
 * fill taken from the solved level below, until max|d| < tol.  `branch` is the
 * sign in front of the square root of Eq. two_branch (+1 or -1); 0 selects
 * sgn(alpha), the physical root of Eq. one_branch.  With alpha = 0 the equation
 * is the linear Poisson equation and branch must be 0.  tol is in the units of
 * kappa*delta.  `stats` may be NULL; it describes the domain solve.
 * On MG_ENOCONV or MG_ENAN the last iterate stays in the handle; after
 * MG_ETIMEOUT the field is undefined and must be set again before the next solve.
 * Errors: MG_EINVAL, MG_ESTATE (no density), MG_ENOCONV, MG_ENAN, MG_ECUDA.
 */
mg_status mg_solve(mg_grid* g, int branch, double alpha, double kappa, double tol,
                   mg_solve_stats* stats);

/* Copy the field out (same addressing as mg_set_density). */
mg_status mg_get_field(const mg_grid* g, int level, int patch, double* out, int on_device);

/* The density contrast delta of (level, patch) as the solver holds it (after
 * mg_set_density or mg_assign_density), addressed as in mg_get_field. */
mg_status mg_get_density(const mg_grid* g, int level, int patch, double* out, int on_device);

/*
 * The fifth force g = -(1/2) grad(phi) (Sec. II.B) by central differences
 * (Sec. III.B), as 3 x cells float64 (x components, then y, then z).  Level 0:
 * 3 x n^3.  Level >= 1: 3 x count x 512 for patch = -1, 3 x 512 for one patch;
 * differences at patch faces use the neighbouring patch or the Dirichlet fill.
 */
mg_status mg_get_force(const mg_grid* g, int level, int patch, double* out, int on_device);

/* Read or replace the options of a handle (the level hierarchy and the grid
 * size stay as created; `coarsest` is not changed by mg_set_options). */
mg_status mg_get_options(const mg_grid* g, mg_options* out);
mg_status mg_set_options(mg_grid* g, const mg_options* opt);

/*
 * Autotuner.  Solves the handle's problem (its density and the field the caller
 * left in it, restored before every trial) with every combination of a sweep
 * pair (nu_pre, nu_post) from {1,1 2,1 1,2 2,2 3,2 2,3 3,3 4,3 3,4 4,4 5,4 4,5
 * 5,5}, for MG_MIXED inner_cycles in {3,4}, and for n <= 64 fuse_coarse in
 * {0,1}.  For MG_MIXED with n >= 256 it then tries, at the winning counts, the
 * shapes of the FP32 sweep: whole colour stages with CTA tiles of tile32 in
 * {0,1,2,4,8} planes, slabs of slab32 in {8,16,32,64} planes, and (n = 256 or
 * 512) half32 = 1.  Each candidate is solved and timed
 * on the device (twice for n <= 64, where the second solve counts).  The fastest
 * candidate that converges to
 * `tol` becomes the handle's options and is returned in *best (may be NULL) with
 * its time in *best_seconds (may be NULL).  With a cache_path, the choice is
 * stored in that JSON file under the key "n=<n>,prec=<fp64|mixed>,device=<name>";
 * with use_cache = 1 a stored choice is applied without any trial.
 * The field left in the handle is the caller's, unchanged.
 * Errors: MG_EINVAL, MG_ESTATE (no density), MG_ENOCONV (no candidate converged),
 * MG_ENOMEM, MG_ECUDA.
 */
mg_status mg_autotune(mg_grid* g, int branch, double alpha, double kappa, double tol,
                      const char* cache_path, int use_cache, mg_options* best,
                      double* best_seconds);

/*
 * The launch order of one FP32 correction sweep in slabs (option slab32; host
 * only, no GPU needed): launch m updates the cells of colour colour[m]
 * (c = ((i+k)&1) + 2((j+k)&1)) on the planes z0[m], ..., z0[m] + nz[m] - 1 (mod n).
 * The n/slab slabs run in order and, within a slab, colours 0 to 3; colour c's
 * slabs sit c planes below colour 0's, and its first c planes come in its last
 * slab.  Every cell then reads the same neighbour values as in four whole colour
 * stages (Sec. III.B's Gauss-Seidel order), and each launch reads planes that the
 * launch before it touched.  Writes 4 n/slab entries into each array (cap entries
 * at most) and their number into *count.
 * Errors: MG_EINVAL (no slab order for this n and slab: slab < 8, n % slab != 0,
 * n / slab < 2, or cap too small; a NULL pointer).
 */
mg_status mg_slab_order(int n, int slab, int* colour, int* z0, int* nz, int cap, int* count);

/* Statistics of the last solve of a refinement level (level >= 1): cycles,
 * status, final residual, the residual after each cycle and the device time of
 * its V-cycles (wall_s). */
mg_status mg_get_level_stats(const mg_grid* g, int level, mg_solve_stats* out);

/* Release the handle and all of its device memory.  NULL is ignored. */
void mg_destroy_grid(mg_grid* g);

/* Message of the last failed call on this thread ("" if none). */
const char* mg_last_error(void);

/*
 * Newtonian potential and total force (Sec. II.B, Eq. newton and the sentence
 * after it).  mg_solve_newton solves the Poisson equation
 *     (phi_N(i+1) + phi_N(i-1) + ... - 6 phi_N(i)) / h^2 = coef * delta,
 * coef = (3/2) Omega_m a in code units, on the domain and on every refinement
 * level of the handle, with the same FAS V-cycles as mg_solve in their linear
 * (alpha = 0) form, into buffers of its own: the scalar field of mg_solve is
 * left untouched, and phi_N persists between calls as the next initial guess.
 * Refinement levels take their Dirichlet shells from phi_N of the level below.
 * `stats` (nullable) describes the domain solve.  Errors as mg_solve, plus
 * MG_EINVAL for a batch handle or a non-finite coef.
 */
mg_status mg_solve_newton(mg_grid* g, double coef, double tol, mg_solve_stats* stats);

/* phi_N of (level, patch), addressed as in mg_get_field.  MG_ESTATE before the
 * first mg_solve_newton. */
mg_status mg_get_newton_field(const mg_grid* g, int level, int patch, double* out, int on_device);

/*
 * Total force -grad Psi with Psi = phi_N + phi / 2, the potential under which
 * particles move in the DGP model: -grad phi_N plus the fifth force of
 * mg_get_force, by the same central differences (evaluated as -1/2 grad of
 * phi + 2 phi_N, including the refinement levels' ghost shells).  Layout and
 * addressing as mg_get_force.  MG_ESTATE before the first mg_solve_newton.
 */
mg_status mg_get_total_force(const mg_grid* g, int level, int patch, double* out, int on_device);

/*
 * Particles to mesh (Sec. VI: the density on the mesh comes from assigning the
 * particles with the triangular-shaped-cloud scheme).  Sets delta = rho - 1 on
 * the domain (level 0, every cell) or on the patches of a refinement level
 * (only cells inside a patch receive mass), then prepares it as mg_set_density.
 *   scheme  MG_TSC (27 cells, W(u) = 3/4 - u^2 for |u| <= 1/2 and
 *           (3/2 - |u|)^2 / 2 for 1/2 < |u| < 3/2) or MG_CIC (8 cells, 1 - |u|),
 *           u the per-axis distance from a cell centre in cells
 *   pos     3 x count doubles, SoA (all x, then all y, then all z), box units;
 *           periodic (folded into [0, 1)); a non-finite coordinate drops the particle
 *   mass    count doubles in units of the total mass of the box (mean density 1),
 *           or NULL for 1/count each
 * The FP64 atomic additions run in no fixed order: the last bits of a cell can
 * vary between runs.  Errors: MG_EINVAL (batch handle, scheme, count <= 0, no
 * patches on the level), MG_ENOMEM, MG_ECUDA.
 */
#define MG_CIC 1
#define MG_TSC 2
mg_status mg_assign_density(mg_grid* g, int level, int scheme, long long count, const double* pos,
                            const double* mass, int on_device);

/*
 * Refinement criterion (Sec. III.B: refine a cell when the effective number of
 * particles in it exceeds N_pc; Sec. V uses N_pc = 9): every 4^3-aligned block
 * of `level` (the domain, or the blocks of that level's patches) holding a cell
 * with (1 + delta) h^3 / particle_mass > npc becomes an 8^3 patch of level + 1,
 * whose origin (twice the block origin) is written to `origins` (3 int32 each,
 * sorted by z, then y, then x).  At most max_count origins are written; *found
 * receives how many there are.  particle_mass is in units of the total mass
 * (1/count for equal masses).  MG_ESTATE if the level has no density.
 */
mg_status mg_refine_blocks(const mg_grid* g, int level, double npc, double particle_mass,
                           int32_t* origins, int max_count, int* found);

/*
 * Batched independent periodic solves (one handle, `count` grids of sides n[s],
 * each valid for mg_create_grid).  Densities and fields are set per solve with
 * mg_set_density / mg_set_field (level 0, patch = solve index).
 */
mg_status mg_create_batch(mg_grid** out, int count, const int* n, const mg_options* opt);

/*
 * Solve every grid of a batch handle to max|d - lambda| < tol.  branch, alpha and
 * kappa hold one entry per solve; `stats` (may be NULL) holds `count` entries.
 * Returns MG_OK when every solve converged, else the first failing status.
 */
mg_status mg_solve_batch(mg_grid* g, const int* branch, const double* alpha, const double* kappa,
                         double tol, mg_solve_stats* stats);

/* ------------------------------------------------------------------------
 * Single-kernel entry points on caller-owned device arrays (periodic n^3,
 * float64, x fastest), ordered on `stream` (a cudaStream_t, NULL = legacy
 * default stream).  They run the same kernels as mg_solve and exist so that
 * each step can be checked on its own.  Errors: MG_EINVAL, MG_ENOMEM, MG_ECUDA.
 * ---------------------------------------------------------------------- */

/*
 * d = L^h phi - f (Sec. III.C residual; L^h of Sec. III.B), h = 1/n.  f may be
 * NULL (f = 0); d may be NULL (norms only).  norms (host, 5 doubles, may be
 * NULL): [sum d, max d, min d, guarded cells, non-finite cells].  Synchronises
 * the stream before it returns.
 */
mg_status mg_op_residual(int n, const double* phi, const double* delta, const double* f,
                         int branch, double alpha, double kappa, double* d, double* norms,
                         void* stream);

/* `sweeps` four-colour Newton-Gauss-Seidel sweeps of L^h phi = f + lambda in place
 * (f may be NULL). */
mg_status mg_op_smooth(int n, double* phi, const double* delta, const double* f, int branch,
                       double alpha, double kappa, double lambda, int sweeps, void* stream);

/* coarse[(n/2)^3] = mean of the 8 children of fine[n^3] (n even). */
mg_status mg_op_restrict(int n, const double* fine, double* coarse, void* stream);

/* fine[n^3] += P(coarse - coarse_ref), trilinear, coarse arrays (n/2)^3. */
mg_status mg_op_prolong_correct(int n, const double* coarse, const double* coarse_ref,
                                double* fine, void* stream);

/* out[3 n^3] = -(1/2) grad phi. */
mg_status mg_op_force(int n, const double* phi, double* out, void* stream);

/*
 * mg_op_residual without any device allocation (the paper has no counterpart:
 * it is a service to callers).  mg_op_residual allocates and frees temporaries
 * with cudaMalloc/cudaFree on every call; those calls synchronise the whole
 * device, and they fail in a process whose device memory is already taken by
 * its own allocator.  Callers in that position (programs that overlap work on
 * several streams, or that hand the card to a framework's memory pool) use this
 * entry point instead.  Same arguments, same results as mg_op_residual.
 *   - Limit: n <= 256 (at most 256^3 cells); larger n returns MG_EINVAL.
 *   - Storage: a fixed, file-scope device array of about 2.6 MB that every device
 *     loading the library holds until the process ends.  All calls on a device
 *     share it and it keeps the last call's contents; calls that overlap on the
 *     GPU race on it, so the caller must order them (one stream, or events).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *     The address is kept for the life of the process: do not call this entry
 *     point again after cudaDeviceReset.
 *   - Like mg_op_residual, the call synchronises `stream` before it returns,
 *     whether or not norms is given, and reports execution errors.
 * Errors: MG_EINVAL (size, branch, non-finite alpha, NULL input), MG_ECUDA.
 */
mg_status mg_op_residual_noalloc(int n, const double* phi, const double* delta, const double* f,
                                 int branch, double alpha, double kappa, double* d, double* norms,
                                 void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MG_H */
