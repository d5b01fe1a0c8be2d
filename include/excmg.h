/*
 * excmg.h -- C ABI of the GB300 (sm_103a) EXCMG solver for the 3D Dirichlet Poisson
 * problem  u_xx + u_yy + u_zz = f in a box, u = g on its boundary  (Section 1, eq. bvp),
 * discretised by the 19-point fourth-order compact scheme with unequal meshsizes
 * (Section 2, eq. compact) and solved by the extrapolation cascadic multigrid method of
 * Algorithm 1 (Section 3.1).  Reference: Pan, He & Hu, arXiv 1507.05063.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Node arrays.  A grid of Nx x Ny x Nz cells on [0,Lx]x[0,Ly]x[0,Lz] has
 * (Nx+1)(Ny+1)(Nz+1) nodes (i hx, j hy, k hz), hx = Lx/Nx etc. (Section 2).  Every
 * node array is float64, dense, x fastest: node (i,j,k) is element
 * i + (Nx+1)*(j + (Ny+1)*k).  All array pointers are DEVICE pointers, owned by the
 * caller, at least 8-byte aligned, and must not overlap unless stated.
 * Levels.  The finest grid is (Nx,Ny,Nz); the coarsest is (Nx0,Ny0,Nz0); every level
 * halves all three cell counts, so Nx/Nx0 = Ny/Ny0 = Nz/Nz0 = 2^(levels-1) with
 * levels >= 3, and Nx0, Ny0, Nz0 must be even (the tri-quartic interpolation cells of
 * Section 3.3 are 2x2x2 coarse elements).  Coarse-level f and g are the finest values
 * at the coarse nodes.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 * Work is enqueued on it; entry points that run CG read convergence flags back and so
 * return only after their work on the stream has finished.
 * Workspace.  Scratch memory is caller-owned device memory of at least the size the
 * matching *_workspace_size query returns, 256-byte aligned.  The library allocates no
 * device memory.  Calls that share a workspace must not run concurrently.
 * Errors.  Every entry point returns an excmg_status and never throws.  Invalid
 * arguments are detected before any work is enqueued.  A CUDA launch or copy error maps
 * to EXCMG_ERR_CUDA (a sticky error leaves the context unusable, as in CUDA itself).
 */
#ifndef EXCMG_H
#define EXCMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EXCMG_OK = 0,
  EXCMG_ERR_INVALID_ARG = 1,   /* sizes, pointers, options or alignment rejected */
  EXCMG_ERR_NOT_CONVERGED = 2, /* a CG loop hit max_iter before its tolerance */
  EXCMG_ERR_CUDA = 3,          /* a CUDA call failed */
  EXCMG_ERR_NONFINITE = 4,     /* NaN/Inf met in a CG reduction (e.g. NaN in f or g) */
  EXCMG_ERR_TIMEOUT = 5,       /* a bounded device wait (a grid barrier of a cooperative
                                  CG launch) ran out; the kernel returned instead */
  EXCMG_ERR_WORKSPACE = 6      /* workspace NULL, too small or misaligned */
} excmg_status;

typedef enum {
  EXCMG_FP64 = 0,  /* CG entirely in float64 */
  EXCMG_MIXED = 1  /* float32 CG on the correction equation inside float64 iterative
                      refinement; residuals, reductions, extrapolation in float64 */
} excmg_precision;

#define EXCMG_MAX_LEVELS 24

/* Kernel kinds reported by options.profile. */
typedef enum {
  EXCMG_K_SPMV_F64 = 0,   /* p = r + beta p, q = A p, p.q            (float64 CG) */
  EXCMG_K_UPDATE_F64 = 1, /* x += alpha p, r -= alpha q, r.r        (float64 CG) */
  EXCMG_K_SPMV_F32 = 2,   /* the same in float32 (MIXED inner solves) */
  EXCMG_K_UPDATE_F32 = 3,
  EXCMG_K_RESIDUAL = 4,   /* r = b - A u in float64, ||r||, ||b|| */
  EXCMG_K_EXP_FINITE = 5, /* w_h = EXP_finite(u_2h, u_4h) */
  EXCMG_K_INIT = 6,       /* boundary data, zero interior (levels 0, 1) */
  EXCMG_K_CORRECT = 7,    /* u += e (MIXED) */
  EXCMG_K_EXP_TRUE = 8,   /* u~_h = EXP_true(u_h, u_2h) */
  EXCMG_K_CG_F64 = 9,     /* all CG steps of a level in one persistent launch (float64);
                             prof_nodes counts nodes x steps */
  EXCMG_K_CG_F32 = 10,    /* the same for a float32 inner solve */
  EXCMG_K_CG_CLUSTER_F64 = 11, /* all CG steps of a small grid in one block cluster (float64) */
  EXCMG_K_CG_CLUSTER_F32 = 12, /* the same in float32 */
  EXCMG_K_CG_RESIDENT_F64 = 13, /* all CG steps of a mid-size grid, vectors resident in the
                                   blocks' shared memory (float64) */
  EXCMG_K_DSOLVE = 14,    /* direct solve of a coarse level (discrete sine transform) */
  EXCMG_K_PROLONG_CMP = 15, /* w_h by a comparison prolongation (options.prolong QUADRATIC
                               or LINEAR) in place of EXP_finite */
  EXCMG_KERNEL_KINDS = 16
} excmg_kernel_kind;

/* Box and grids (Section 2: hx = Lx/Nx ...; Algorithm 1: coarsest grid H, L levels). */
typedef struct {
  double Lx, Ly, Lz;  /* box lengths, > 0 */
  int Nx, Ny, Nz;     /* finest-grid cells per direction */
  int Nx0, Ny0, Nz0;  /* coarsest-grid cells per direction (even) */
} excmg_grid;

/* Solver options.  Fill with excmg_default_options() and override. */
typedef struct {
  int precision;           /* excmg_precision */
  double eps;              /* relative-residual tolerance on levels >= 2: CG stops when
                              ||A u - b||_2 <= eps ||f_h||_2 (the WHILE test of Algorithm 1),
                              ||f_h|| as options.rhs_norm reads it */
  double eps_coarse;       /* same test on levels 0 and 1 when DSOLVE is CG */
  int max_iter;            /* cap on CG iterations per level (per inner solve) */
  double inner_tol;        /* MIXED: inner float32 CG stops at ||r|| <= inner_tol ||r0|| */
  int max_refine;          /* MIXED: cap on refinement steps per level */
  const int* fixed_iters;  /* HOST array of `levels` counts or NULL: run exactly that
                              many CG iterations on each level (FP64 only; parity tests) */
  int tile_z;              /* z-slab depth of the stencil kernels; 0 = library default */
  int chunk;               /* CG iterations enqueued between convergence reads; 0 = auto */
  long long mixed_min_nodes; /* MIXED: grids with fewer nodes use float64 CG (latency-
                              bound there, float32 saves nothing); 0 = library default
                              2^21; 1 = float32 inner solves on every grid */
  int profile;             /* nonzero: time every kernel launch of excmg_solve / excmg_cg
                              with CUDA events on the caller's stream (stats.prof_*);
                              single-problem calls only; adds two event records per launch */
  int dsolve;              /* excmg_dsolve: how levels 0 and 1 are solved (DSOLVE of
                              Algorithm 1) */
  double eps_ratio;        /* per-level tolerance: level l >= 2 of L levels stops at
                              eps * eps_ratio^(L-1-l), so the finest level uses eps and each
                              coarser one eps_ratio times more (64 = 2^6 follows the
                              sixth-order error of u~ from level to level); 1 (the default)
                              or 0: the uniform eps of Algorithm 1 */
  int prolong;             /* excmg_prolong: how the initial guess w_h of levels >= 2 is
                              formed (the initial guess of Algorithm 1); default QUARTIC */
  double* history;         /* HOST array or NULL: the residual history of the finest
                              level (the relative residual against the CG step, as in the
                              figure of Section 5 that plots it): history[k] =
                              ||r_k||_2 / ||b||_2 after k steps, r_k CG's recursively
                              updated residual (the one the stopping test reads), for
                              k = 0 .. min(iters, history_len - 1); later entries are left
                              unchanged.  excmg_solve and excmg_cg (its one level), FP64
                              only; the workspace grows by history_len doubles */
  int history_len;         /* entries of `history` (>= 1 when history is set) */
  int rhs_norm;            /* excmg_rhs_norm: the reading of ||f_h|| in the stopping test */
  double wait_timeout_ms;  /* bound on every device-side wait of a cooperative CG launch
                              (its grid barriers and tensor-copy completions): a wait that
                              runs out ends the launch with EXCMG_ERR_TIMEOUT; 0 = 20000 */
  int test_phantom_blocks; /* TEST ONLY, 0 otherwise: adds this many members that are never
                              launched to the block team of each streaming cooperative CG
                              launch (float64 grids too large for the shared-memory engine,
                              about 2^19 nodes and up; float32 inner solves of MIXED), so
                              that its first grid barrier cannot
                              complete and its wait must run out (with a short
                              wait_timeout_ms, to check that the call returns
                              EXCMG_ERR_TIMEOUT and the context stays usable) */
  int autotune;            /* launch-shape tuning: 1 = before a single solve, time candidate
                              slab depths of every level's residual and tiled CG engine that
                              the cache (per level grid, engine class and device, kept for
                              the process) lacks, and keep the fastest; 0 (default) = use the
                              cache where it holds the level, the models elsewhere; -1 = the
                              models only.  options.tile_z > 0 overrides both */
  int res_rows;            /* y-rows per thread of the residual kernel: 0 (default) = the
                              tuning cache's or the model's choice per level (the model:
                              4 on grids of 2^26 nodes and more, else 1), 1 or 4 = that for
                              every level; other values are EXCMG_ERR_INVALID_ARG.  Four
                              rows share neighbour sums (fewer float64 instructions per
                              node) at a lower occupancy. */
} excmg_options;

/* One entry of the launch-shape cache (options.autotune): a level grid and engine class
   with the tuned and the modelled slab depths and their measured times. */
typedef struct {
  int N[3];                     /* the level's cells */
  int f32;                      /* 1: its CG is the float32 engine of MIXED inner solves */
  int res_tz, res_tz_model;     /* residual slab depth: tuned, modelled */
  double res_ms, res_ms_model;  /* one residual launch at each (ms) */
  int cg_tz, cg_tz_model;       /* slab depth of its CG engine (0: the engine is not tiled) */
  double cg_ms, cg_ms_model;    /* one CG step at each (ms) */
  int res_rows, res_rows_model; /* y-rows per thread of its residual launch (1 or 4); res_ms
                                   is at (res_rows, res_tz), res_ms_model at the model's */
} excmg_tuning;

/* Copies up to `max` cache entries to out (NULL: none) and returns how many there are. */
int excmg_tuning_entries(excmg_tuning* out, int max);
/* Empties the launch-shape cache. */
void excmg_tuning_clear(void);

/* ||f_h||_2 in the WHILE test ||A_h u_h - f_h|| > eps ||f_h|| of Algorithm 1.  The paper
   defines f_h (Section 2, after eq. FD) as the right-hand side vector of eq. (compact),
   but its printed tables fit two different readings:
   LIFT (default): the 2-norm of the assembled right-hand side b of eq. (FD), Dirichlet
     lift included -- this reproduces the finest-grid CG step counts of Table 11;
   FORCING: the 2-norm of (6 f + the six face values of f)/2 over the interior nodes, the
     right-hand side of eq. (compact) alone -- this reproduces the errors of Tables 1-10
     on the 128^3 meshes, where the algebraic error shows, and takes more CG steps.
     Where that vector is zero (f = 0, e.g. Example 2) FORCING uses LIFT: no relative
     test against a zero norm can pass.
   stats.relres and options.history are relative to the same norm. */
typedef enum { EXCMG_RHS_NORM_LIFT = 0, EXCMG_RHS_NORM_FORCING = 1 } excmg_rhs_norm;

/* DSOLVE of Algorithm 1 (levels 0 and 1).  DIRECT: the exact discrete solution by the
   three-dimensional discrete sine transform, which diagonalises the 19-point operator on
   the box (grids whose interior fits one block's shared memory, about 9,000 unknowns;
   larger coarse grids fall back to CG); stats.iters = 0 for these levels and relres the
   residual of the direct solution.  CG: CG from zero to eps_coarse. */
typedef enum { EXCMG_DSOLVE_DIRECT = 0, EXCMG_DSOLVE_CG = 1 } excmg_dsolve;

/* Initial guess of levels >= 2 (Algorithm 1, before the CG loop).  QUARTIC: EXP_finite(u_2h, u_4h) --
   extrapolation to the grid-2h nodes (eqs. jiedian, zhongdian), then tri-quartic
   interpolation over cells of 2x2x2 grid-4h elements (eq. inter); the method of the paper.
   The other two exist to measure what EXP_finite saves: QUADRATIC keeps the extrapolation
   and interpolates tri-quadratically over cells of 2x2x2 grid-2h elements (the
   interpolation of the earlier EXCMG for linear finite elements, which the first remark of
   Section 3.3 finds too inaccurate for the fourth-order scheme); LINEAR is the cascadic
   multigrid prolongation of Section 3: trilinear interpolation of u_2h alone, no
   extrapolation.  All three write the Dirichlet data on the boundary. */
typedef enum { EXCMG_PROLONG_QUARTIC = 0, EXCMG_PROLONG_QUADRATIC = 1,
               EXCMG_PROLONG_LINEAR = 2 } excmg_prolong;

/* Per-solve statistics, valid when the call returns. */
typedef struct {
  int levels;
  int N[EXCMG_MAX_LEVELS][3];        /* cells per level */
  int iters[EXCMG_MAX_LEVELS];       /* CG iterations per level (summed over refinements) */
  int refinements[EXCMG_MAX_LEVELS]; /* MIXED: refinement steps per level */
  double relres[EXCMG_MAX_LEVELS];   /* final ||r||/||f_h|| per level (recursive residual
                                        for FP64; true float64 residual for MIXED; ||f_h||
                                        as options.rhs_norm reads it) */
  long long launches;                /* kernels this call launched (all levels) */
  /* options.profile: per kernel kind (excmg_kernel_kind), summed CUDA-event time of its
     launches that did work, their count, and the node count they covered in total
     (CG launches issued after convergence return at once and are not counted) */
  double prof_ms[EXCMG_KERNEL_KINDS];
  long long prof_launches[EXCMG_KERNEL_KINDS];
  double prof_nodes[EXCMG_KERNEL_KINDS];
  /* options.profile, single solves: the same launch times summed per level, and over all
     launches (EXP_true counts to the finest level; the direct DSOLVE of levels 0 and 1 is
     one launch, counted to level 0) */
  double ms_level[EXCMG_MAX_LEVELS];
  double ms_total;
} excmg_stats;

/* Writes the defaults: precision FP64, eps 1e-9, eps_coarse 1e-12, max_iter 100000,
   inner_tol 1e-4, max_refine 50, fixed_iters NULL, tile_z 0, chunk 0,
   mixed_min_nodes 0, profile 0, dsolve DIRECT, eps_ratio 1 (uniform tolerance),
   prolong QUARTIC, history NULL, history_len 0, rhs_norm LIFT, wait_timeout_ms 0
   (20 s), test_phantom_blocks 0, autotune 0, res_rows 0. */
void excmg_default_options(excmg_options* opt);

/* Human-readable name of a status code (static string). */
const char* excmg_status_string(excmg_status s);

/* Number of levels of `grid`, or -1 if the grid is invalid. */
int excmg_num_levels(const excmg_grid* grid);

/* Bytes of workspace excmg_solve needs for `grid` and `opt` (0 if invalid). */
size_t excmg_workspace_size(const excmg_grid* grid, const excmg_options* opt);

/*
 * excmg_solve -- Algorithm 1.  Levels 0 and 1: CG from zero (eps_coarse).  Each finer
 * level: w_h = EXP_finite(u_2h, u_4h) (Section 3.3: eqs. jiedian and zhongdian on the
 * nodes of grid 2h, tri-quartic Lagrange interpolation eq. inter on every cell of 2x2x2
 * elements of grid 4h), then CG from w_h (interior) until the relative residual is at
 * most eps.  On the finest level, optionally u~_h = EXP_true(u_h, u_2h) (eqs. t1,
 * chenlin; the optional last step).
 *   f        [in]  finest-grid node array: the Poisson right-hand side on ALL nodes
 *                  (the compact RHS uses f at face neighbours, which may be boundary
 *                  nodes).
 *   g        [in]  finest-grid node array; only boundary entries are read (Dirichlet
 *                  data).
 *                  f and g may be device memory, or page-locked host memory mapped into
 *                  the device's address space (cudaHostAlloc, or cudaHostRegister with
 *                  cudaHostRegisterMapped; the same address on host and device): the
 *                  kernels then read them over the host link while they compute, with
 *                  no separate copy.  Any other pointer returns EXCMG_ERR_INVALID_ARG.
 *   u        [out] finest-grid node array in device memory: the FD solution u_h,
 *                  boundary = g.
 *   u_tilde  [out] NULL, or a finest-grid node array in device memory receiving
 *                  EXP_true(u_h, u_2h).
 *   ws, ws_bytes   workspace of at least excmg_workspace_size(grid, opt) bytes.
 *   stats    [out] NULL or host struct.
 * Returns EXCMG_ERR_NOT_CONVERGED if any level hit max_iter (u then holds the last
 * iterate), EXCMG_ERR_NONFINITE if a reduction turned non-finite.
 */
excmg_status excmg_solve(const excmg_grid* grid, const double* f, const double* g,
                         const excmg_options* opt, double* u, double* u_tilde,
                         void* ws, size_t ws_bytes, excmg_stats* stats, void* stream);

/*
 * excmg_grad -- gradient of a node array (Section 5, text of Example 1): on x = 0 and
 * x = Lx the one-sided fourth-order five-point formulas; at interior x-nodes of every
 * x-line the compact system (1/6, 4/6, 1/6) u_x = (u_{i+1} - u_{i-1}) / (2 hx), solved
 * by the Thomas algorithm; likewise along y and z.  Needs Nx, Ny, Nz >= 4 (the five-
 * point formula); Nx0.. are ignored.  ux, uy, uz [out]: node arrays, all nodes.
 * No workspace: the forward sweep is stored in the outputs.
 */
excmg_status excmg_grad(const excmg_grid* grid, const double* u, double* ux, double* uy,
                        double* uz, void* stream);

/*
 * excmg_solve_batched -- `nprob` independent problems (each its own grid, f, g) solved by
 * Algorithm 1 together: each CG step of every active problem runs in ONE launch of the
 * stencil kernels over the union of all problems' tiles; problems are aligned on their
 * finest level.  Problems whose finest grid has 2^18 nodes or more run first, one after
 * another, as single solves (each fills the GPU by itself and takes a single solve's CG
 * engines); the others share the batch's launches.  The results are those of single
 * solves up to rounding.  grids[nprob]: host array; f, g, u: host arrays of device pointers.
 * opt: shared options (fixed_iters must be NULL).  stats: NULL or host array[nprob].
 * Workspace: excmg_workspace_size_batched().  1 <= nprob <= 128.
 */
size_t excmg_workspace_size_batched(int nprob, const excmg_grid* grids,
                                    const excmg_options* opt);
excmg_status excmg_solve_batched(int nprob, const excmg_grid* grids,
                                 const double* const* f, const double* const* g,
                                 const excmg_options* opt, double* const* u, void* ws,
                                 size_t ws_bytes, excmg_stats* stats, void* stream);

/*
 * excmg_adjoint -- gradients of a scalar loss L(u) through the discrete solve
 * u_I = A^{-1} b(f, g), u_B = g, with A the SPD form of eq. (FD) (A = -(printed LHS)):
 *   lambda = A^{-1} (dL/du)_I          (CG on the finest grid, tolerance eps, from 0;
 *                                        A is symmetric so A^T = A)
 *   dL/df  = -R^T lambda               (R: the 7-point right-hand-side operator
 *                                        (6 f_c + sum of face f)/2 of eq. compact)
 *   dL/dg  = LHS_IB^T lambda + dL/du   on boundary nodes (LHS_IB: the boundary columns
 *                                        of the printed left-hand side), 0 inside.
 * The paper has no adjoint; this is the exact transpose of the discrete map.
 *   dLdu [in]: finest node array.  dLdf, dLdg [out]: finest node arrays.
 *   stats: iters[0], relres[0] of the lambda solve.
 * Workspace: excmg_workspace_size_adjoint().  MIXED precision refines the lambda solve.
 */
size_t excmg_workspace_size_adjoint(const excmg_grid* grid, const excmg_options* opt);
excmg_status excmg_adjoint(const excmg_grid* grid, const double* dLdu,
                           const excmg_options* opt, double* dLdf, double* dLdg,
                           void* ws, size_t ws_bytes, excmg_stats* stats, void* stream);

/* ---- single steps of the path, exported for parity tests and custom drivers ---- */

/*
 * excmg_exp_finite -- EXP_finite(u_2h, u_4h) of Algorithm 1 / Section 3.3 onto
 * grid h = `grid`'s finest level: u2h and u4h are node arrays of the grids with
 * Nx/2 and Nx/4 cells.  Writes w (node array of grid h) on all nodes; if g is not NULL
 * the boundary nodes of w are set to g (the CG start), otherwise they keep their
 * interpolated values.  Needs Nx, Ny, Nz divisible by 8.
 */
excmg_status excmg_exp_finite(const excmg_grid* grid, const double* u2h, const double* u4h,
                              const double* g, double* w, void* stream);

/*
 * excmg_exp_true -- EXP_true(u_h, u_2h) of Algorithm 1, its optional last step (Section 3.3): eq. (t1)
 * (16 u_h - u_2h)/15 at the nodes of grid 2h, eq. (chenlin) u_h + (d_a + d_b)/30 along
 * every edge, face diagonal or space diagonal through the other nodes (averaged over the
 * diagonals), d = u_h - u_2h.  uh: grid h node array; u2h: Nx/2 grid.  Needs Nx, Ny, Nz
 * even.
 */
excmg_status excmg_exp_true(const excmg_grid* grid, const double* uh, const double* u2h,
                            double* ut, void* stream);

/* Bytes of workspace excmg_cg and excmg_residual need on the grid Nx x Ny x Nz
   (Nx0.. ignored; each N >= 2); 0 if invalid. */
size_t excmg_workspace_size_level(const excmg_grid* grid, const excmg_options* opt);

/*
 * excmg_cg -- CG on the grid Nx x Ny x Nz alone (the CG loop of Algorithm 1; Nx0.. ignored):
 * from the interior values of u (boundary entries of u must already hold g) until
 * ||r|| <= opt->eps ||b|| (or exactly opt->fixed_iters[0] iterations; MIXED refines with
 * float32 inner solves).  u [in/out].  Workspace: excmg_workspace_size_level().
 * stats: iters[0], refinements[0], relres[0].
 */
excmg_status excmg_cg(const excmg_grid* grid, const double* f, const excmg_options* opt,
                      double* u, void* ws, size_t ws_bytes, excmg_stats* stats,
                      void* stream);

/*
 * excmg_residual -- r = b - A u_I = LHS(u) - RHS(f) at interior nodes (0 on the
 * boundary), eq. (compact) / (FD), in float64; also returns ||r||_2 and ||b||_2 (b with
 * its Dirichlet lift taken from u's boundary entries) in *rnorm, *bnorm (host).
 * Workspace: excmg_workspace_size_level().
 */
excmg_status excmg_residual(const excmg_grid* grid, const double* f, const double* u,
                            double* r, double* rnorm, double* bnorm, void* ws,
                            size_t ws_bytes, void* stream);

/* ---- an entry point for callers that cannot allocate device memory ----
 *
 * excmg_cg_noalloc -- the same computation as excmg_cg (float64 CG on the grid
 * Nx x Ny x Nz from the interior of u, with the same outputs and status codes), but it
 * takes no workspace: its scratch is a device array built into the library.  Options
 * are checked as for excmg_cg; precision must be EXCMG_FP64, and options.history and
 * options.profile must be unset (EXCMG_ERR_INVALID_ARG otherwise: they need host-side
 * buffers and events that this entry point does not keep).
 * The paper has no counterpart; this exists for callers that must not allocate device
 * memory -- an application or framework that owns all device memory through its own
 * pool, code that cannot afford cudaMalloc's implicit synchronisation, or a binding
 * with no access to a CUDA allocator.  Those callers pass inputs and outputs only.
 *   Limit: the scratch is EXCMG_NOALLOC_SCRATCH_BYTES (16 MiB) per device, held from the
 *   moment the library is loaded until the process exits; it holds four float64 node
 *   arrays plus ~66 KB, i.e. grids up to about 520,000 nodes (80 x 80 x 80 cells does
 *   not fit, 64 x 64 x 64 does).  A larger grid returns EXCMG_ERR_WORKSPACE before any
 *   work is enqueued.  Only EXCMG_FP64 is accepted.
 *   Set-up: the first call on each device looks up the scratch's device address (with
 *   that device current) and caches it.
 *   Sharing: every call uses the same scratch and leaves its last contents there (the
 *   call clears what must start at zero itself).  Calls whose work overlaps on the GPU
 *   -- on different streams or from different host threads -- race on the scratch and
 *   must be serialised by the caller.
 */
#define EXCMG_NOALLOC_SCRATCH_BYTES (16u << 20)
excmg_status excmg_cg_noalloc(const excmg_grid* grid, const double* f,
                              const excmg_options* opt, double* u, excmg_stats* stats,
                              void* stream);

#ifdef __cplusplus
}
#endif

#endif /* EXCMG_H */
