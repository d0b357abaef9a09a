/*
 * mcwind -- mass-consistent wind downscaling on one GB300 (sm_103a).
 *
 * The C boundary of a multigrid solver for the Lagrange multiplier of
 * Mandel et al., "Simple finite elements and multigrid for efficient
 * mass-consistent wind downscaling in a coupled fire-atmosphere model":
 *
 *   Eq. 1  min 1/2 int (u-u0).A(u-u0)  s.t. div u = 0 in Omega, u.n = 0 on Gamma
 *   Eq. 3  u = u0 + A^{-1} grad lambda
 *   Eq. 4  -div A^{-1} grad lambda = div u0,  lambda = 0 on the top and the
 *          lateral faces, natural condition on the terrain surface Gamma
 *   Eq. 5  int A^{-1} grad lambda . grad mu = - int grad mu . u0
 *   Eq. 6-7 (Sec. 3) multigrid: Gauss-Seidel smoothing in vertical columns,
 *          variational coarse correction K_c = P^T K P, adaptive
 *          semicoarsening, direct solve on the coarsest grid.
 *
 * A = diag(a1^2, a2^2, a3^2) with the caller's penalty constants a[0..2]
 * (Sec. 2, after Eq. 1).  Discretization: isoparametric trilinear
 * hexahedra on a logically Cartesian, terrain-following node grid
 * (Sec. 2), 2x2x2 Gauss quadrature for the left side of Eq. 5.
 *
 * Grids and layouts.  A problem has nx x ny x nz cells and
 * (nx+1)(ny+1)(nz+1) nodes.  Every nodal array at this boundary is
 * row-major [k][j][i] with i fastest (k = 0 is the ground), float64, and a
 * vector field is [3][k][j][i] (components x, y, z).  The free unknowns are
 * the nodes with 1 <= i <= nx-1, 1 <= j <= ny-1, 0 <= k <= nz-1; lambda is
 * written as 0 at every other node.
 *
 * Memory and streams.  Pointers named "device" are CUDA device (or
 * managed) memory on the current device; "host" pointers are ordinary
 * host memory.  The caller owns every buffer, including the workspace
 * whose size mcwind_plan_create reports; the library never allocates device
 * memory.  Work is enqueued on the caller's stream (a cudaStream_t passed as
 * void*; NULL is the legacy default stream).  The library keeps the
 * workspace pointer and the geometry pointers given to mcwind_assemble
 * until the plan is destroyed or assembled again: they must stay valid and
 * unchanged.  A plan is not re-entrant: do not use one plan from two host
 * threads or on two streams at once.
 *
 * Errors.  Every int-returning call returns MCWIND_OK (0) or a negative
 * MCWIND_E* code; mcwind_strerror names it.  No exception crosses the
 * boundary.  On MCWIND_ECUDA the CUDA error is reported by
 * mcwind_last_cuda_error().
 */
#ifndef MCWIND_H
#define MCWIND_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcwind_plan_s* mcwind_plan;

enum {
  MCWIND_OK = 0,
  MCWIND_EINVAL = -1,     /* bad argument: size, null pointer, option, level */
  MCWIND_EGEOM = -2,      /* an element has detJ <= 0 at a quadrature point */
  MCWIND_ENONFINITE = -3, /* u0 (hence the load vector) is not finite */
  MCWIND_ENOTCONV = -4,   /* max_cycles reached above rtol; lambda and stats are written */
  MCWIND_ECUDA = -5,      /* a CUDA call failed */
  MCWIND_ESTATE = -6,     /* call out of order (e.g. solve before assemble) */
  MCWIND_ETIMEOUT = -7,   /* a kernel's bounded device wait ran out (a copy that did not
                             arrive within its limit); the solve stops, lambda unwritten */
  MCWIND_ESHIFT = -8      /* MCWIND_OP_SEPARABLE on a grid that is not in shift form */
};

enum { MCWIND_PREC_F64 = 0, MCWIND_PREC_MIXED = 1 };
enum { MCWIND_RHS_GAUSS8 = 0, MCWIND_RHS_CENTER1 = 1 };
enum { MCWIND_RULE_PAPER = 0, MCWIND_RULE_OPERATOR = 1 };
enum { MCWIND_AT_CENTERS = 0, MCWIND_AT_GAUSS = 1 };
enum { MCWIND_FORWARD = 0, MCWIND_BACKWARD = 1 };
enum { MCWIND_ACCEL_NONE = 0, MCWIND_ACCEL_CG = 1 };
enum { MCWIND_U0_NODES = 0, MCWIND_U0_CENTERS = 1 };
enum { MCWIND_ARITH_F64 = 0, MCWIND_ARITH_DFLOAT = 1 };
enum { MCWIND_OP_STORED = 0, MCWIND_OP_SEPARABLE = 1 };

#define MCWIND_WARM 1u        /* mcwind_solve flag: start from the caller's lambda */
#define MCWIND_HIST 256

typedef struct {
  /* Gauss-Seidel sweeps before and after the coarse correction (Sec. 3
     uses four smoothing steps in a cycle: default 2 and 2). */
  int nu_pre, nu_post;
  /* Semicoarsening ratio (Sec. 3): MCWIND_RULE_PAPER uses h3/(h1 a3) as
     printed; MCWIND_RULE_OPERATOR (default) uses a3 h3/(a1 h1), the ratio
     of the operator's horizontal to vertical coupling strengths when
     A = diag(a^2).  The two agree when a3 = a1. */
  int coarsen_rule;
  /* Stop coarsening at a level with at most this many free nodes, which is
     then solved directly (Sec. 3).  Default 1024, at most 4096. */
  int coarsest_max;
  /* MCWIND_PREC_F64: every step in float64.  MCWIND_PREC_MIXED: float32
     V-cycles inside a float64 residual / update loop. */
  int precision;
  /* MCWIND_RHS_GAUSS8 (default): right side of Eq. 5 by 2x2x2 Gauss with u0
     interpolated from the nodes; MCWIND_RHS_CENTER1: one point at the
     element center with u0 there (Sec. 2). */
  int rhs_quad;
  /* 1 (default): post-smoothing visits the nodes in the reverse order of
     pre-smoothing (column groups 3..0, each column top-down), which makes
     the cycle symmetric; 0: the same order as pre-smoothing. */
  int post_reverse;
  /* MCWIND_ACCEL_NONE (default): the multigrid iteration of Sec. 3, one
     V-cycle per iteration.  MCWIND_ACCEL_CG: conjugate gradients with one
     V-cycle as the preconditioner per iteration (needs post_reverse = 1, the
     symmetric cycle); same solution, fewer cycles when the cycle alone
     converges slowly. */
  int accel;
  /* 1 (default): each solver iteration is captured once as a CUDA graph
     (on a stream the plan creates) and replayed on the caller's stream;
     0: direct launches.  Same kernels, same order, same results.  While the
     profiler is on, direct launches are used. */
  int use_graphs;
  /* MCWIND_U0_NODES (default): u0 arrays are nodal [3][nz+1][ny+1][nx+1] and
     interpolated trilinearly.  MCWIND_U0_CENTERS: u0 is one vector per element
     center, [3][nz][ny][nx] (the paper's representation of the wind, Sec. 2),
     constant over the element in the load vector and in the recovery.  The
     gradient entry points require MCWIND_U0_NODES. */
  int u0_at;
  /* Arithmetic of the 2x2x2-Gauss element kernels (stiffness and load
     vector).  MCWIND_ARITH_DFLOAT (default): pairs of floats (about 48
     significant bits) on the float pipe, which issues 61 times the float64
     rate on GB300, for the element values and for their sums into the
     stencil and the load vector (each entry is rounded to float64 once, by
     the last element that adds to it); MCWIND_ARITH_F64: float64 throughout.
     The Galerkin products of the coarser levels sum in float pairs either
     way (their interpolation weights make every product exact); the stored
     operators and the solve are float64 (float32 inside the float64
     refinement of MCWIND_PREC_MIXED).  With MCWIND_OP_SEPARABLE the same
     choice applies to the column factors' Gauss sums, the finest and
     coarsest float64 rows expanded from the factors, and the load vector
     (float pairs from its own factors; float64 element by element). */
  int element_arith;
  /* V-cycles between two convergence checks, 1..8; 0 (default) = 6 with
     MCWIND_PREC_MIXED, 1 with MCWIND_PREC_F64 (mcwind_plan_query reports
     the value in use).  In mixed precision the cycles of one check run back
     to back on the float32 correction (each from the previous one's result,
     as in the plain multigrid iteration) before the float64 update and
     residual, which are computed once per check: a float64 residual costs
     about as much as a float32 cycle on GB300 (its 27 multiply-adds per node
     run at the float64 rate), and the float32 correction keeps converging
     for 6 cycles on the benchmark's grids.  Solves stop at a check, so the
     cycle count is a multiple of this (or max_cycles).  Ignored with
     MCWIND_ACCEL_CG (one cycle per iteration). */
  int cycles_per_check;
  /* Form of the float32 cycle's operators (MCWIND_PREC_MIXED).
     MCWIND_OP_STORED (default): the 27 coefficients of every node are stored
     on every level, float64 and a float32 copy (general hexahedra).
     MCWIND_OP_SEPARABLE: for a terrain-following grid in shift form (X and Y
     the same in every layer, z = z_s(x, y) + zeta_k, Sec. 2) the stiffness of
     Eq. 5 is exactly sum_t H_t (x) V_t, four horizontal 9-point operators on
     the node columns times four vertical tridiagonal ones on the layers (the
     element Jacobian splits into the terrain's slopes and the layer
     thickness), and the Galerkin products of Eq. 7 keep that form.  The
     float32 cycle then stores 36 values per column and 12 per layer on every
     level and rebuilds each row as it smooths; float64 operators are kept
     for the finest level (the float64 residual of the refinement) and the
     coarsest (its direct solve) only.  Needs MCWIND_PREC_MIXED;
     mcwind_assemble returns MCWIND_ESHIFT when the grid is not in shift form
     (to 1e-10 of the coordinates' magnitude). */
  int op_form;
} mcwind_options;

typedef struct {
  int cycles;            /* V-cycles run (one per conjugate-gradient iteration with CG) */
  int status;            /* MCWIND_OK or MCWIND_ENOTCONV */
  double norm_f;         /* ||f_F||_2, f the load vector of Eq. 5 */
  double rel_res;        /* final ||f_F - K_FF lambda_F||_2 / ||f_F||_2 */
  double rate;           /* geometric mean residual reduction per cycle, from cycle 3 on */
  double res_hist[MCWIND_HIST]; /* relative residual before cycle 1 (index 0), then after each;
                                   between two checks (cycles_per_check > 1) the entries are
                                   the geometric interpolation of the checked values */
} mcwind_stats;

/* Fill *opt with the defaults listed above. */
void mcwind_default_options(mcwind_options* opt);

/* Plan the multigrid hierarchy (host only, no CUDA call).
 * nx, ny, nz >= 2 cells; a[3] > 0 (host); h1 > 0 is the horizontal node
 * spacing and h3 (host, nz entries > 0) the thickness of each layer from
 * the ground up (means over the columns on a terrain-following grid): the
 * inputs of the semicoarsening rule of Sec. 3.  opt may be NULL (defaults).
 * On success *out is a new plan and *workspace_bytes the device workspace
 * it needs.  EINVAL on bad sizes or options. */
int mcwind_plan_create(int nx, int ny, int nz, const double a[3], double h1, const double* h3,
                       const mcwind_options* opt, mcwind_plan* out, size_t* workspace_bytes);

/* The plan's options as they stand (host output; mcwind_plan_set_tuning
 * changes nu_pre and nu_post; a cycles_per_check of 0 is reported as the
 * interval in use) and its device workspace bytes.  Either output may be
 * NULL.  Host only.  EINVAL on a NULL plan. */
int mcwind_plan_query(mcwind_plan plan, mcwind_options* opt, size_t* workspace_bytes);

/* Number of grid levels (finest = 0); negative code on a NULL plan. */
int mcwind_plan_num_levels(mcwind_plan plan);

/* Level description (host outputs; any output pointer may be NULL):
 * dims[3] = node counts (Nx, Ny, Nz); for level < num_levels-1, *hx/*hy = 1
 * when the transfer to the next level halves that horizontal direction and
 * kmap[0 .. Nz_next-1] = the fine k of each coarse node layer (kmap must
 * hold Nz_next ints).  The last level reports hx = hy = 0, no kmap. */
int mcwind_plan_level(mcwind_plan plan, int level, int dims[3], int* hx, int* hy, int* kmap);

/* Assemble (Sec. 2; Eq. 5 left side; Eq. 7 second row on every level).
 * workspace: device, >= workspace_bytes, 256-byte aligned.  X, Y, Z: device
 * node coordinates [nz+1][ny+1][nx+1].  Builds the 27-point stiffness
 * stencil by 2x2x2 Gauss quadrature, the Galerkin operators of all coarser
 * levels and the coarsest direct solver (MCWIND_OP_SEPARABLE: the column and
 * layer factors of every level, the finest and coarsest float64 rows).  The
 * plan keeps the X, Y, Z pointers: they must stay valid and unchanged until
 * the plan is assembled again or destroyed (the load vector, the recovery,
 * the weak divergence and the gradient calls read them).  Synchronizes the
 * stream once at the end to report EGEOM when an element is inverted or
 * degenerate and ESHIFT when a separable plan's grid is not in shift form. */
int mcwind_assemble(mcwind_plan plan, void* workspace, const double* X, const double* Y,
                    const double* Z, void* stream);

/* Solve K_FF lambda_F = f_F (Eq. 5) by V-cycles (Sec. 3) until
 * ||f_F - K_FF lambda_F|| <= rtol ||f_F|| or max_cycles (0..MCWIND_HIST-1).
 * u0: device [3][nz+1][ny+1][nx+1].  lambda: device [nz+1][ny+1][nx+1];
 * read as the first iterate when flags & MCWIND_WARM (its fixed-node
 * entries are ignored), always written (0 at fixed nodes).  stats: host,
 * may be NULL.  Reads the residual norm back after every cycle (one stream
 * synchronization per cycle).  Returns OK, ENOTCONV (lambda and stats still
 * written), ENONFINITE (u0 not finite), ESTATE (not assembled), ETIMEOUT (a
 * kernel's bounded wait ran out; the status stays set until the plan is
 * assembled again). */
int mcwind_solve(mcwind_plan plan, const double* u0, double* lambda, double rtol, int max_cycles,
                 unsigned flags, mcwind_stats* stats, void* stream);

/* Solve K_FF x_F = f_F for the caller's load vector instead of Eq. 5's:
 * f device [nz+1][ny+1][nx+1] (fixed-node entries ignored), x as lambda in
 * mcwind_solve (read when flags & MCWIND_WARM, always written).  Same
 * iteration, stopping test (relative to ||f_F||), codes and stats. */
int mcwind_solve_rhs(mcwind_plan plan, const double* f, double* x, double rtol, int max_cycles,
                     unsigned flags, mcwind_stats* stats, void* stream);

/* Recover the wind, Eq. 3: u = u0 + A^{-1} grad lambda.
 * where = MCWIND_AT_CENTERS: u device [3][nz][ny][nx] at element centers
 * (u0 there is the mean of the 8 corners); MCWIND_AT_GAUSS: u device
 * [3][8][nz][ny][nx] at the 2x2x2 Gauss points, g = gx + 2 gy + 4 gz with
 * gx = 0 at xi = -1/sqrt(3).  u0, lambda: device nodal, as in mcwind_solve. */
int mcwind_recover(mcwind_plan plan, const double* u0, const double* lambda, double* u,
                   int where, void* stream);

/* Gradients of a loss l(u) with u the wind at the element centers (Eq. 3,
 * mcwind_recover with MCWIND_AT_CENTERS) and lambda from Eq. 5 (2x2x2 load
 * vector), by the adjoint method; the same self-adjoint multigrid solves the
 * adjoint system.  With gu = dl/du (device [3][nz][ny][nx]):
 *   1. mcwind_recover_adjoint: h = G^T A^{-1} gu (device nodal) and
 *      du0 = C^T gu (device [3][nz+1][ny+1][nx+1]), G the gradient and C the
 *      corner mean at the centers;
 *   2. mu = K_FF^{-1} h_F by mcwind_solve_rhs;
 *   3. mcwind_adjoint_finish: du0 -= I^T B^T mu (I: nodes to Gauss points, B
 *      the weak divergence), so du0 = dl/du0; and dloga (host, 3) =
 *      dl/d(log a_d) = 2 a_d^-2 (mu^T K_d lambda - sum_centers gu_d d_d lambda),
 *      K_d the stiffness of the d-th derivative term.  Synchronizes once.
 * lambda and mu must be 0 at fixed nodes (as mcwind_solve writes them). */
int mcwind_recover_adjoint(mcwind_plan plan, const double* gu, double* h, double* du0,
                           void* stream);
int mcwind_adjoint_finish(mcwind_plan plan, const double* mu, const double* lambda,
                          const double* gu, double* du0, double* dloga, void* stream);

/* Load vector f of Eq. 5 (right side; plan's quadrature) at every node,
 * device [nz+1][ny+1][nx+1]; 0 at fixed nodes. */
int mcwind_rhs(mcwind_plan plan, const double* u0, double* f, void* stream);

/* Discrete weak divergence (B u)_m = sum_e sum_g detJ grad N_m(g) . u_e(g),
 * the constraint operator of Eq. 5, for u given at the Gauss points, device
 * [3][8][nz][ny][nx]; out device nodal, every node. */
int mcwind_weak_div(mcwind_plan plan, const double* ug, double* out, void* stream);

/* ---- the steps of one V-cycle, one level at a time (Sec. 3) ----------
 * Vectors are device float64 [Nz][Ny][Nx] of the level's node dims.
 * precision selects the float64 or the float32 kernels (float32 needs a
 * plan created with MCWIND_PREC_MIXED); float32 work converts at entry and
 * exit.  These calls use the level's internal buffers: they must not run
 * while mcwind_solve runs on the same plan.  With MCWIND_OP_SEPARABLE the
 * float32 calls use the separable operator; the float64 residual and
 * smoother exist on the finest and the coarsest level only (EINVAL
 * elsewhere), the float64 V-cycle not at all, and the stencil export
 * rebuilds the rows from the float64 or float32 factors. */

/* Export the level's stencil: out device [27][Nz][Ny][Nx], plane
 * s = (di+1) + 3(dj+1) + 9(dk+1) holding the coefficient of node
 * (i+di, j+dj, k+dk) in row (i, j, k) of K_FF (0 outside the free block). */
int mcwind_level_stencil(mcwind_plan plan, int level, int precision, double* out, void* stream);

/* r = f - K x at the free nodes, 0 elsewhere. */
int mcwind_level_residual(mcwind_plan plan, int level, int precision, const double* x,
                          const double* f, double* r, void* stream);

/* sweeps Gauss-Seidel sweeps on K x = f in place (column groups by (i mod 2)
 * + 2 (j mod 2); MCWIND_FORWARD: groups 0..3, columns bottom-up;
 * MCWIND_BACKWARD: groups 3..0, columns top-down). */
int mcwind_level_smooth(mcwind_plan plan, int level, int precision, double* x, const double* f,
                        int sweeps, int direction, void* stream);

/* f_c = P^T r (Eq. 7 first row) from level to level+1. */
int mcwind_level_restrict(mcwind_plan plan, int level, int precision, const double* r,
                          double* fc, void* stream);

/* f_c = P^T (f - K x) (Eq. 7 first row) from level to level+1, the residual
 * not stored where the float32 separable cycle fuses the two (a transfer
 * that keeps the columns). */
int mcwind_level_residual_restrict(mcwind_plan plan, int level, int precision, const double* x,
                                   const double* f, double* fc, void* stream);

/* x += P e_c (Eq. 7 last row) from level+1 to level. */
int mcwind_level_prolong(mcwind_plan plan, int level, int precision, const double* ec, double* x,
                         void* stream);

/* x = K_c^{-1} f on the coarsest level (direct; 0 at fixed nodes). */
int mcwind_coarse_solve(mcwind_plan plan, const double* f, double* x, void* stream);

/* One V-cycle on level 0 (x in place): the pre-smoothing, restriction,
 * recursive coarse correction, prolongation and post-smoothing of Sec. 3. */
int mcwind_vcycle(mcwind_plan plan, int precision, double* x, const double* f, void* stream);

/* Residual norms without allocating anything.  For callers that cannot
 * call cudaMalloc at the point where they check a solution: a host model that
 * hands all device memory to its own pool at start-up and forbids later
 * allocations, or a latency-bound loop in which an allocation (which may
 * synchronize the whole device) is not allowed.  The paper has no
 * counterpart: this is the solver's float64 convergence check exposed on its
 * own.  norms (device, 2 doubles) receives ||f_F||_2 and
 * ||f_F - K_FF lambda_F||_2 with K_FF the plan's assembled finest operator;
 * f and lambda are device [nz+1][ny+1][nx+1] (entries at fixed nodes are
 * ignored: lambda counts as 0 there).  Nothing is allocated and the stream is
 * not synchronized.  The per-block partial sums live in a static device
 * array of 2 x 131072 doubles (2 MiB, held by every GPU that loads the
 * library until the process exits): the finest grid may need at most
 * 131072 blocks of 32 x 4 node columns, i.e. ceil(H/32) * ceil((ny+1)/4) * 2
 * <= 131072 with H = (nx+2)/2 rounded up to 32; larger plans get
 * MCWIND_EINVAL before any device work.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current: make that first call before any stream capture.  Every call shares
 * the array and overwrites what it reads; calls that overlap on the GPU race
 * on it.  ESTATE if the plan is not assembled. */
int mcwind_residual_norm_noalloc(mcwind_plan plan, const double* f, const double* lambda,
                                 double* norms, void* stream);

/* ---- many independent domains ---------------------------------------------
 * A batch groups n assembled plans (independent domains of any sizes) whose
 * solves run together.  One solve is ONE CUDA graph launch and one
 * device-to-host read: per-domain set-up branches, then a conditional WHILE
 * node whose body holds a conditional IF node per domain (its
 * cycles_per_check V-cycles, refinement update and float64 residual) and a
 * bookkeeping kernel that computes every domain's relative residual on the
 * device, keeps iterating exactly the domains still above rtol and ends the
 * loop when none is, or when the next check would pass max_cycles (so each
 * domain gets exactly the result of its own mcwind_solve).  The graph is
 * built on the first solve and rebuilt when the arguments (tolerance, cycle
 * limit, flags, buffers) or a plan's workspace or tuning change.  Plans must
 * use the plain multigrid iteration (accel = MCWIND_ACCEL_NONE), stay
 * assembled and keep their workspaces while the batch lives; a plan belongs
 * to at most one batch.  Host arrays of device pointers are passed per
 * domain. */
typedef struct mcwind_batch_s* mcwind_batch;

/* Device workspace bytes a batch of n domains needs (the per-domain
 * residual histories and the graph's bookkeeping; about 2.1 KB per domain). */
size_t mcwind_batch_workspace_bytes(int n);

/* plans: host array of n assembled plans.  workspace: device, >=
 * mcwind_batch_workspace_bytes(n), 256-byte aligned, caller-owned. */
int mcwind_batch_create(int n, const mcwind_plan* plans, void* workspace, mcwind_batch* out);

/* Solve every domain d: u0[d], lambda[d] as in mcwind_solve.  Checks every
 * cycles_per_check cycles of the first plan (give the plans one setting), up
 * to the last check within max_cycles.  stats: host, n entries, may be NULL.
 * Returns OK, ENOTCONV (some domain above rtol), ENONFINITE (some domain's
 * wind is not finite; the others are solved), ETIMEOUT (a kernel's bounded
 * wait ran out), EINVAL. */
int mcwind_batch_solve(mcwind_batch batch, const double* const* u0, double* const* lambda,
                       double rtol, int max_cycles, unsigned flags, mcwind_stats* stats,
                       void* stream);

void mcwind_batch_destroy(mcwind_batch batch);

/* Change the smoothing sweeps and the smoother's thread-block height (column
 * rows per block: 1, 2, 4 or 8; default 4; the separable form's staged
 * smoother always uses 4) of an existing plan.  Used by the batch autotuner;
 * invalidates the plan's captured iteration graph. */
int mcwind_plan_set_tuning(mcwind_plan plan, int nu_pre, int nu_post, int gs_block_rows);

/* Self-test of the bounded device waits: one block waits, with the same
 * bounded wait as the solver's kernels, on a barrier that nothing completes.
 * The wait gives up after limit_us microseconds (1 .. 1e6), sets the plan's
 * status word and the kernel returns; the call then returns MCWIND_ETIMEOUT,
 * as a solve on this plan does until it is assembled again.  The GPU context
 * stays usable throughout.  Synchronizes the stream.  The paper has no
 * counterpart: this tests how the library reports a copy that never arrives. */
int mcwind_plan_wait_selftest(mcwind_plan plan, int limit_us, void* stream);

/* ---- measurement --------------------------------------------------------
 * Kernel classes timed by the optional profiler (CUDA events recorded on the
 * caller's stream around each launch of the class while profiling is on). */
enum {
  MCWIND_K_ASSEMBLE = 0,    /* element stiffness, 2x2x2 Gauss, scatter */
  MCWIND_K_RAP,             /* Galerkin stages K_c = P^T K P (of the factors when separable) */
  MCWIND_K_SETUP,           /* stencil finalize, float32 copy, coarsest inverse, factors */
  MCWIND_K_RHS,             /* load vector of Eq. 5 */
  MCWIND_K_OUTER_RESIDUAL,  /* float64 residual + norm on the finest level */
  MCWIND_K_SMOOTH_FINE,     /* Gauss-Seidel on the finest level */
  MCWIND_K_SMOOTH_COARSE,   /* Gauss-Seidel on coarser levels */
  MCWIND_K_RESIDUAL_FINE,   /* cycle residual on the finest level */
  MCWIND_K_RESIDUAL_COARSE, /* cycle residual on coarser levels */
  MCWIND_K_RESTRICT,        /* f_c = P^T r, all levels */
  MCWIND_K_PROLONG,         /* x += P e_c, all levels */
  MCWIND_K_COARSE_SOLVE,    /* dense solve on the coarsest level */
  MCWIND_K_UPDATE,          /* float64 update of the mixed refinement */
  MCWIND_K_RECOVER,         /* u = u0 + A^{-1} grad lambda */
  MCWIND_K_KRYLOV,          /* conjugate-gradient vector updates and dots */
  MCWIND_K_OTHER,           /* layout conversion, norms, memsets */
  MCWIND_K_KINDS
};

/* Number of CUDA kernels this library has launched in this process (all
 * plans, all threads); a monotone counter. */
long long mcwind_launch_count(void);

/* enable = 1: reset the plan's profile and time every kernel class from now
 * on; enable = 0: stop timing (the profile is kept). */
int mcwind_profile(mcwind_plan plan, int enable, void* stream);

/* Synchronize the stream, then write per class k < nkinds the summed device
 * time in ms (ms[k]) and the number of launches timed (launches[k]); returns
 * MCWIND_K_KINDS or a negative code.  Host outputs. */
int mcwind_profile_read(mcwind_plan plan, double* ms, long long* launches, int nkinds,
                        void* stream);

void mcwind_plan_destroy(mcwind_plan plan);
const char* mcwind_strerror(int code);
/* The last CUDA error seen by this thread inside the library (cudaError_t). */
int mcwind_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MCWIND_H */
