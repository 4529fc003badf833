/*
 * pbm.h - C ABI of the reduced-Newton MG-MINRES library for the variable-thickness-sheet (VTS)
 * minimum-compliance problem solved by the penalty-barrier multiplier (PBM) method.
 *
 * Paper: M. Brune, M. Kocvara, "On barrier and modified barrier multigrid methods for 3d topology
 * optimization" (arXiv:1904.06556).
 *
 * Conventions shared by every call
 *   - Grids are structured nx x ny x nz arrays of cubes of edge h (Section 6) with trilinear (Q1)
 *     displacements and one density per element.
 *       node id  = i + (nx+1) * (j + (ny+1) * k),   0 <= i <= nx, 0 <= j <= ny, 0 <= k <= nz
 *       dof      = 3 * node + c,                     c = 0, 1, 2  (x, y, z displacement)
 *       element  = i + nx * (j + ny * k)
 *       local node of an element: a = ix + 2 iy + 4 iz at node (i+ix, j+iy, k+iz); local dof 3a + c.
 *     Displacement vectors hold every node (n = 3 (nx+1)(ny+1)(nz+1) entries). Supported
 *     (Dirichlet) dofs are eliminated: their rows and columns of K(rho) and S are those of the
 *     identity, and every right-hand side must be zero there.
 *   - Vectors of the reduced Newton system (eq. (system)) have n + 1 entries: the n displacement
 *     dofs followed by the scalar alpha.
 *   - Every pointer argument named *_dev is a device pointer to memory the CALLER owns and keeps
 *     alive until the work on `stream` has finished; the library never frees it. Arrays are dense
 *     and contiguous (no strides); double pointers must be 8-byte aligned, float pointers 4-byte.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream. Calls
 *     enqueue work and return without synchronising, except where a call returns host scalars or
 *     says otherwise. Calls on one grid handle must not run concurrently from several host threads.
 *   - Every call returns an int status: PBM_OK (0) or a negative error code. On error nothing is
 *     guaranteed about the outputs, and pbm_last_error() gives a one-line message (per host
 *     thread). A CUDA error during a call is reported as PBM_ECUDA.
 *   - All work runs on the CUDA device that is current when the grid is created; the library
 *     makes that device current itself on every call.
 */
#ifndef PBM_H
#define PBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pbm_grid pbm_grid; /* opaque handle: grid, multigrid hierarchy and workspace */

enum pbm_status {
    PBM_OK = 0,
    PBM_EINVAL = -1,       /* invalid argument (sizes, null pointers, unsupported combination)  */
    PBM_ENOMEM = -2,       /* device or host allocation failed                                  */
    PBM_ECUDA = -3,        /* a CUDA runtime call or kernel launch failed                       */
    PBM_EBREAKDOWN = -4,   /* MINRES: v^T M^{-1} v < 0, the preconditioner is not SPD           */
    PBM_ENOTCONV = -5,     /* iteration limit reached before the tolerance                      */
    PBM_ETIMEOUT = -6,     /* a bounded device-side wait gave up                                */
    PBM_ELINESEARCH = -7,  /* Armijo backtracking failed                                        */
    PBM_ENONFINITE = -8,   /* a NaN or Inf was found in an input or a reduction                 */
    PBM_ESTATE = -9        /* call out of order (e.g. S applied before pbm_set_state)           */
};

enum pbm_support {         /* Section 6: supports of the two test problems                       */
    PBM_CANTILEVER = 0,    /* every node of the face x = 0 fixed in all directions              */
    PBM_BRIDGE_CORNERS = 1,/* the four corner nodes of the bottom face z = 0 fixed               */
    PBM_BRIDGE_EDGES = 2,  /* the two bottom edges {x = 0, z = 0} and {x = nx, z = 0} fixed      */
    PBM_FREE = 3           /* no support (K singular; for operator tests only)                  */
};

enum pbm_precision {
    PBM_FP64 = 0,          /* every operator, smoother, transfer and Krylov vector in FP64      */
    PBM_MIXED = 1          /* FP32 operator / smoother / transfers / inner Krylov vectors inside
                              an FP64 iterative refinement; FP64 dots, scalars and coarsest solve */
};

enum pbm_op {
    PBM_OP_K = 0,          /* K(rho) of eq. (1), rho from pbm_set_density                        */
    PBM_OP_S = 1           /* reduced Newton matrix S of eq. (S), from pbm_set_state             */
};

enum pbm_epilogue {        /* what a fused operator launch writes (pbm_apply_fine_f32)           */
    PBM_EPI_APPLY = 0,     /* y = A x                                                            */
    PBM_EPI_RESID = 1,     /* y = b - A x                                                        */
    PBM_EPI_JACOBI = 2     /* y = x + omega D^{-1} (b - A x), one damped-Jacobi sweep             */
};

enum pbm_smoother {        /* smoothing of the multigrid V-cycle (Section 5.2; the paper uses Gauss-Seidel) */
    PBM_SMOOTHER_JACOBI = 0,    /* damped Jacobi x += omega_k D^{-1} (b - A x), omega_k = theta / lambda_k */
    PBM_SMOOTHER_CHEBYSHEV = 1, /* Chebyshev acceleration of Jacobi (Saad, Iterative Methods, Alg. 12.1) on
                                   the interval [0.1, 1.4] lambda_k of D^{-1} A: each pass of nu steps damps
                                   that interval by the Chebyshev polynomial of degree nu (and every
                                   eigenvalue up to 1.5 lambda_k); same operator applications per step as a
                                   Jacobi sweep                                                          */
    PBM_SMOOTHER_GAUSS_SEIDEL = 2  /* the paper's (point) Gauss-Seidel, made parallel: multicolour sweeps over
                                   24 dof colours 3 ((i mod 2) + 2 (j mod 2) + 4 (k mod 2)) + component (and
                                   alpha as a 25th for S), x_c += D_c^{-1} (b - A x)_c colour after colour
                                   (no two dofs of a colour are coupled); forward before the coarse
                                   correction, backward after it. One operator application per colour, so
                                   24 (25) per sweep. Not for batched solves.                            */
};

typedef struct pbm_grid_desc {
    int nx, ny, nz;        /* fine elements per direction, >= 1                                   */
    int levels;            /* multigrid levels >= 1; nx, ny, nz divisible by 2^(levels-1)       */
    int support;           /* enum pbm_support                                                   */
    int precision;         /* enum pbm_precision                                                 */
    double E, nu;          /* isotropic material, E > 0, -1 < nu < 0.5                          */
    double h;              /* fine element edge > 0                                             */
    int pre_sweeps;        /* smoothing steps before / after the coarse correction (Chebyshev:
                              at most 9 each)                                                    */
    int post_sweeps;
    double jacobi_theta;   /* Jacobi weight on level k is theta / lambda_k (lambda_k: Lanczos
                              estimate of lambda_max(D_k^{-1} A_k)); 0 < theta < 2               */
    int lanczos_steps;     /* Lanczos steps of that estimate, 2..64                              */
    double inner_rtol;     /* PBM_MIXED: relative tolerance of each inner (FP32) MINRES solve    */
    int smoother;          /* enum pbm_smoother                                                   */
} pbm_grid_desc;

typedef struct pbm_grid_info {
    int levels;
    int nx[16], ny[16], nz[16];   /* per level, 0 = finest                                       */
    int64_t n[16];                /* 3 * nodes per level                                        */
    int64_t m[16];                /* elements per level                                          */
    int64_t n_free;               /* free displacement dofs of the fine level (the paper's n)    */
    double omega[16];             /* current Jacobi weights (0 until an operator is set up)      */
    double lambda_max[16];        /* current Lanczos estimates                                   */
    int64_t device_bytes;         /* device memory held by the handle                            */
    int fine_chunk[4];            /* element layers per thread of the fine operator's column pass,
                                     chosen by timing at creation: FP64 K, FP64 S, FP32 K, FP32 S
                                     (FP32: batched solves; 0 where the precision is not used)    */
    int fp32_tile[2][5];          /* plan of the single-pass FP32 fine operator, for K and for S:
                                     {TX, TY, DZ} node columns x node columns x planes per CTA,
                                     threads per CTA, plan index (pbm_set_fp32_plan)               */
    int coarse_plan[2][16];       /* form of the FP32 operator of coarse level k, for K and for S
                                     (pbm_set_fp32_coarse_plan): set for 1 <= k <= levels - 2 on
                                     PBM_MIXED grids, 0 elsewhere                                 */
} pbm_grid_info;

/* Newton state of the dual VTS problem (eq. (aug_lagr)): variables xi = (u, alpha, nu_lo, nu_up),
 * multipliers (rho, mu_lo, mu_up), penalties (p, q_lo, q_up; scalars, as Algorithm 1 updates them
 * uniformly) and the problem data V, rho_lo, rho_up. */
typedef struct pbm_state {
    double* u_dev;         /* n, zero on supported dofs                                          */
    double* nu_lo_dev;     /* m                                                                  */
    double* nu_up_dev;     /* m                                                                  */
    double* rho_dev;       /* m, > 0                                                             */
    double* mu_lo_dev;     /* m, > 0                                                             */
    double* mu_up_dev;     /* m, > 0                                                             */
    double alpha;
    double p, q_lo, q_up;  /* > 0                                                                */
    double V, rho_lo, rho_up;
} pbm_state;

typedef struct pbm_solve_info {
    int status;            /* same as the return value                                           */
    int iterations;        /* MINRES iterations (all inner iterations for PBM_MIXED)             */
    int outer;             /* refinement steps (PBM_MIXED), 1 for PBM_FP64                       */
    double relres;         /* true ||b - A x||_2 / ||b||_2 at exit, FP64 operator                */
    double setup_ms;       /* operator hierarchy set-up inside this call (0 if already built)    */
    double solve_ms;       /* host wall time of the solve                                        */
} pbm_solve_info;

typedef struct pbm_newton_info {
    int status;
    int minres_iterations;
    int halvings;          /* Armijo step halvings                                               */
    double kappa;          /* accepted step length                                               */
    double res_pbm;        /* eq. (resIP) at the state BEFORE the step                           */
    double slope;          /* grad L^T dxi (must be < 0)                                         */
    double lagrangian_old, lagrangian_new;
    double minres_relres;
    int resolves;          /* re-solves with a tightened eps_mr after a non-descent direction         */
    int stalled;           /* 1: no descent direction even at the floor; the step was not taken     */
    double eps_mr;         /* MINRES tolerance of the last solve                                     */
} pbm_newton_info;

/* Timing of the fine-level operator kernel (K(w) x or S x with any of its fused epilogues: plain
 * apply, residual b - A x, damped-Jacobi sweep, Chebyshev step), accumulated per handle while profiling is on. */
typedef struct pbm_profile_stats {
    int64_t launches;      /* fine-level operator launches timed                                  */
    double total_ms;       /* sum of their durations, CUDA events on the launch stream            */
    double bytes;          /* sum of their algorithmic HBM bytes: every input vector and element
                              array read once, the output written once                           */
    double flops;          /* sum of their arithmetic operations (add, mul, FMA each counted 1)  */
} pbm_profile_stats;

/* Fills `d` with defaults: FP64, E = 1, nu = 0.3, h = 1, 2 + 2 sweeps, theta = 1.2, 10 Lanczos
 * steps, inner_rtol = 1e-4. */
int pbm_default_desc(pbm_grid_desc* d, int nx, int ny, int nz, int levels, int support);

/* Builds the grid and its level hierarchy (Section 6: regular 8-way refinement of a coarse mesh,
 * here read from the fine grid down), the element matrix K_e of Section 5.2 / eq. (1) (Q1,
 * isotropic, exact integration), the supports, and allocates every device buffer the solves need.
 * Errors: PBM_EINVAL (sizes not divisible, levels > 16, coarsest grid with more than 1500 dofs,
 * bad material), PBM_ENOMEM. */
int pbm_create_grid(const pbm_grid_desc* d, pbm_grid** out);

/* Releases every buffer of the handle. Waits for the device work the handle enqueued. */
int pbm_destroy_grid(pbm_grid* g);

/* One-line description of the last error on this host thread ("" if none). */
const char* pbm_last_error(void);

/* Sizes, current Jacobi weights and memory of the handle (host struct). */
int pbm_grid_info_get(const pbm_grid* g, pbm_grid_info* out);

enum pbm_map {
    PBM_MAP_FIXED_DOFS = 0,    /* uint8[n_level]: 1 where the dof is supported                    */
    PBM_MAP_ELEM_NODES = 1,    /* int32[m_level * 8]: node ids of every element, local order a    */
    PBM_MAP_PROLONG = 2,       /* level >= 1: for every node of level-1 (the finer grid), 8 int32
                                  coarse parent node ids then 8 double weights, packed as
                                  int32[nodes_fine*8] followed by double[nodes_fine*8]; unused
                                  slots have id -1 and weight 0; supports are NOT applied         */
    PBM_MAP_KE = 3             /* double[576]: element matrix of the level (row-major 24 x 24)    */
};
/* Copies an integer map or table of `level` into host memory `host_dst` (caller-allocated, sized
 * as listed above). Synchronous. Errors: PBM_EINVAL. */
int pbm_get_maps(const pbm_grid* g, int level, int which, void* host_dst);

/* rho_dev: m FP64 element densities (eq. (1)). Copied into the handle (the caller may free it
 * after the stream has passed this call); marks the K(rho) hierarchy stale. Checks that every
 * value is finite and >= 0 (this synchronises `stream`): PBM_ENONFINITE / PBM_EINVAL. */
int pbm_set_density(pbm_grid* g, const double* rho_dev, void* stream);

/* y = A_level x with A_0 = K(w) on the fine level, eq. (1): K(w) = sum_i w_i K_i with supported
 * rows/columns the identity; and for level >= 1 the Galerkin operator A_level = R A_{level-1} P of
 * Section 5.1 (R = P^T, P the trilinear prolongation of Section 5.2) built from K(rho) of the density
 * set by pbm_set_density, supported rows/columns of that level the identity.
 *   level 0: w_dev m element weights (NULL = the density set by pbm_set_density); x_dev, y_dev n.
 *   level k >= 1: w_dev must be NULL; x_dev, y_dev hold 3 (nx/2^k + 1)(ny/2^k + 1)(nz/2^k + 1)
 *   entries. If the K(rho) hierarchy is not current (no K solve or V-cycle since the last
 *   pbm_set_density, or an S hierarchy replaced it) it is built first, on `stream`. (The set-up of
 *   a PBM_MIXED grid builds its coarse operators in FP32, for the FP32 V-cycle; the first FP64 read
 *   of a coarse level after a set-up builds the FP64 ones on `stream`.)
 * x and y must not overlap. FP64 throughout. Errors: PBM_EINVAL (level out of range, weights given
 * for a coarse level), PBM_ESTATE (no density set and no weights). */
int pbm_apply_K(pbm_grid* g, const double* w_dev, const double* x_dev, double* y_dev, int level, void* stream);

/* Same operator in FP32 (the kernel the mixed path runs); w_dev must not be NULL. */
int pbm_apply_K_f32(pbm_grid* g, const float* w_dev, const float* x_dev, float* y_dev, void* stream);

/* One FP32 fine-level application of the operator `op` (PBM_OP_K: K(rho) of eq. (1) with the density
 * of pbm_set_density; PBM_OP_S: S of eq. (S) at the state of pbm_set_state) with one of the fused
 * epilogues the mixed-precision V-cycle uses (Section 5.1):
 *   PBM_EPI_APPLY  y = A x                       dot: y . x
 *   PBM_EPI_RESID  y = b - A x                   dot: y . y
 *   PBM_EPI_JACOBI y = x + omega_0 D_0^{-1} (b - A x), omega_0 and D_0 the fine level's Jacobi weight
 *                  and diagonal of the current hierarchy (pbm_grid_info_get, pbm_get_diag)   dot: y . b
 * Only for PBM_MIXED grids, whose FP32 copies of the operator data are made when the operator's
 * hierarchy is set up (pbm_set_state for S; a K solve or pbm_vcycle for K): PBM_ESTATE otherwise.
 * x_dev, b_dev (NULL for APPLY), y_dev: FP32 device vectors of n (K) or n + 1 (S) entries, y not
 * overlapping x or b. dot_host: NULL, or receives the epilogue's FP64-reduced dot product (this
 * synchronises `stream`). Errors: PBM_EINVAL, PBM_ESTATE. */
int pbm_apply_fine_f32(pbm_grid* g, int op, int epilogue, const float* x_dev, const float* b_dev, float* y_dev,
                       double* dot_host, void* stream);

/* The same on level `level` of the current hierarchy (0 = fine; level >= 1: the Galerkin operator
 * A_level = P^T A_(level-1) P of Section 5.1 as the FP32 V-cycle applies it (built in FP32 from the
 * FP32 copies of the weights and u), with the alpha border for S, and that level's Jacobi weight and
 * diagonal). Vectors have n_level (+ 1 for S) entries. Errors as
 * above, and PBM_EINVAL for a level out of range. */
int pbm_apply_level_f32(pbm_grid* g, int level, int op, int epilogue, const float* x_dev, const float* b_dev,
                        float* y_dev, double* dot_host, void* stream);

/* Tile plans of the single-pass FP32 fine operator (CTA size, register budget, TX x TY node columns
 * by DZ planes per CTA; listed by pbm_grid_info_get's fp32_tile). pbm_create_grid times every plan
 * on PBM_MIXED grids and keeps the fastest per operator; pbm_set_fp32_plan overrides that choice
 * for `op` (PBM_OP_K or PBM_OP_S) with plan 0 <= plan < pbm_fp32_plan_count(). Every plan computes
 * the same operator; only the reduction order of the dot products and alpha row depends on it.
 * Plan pbm_fp32_tc_plan() (the last) runs the element contraction K_e x_e of every element layer
 * on the tensor cores (tcgen05 MMA, TF32 operands split into a rounded high part and the FP32
 * remainder, FP32 accumulation: products as accurate as FP32 arithmetic); the others run the
 * factored element matrix on the CUDA cores. A wait of the tensor-core plan that gives up (after
 * one second) leaves a NaN in y[0]. Errors: PBM_EINVAL. */
int pbm_fp32_plan_count(void);
int pbm_fp32_tc_plan(void);
int pbm_set_fp32_plan(pbm_grid* g, int op, int plan);

/* Forms of the FP32 operator of a coarse level 1 <= level <= levels - 2 (the Galerkin element
 * matrices of Section 5.1, stored; the coarsest level is solved directly): plan -1 is two passes
 * (element rows, then node sums) with the 24 rows of each element split over eight threads, -2
 * the two passes with one thread per element (each stored entry loaded once), and
 * 0 <= plan < pbm_fp32_coarse_plan_count() a tile plan of the single marching pass.
 * pbm_create_grid times them on PBM_MIXED grids per level and operator (levels of 32768 elements
 * or more: the two-pass forms only) and keeps the fastest; pbm_set_fp32_coarse_plan overrides the
 * choice for `op` on `level`. Every form computes the same operator; only the summation order
 * differs. Errors: PBM_EINVAL (op, level or plan out of range), PBM_ESTATE (not a PBM_MIXED grid). */
int pbm_fp32_coarse_plan_count(void);
int pbm_set_fp32_coarse_plan(pbm_grid* g, int op, int level, int plan);

/* Copies the Jacobi diagonal of level `level` of the current hierarchy (K or S, the last one set
 * up) into diag_dev: n_level + 1 FP64 entries (the last is the alpha entry of S, 1 for K);
 * supported dofs hold 1. On a PBM_MIXED grid a coarse level's FP64 diagonal comes from its FP64
 * matrices, built by the first such call after a set-up (on `stream`). Errors: PBM_EINVAL,
 * PBM_ESTATE (no hierarchy). */
int pbm_get_diag(const pbm_grid* g, int level, double* diag_dev, void* stream);

/* Sets the Newton state and builds what S needs (Section 3.2): the per-element factors rho', rho'',
 * mu''_lo, mu''_up, the Schur weights d_i = 1/(1/rho'' + 1/mu''_lo + 1/mu''_up) and rhs weights
 * eps_i, then the Galerkin hierarchy of S (Section 5.1: A_{k-1} = P^T A_k P, identity on alpha),
 * the Jacobi diagonals, weights and the coarsest factorisation. The state's arrays are read
 * during this call only (on `stream`). Synchronises `stream` (host reads the Lanczos scalars).
 * Errors: PBM_EINVAL (null array), PBM_ENONFINITE (non-finite or non-positive factor). */
int pbm_set_state(pbm_grid* g, const pbm_state* st, void* stream);

/* y = S x, eq. (S) in closed form: S = [K(rho'), 0; 0, 0] + sum_i d_i g_i g_i^T, g_i = [K_i u; -1],
 * supported rows/columns the identity. x_dev, y_dev: n + 1 FP64, no overlap. Needs pbm_set_state. */
int pbm_apply_S(pbm_grid* g, const double* x_dev, double* y_dev, void* stream);

/* Right-hand side of the reduced system, eq. (system): rhs = [f - K(rho' - eps) u ;
 * -V + sum_i (rho'_i - eps_i)], zero on supported dofs. f_dev: n (zero on supported dofs);
 * rhs_dev: n + 1. If norms_host is not NULL it receives {||res_1||_2, res_2, ||res_3||_2} of
 * eq. (lagr_grad_a) at the state (res_1 on free dofs), which synchronises `stream`. */
int pbm_reduced_rhs(pbm_grid* g, const double* f_dev, double* rhs_dev, double* norms_host, void* stream);

/* x = M^{-1} b: one V-cycle (Section 5.1; correction scheme, the grid's smoothing (damped Jacobi or
 * Chebyshev, pbm_grid_desc.smoother), restriction P^T, 27-point prolongation, identity transfer of
 * alpha, exact coarsest solve) for the operator `op`; in FP32 on PBM_MIXED grids (b and x are cast).
 * Vectors have n + 1 entries for PBM_OP_S and n for PBM_OP_K. For PBM_OP_K the K(rho) hierarchy is
 * built first if stale (synchronises `stream`). */
int pbm_vcycle(pbm_grid* g, int op, const double* b_dev, double* x_dev, void* stream);

/* Solves A x = b, A = K(rho) or S, by MINRES preconditioned with one V-cycle (Section 5) until the
 * true residual satisfies ||b - A x||_2 <= rtol ||b||_2 (eq. (cgstop), 2-norm over all entries) or
 * maxit iterations. x_dev is the initial guess on entry (pass zeros for none) and the solution on
 * exit. PBM_MIXED grids run FP64 iterative refinement around FP32 inner solves of relative
 * tolerance desc.inner_rtol. Synchronises `stream`. info may be NULL. Errors: PBM_ENOTCONV,
 * PBM_EBREAKDOWN, PBM_ESTATE. */
int pbm_minres_solve(pbm_grid* g, int op, const double* b_dev, double* x_dev, double rtol, int maxit,
                     pbm_solve_info* info, void* stream);

/* ---- damped optimality criteria (Section 4.2, Algorithm DOC) ---------------------------------
 * One DOC iteration: the equilibrium displacement u of K(rho) u = f by MG-MINRES to the true
 * relative residual eps_mr (the paper uses 1e-4), then the volume multiplier alpha by bisection on
 * [0, 10^4]: each trial density is rho_i^+ = min(max(rho_i (u^T K_i u)^q / alpha, rho_lo), rho_up),
 * the lower end moves up while sum(rho^+) > V and the upper end down otherwise, until
 * (hi - lo)/(hi + lo) <= tau_alpha; rho^+ is the last trial's density. */
typedef struct pbm_doc_params {
    double V, rho_lo, rho_up;  /* volume bound and density bounds                                     */
    double q;                  /* damping exponent (the paper: 1/2)                                  */
    double eps_doc;            /* stop when ||rho^+ - rho||_inf <= eps_doc (pbm_doc_solve)            */
    double tau_alpha;          /* bisection tolerance (<= 0: eps_doc / 10)                            */
    double eps_mr;             /* MINRES tolerance of the equilibrium solves                          */
    int maxit;                 /* MINRES iterations per solve                                         */
    int max_iter;              /* DOC iterations (pbm_doc_solve)                                      */
} pbm_doc_params;

typedef struct pbm_doc_info {
    int status;
    int iterations;            /* DOC iterations done                                                 */
    int minres;                /* MINRES iterations, summed                                           */
    int trials;                /* bisection trials of the last iteration                              */
    double alpha;              /* volume multiplier of the last trial                                 */
    double change;             /* ||rho^+ - rho||_inf of the last iteration                           */
    double compliance;         /* f^T u of the last equilibrium solve                                 */
    double minres_relres;      /* true relative residual of the last solve                            */
} pbm_doc_info;

/* Defaults: q = 1/2, eps_doc = 1e-3, tau_alpha = eps_doc / 10, eps_mr = 1e-4, maxit = 500,
 * max_iter = 1000; V, rho_lo, rho_up are the caller's. */
int pbm_default_doc_params(pbm_doc_params* p);

/* One DOC iteration from the densities rho_dev (m, FP64, in/out: rho^+ on return) and the
 * displacement u_dev (n, in: initial guess of the solve, out: u of K(rho) u = f). f_dev: n load.
 * Synchronises. Errors: PBM_EINVAL, PBM_ENOTCONV (solve or bisection), PBM_EBREAKDOWN. */
int pbm_doc_step(pbm_grid* g, double* rho_dev, const double* f_dev, double* u_dev, const pbm_doc_params* p,
                 pbm_doc_info* info, void* stream);

/* Algorithm DOC: iterations of pbm_doc_step until ||rho^+ - rho||_inf <= eps_doc (rho_dev then holds
 * the last density, whose change was below the tolerance) or max_iter. Errors: as pbm_doc_step, and
 * PBM_ENOTCONV when max_iter is reached. */
int pbm_doc_solve(pbm_grid* g, double* rho_dev, const double* f_dev, double* u_dev, const pbm_doc_params* p,
                  pbm_doc_info* info, void* stream);

/* ---- interior-point Newton system (Section 4.1) ----------------------------------------------
 * The primal-dual interior-point method's Newton step on the perturbed KKT system of eq. (1)
 * (barrier parameters r, s), reduced by two Schur complements to eq. (S_IP):
 *   S_IP = [K(rho), 0; 0, 0] + sum_i d_i [K_i u; 1][K_i u; 1]^T,
 *   d_i = 1 / (nu_lo_i / (rho_i - rho_lo) + nu_up_i / (rho_up - rho_i)).
 * It has the structure of the PBM matrix S (the alpha border has the opposite sign), so the same
 * operator kernels, Galerkin hierarchy and MG-MINRES solve it. The right-hand side and the
 * recovered increments are those of the Newton step J dz = -res with J the Jacobian eq. (gradres):
 *   rhs = [f - K(rho + d c) u ; V - sum(rho + d c)],  c_i = res_3 - res_4/(rho_i - rho_lo) + res_5/(rho_up - rho_i),
 *   drho = d (K_i u . du + dalpha + c),  dnu_up by the form of eq. (Delta_onu),  dnu_lo by eq. (Delta_unu),
 * with res_3 = 1/2 u^T K_i u + alpha + nu_lo - nu_up, res_4 = nu_lo (rho - rho_lo) - r,
 * res_5 = nu_up (rho_up - rho) - s. Supported dofs are eliminated as everywhere. */
typedef struct pbm_ip_state {
    const double* u_dev;      /* n: displacement (supported dofs ignored)                           */
    double alpha;             /* volume multiplier                                                    */
    const double* rho_dev;    /* m: densities, strictly rho_lo < rho_i < rho_up                       */
    const double* nu_lo_dev;  /* m: bound multipliers, > 0                                            */
    const double* nu_up_dev;  /* m: > 0                                                               */
    double V, rho_lo, rho_up; /* volume bound and density bounds                                      */
    double r, s;              /* barrier parameters of the lower and upper bounds, > 0                */
} pbm_ip_state;

/* Sets the interior-point state: the per-element coefficients above and the Galerkin hierarchy,
 * Jacobi diagonals, weights and coarsest factorisation of S_IP. The state's arrays are read during
 * this call only. Replaces any PBM state of the grid (pbm_set_state replaces this one). Synchronises
 * `stream`. Errors: PBM_EINVAL (null array, a point that is not strictly feasible, r or s <= 0). */
int pbm_ip_set_state(pbm_grid* g, const pbm_ip_state* st, void* stream);

/* y = S_IP x (n + 1 FP64 entries each, alpha last; supported rows and columns the identity). */
int pbm_ip_apply_S(pbm_grid* g, const double* x_dev, double* y_dev, void* stream);

/* rhs (n + 1) of the reduced system at the state; f_dev: n load vector. */
int pbm_ip_reduced_rhs(pbm_grid* g, const double* f_dev, double* rhs_dev, void* stream);

/* Solves S_IP dz = rhs by MG-MINRES as pbm_minres_solve does (true relative residual <= rtol;
 * dz_dev holds the initial guess on entry). Synchronises. Errors as pbm_minres_solve. */
int pbm_ip_solve(pbm_grid* g, const double* rhs_dev, double* dz_dev, double rtol, int maxit, pbm_solve_info* info,
                 void* stream);

/* The density and multiplier increments (m entries each) from the reduced solution dz = [du; dalpha]. */
int pbm_ip_recover(pbm_grid* g, const double* dz_dev, double* drho_dev, double* dnu_lo_dev, double* dnu_up_dev,
                   void* stream);

/* One Newton step of Algorithm 2 on the augmented Lagrangian: builds S and its rhs at `st`,
 * solves the reduced system to relative residual eps_mr, recovers (dnu_lo, dnu_up) by
 * eq. (deltanu), backtracks (Armijo, c1 = 1e-4, halving, at most 30 halvings) and updates
 * st->u_dev, st->alpha, st->nu_lo_dev, st->nu_up_dev in place. f_dev: n load vector. Synchronises.
 * A direction that is not one of descent (grad L^T dxi >= 0: the failure of inexact solves that
 * Section 6 reports for the largest bridge examples) is solved again from zero with eps_mr / 10, down
 * to the floor 1e-9 of Section 5.3 (info->resolves counts them); if it is still not a descent
 * direction there the step is not taken (info->stalled = 1, PBM_ELINESEARCH).
 * Errors: PBM_ELINESEARCH (no acceptable step; state unchanged), PBM_ENOTCONV (the step was taken
 * with a solve that did not reach the tolerance), PBM_EBREAKDOWN. */
int pbm_newton_step(pbm_grid* g, pbm_state* st, const double* f_dev, double eps_mr, pbm_newton_info* info,
                    void* stream);

/* Parameters of one Newton step (pbm_newton_step_ex); pbm_default_newton_params gives the values
 * pbm_newton_step uses for the ones it does not take. */
typedef struct pbm_newton_params {
    double eps_mr;         /* MINRES relative tolerance of the reduced system, > 0                   */
    double eps_mr_min;     /* floor of the non-descent re-solves (Section 5.3: 1e-9); a value above
                              eps_mr means no re-solve                                            */
    int max_halvings;      /* Armijo step halvings before PBM_ELINESEARCH, >= 0 (reading: 30)     */
    int maxit;             /* MINRES iterations per solve, >= 1 (10000)                            */
} pbm_newton_params;

int pbm_default_newton_params(pbm_newton_params* p);

/* pbm_newton_step with every parameter given. Errors as pbm_newton_step, and PBM_EINVAL. */
int pbm_newton_step_ex(pbm_grid* g, pbm_state* st, const double* f_dev, const pbm_newton_params* prm,
                       pbm_newton_info* info, void* stream);

/* Parameters of Algorithm 1 (PBM outer loop). pbm_default_pbm_params gives the paper's values
 * (Section 3.3, Section 5.3): eps_pbm 1e-5, beta = gamma = 0.3, p_min 1e-8, eps_nwt 1 and its
 * floor 1e-3, eps_mr = 1e-4 sqrt(n) (eps_mr <= 0 selects it) reduced tenfold down to eps_mr_min
 * whenever a Newton step reduces res_PBM by less than 10 percent. */
typedef struct pbm_pbm_params {
    double eps_pbm;        /* stop when |delta / d| < eps_pbm (duality gap over dual objective)  */
    double beta;           /* multiplier safeguard: beta x <= x+ <= x / beta, 0 < beta < 1       */
    double gamma;          /* penalty reduction p+ = max(gamma p, p_min), 0 < gamma < 1          */
    double p_min;
    double eps_nwt, eps_nwt_min;  /* Newton tolerance on res_PBM and its floor                   */
    double eps_mr, eps_mr_min;    /* MINRES relative tolerance (<= 0: 1e-4 sqrt(n)) and floor    */
    int max_outer, max_newton;    /* outer iterations; Newton steps per Newton loop              */
    int max_halvings;             /* Armijo step halvings per Newton step (30)                   */
} pbm_pbm_params;

typedef struct pbm_pbm_info {
    int status;
    int outer, newton, minres;    /* outer iterations, Newton steps, MINRES iterations in total */
    double gap_ratio;             /* |delta / d| at the end of the last outer iteration         */
    double compliance;            /* 1/2 f^T u at exit                                           */
    double volume;                /* sum rho at exit                                              */
    double eps_mr;                /* MINRES tolerance in use at exit                              */
    int resolves;                 /* Newton systems solved again after a non-descent direction    */
    int stalls;                   /* Newton loops ended early because no descent direction was
                                     found at eps_mr_min (Section 6: the iterate is accepted)      */
} pbm_pbm_info;

int pbm_default_pbm_params(pbm_pbm_params* p);

/* Algorithm 1: the PBM method for the VTS problem (eq. (1)) in its dual form, from the state *st
 * (for the paper's initial point: u = 0, alpha = 1, nu = e, rho = V/m, mu = e, p = q = 1). Each
 * outer iteration runs Newton steps (Algorithm 2, pbm_newton_step) until res_PBM < eps_nwt, then
 * evaluates the duality gap delta (eq. (gap)) and d, stops when |delta / d| < eps_pbm, else updates
 * the multipliers (rho, mu_lo, mu_up with the beta safeguard), the penalties and eps_nwt. The run
 * ends with a Newton loop at 10 eps_pbm and a final density update. st is updated in place; st->rho
 * holds the optimal densities on exit. A Newton direction that is not one of descent is solved again
 * with eps_mr / 10 (down to eps_mr_min); a Newton loop that finds no descent direction at the floor
 * ends at its current iterate, which is accepted as Section 6 does for its stalled runs
 * (info->stalls). Synchronises. Errors: PBM_ENOTCONV (max_outer or max_newton reached),
 * PBM_ELINESEARCH, PBM_EBREAKDOWN, PBM_EINVAL. */
int pbm_solve(pbm_grid* g, pbm_state* st, const double* f_dev, const pbm_pbm_params* prm, pbm_pbm_info* info,
              void* stream);

/* Per-element compliances c_i = 1/2 u^T K_i u (the constraint terms of the dual, eq. (dual), and
 * minus the derivative of 1/2 f^T u w.r.t. rho_i at equilibrium). u_dev: n (masked internally);
 * c_dev: m. If f_dev and fTu_host are both non-NULL, *fTu_host receives f^T u (synchronises). */
int pbm_compliance_grad(pbm_grid* g, const double* u_dev, double* c_dev, const double* f_dev, double* fTu_host,
                        void* stream);

/* Number of CUDA kernels this library has launched in the process so far (all handles, all
 * threads). Lets a caller count the device work of a region of code. Never fails. */
int64_t pbm_kernel_launches(void);

/* on != 0: from now on, bracket every fine-level operator launch of `g` in its working precision
 * (FP64 grids: the FP64 kernels; PBM_MIXED grids: the FP32 kernels of the inner solves, not the
 * FP64 residual applies of the refinement) with a pair of CUDA events on its stream (two event
 * records per launch; off by default). on == 0: stop. */
int pbm_profile(pbm_grid* g, int on);

/* Copies the statistics of operator `op` (PBM_OP_K: the K(w) kernel, PBM_OP_S: the S kernel)
 * accumulated since its last read into `out` and resets them. Waits for the recorded events.
 * Errors: PBM_EINVAL (null argument, unknown operator). */
int pbm_profile_read(pbm_grid* g, int op, pbm_profile_stats* out);

/* ---- batched solves --------------------------------------------------------------------------
 * A batch advances several independent systems (grid handles of any sizes, FP64 or all mixed, with
 * the same smoothing sweeps) together: every stage of the MINRES iteration and the V-cycle is one
 * launch over all systems' work, and the iteration runs as a CUDA-graph loop until every system has
 * finished: many design instances and load cases solved together. Each system keeps its own hierarchy, scratch and scalars, so the results equal those of separate solves up to the
 * iteration at which each system stops. */
typedef struct pbm_batch pbm_batch;

/* grids: n handles on one device. op: PBM_OP_K or PBM_OP_S (every system's operator must be set up
 * before each solve: pbm_set_density + a solve or pbm_vcycle for K, pbm_set_state for S). The
 * batch stores the grids' buffer addresses: destroy it before any of its grids. Errors: PBM_EINVAL
 * (mixed precisions, different sweeps, a repeated grid), PBM_ENOMEM. */
int pbm_batch_create(pbm_grid* const* grids, int n, int op, pbm_batch** out);
int pbm_batch_destroy(pbm_batch* b);

/* Solves A_s x_s = b_s for every system s (b_dev[s], x_dev[s]: device vectors of that system's
 * length, x the initial guess on entry) to the true relative residual rtol, as pbm_minres_solve does
 * for one system (mixed grids: FP64 refinement around batched FP32 inner solves, with the
 * single-system FP32-preconditioned FP64 stage for any system the refinement cannot finish).
 * infos: n results or NULL. Synchronises. Returns the first non-OK status of any system. */
int pbm_batch_minres_solve(pbm_batch* b, const double* const* b_dev, double* const* x_dev, double rtol, int maxit,
                           pbm_solve_info* infos, void* stream);

/* y = K(w) x, exactly as pbm_apply_K computes it (FP64, supported rows and columns the identity),
 * for callers that cannot allocate device memory and so cannot create a grid handle: loops that must
 * not allocate after start-up, host frameworks whose own allocator owns all device memory, and
 * plug-ins running inside such hosts. The paper has no counterpart; this is an interface for such
 * callers. The call allocates nothing (no cudaMalloc, cudaFree or allocating library routine): the
 * scratch of its kernels is one fixed 32 MiB array in the library's device code, which every GPU that
 * loads the library holds until the process exits.
 *   nx, ny, nz, support, E, nu, h: the grid as in pbm_grid_desc (no multigrid levels are needed).
 *   w_dev: m FP64 element weights; x_dev, y_dev: n FP64 entries, caller-owned, not overlapping, all
 *   three on the current device (the call runs there; arrays on another device are rejected).
 *   stream: as elsewhere (work is enqueued, nothing synchronises).
 * The first call on a device looks up the array's device address on that device and keeps it; make
 * that first call before any stream capture, and do not call the library again after a
 * cudaDeviceReset of that device. Every call shares the array and finds it as the previous call left
 * it, so calls whose work overlaps on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.
 * Errors: PBM_EINVAL (null pointer, bad sizes or material, arrays that are not device memory of the
 * current device, or a grid whose scratch exceeds the array: grids of up to about 170,000 elements always fit),
 * PBM_ECUDA. */
int pbm_apply_K_noalloc(int nx, int ny, int nz, int support, double E, double nu, double h, const double* w_dev,
                        const double* x_dev, double* y_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PBM_H */
