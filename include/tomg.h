/*
 * tomg -- multigrid-preconditioned conjugate-gradient solve of the SIMP-penalised
 * linear-elasticity system K(rho) u = f on structured quad4 (2D) / hex8 (3D) grids,
 * for NVIDIA GB300 (sm_103a).  C ABI: plain pointers and sizes, no C++ or torch types.
 *
 * The calls follow the problem statement of Peetz & Elbanna, "On the use of multigrid
 * preconditioners for topology optimization" (Sec. 2.1 Eq. 1-2, Sec. 3.1-3.2, Sec. 4):
 *   grid dims, density rho, E0 / Emin / p / nu, loads f, fixed DOFs, tolerance and
 *   preconditioner type in; displacements u, compliance f^T u and iteration count out.
 *
 * Conventions (the paper fixes none of them):
 *   nodes    n = i + (nx+1) (j + (ny+1) k), x fastest; DOF = dim * n + c (interleaved)
 *   elements e = i + nx (j + ny k); unit elements; local node a = (a&1, a>>1&1, a>>2&1)
 *   vectors of several right-hand sides are column-major n x nrhs (RHS r at offset r*n)
 *
 * Errors: every call returns a tomg_status; nothing throws across the ABI.  On an error the
 * message is available from tomg_last_error() (thread-local).  Pointers flagged "on_device"
 * must be device pointers on the context's device, ordered with respect to the context's
 * stream (the caller synchronises its own producers).  Inputs are copied; outputs are
 * caller-owned.  Handles are not thread-safe: one thread per problem at a time.
 */
#ifndef TOMG_H
#define TOMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tomg_ctx tomg_ctx;
typedef struct tomg_problem tomg_problem;

typedef enum {
  TOMG_OK = 0,
  TOMG_NOT_CONVERGED = 1,   /* max_iter reached; u, iterations and residual still written   */
  TOMG_E_INVALID = -1,      /* bad argument (size, index, NaN density, missing setup ...)   */
  TOMG_E_OOM = -2,          /* device allocation failed                                      */
  TOMG_E_CUDA = -3,         /* CUDA runtime error (message in tomg_last_error)               */
  TOMG_E_BREAKDOWN = -4,    /* p^T A p <= 0, NaN, or a non-SPD coarse operator               */
  TOMG_E_TIMEOUT = -5,      /* a bounded device wait expired                                  */
  TOMG_E_BUDGET = -6        /* serving: request larger than the memory budget                */
} tomg_status;

/* Preconditioner hierarchy (Sec. 3.2; Sec. 4 for AMG and the hybrid of Sec. 4.3). */
typedef enum {
  TOMG_PC_GMG = 0,      /* geometric levels: bilinear/trilinear P, Galerkin P^T A P          */
  TOMG_PC_AMG = 1,      /* smoothed aggregation from the fine operator, rigid-body modes      */
  TOMG_PC_HYBRID = 2,   /* n_geo_levels geometric levels, smoothed aggregation below          */
  TOMG_PC_JACOBI = 3    /* point-block Jacobi only (no hierarchy)                             */
} tomg_pc;

/* Arithmetic of the V-cycle; the outer Krylov loop, its residual and dots are always FP64. */
typedef enum {
  TOMG_PREC_FP64 = 0,         /* FP64 V-cycle inside FP64 PCG                                 */
  TOMG_PREC_FP32_VCYCLE = 1,  /* FP32 V-cycle inside FP64 flexible CG (Notay 2000)            */
  TOMG_PREC_TC_VCYCLE = 2,    /* as FP32_VCYCLE, with the hex8 level-0 element contractions on
                                 the tensor cores: each element row scaled by a power of two
                                 and split into two FP16 parts, against the exact integer
                                 parts 72 K_l, 72 K_m of Ke = lambda K_l + mu K_m, FP32
                                 accumulation (FP32 accuracy); quad4 problems run exactly as
                                 FP32_VCYCLE                                                   */
  TOMG_PREC_3XTF32_VCYCLE = 2 /* former name of TOMG_PREC_TC_VCYCLE                           */
} tomg_prec;

typedef struct {
  int pc;              /* tomg_pc                                              default GMG  */
  int prec;            /* tomg_prec                                            default FP64 */
  double rtol;         /* stop when ||b - K u||_2 <= rtol ||b||_2 (true residual)  1e-8     */
  int max_iter;        /* outer iterations                                         1000     */
  int n_levels;        /* GMG levels incl. the fine grid; 0 = from max_coarse_dofs  0       */
  int max_coarse_dofs; /* coarsest level has fewer DOFs than this                   2000    */
  int n_geo_levels;    /* hybrid: geometric levels incl. the fine grid             3        */
  int smoother;        /* 0 = weighted point-block Jacobi (Sec. 4.1); 1 = point-block
                          Jacobi-preconditioned Chebyshev polynomial (the paper's Chebyshev
                          smoother study, Sec. 4.1), degree cheb_degree on
                          [cheb_lower, cheb_upper] x lambda_max(D^-1 A) of each level;
                          2 = gmres_steps steps of point-block-Jacobi right-preconditioned
                          GMRES (the paper's GMRES smoother, Sec. 4.1), before the coarse
                          correction from x = 0, after it from the corrected iterate; the
                          cycle then depends on its input, so the CG loop is flexible CG in
                          every precision                                             0        */
  double omega;        /* Jacobi weight (Sec. 4.1)                                 0.5      */
  int n_pre, n_post;   /* smoothing sweeps (one each)                              1, 1     */
  double soc_beta;     /* strength-of-connection threshold (Eq. 10)                0.003    */
  int check_every;     /* use_graph < 2: outer iterations between host polls       4        */
  int use_graph;       /* 2: whole solve = one graph with a device-side while loop;
                          1: one captured graph per iteration; 0: plain launches   2        */
  int max_levels;      /* cap on the number of levels                              25       */
  int concurrency;     /* solve slots: right-hand sides solved concurrently        4        */
  int cheb_degree;     /* Chebyshev smoother: operator applies per smoothing, 1..8  2       */
  double cheb_lower;   /* Chebyshev interval, fractions of the 20-step power-iteration
                          estimate of lambda_max(D^-1 A): lower                     0.1      */
  double cheb_upper;   /*                                   upper                     1.1      */
  int adaptive_geo;    /* hybrid only: adaptive geometric level count across the design
                          updates of a problem (Sec. 4.4): the first setup uses n_geo_levels
                          (6 in the paper); every solve that needs more than adaptive_iters
                          outer iterations makes the next setup use one geometric level
                          fewer, down to adaptive_min_geo                          0 (off)  */
  int adaptive_iters;  /*                                                          200      */
  int adaptive_min_geo;/*                                                          2        */
  int krylov;          /* outer Krylov method: 0 = CG (PCG with the FP64 V-cycle, flexible CG
                          with the FP32 one); 1 = flexible GMRES(gmres_restart), the paper's
                          outer solver (Sec. 4), host-driven, one right-hand side at a time,
                          iterations = preconditioner applications                    0        */
  int gmres_restart;   /* FGMRES restart length m, 1..200                             30       */
  int gmres_steps;     /* GMRES smoother: Arnoldi steps (operator applies) per smoothing,
                          1..8                                                        2        */
  int block_rhs;       /* block solve of several right-hand sides (Sec. 2.2, 4.2: load cases
                          and adjoint right-hand sides on one hierarchy): with R = block_rhs
                          >= 2, tomg_solve advances up to R right-hand sides together in one
                          flexible-CG loop, one captured graph whose every kernel launch
                          covers all of them (per-right-hand-side scalars, reductions and
                          convergence: a converged right-hand side stops updating while the
                          others go on); each result is bit-identical to its solve alone
                          (the same sums in the same order per right-hand side).  Needs hex8, prec
                          TOMG_PREC_TC_VCYCLE, the Jacobi or Chebyshev smoother and krylov 0;
                          R <= 64.  0 or 1: solve slots (concurrency)                  0        */
  int fp64_tc;         /* hex8: the outer loop's FP64 K p and residuals with the element
                          contractions on the tensor cores, exact integer products of 11-bit
                          digits of each element's fixed-point displacements against the
                          integer matrix C of Ke = c C (nu with a rational lambda / mu, e.g.
                          0.3), FP64 scaling and node sums; 0: the assembled FP64 stencil on
                          the FP64 pipe.  Ignored where nu admits no such C           1        */
  int fuse_transfers;  /* V-cycle with the Chebyshev smoother (Algorithm 1, Sec. 3.2): 1 =
                          the prolongation of the coarse correction computed inside the first
                          post-smoothing step of the geometric levels that support it (3^d
                          stencils, the FP32 tensor-core hex8 operator), and the first step
                          from x = 0 inside the second on hex8 level 0; bit-identical results
                          to the separate kernels.  Off by default: forming x + P xc at every
                          node a smoothing kernel reads costs those kernels more than the
                          separate streaming passes (3D cantilever 192x96x96: 25.9 against
                          24.0 ms per solve).  0: separate transfer launches           0        */
} tomg_options;

typedef struct {
  int iterations;        /* outer iterations (updates of u)                               */
  double rel_residual;   /* true ||b - K u||_2 / ||b||_2 in FP64, b = f on free DOFs       */
  double compliance;     /* f^T u (Eq. 1)                                                  */
  double setup_ms;       /* hierarchy build of the last tomg_setup                         */
  double solve_ms;       /* this right-hand side's solve, device time                      */
  int status;            /* tomg_status of this right-hand side                            */
} tomg_result;

typedef struct {
  int kind;              /* 0 matrix-free element operator, 1 structured 3^d stencil, 2 BSR */
  int block;             /* DOFs per node on this level                                     */
  int64_t n_nodes;       /* nodes (aggregates on AMG levels)                                */
  int64_t n_dofs;        /* block * n_nodes                                                 */
  int64_t nnzb;          /* stored blocks (stencil: 3^d per node incl. out-of-grid zeros)   */
  int nx, ny, nz;        /* element counts on geometric levels, 0 on AMG levels             */
  int geometric;         /* 1 if the transfer to the next level is geometric                */
} tomg_level_info;

/* ---- context ------------------------------------------------------------------------- */
/* Create a context on CUDA device `device`.  `cuda_stream` (a cudaStream_t, may be NULL)
 * is used for all work; NULL creates a private non-blocking stream. */
tomg_status tomg_ctx_create(tomg_ctx** out, int device, void* cuda_stream);
tomg_status tomg_ctx_destroy(tomg_ctx* ctx);
const char* tomg_last_error(void);
void tomg_options_default(tomg_options* opt);

/* ---- problem (Sec. 2.1) -------------------------------------------------------------- */
/* A structured grid problem.  dim = 2 (quad4, plane stress, nz ignored) or 3 (hex8).
 * E(rho) = Emin + (E0 - Emin) rho^penal (Eq. 2); nu = Poisson ratio.
 * E_INVALID for non-positive sizes, E0 <= 0, Emin < 0, nu outside (-1, 0.5). */
tomg_status tomg_problem_create(tomg_ctx* ctx, int dim, int nx, int ny, int nz, double E0,
                                double Emin, double penal, double nu, tomg_problem** out);
tomg_status tomg_problem_destroy(tomg_problem* prob);
/* Problem sizes: DOFs, nodes, elements (any pointer may be NULL). */
tomg_status tomg_problem_sizes(const tomg_problem* prob, int64_t* n_dofs, int64_t* n_nodes,
                               int64_t* n_elems);
/* Fixed (zero-displacement) DOFs, `count` indices in [0, n_dofs), host array, copied.
 * Duplicates are allowed.  E_INVALID on an index out of range.  Invalidates the setup. */
tomg_status tomg_set_fixed_dofs(tomg_problem* prob, const int64_t* dofs, int64_t count);
/* Element densities rho (n_elems doubles, host or device), copied.  E_INVALID if any value
 * is negative or NaN (checked on the device for device input).  Marks the hierarchy stale. */
tomg_status tomg_set_density(tomg_problem* prob, const double* rho, int on_device);

/* ---- preconditioner setup (Sec. 3.2, Eq. 9; Sec. 4) ------------------------------------ */
/* Builds (or refreshes) the hierarchy for the current density: SIMP moduli, Galerkin coarse
 * operators, point-block smoother diagonals, AMG aggregation / prolongators, coarse dense
 * Cholesky.  opt = NULL uses the defaults. */
tomg_status tomg_setup(tomg_problem* prob, const tomg_options* opt);

/* ---- solve (Sec. 3.1, Sec. 4) -------------------------------------------------------------
 * Solves K(rho) u = f for `nrhs` right-hand sides (f and u column-major n x nrhs, host or
 * device per on_device).  u is read as the initial guess (warm start; zeros for a cold
 * start) and overwritten with the solution; fixed DOFs of u are returned as 0.  results has
 * nrhs entries.  Returns the worst status over the right-hand sides. f = 0 gives u = 0 in 0
 * iterations.  Requires a setup for the current density (E_INVALID otherwise). */
tomg_status tomg_solve(tomg_problem* prob, int nrhs, const double* f, double* u, int on_device,
                       tomg_result* results);

/* ---- serving: continuous batching of design updates ---------------------------------------
 * The paper's optimisation loop solves the same kind of system once per design iteration,
 * warm-started from the previous displacements (Sec. 4).  A server runs such requests for many
 * problems at once: `max_slots` worker threads take requests in arrival order as soon as a
 * slot is free and the request's estimated device footprint fits `hbm_budget_bytes`; each
 * problem runs on its own stream, so requests in flight overlap on the GPU.  A problem's
 * updates are applied in submission order, never two at a time.  Its previous solution stays
 * on the device and is the next update's initial guess.  Results are independent of the mix
 * (fixed-order reductions, private buffers).  Destroy the server before its problems. */
typedef struct tomg_server tomg_server;
tomg_status tomg_server_create(tomg_ctx* ctx, size_t hbm_budget_bytes, int max_slots,
                               tomg_server** out);
/* One design update: rho (n_elems doubles, host) and f (n_dofs x nrhs column-major, host) are
 * copied; u (host, nullable) receives the solution when the request completes.  opt = NULL
 * uses the defaults.  E_BUDGET if the request alone exceeds the budget. */
tomg_status tomg_server_submit(tomg_server* srv, tomg_problem* prob, const double* rho, int nrhs,
                               const double* f, double* u, const tomg_options* opt,
                               uint64_t* ticket);
/* Waits for a ticket (timeout_ms < 0: no limit); E_TIMEOUT if it is still running after the
 * limit (the ticket stays valid), E_INVALID for an unknown ticket.  results: nrhs entries.
 * Returns the request's status. */
tomg_status tomg_server_wait(tomg_server* srv, uint64_t ticket, int timeout_ms,
                             tomg_result* results);
/* Request latency percentiles (submission to completion), completed requests per second
 * (first submission to last completion), and the peak concurrency / estimated bytes in flight. */
tomg_status tomg_server_stats(tomg_server* srv, double* p50_ms, double* p99_ms,
                              double* solves_per_s, int64_t* completed, int* peak_active,
                              size_t* peak_bytes);
/* Waits (timeout_ms < 0: no limit) until `prob` has no queued or running request, then frees
 * the warm start the server keeps for it and stops counting its device memory against the
 * budget: the client is done with this problem (destroy it, or keep it outside the server).
 * While a problem is resident, i.e. after its first update and until it is retired, its
 * measured device bytes (hierarchy, solve slots, warm start) count against the budget; a
 * request of a problem that is not resident yet is admitted only when its estimated footprint
 * fits beside them.  E_TIMEOUT if requests remain after the limit. */
tomg_status tomg_server_retire(tomg_server* srv, tomg_problem* prob, int timeout_ms);
tomg_status tomg_server_destroy(tomg_server* srv);

/* ---- hierarchy introspection and single steps (parity checking) ------------------------- */
tomg_status tomg_num_levels(const tomg_problem* prob, int* n_levels);
tomg_status tomg_level_info_get(const tomg_problem* prob, int level, tomg_level_info* info);
/* Level operator as block CSR (row_ptr n_nodes+1, col nnzb, val nnzb*block*block, row-major
 * blocks), FP64, host arrays.  Call with NULL arrays to get nnzb only.  Stencil levels drop
 * their out-of-grid blocks, so nnzb may be smaller than tomg_level_info.nnzb.  Level 0 is
 * assembled on the fly from the matrix-free operator. */
tomg_status tomg_level_export(tomg_problem* prob, int level, int64_t* nnzb, int64_t* row_ptr,
                              int64_t* col, double* val);
/* Prolongation P of level -> level+1 as block CSR (fine rows, coarse block columns, blocks
 * block(level) x block(level+1)), host arrays; NULL arrays return nnzb only. */
tomg_status tomg_prolongation_export(tomg_problem* prob, int level, int64_t* nnzb,
                                     int64_t* row_ptr, int64_t* col, double* val);
/* AMG levels: aggregate id of every node of `level` (-1 = unaggregated), host array. */
tomg_status tomg_aggregates_export(tomg_problem* prob, int level, int64_t* agg);
/* The point-block smoother's inverse diagonal blocks D_b^-1 of `level` (Alg. 1, Sec. 3.2):
 * n_nodes blocks of block x block, row-major, FP64, host array (levels below the coarsest). */
tomg_status tomg_block_diag_inv_export(tomg_problem* prob, int level, double* dinv);
/* y = A_level x in the given tomg_prec (FP32 math for FP32_VCYCLE), double in/out. */
tomg_status tomg_level_apply(tomg_problem* prob, int level, int prec, const double* x, double* y,
                             int on_device);
/* y = K x on the fine grid in FP64, exactly as the outer Krylov loop applies it (Sec. 3.1;
 * K = M K(rho) M + (I - M) with the SIMP moduli of Eq. 2): the assembled FP64 fine stencil of
 * the current setup.  x, y: n doubles, host or device (on_device), DOF-interleaved.  Needs a
 * setup; E_INVALID otherwise. */
tomg_status tomg_outer_apply(tomg_problem* prob, const double* x, double* y, int on_device);
/* z = M r: one V-cycle of the current setup (its precision), double in/out. */
tomg_status tomg_vcycle(tomg_problem* prob, const double* r, double* z, int on_device);
/* Coarsest-level direct solve x = A_c^{-1} b (FP64), host or device arrays. */
tomg_status tomg_coarse_solve(tomg_problem* prob, const double* b, double* x, int on_device);
/* SIMP moduli E_e (Eq. 2) of the current density, n_elems doubles. */
tomg_status tomg_moduli(tomg_problem* prob, double* E, int on_device);
/* Element stiffness matrix of the problem for E = 1 (dim*2^dim squared, row-major). */
tomg_status tomg_element_stiffness(const tomg_problem* prob, double* Ke);
/* Timing of the level-0 SIMP element operator kernel (Sec. 2.1 Eq. 2 inside the K apply):
 * op 0 = y = A x, 1 = residual b - A x, 2 = one weighted block-Jacobi sweep, in the V-cycle's
 * kernels of precision prec (a tomg_prec); op 3 = the outer FP64 q = K p with the per-block
 * partials of p . q, exactly as the Krylov loop launches it (prec ignored).
 * Launches it `reps` times on the context stream, each launch bracketed by CUDA events; with
 * cold_l2 != 0 a 256 MB buffer is written before every launch (outside the events) so the
 * kernel reads its inputs from HBM.  Writes the mean device time per launch (ms).  Needs a
 * setup; reps in [1, 10000]. */
tomg_status tomg_time_fine_operator(tomg_problem* prob, int op, int prec, int reps, int cold_l2,
                                    double* ms_per_launch);
/* Test hook of the failure path of the tensor-core element kernel (TOMG_PREC_TC_VCYCLE).  With
 * polls > 0, launches made after this call wait for their MMAs on a barrier that nothing
 * arrives on and give up after `polls` polls, exactly as after a real timeout: the kernel
 * records the failure, waits with the default limit (2^22 polls) for the MMAs it has in flight
 * on their own barrier, frees its tensor memory and returns; the next tomg_level_apply or
 * tomg_solve of the problem reports TOMG_E_TIMEOUT and clears the record.  polls <= 0 restores
 * normal launches.  No fault is involved.  Process-wide, not thread-safe; for tests only. */
tomg_status tomg_debug_tc_wait_limit(int polls);
/* Test hook of the failure path of the grid barriers in the two single-launch (cooperative)
 * kernels of the setup: the MIS-2 rounds of the aggregation and the coarsest level's Cholesky
 * factorisation and inverse (Sec. 3.2).  With polls > 0, launches made after this call give up
 * a barrier wait at its `polls`-th poll (default 2^24 polls; polls = 1 gives up at once,
 * without looking at the barrier, so with more than one block the wait always runs out); the
 * block that gives up records it, every other block leaves at its next wait, and the
 * tomg_setup in progress reports TOMG_E_TIMEOUT.
 * polls <= 0 restores the defaults.  No fault is involved.  Process-wide, not thread-safe; for
 * tests only. */
tomg_status tomg_debug_grid_wait_limit(int polls);
/* Allocation-free y = A_0 x with FP32 arithmetic: the same computation as
 * tomg_level_apply(prob, 0, TOMG_PREC_FP32_VCYCLE, x, y, 1), for callers that must not
 * allocate device memory where they apply the operator (memory owned by another allocator,
 * loops that cannot take the device-wide synchronisation of cudaFree).  The paper has no
 * counterpart; this is a library service.
 *   x, y      device arrays of n_dofs doubles (on the context's device), caller-owned
 *   limits    n_dofs <= 1,048,576, else TOMG_E_INVALID with a message; needs a density
 *             (tomg_set_density), not a tomg_setup
 *   memory    allocates nothing: the FP32 copies of x and A x live in one fixed 8 MiB
 *             __device__ array that every GPU loading the library keeps until process exit.
 *             The first call on a device looks up that array's address (cudaGetSymbolAddress);
 *             make that first call before any stream capture.
 *   ordering  asynchronous on the context stream; y is ready once that stream is synchronised.
 *             All calls share the array: calls that overlap on the GPU (other streams, other
 *             contexts on the same device) race and must be serialised by the caller.
 *             Every array entry a call reads is written earlier in the same call. */
tomg_status tomg_fine_apply_f32_noalloc(tomg_problem* prob, const double* x, double* y);
/* ---- the steps either side of the solve in a design iteration (Sec. 2.1) ------------------
 * Linear density filter (Eq. 1, rho = S alpha; radius 1.5 element sizes in Sec. 4):
 *   rho_e = sum_j w_ej alpha_j / sum_j w_ej,  w_ej = max(0, radius - |c_e - c_j|)
 * over the element centroids c of the problem's grid; transpose != 0 applies S^T instead (the
 * chain rule dF/dalpha = S^T dF/drho of Eq. 3).  in, out: n_elems doubles, host or device
 * (on_device), caller-owned, may not alias.  E_INVALID for radius outside (0, 3]. */
tomg_status tomg_density_filter(tomg_problem* prob, double radius, int transpose,
                                const double* in, double* out, int on_device);
/* Compliance sensitivities (Eq. 3): dF/drho_e = -p rho_e^(p-1) (E0 - Emin) u_e^T Ke u_e for the
 * problem's current density (tomg_set_density) and displacements u (n_dofs doubles, e.g. the
 * output of tomg_solve); out: n_elems doubles.  Host or device arrays (on_device). */
tomg_status tomg_compliance_sensitivity(tomg_problem* prob, const double* u, double* out,
                                        int on_device);

/* ---- linear buckling, the stability problem (Sec. 2.2 Eq. 4-5; Sec. 3.3 Algorithm 2) --------
 * Stress stiffness for the displacements u of the current density: element stresses at the
 * element centres sigma_e = E_sigma(rho_e) D_0 B u_e with E_sigma = E0 rho^p for rho >= 0.1 and 0
 * below (Eq. 5); K_sigma = -sum_e (sum_ij sigma_e,ij L_ij) (x) I, L_ij the integrals of products of
 * shape-function derivatives, masked at fixed DOFs (the sign makes compression give positive
 * eigenvalues).  y = K_sigma x: u, x, y n_dofs doubles, host or device (on_device). */
tomg_status tomg_stress_stiffness_apply(tomg_problem* prob, const double* u, const double* x,
                                        double* y, int on_device);
/* The n_eig largest eigenpairs of K_sigma Phi = lambda K Phi (lambda_max = 1 / P_critical) by
 * generalized Davidson (Algorithm 2) with the current setup's V-cycle as preconditioner (its
 * precision): search space j_min..j_max (10..25 in the paper), converged when every pair has
 * ||K_sigma q - theta K q|| <= tol |theta| ||K q||.  lambdas: n_eig doubles, descending (host);
 * modes: NULL or n_dofs x n_eig column-major, K-orthonormal (host or device per on_device);
 * iterations: preconditioner applications (nullable).  Needs a setup; 1 <= n_eig <= 16,
 * n_eig < j_min < j_max <= 64.  NOT_CONVERGED after max_iter with the current Ritz pairs. */
tomg_status tomg_buckling(tomg_problem* prob, const double* u, int n_eig, int j_min, int j_max,
                          double tol, int max_iter, double* lambdas, double* modes, int on_device,
                          int* iterations);

/* Right-hand sides of the stability adjoint equations K v_k = g_k (Sec. 2.2, Eq. 7):
 *   g_k = Phi_k^T (dK_sigma/du) Phi_k = -sum_e E_sigma(rho_e) (D_0 B)^T w_e(Phi_k),
 *   w_e,v = sum_ab L_ij[a, b] Phi_a . Phi_b summed over the index pairs (i, j) of Voigt
 *           component v (both orders for a shear component),
 * masked at fixed DOFs, for the problem's current density.  K_sigma is linear in u, so g does
 * not depend on u.  modes: n_dofs x n_modes column-major (e.g. from tomg_buckling); g: n_dofs
 * x n_modes column-major, ready for tomg_solve.  Host or device arrays (on_device),
 * caller-owned, may not alias.  E_INVALID for n_modes outside 1..16. */
tomg_status tomg_buckling_adjoint_rhs(tomg_problem* prob, int n_modes, const double* modes,
                                      double* g, int on_device);
/* Sensitivities of the buckling eigenvalues (Sec. 2.2, Eq. 6) and of their p-norm aggregate
 * F = (sum_k lambda_k^p)^(1/p) (Eq. 8-9) with respect to the densities rho:
 *   dlambda_k/drho_e = E_sigma'(rho_e) Phi_k,e^T K_sigma,e^1 Phi_k,e
 *                      - lambda_k E'(rho_e) Phi_k,e^T Ke Phi_k,e - E'(rho_e) v_k,e^T Ke u_e,
 *   dF/drho_e = F^(1-p) sum_k lambda_k^(p-1) dlambda_k/drho_e,
 * for K-normalised modes Phi_k (as tomg_buckling returns them), the displacements u and the
 * adjoint solutions v_k of K v_k = g_k (tomg_buckling_adjoint_rhs, then tomg_solve).
 * K_sigma,e^1 is the element stress stiffness at unit stress modulus, E' the derivative of the
 * SIMP modulus of K (Eq. 2), E_sigma' that of Eq. 5 (0 below rho = 0.1).  The paper prints the
 * adjoint term as +v^T E_sigma' (dK/dE) u; this is the derivation's -v^T E' (dK/dE) u.
 * lambdas: host, n_modes; u: n_dofs; modes, adjoints: n_dofs x n_modes column-major;
 * dlambda: NULL or n_elems x n_modes column-major; dF: NULL or n_elems; F: NULL or a host
 * scalar.  Arrays other than lambdas and F on host or device (on_device).  E_INVALID for
 * n_modes outside 1..16, pnorm < 1 or a p-norm that is not positive and finite.  dF/drho is
 * the chain rule's first factor: tomg_density_filter with transpose gives dF/dalpha. */
tomg_status tomg_buckling_sensitivity(tomg_problem* prob, const double* u, int n_modes,
                                      const double* lambdas, const double* modes,
                                      const double* adjoints, double pnorm, double* dlambda,
                                      double* dF, double* F, int on_device);

/* Adaptive hybrid hierarchy (Sec. 4.4): the geometric level count (including the fine grid)
 * the next tomg_setup of this problem will use, 0 before the first setup with adaptive_geo. */
tomg_status tomg_adaptive_geo_levels(const tomg_problem* prob, int* n_geo_levels);
/* Number of kernels this library launched since the context was created. */
tomg_status tomg_kernel_launches(const tomg_ctx* ctx, int64_t* count);

#ifdef __cplusplus
}
#endif
#endif /* TOMG_H */
