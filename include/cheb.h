/*
 * cheb.h - C ABI of the B300 Chebyshev-collocation diffusion solver.
 *
 * The library solves -div(K grad u) = f on a box [lo, hi] (1-D, 2-D or 3-D)
 * by collocation at the Chebyshev-Gauss-Lobatto (CGL) points with per-face
 * Dirichlet / Neumann data (Quecedo & Segurado, "An FFT-based solver with
 * general boundary conditions for stationary diffusion problems based on
 * Chebyshev collocation", Sec. 2).  Every numerical step runs in the
 * library's own CUDA kernels for sm_103a; the header uses plain pointers
 * and sizes only.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grid: n[a] points along axis a (x = 0, y = 1, z = 2), N_a = n[a] - 1.
 *    Node j of axis a sits at t_j = (hi-lo)/2 cos(pi j / N_a) + (hi+lo)/2
 *    (Sec. 2.2, affine mapping): node 0 is the hi end, node N_a the lo end.
 *    Unused axes of 1-D / 2-D problems have n = 1.  Active axes need n >= 3.
 *  - Fields: row-major [nz][ny][nx] arrays (x fastest), device memory,
 *    double (FP64) or float (FP32) as the call states.  The caller owns
 *    every field buffer; buffers of one call must not overlap unless stated.
 *  - Faces: id f = 2a + side, side 0 = lo, side 1 = hi: x-, x+, y-, y+, z-, z+.
 *    Face data of face f is a device array shaped like a field with axis a
 *    removed (x faces [nz][ny], y faces [nz][nx], z faces [ny][nx]).
 *  - Boundary rows (Sec. 2 "Extension to the three-dimensional setting":
 *    equations at boundary nodes are replaced by the boundary conditions):
 *    each boundary node has ONE owner face; Dirichlet faces beat Neumann
 *    and flux faces, and among the others the lowest axis wins.  A Dirichlet
 *    row reads u_p = g; a Neumann row reads n.grad u = g with n the outward
 *    normal (+d_a u on the hi face, -d_a u on the lo face); a flux row reads
 *    -K_p n.grad u = g.
 *  - Streams: every call is ordered on the plan's stream.  Calls that
 *    return data to the host (solves, norms) synchronise that stream.
 *  - Errors: every function returns a cheb_status; no call aborts the
 *    process.  CHEB_ERR_ARG leaves outputs untouched.  CHEB_ERR_CUDA
 *    reports a failed CUDA call (message in cheb_last_error()).
 */
#ifndef CHEB_H
#define CHEB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cheb_plan_s* cheb_plan;

/* Face types: Dirichlet u = g; Neumann n.grad u = g; flux -K n.grad u = g
 * (the heat-flux condition q_N = -k grad T . n of Sec. 3.4, with the
 * conductivity at the boundary node). */
enum cheb_bc { CHEB_DIRICHLET = 0, CHEB_NEUMANN = 1, CHEB_FLUX = 2 };

/* arithmetic of an operator application (buffer element type) */
enum cheb_prec { CHEB_FP64 = 0, CHEB_FP32 = 1 };

/* solve mode: plain FP64 LGMRES, or FP32 inner LGMRES inside an FP64
 * iterative-refinement loop */
enum cheb_solve_mode { CHEB_SOLVE_FP64 = 0, CHEB_SOLVE_MIXED = 1 };

/* per-axis line-derivative route: FFT-based DCT-I + recurrence, or the
 * dense differentiation matrix.  CHEB_ROUTE_AUTO lets the plan choose.
 * CHEB_ROUTE_TENSOR (FP32 operator apply only): the dense matrix on the
 * tensor cores (split-TF32 tcgen05 contractions, FP32-level accuracy);
 * needs a 2-D or 3-D grid, 33 <= n <= 257 on the axis and at least 128
 * lines; the other FP32 line operations of that axis (derivative, adjoint)
 * then use the power-of-two transform route where it exists, else the
 * dense one, else the chirp transform. */
enum cheb_route { CHEB_ROUTE_AUTO = -1, CHEB_ROUTE_TRANSFORM = 0, CHEB_ROUTE_DENSE = 1, CHEB_ROUTE_TENSOR = 2 };

enum cheb_status {
  CHEB_OK = 0,
  CHEB_ERR_NOT_CONVERGED = 1,   /* solve stopped at maxiter; best iterate written */
  CHEB_ERR_ARG = -1,            /* invalid argument (null pointer, bad size, ...) */
  CHEB_ERR_CUDA = -2,           /* a CUDA runtime call failed */
  CHEB_ERR_NOMEM = -3,          /* device allocation failed */
  CHEB_ERR_NONFINITE = -4,      /* NaN / Inf met in a residual norm */
  CHEB_ERR_SINGULAR_BC = -5,    /* no Dirichlet face: A is singular */
  CHEB_ERR_UNSUPPORTED = -6     /* size / route combination not supported */
};

/* Create a plan for one grid.
 *   dim      1, 2 or 3 (the first dim axes are active)
 *   n        points per axis, n[a] >= 3 for a < dim, n[a] = 1 otherwise
 *            (route TRANSFORM needs 2 <= n - 1 <= 256: a power of two n - 1 >= 4
 *             runs one FFT of length 2(n - 1) per line pair, any other n - 1 the
 *             chirp form (Bluestein's convolution, FFT length the power of two
 *             >= 4(n - 1) - 1); route DENSE needs n <= 129.  Without a forced
 *             route an axis takes the power-of-two transform, else dense, else
 *             the chirp transform)
 *   lo, hi   interval of each axis (hi > lo); entries of unused axes ignored
 *   bc_type  six CHEB_DIRICHLET / CHEB_NEUMANN / CHEB_FLUX values, faces
 *            x-,x+,y-,y+,z-,z+ (flux faces exclude CHEB_ROUTE_TENSOR)
 *   stream   cudaStream_t to order the plan's work on (NULL = legacy stream)
 * The plan owns its device tables and, once a solve runs, its Krylov
 * workspace; cheb_plan_destroy frees them.  A pure-Neumann set is accepted
 * here (cheb_apply is defined for it) but cheb_solve rejects it with
 * CHEB_ERR_SINGULAR_BC (also when every face is Neumann or flux). */
int cheb_plan_create(cheb_plan* out, int dim, const int n[3], const double lo[3],
                     const double hi[3], const int bc_type[6], void* stream);
int cheb_plan_destroy(cheb_plan plan);
int cheb_plan_set_stream(cheb_plan plan, void* stream);

/* Force the line-derivative route of one axis (CHEB_ROUTE_*), both
 * precisions; fails with CHEB_ERR_UNSUPPORTED when the axis size does not
 * allow it.  get_route reports the FP64 route. */
int cheb_plan_set_route(cheb_plan plan, int axis, int route);
int cheb_plan_get_route(cheb_plan plan, int axis, int* route);
/* The FP32 route of one axis alone (CHEB_ROUTE_TRANSFORM, _DENSE, _TENSOR
 * or _AUTO); same errors as cheb_plan_set_route.  get_route32 reports it. */
int cheb_plan_set_route32(cheb_plan plan, int axis, int route);
int cheb_plan_get_route32(cheb_plan plan, int axis, int* route);

/* Line-tile height of the transform and dense line passes of one axis in
 * precision prec: 8 or 16 lines per CTA (default 16; 8 doubles the CTA count
 * of small grids).  The tensor route has its own tiling. */
int cheb_plan_set_tile(cheb_plan plan, int axis, int prec, int lines);
int cheb_plan_get_tile(cheb_plan plan, int axis, int prec, int* lines);

/* Autotuner: for every active axis whose size allows more than one choice,
 * time the operator line pass with each route the size allows - transform
 * and dense, each with line tiles of 8 and 16 lines, and for FP32 tensor
 * (CHEB_ROUTE_TENSOR) - FP64 and FP32 separately, on the plan's grid and
 * stream, and keep the fastest (route, tile).  cache_path (nullable) names a
 * text file of earlier decisions, one line per (GPU name, axis size,
 * precision); hits skip the timing and new decisions are appended.
 * routes_out[6] (nullable) receives the FP64 routes of axes x, y, z then the
 * FP32 routes (cheb_plan_get_tile reports the tiles).  Allocates three
 * temporary fields when timing; synchronises the plan's stream. */
int cheb_autotune(cheb_plan plan, const char* cache_path, int routes_out[6]);

/* Host copy of the CGL coordinates of one axis (n[axis] doubles, node 0 =
 * hi end).  Callers sample f, K and face data at these points. */
int cheb_nodes(cheb_plan plan, int axis, double* out_host);

/* Number of grid points nx*ny*nz. */
size_t cheb_plan_size(cheb_plan plan);

/* One first-derivative line pass (Alg. 1 semantics; Sec. 2.2):
 * du = d u / d t_axis at every node, computed per line as forward DCT-I
 * to Chebyshev coefficients, the backward derivative recurrence
 * b_{k-1} = b_{k+1} + 2k a_k (k = N..1, b_0 halved) and the inverse DCT-I,
 * times 2/(hi-lo).  u, du: device fields of type prec; must not overlap. */
int cheb_deriv(cheb_plan plan, int prec, int axis, const void* u, void* du);

/* Transposed line pass: du = D_axis^T u (used by the discrete adjoint). */
int cheb_deriv_t(cheb_plan plan, int prec, int axis, const void* u, void* du);

/* Operator apply with boundary rows (Alg. 3; Eq. (eq1) of Sec. 3.3):
 *   interior node p:  (Au)_p = -sum_a [D_a (K * D_a u)]_p
 *   boundary node p:  Dirichlet u_p, Neumann +-(D_a u)_p, flux -+K_p (D_a u)_p
 *                     (owner face's axis and outward sign)
 * K, u, Au: device fields of type prec.  Au must not alias K or u. */
int cheb_apply(cheb_plan plan, int prec, const void* K, const void* u, void* Au);

/* Transposed operator: ATlam = A^T lam with A as in cheb_apply (the
 * discrete adjoint; boundary rows transposed too).  Same buffer rules. */
int cheb_adjoint_apply(cheb_plan plan, int prec, const void* K, const void* lam, void* ATlam);

/* Right-hand side with boundary rows: b_p = f_p at interior nodes and the
 * owner face's datum at boundary nodes (Eqs. (eq:residualN), (eq:boundaryN)).
 * f, b: FP64 device fields (may alias); face_vals[f]: FP64 device face
 * arrays (entries of unused axes ignored). */
int cheb_rhs(cheb_plan plan, const double* f, const double* const face_vals[6], double* b);

/* ------------------------------------------------------------------------
 * Solves
 * ------------------------------------------------------------------------ */

/* Preconditioner of the Krylov solves.  The paper solves the collocation
 * system with LGMRES and no preconditioner (CHEB_PRECOND_NONE).  FDM is
 * the exact inverse of the constant-coefficient collocation operator with
 * the same boundary rows (conductivity kref), applied by fast
 * diagonalization; the solve runs on M^{-1} A u = M^{-1} b. */
enum cheb_precond { CHEB_PRECOND_NONE = 0, CHEB_PRECOND_FDM = 2 };

/* System the Krylov solver works on.  REPLACE: the boundary equations
 * replace the collocation rows at boundary nodes (cheb_apply).  ELIMINATE:
 * the paper's formulation (Sec. 2.3.1): the boundary unknowns are eliminated
 * through the boundary rows, x_r = G x_k + H g, and the solver runs on the
 * reduced interior system (A_kk + A_kr G) x_k = f_k - A_kr H g, applied
 * matrix-free (the boundary values of a Krylov vector come from the per-line
 * elimination of the preconditioner's tables); FP64 forward solves only.
 * Both give the same discrete solution; the reduced system is better
 * conditioned. */
enum cheb_formulation { CHEB_FORM_REPLACE = 0, CHEB_FORM_ELIMINATE = 1 };

typedef struct cheb_solve_opts {
  int mode;            /* CHEB_SOLVE_FP64 or CHEB_SOLVE_MIXED */
  double rtol;         /* stop when ||M^{-1}(b - A u)|| <= rtol ||M^{-1} b|| (M = I
                          without preconditioner) */
  double atol;         /* ... or when ||M^{-1}(b - A u)|| <= atol */
  int restart;         /* m: new Krylov directions per LGMRES cycle */
  int augment;         /* k: error-approximation vectors carried between cycles;
                          restart + augment + 1 <= 40 */
  int maxiter;         /* cap on Arnoldi steps (all precisions) */
  double inner_rtol;   /* MIXED: relative tolerance of each FP32 inner solve; a
                          refinement that needs less takes max(inner_rtol,
                          rtol / (2 eta)), eta the current outer residual */
  int inner_maxiter;   /* MIXED: cap on Arnoldi steps of one inner solve */
  int max_refinements; /* MIXED: cap on FP64 refinement steps */
  int reorth;          /* 1: Gram-Schmidt twice per Arnoldi step */
  int precond;         /* CHEB_PRECOND_* */
  double kref;         /* FDM conductivity; <= 0: geometric mean of K */
  int verbose;         /* 1: progress lines on stderr */
  int use_graph;       /* 1: Arnoldi cycles after a full-length cycle run as captured
                          CUDA graphs (one host synchronisation per cycle); graphs
                          are cached per operator and shape */
  int recycle;         /* MIXED: 1 = each refinement's FP32 inner solve starts with
                          the augmentation vectors (and their images under the
                          preconditioned operator) of the previous one; the
                          operator is the same within one solve, so they remain
                          valid.  0 = every inner solve starts without them (the
                          default: measured faster on the two-phase hierarchy) */
  int formulation;     /* CHEB_FORM_REPLACE or CHEB_FORM_ELIMINATE */
  double coarse_rtol;  /* hierarchies: rtol of the levels below the finest (their
                          solutions only start the next level); 0 = rtol */
  int batch_mode;      /* cheb_solve_batched / cheb_picard_batched: CHEB_BATCH_* */
  int precond_matrices; /* FP32 FDM applications on the tensor cores: CHEB_PMAT_TF32
                          (the default) uses the eigenvector matrices rounded to TF32,
                          two TF32 products per step; CHEB_PMAT_FP32 the matrices to
                          FP32 accuracy (split pair), three products.  Either way the
                          field is contracted to FP32 accuracy, so the preconditioner
                          is a fixed linear map; TF32 matrices change it by about 2^-11
                          relative and leave the solve's tolerance as it is (the FP64
                          refinement and its stopping test keep their form).  FP64
                          applications always use FP64 matrices. */
} cheb_solve_opts;

/* Precision of the FP32 preconditioner's eigenvector matrices (opts.precond_matrices). */
enum cheb_pmat { CHEB_PMAT_TF32 = 0, CHEB_PMAT_FP32 = 1 };

/* How a batch iterates: LOCKSTEP = every instance in one iteration stream
 * (batched line passes over an (instance, line-tile) work list, batched
 * Gram-Schmidt and Givens kernels with a per-instance converged mask, the
 * preconditioner's lift, face and boundary-line steps batched over the
 * instances, one captured graph per Arnoldi step; needs n <= 129 on every axis, a
 * Dirichlet face per instance, plans of one dimension and device, the
 * row-replaced formulation and reorth 0); CONCURRENT = one host thread and
 * stream per instance running the single-instance solver; AUTO = LOCKSTEP
 * where allowed and the batch has at least 32 instances or at most 200,000
 * points per instance on average (where it measured faster), else
 * CONCURRENT. */
enum cheb_batch_mode { CHEB_BATCH_AUTO = 0, CHEB_BATCH_LOCKSTEP = 1, CHEB_BATCH_CONCURRENT = 2 };

typedef struct cheb_solve_info {
  int status;              /* return code of the solve */
  int iterations;          /* Arnoldi steps, all precisions */
  int cycles;              /* LGMRES restart cycles */
  int refinements;         /* MIXED: FP64 refinement steps taken */
  int applies_fp64;        /* operator applications in FP64 */
  int applies_fp32;        /* operator applications in FP32 */
  double rel_residual;     /* final ||M^{-1}(b - A u)|| / ||M^{-1} b|| */
  double rel_residual_inner; /* MIXED: last inner relative residual */
  double seconds;          /* wall time of the call */
  double kref;             /* FDM conductivity used */
  int graph_captures;      /* Arnoldi-cycle graphs captured (use_graph) */
  int host_syncs;          /* host synchronisations of the LGMRES cycles
                              (residual norm, Arnoldi checkpoints, update norm) */
  int discarded_steps;     /* Arnoldi steps run past the converged one (their
                              work is discarded; see cheb_solve) */
} cheb_solve_info;

/* Defaults: MIXED, rtol 1e-12, restart 30, augment 3, maxiter 2000,
 * inner_rtol 1e-4, inner_maxiter 400, max_refinements 30, FDM, kref auto,
 * use_graph 0, recycle 0, formulation REPLACE, coarse_rtol 0 (= rtol),
 * batch_mode AUTO, precond_matrices TF32. */
void cheb_solve_opts_default(cheb_solve_opts* opts);

/* Solve A u = b (Alg. 2 with the Krylov solver LGMRES; boundary rows as in
 * cheb_apply).  K, b: FP64 device fields; u: FP64 device field, in: initial
 * guess (e.g. a prolonged coarse solution, Alg. 4), out: solution.  opts may
 * be NULL (defaults); info may be NULL.  Returns CHEB_OK,
 * CHEB_ERR_NOT_CONVERGED (u holds the last iterate) or an error.  The plan
 * allocates its Krylov workspace at the first solve (about
 * (restart + 2 augment + 5) fields of the working precision) and keeps it.
 * The Hessenberg matrix and its Givens rotations are updated on the device
 * (FP64); the host reads them at checkpoints: at the end of every LGMRES
 * cycle, and earlier only when the residual estimates, extrapolated at
 * their observed reduction rate, reach the tolerance.  A cycle far from the
 * tolerance therefore costs one synchronisation; a few Arnoldi steps past
 * the converged one may run and are discarded.  (With use_graph the cycles
 * run as captured graphs, one synchronisation each.) */
int cheb_solve(cheb_plan plan, const double* K, const double* b, double* u,
               const cheb_solve_opts* opts, cheb_solve_info* info);

/* Picard iteration for K = K0 (1 + beta |grad u|^2) (Sec. 2.3, Picard:
 * the nonlinearity is evaluated at the previous iterate): repeat
 * K^m = K0 (1 + beta |grad u^m|^2) (gradients by line passes, FP64), solve
 * A(K^m) u* = b warm-started from u^m (cheb_solve with opts) and relax
 * u^{m+1} = omega u* + (1 - omega) u^m (0 < omega <= 1; omega = 1 is the
 * plain iteration), until ||u^{m+1} - u^m|| / ||u^{m+1}|| <= tol or maxit.  u: FP64
 * device field, in: initial guess, out: last iterate.  info sums the inner
 * solves; picard_iters / picard_delta (nullable) receive the outer count and
 * the last relative change.  Returns CHEB_ERR_NOT_CONVERGED at maxit. */
int cheb_picard_solve(cheb_plan plan, const double* K0, const double* b, double* u, double beta,
                      double omega, double tol, int maxit, const cheb_solve_opts* opts,
                      cheb_solve_info* info, int* picard_iters, double* picard_delta);

/* Jacobian action of Newton's linearisation (Sec. 2.3, Newton; Sec. 3.4):
 *   interior node p:  (J du)_p = -sum_a [D_a (K * D_a du + C_a * du)]_p
 *   boundary node p:  Dirichlet du_p, Neumann +-(D_a du)_p, flux
 *                     -+(K_p (D_a du)_p + C_a,p du_p) (owner face's axis, outward sign)
 * For a conductivity law k(u) this is the derivative of A(k(u)) u at u along
 * du when K = k(u) and C_a = k'(u) d_a u (the paper's J(T) dT =
 * div(-k grad dT - k' dT grad T)).  K, du, Jdu and C[a] for a < dim: device
 * fields of type prec (entries of unused axes ignored); Jdu must not alias K
 * or du.  Axes on CHEB_ROUTE_TENSOR use their transform or dense route here. */
int cheb_jacobian_apply(cheb_plan plan, int prec, const void* K, const void* const C[3], const void* du,
                        void* Jdu);

/* Newton's method for the temperature-dependent conductivity
 * k(u) = K0 / (1 + alpha u) (Sec. 2.3, Newton; the reciprocal law of Sec. 3.4)
 * with boundary rows as in cheb_apply at K = k(u) (a flux face imposes
 * -k(u) n.grad u = g).  Repeat: K = k(u^m), C_a = k'(u^m) d_a u^m; solve
 * J(u^m) du = b - A(K) u^m (cheb_jacobian_apply) by LGMRES left-preconditioned
 * with the constant-coefficient inverse at the geometric mean of K, to a
 * relative tolerance of opts->inner_rtol (MIXED: FP32 LGMRES whose error the
 * next step's FP64 nonlinear residual corrects; FP64: FP64 LGMRES); then
 * u^{m+1} = u^m + du; until ||du|| / ||u^{m+1}|| <= tol, or until the
 * preconditioned nonlinear residual ||M^{-1} R(u)|| <= opts->rtol ||M^{-1} b||
 * before a step (a prolonged guess that already resolves the solution costs
 * no linear solve), or maxit steps.  alpha = 0 is the linear problem.  K0, b:
 * FP64 device fields; u: FP64 device field, in: initial guess (e.g. a
 * prolonged coarse solution, Alg. 4), out: last iterate.  info sums the linear
 * solves (rel_residual: the last preconditioned relative nonlinear residual);
 * newton_iters / newton_delta (nullable) receive the step count and the last
 * relative step (0 when the residual test stopped it).  Returns
 * CHEB_ERR_NOT_CONVERGED at maxit.
 * Allocates six FP64 fields of scratch for the call (and four FP32 fields in
 * MIXED), plus the plan's Krylov workspace. */
int cheb_newton_solve(cheb_plan plan, const double* K0, double alpha, const double* b, double* u, double tol,
                      int maxit, const cheb_solve_opts* opts, cheb_solve_info* info, int* newton_iters,
                      double* newton_delta);

/* Batches of independent instances (each its own plan, any sizes).
 * opts->batch_mode picks the iteration (CHEB_BATCH_*).  LOCKSTEP copies the
 * instances' K, b and u into one concatenated workspace (allocated for the
 * call: about (restart + 2 augment + 5) FP32 and 8 FP64 words per DOF of the
 * batch), iterates all instances together, each leaving the iteration when
 * it converges, and copies u back; it waits for the plans' streams first and
 * runs on a private stream, and the plans must not be used by other calls
 * until it returns (their preconditioners carry the call's mask).  info.graph_captures counts the step graphs it
 * captured.  CONCURRENT runs one host thread per instance on its plan's
 * stream (plans on the legacy NULL stream get a private stream for the
 * call).  Arrays have `count` entries; infos / picard_iters may be NULL.
 * Returns the most severe status; the first error message is kept. */
int cheb_solve_batched(int count, const cheb_plan* plans, const double* const* K,
                       const double* const* b, double* const* u, const cheb_solve_opts* opts,
                       cheb_solve_info* infos);
int cheb_picard_batched(int count, const cheb_plan* plans, const double* const* K0,
                        const double* const* b, double* const* u, double beta, double omega,
                        double tol, int maxit, const cheb_solve_opts* opts,
                        cheb_solve_info* infos, int* picard_iters);

/* Discrete adjoint solve: lambda = A^{-T} dJdu with A = A(K) as in
 * cheb_apply (LGMRES on A^T, preconditioned by M^{-T}; same options and
 * modes as cheb_solve).  lambda: FP64 device field, in: initial guess, out:
 * solution.  When dJdK is not NULL it is incremented by
 * sum_a (D_a^T P_int lambda) * (D_a u), the gradient of J(u(K)) with respect
 * to nodal K for the forward solution u (P_int zeroes boundary rows; K enters
 * A only through the interior rows).  The gradient with respect to b is
 * lambda itself (f on interior rows, boundary data on boundary rows). */
int cheb_adjoint_solve(cheb_plan plan, const double* K, const double* u, const double* dJdu,
                       const cheb_solve_opts* opts, double* lambda, double* dJdK,
                       cheb_solve_info* info);

/* Modal prolongation (Sec. 2.3.3, Alg. 4): per axis, coarse nodal values
 * -> Chebyshev coefficients (DCT-I), zero-padded to the fine degree, ->
 * fine nodal values (inverse DCT-I).  The fine plan must have N_f = 2 N on
 * every active axis (3 <= N, N_f <= 256; CHEB_ERR_UNSUPPORTED otherwise)
 * and the same box; N not a power of two runs the chirp form.  u_c:
 * coarse device field, u_f: fine device field, both of type prec.  Uses two
 * scratch arrays owned by the fine plan (allocated at the first call). */
int cheb_prolong(cheb_plan coarse, cheb_plan fine, int prec, const void* u_c, void* u_f);

/* cheb_prolong for callers that cannot allocate device memory (code running
 * inside a custom allocator, a memory-capped sandbox, or any process that
 * must not call cudaMalloc from this library).  No counterpart in the paper.
 * Same arguments and result as cheb_prolong, but it calls no cudaMalloc,
 * cudaFree or other allocating routine: the intermediate arrays live in one
 * fixed 16 MiB device array inside the library, which every GPU that loads
 * the library keeps until the process exits.  Grids whose intermediates
 * exceed 16 MiB are rejected with CHEB_ERR_UNSUPPORTED: 3-D grids up to
 * 65^3 -> 129^3 fit in FP64 and FP32, 129^3 -> 257^3 does not.  The first call on
 * a device looks up the array's device address for that device (a
 * cudaGetSymbolAddress call), so make that first call before any stream
 * capture.  The current device must be the one the plans were created on
 * (else CHEB_ERR_ARG).  All calls share the one array and nothing in it needs
 * to start at zero; calls that overlap on the GPU (other streams, other host
 * threads) race on it, so order them on one stream. */
int cheb_prolong_noalloc(cheb_plan coarse, cheb_plan fine, int prec, const void* u_c, void* u_f);

/* out = ||a - b||_2 / ||a||_2 for FP64 device fields on the plan's grid (the
 * refinement indicator e_ref of Sec. 2.3.3 with a the fine solution and b
 * the prolonged coarse solution).  Synchronises. */
int cheb_rel_diff(cheb_plan plan, const double* a, const double* b, double* out);

/* Hierarchical refinement (Alg. 4) over `levels` plans of doubling N:
 * solve level 0 from the guess in u[0]; for each further level prolong the
 * previous solution into u[l] as the initial guess, solve, and report
 * e_ref[l] = ||u_l - P u_{l-1}|| / ||u_l|| (e_ref[0] = 0).  K[l], b[l], u[l]:
 * FP64 device fields of level l.  infos, e_ref: arrays of `levels` entries
 * (may be NULL).  Returns the last level's status. */
int cheb_solve_hierarchy(int levels, const cheb_plan* plans, const double* const* K,
                         const double* const* b, double* const* u, const cheb_solve_opts* opts,
                         cheb_solve_info* infos, double* e_ref);

/* Volume-averaged flux of the homogenisation study (Sec. 3.3, effective
 * conductivity): out = (1/|Omega|) int_Omega K d_axis u, the integral by the
 * tensor Clenshaw-Curtis rule on the CGL nodes (exact for the interpolant's
 * polynomial degree), d_axis u by one FP64 line pass.  With q = -K grad u and
 * the imposed macroscopic gradient G along axis, K_num = -<q_axis>/G =
 * out / G.  K, u: FP64 device fields; synchronises the plan's stream. */
int cheb_flux_average(cheb_plan plan, int axis, const double* K, const double* u, double* out);

/* Hierarchical refinement driven by the finest level's data alone: the
 * coarse levels' K and b are recomputed from the fine K and b by injection
 * (CGL grids nest: coarse node j is fine node 2j per level, with the same
 * owner face), solved as in cheb_solve_hierarchy from a zero coarsest guess,
 * and kept only in the coarse plans' workspaces; u (fine, FP64) receives the
 * finest solution.  plans: `levels` plans of doubling N (as for
 * cheb_prolong), the last one the fine grid of K, b, u.  The solution does
 * not depend on the coarse levels (they only start the iterations), so its
 * derivatives are those of the fine solve: cheb_adjoint_solve on the fine
 * plan gives them.  infos, e_ref: arrays of `levels` entries (nullable). */
int cheb_solve_hierarchy_fine(int levels, const cheb_plan* plans, const double* K, const double* b, double* u,
                              const cheb_solve_opts* opts, cheb_solve_info* infos, double* e_ref);

/* z = M^{-T} y (transposed FDM preconditioner, used by the adjoint solve). */
int cheb_precond_apply_t(cheb_plan plan, int prec, double kref, const void* y, void* z);

/* z = M^{-1} r for the FDM preconditioner with conductivity kref > 0
 * (device fields of type prec; FP32 with the eigenvector matrices to FP32
 * accuracy, i.e. cheb_precond_apply_m with CHEB_PMAT_FP32). */
int cheb_precond_apply(cheb_plan plan, int prec, double kref, const void* r, void* z);

/* Same with the FP32 matrix precision given (matrices: CHEB_PMAT_*; ignored
 * for CHEB_FP64 and on grids the tensor-core contraction does not cover).
 * CHEB_PMAT_TF32 is the preconditioner the FP32 inner solves apply by default.
 * CHEB_ERR_ARG for an unknown matrices value. */
int cheb_precond_apply_m(cheb_plan plan, int prec, int matrices, double kref, const void* r, void* z);

/* ------------------------------------------------------------------------
 * Instrumentation
 * ------------------------------------------------------------------------ */

/* Number of kernels this library has launched in the process. */
long long cheb_launch_count(void);

/* Per-phase device timing with CUDA events recorded on the plan streams:
 * enable (on = 1) or disable, resetting the totals.  Phases: 0 FP64 operator
 * applies, 1 FP32 applies, 2 FP64 preconditioner, 3 FP32 preconditioner,
 * 4 FP64 Gram-Schmidt, 5 FP32 Gram-Schmidt, 6 prolongation, 7 other. */
int cheb_profile_enable(int on);
/* Totals since enabling: ms[8] milliseconds and counts[8] timed intervals
 * (either may be NULL).  Waits for the recorded events. */
int cheb_profile_read(double* ms, long long* counts);

/* Measured throughput of the CUDA-core fused multiply-add pipe of the
 * current device in precision prec (CHEB_FP64 or CHEB_FP32), in TFLOP/s
 * (one FMA = two flops): independent FMA chains in every thread of a grid
 * that fills every SM, about 20 ms per launch, five launches timed with CUDA
 * events.  A measurement helper for the ALU-bound kernels' rooflines (the
 * paper has no counterpart); allocates a few KB, synchronises its own
 * stream.  ms_per_launch (nullable) receives the launch time. */
int cheb_fma_peak(int prec, double* tflops, double* ms_per_launch);

/* Failure-detection self-test of the tensor-core kernels' bounded waits:
 * one CTA allocates tensor memory like the contraction kernels, waits on a
 * barrier that nothing completes with a limit of wait_cycles SM clocks
 * (1 .. 2^31), gives up, raises the device error word and frees its tensor
 * memory.  Returns CHEB_ERR_CUDA with the same message a real give-up
 * produces (the expected outcome), CHEB_OK if the wait did not give up.
 * The context stays usable.  Runs on the legacy stream and synchronises
 * it.  A test hook; the paper has no counterpart. */
int cheb_selftest_bounded_wait(long long wait_cycles);

/* Human-readable text of a status code, and the message of the last failed
 * call on the calling thread. */
const char* cheb_status_str(int status);
const char* cheb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CHEB_H */
