/*
 * dcg.h -- C ABI of the GB300 deflated-CG library (libdcg.so).
 *
 * The library solves the symmetric positive definite system
 *
 *     A x = f,   A = (1/dt) M_dev + K_div,
 *
 * that one implicit-Euler step of the pseudo-stress Stokes problem produces
 * (Section 2.3, Eq. weak_IE; Section 3, Eq. pb_study; the system is the
 * paper's A* = M + dt*A divided by dt). M_dev is the matrix of the form
 * (nu^-1 dev sigma, dev tau), K_div that of (div sigma, div tau) (Section 2.2,
 * forms M and A; component form Eq. component_form). Each of the d*d tensor
 * components is a continuous Q1 nodal field on the uniform mesh of [0,1]^d
 * with n elements per side; every boundary node is eliminated (homogeneous
 * Dirichlet), leaving m = n-1 interior nodes per axis.
 *
 * Solvers: plain CG, and the flexible deflated CG of Algorithm 2 with
 * deflation space V = (1/sqrt d)(v kron I) (Eq. Vmatrix), whose inner system
 * V^T A V (a Laplacian, Corollary 1) is solved by the W-cycle multigrid of
 * Algorithms 3-4 with the RAS smoother of Section 4.2.
 *
 * Vector layout (all vectors): node-major. Interior nodes are numbered
 * lexicographically with x fastest (then y, then z); each node holds its d*d
 * components in the paper's row-major order [s11 s12 .. s1d s21 .. sdd]
 * (Section 3.1). Length N = d*d*(n-1)^d doubles. Scalar (inner) vectors have
 * one double per interior node, same node order.
 *
 * Matrix layout: block sparse rows with b x b blocks, b = d*d, one block row
 * per interior node; block (a, c) is stored for every pair of nodes sharing
 * an element (3^d neighbourhood clipped at the boundary), columns ascending,
 * numerical zeros kept; blocks row-major doubles; row_ptr/col_idx int32.
 *
 * Ownership: the caller owns every pointer it passes (right-hand sides,
 * solutions, host arrays); the library never frees them and keeps no
 * reference after the call returns. The library owns everything inside a
 * dcg_problem (device memory allocated with cudaMalloc in dcg_assemble /
 * dcg_setup) and frees it in dcg_destroy.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream). Work is enqueued on it; calls that must read a scalar
 * back (convergence tests) synchronise that stream.
 *
 * Errors: every int-returning call returns a DCG_* status and never throws
 * across the ABI. On DCG_ERR_CUDA the message of the failing CUDA call is
 * available from dcg_last_error().
 */
#ifndef DCG_H
#define DCG_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define DCG_OK                 0
#define DCG_ERR_INVALID_ARG    1  /* n < 2, dt <= 0, nu <= 0, tol <= 0, NULL, bad option */
#define DCG_ERR_NOT_CONVERGED  2  /* max_it reached; x holds the last iterate, stats filled */
#define DCG_ERR_BREAKDOWN      3  /* (d, M_D d) <= 0 or non-finite (also a non-finite
                                     right-hand side or initial guess); x holds the last iterate */
#define DCG_ERR_CUDA           4  /* a CUDA call failed; see dcg_last_error() */
#define DCG_ERR_OOM            5  /* device allocation failed */
#define DCG_ERR_UNSUPPORTED    6  /* configuration outside what the kernels implement */
#define DCG_ERR_STATE          7  /* call order violated (e.g. solve before setup) */

/* ---- option values ----------------------------------------------------- */
#define DCG_INNER_FIXED     0  /* tau_c = c * tol (Eq. fixed_tol, c = c_F) */
#define DCG_INNER_ADAPTIVE  1  /* tau_c = c * tol ||f|| / ||r_i|| (Eq. tol, c = c_A) */
#define DCG_INNER_EXACT     2  /* inner system solved directly (fast diagonalisation) */

#define DCG_FCG1     0  /* flexible CG truncated to one direction (m_i = 1) */
#define DCG_FR       1  /* classical CG coefficients on the deflated system */
#define DCG_FCG_INF  2  /* FCG of Algorithm 1 with directions stored; untruncated while a
                           pass has at most fcg_max_dirs iterations, then the
                           truncation-restart rule of the remark after Table 4 */
#define DCG_GMRES    3  /* GMRES on the deflated system (remarks in Sections 4.3 and 5.1):
                           Arnoldi with classical Gram-Schmidt applied twice, restart
                           length fcg_max_dirs, inner tolerance of Eq. tol from the
                           least-squares residual norm; host-driven loop */

#define DCG_FP64   0  /* everything in FP64 */
#define DCG_MIXED  1  /* W-cycle (stencils, transfers, RAS) in FP32; outer CG FP64 */

#define DCG_INV_FP32  0  /* RAS patch inverses stored FP32 (mixed mode) */
#define DCG_INV_BF16  1  /* RAS patch inverses and box residuals in BF16, products on tcgen05
                             tensor cores with FP32 accumulation (mixed mode) */

#define DCG_RAS_MULTIPLICITY  0  /* D_i = 1/multiplicity (Section 4.2) */
#define DCG_RAS_RESTRICTED    1  /* D_i = 1 on the core tile, 0 on the overlap */

typedef struct dcg_problem dcg_problem;

/* Uniform mesh of [0,1]^dim with n elements per side. */
typedef struct {
  int dim;  /* 2 or 3 */
  int n;    /* elements per side, >= 2 */
} dcg_mesh;

/* Solver options (Algorithm 2 inputs m1, m2, tol, n_max; Section 4.2 blocks).
 * dcg_default_options() fills the defaults given in brackets. */
typedef struct {
  int max_levels;    /* multigrid levels incl. the coarsest [4]; coarsen while
                        n_k is even and n_k >= 8 */
  int patch;         /* RAS core tile, nodes per axis [4] */
  int overlap;       /* RAS overlap layers, 2*overlap <= patch [1] */
  int m1, m2;        /* pre / post smoothing steps [2, 2] */
  int inner_rule;    /* DCG_INNER_* [FIXED] */
  double c;          /* c_F or c_A [0.01] */
  int inner_nmax;    /* W-cycle cap per inner solve, Algorithm 3 n_max [100] */
  int recurrence;    /* DCG_FCG1 / DCG_FR / DCG_FCG_INF / DCG_GMRES [FCG1] */
  int precision;     /* DCG_FP64 / DCG_MIXED [FP64] */
  int ras_inverse;   /* DCG_INV_* (mixed only) [FP32] */
  int ras_weights;   /* DCG_RAS_* [MULTIPLICITY] */
  int deflate;       /* 1 = deflated CG, 0 = plain CG [1] */
  int max_restarts;  /* true-residual restarts after reconstruction [3] */
  int fcg_max_dirs;  /* DCG_FCG_INF: m_max of the truncation-restart rule
                        m_i = max{1, mod(i, m_max + 1)} (remark after Table 4):
                        direction d_i is orthogonalised against the m_i most
                        recent directions, so a pass of at most m_max
                        iterations is the untruncated FCG(inf). Directions
                        d and M_D d are kept in 2 * m_max device vectors of N
                        doubles. DCG_GMRES: the restart length (m_max + 1
                        basis vectors). 0 = min(256, the count that fits
                        8 GiB) [0] */
  int check_every;   /* plain CG only: iterations between host convergence
                        reads (deflated CG reads every iteration) [1] */
  int stall_window;  /* deflated CG: a pass whose recursive residual has not
                        fallen below 0.99 x its best value for
                        max(stall_window, its/4) iterations ends, is
                        reconstructed and restarted from its true residual
                        (such restarts do not count against max_restarts);
                        0 = off [200] */
  int device_loop;   /* deflated CG with W-cycle inner solves on the
                        assembled operator: 1 = the whole solve is captured
                        once into a CUDA graph whose loops (restarts, outer
                        iterations, W-cycles of each inner solve) are
                        conditional nodes driven by device-side tests, so a
                        solve is one graph launch with no host round trip per
                        iteration (re-captured when f, x, tol or max_it
                        change; kernel-class timing uses the host-driven loop);
                        a nonzero initial guess is then handled through the
                        residual equation A e = f - A x0. 0 = host-driven
                        loop with one convergence read per outer iteration
                        and per W-cycle [1] */
} dcg_options;

typedef struct {
  int status;            /* DCG_* of the solve */
  int outer_its;         /* outer (F)CG iterations, restarts included */
  int total_mg_cycles;   /* all W-cycles (paper's "Tot") */
  int iter_mg_cycles;    /* W-cycles inside outer iterations */
  int restarts;          /* true-residual restarts */
  double avg_inner;      /* iter_mg_cycles / outer_its (paper's "Inn") */
  double true_relres;    /* ||f - A x||_2 / ||f||_2 in FP64 */
  double solve_ms;       /* wall time of the solve on the stream */
  int fcg_truncated;     /* DCG_FCG_INF: directions built from fewer than all
                            previous ones of their pass (m_i < i) */
} dcg_stats;

/* Fills opts with the defaults given in brackets above (Algorithm 2's inputs
 * as the paper's 2D experiments set them: W-cycle, m1 = m2 = 2, c_F = 0.01). */
void dcg_default_options(dcg_options* opts);
/* Name of a DCG_* status code (static string; no counterpart in the paper). */
const char* dcg_status_string(int status);
/* Message of the last failing call on the calling thread (the failing CUDA
 * call for DCG_ERR_CUDA); no counterpart in the paper. */
const char* dcg_last_error(void);

/* Assemble A on the current device (Section 3.1 block structure; forms of
 * Section 3.2.1 on Q1). nu_elem: NULL for the uniform viscosity `nu`, else a
 * host array of n^dim per-element viscosities (elements lexicographic, x
 * fastest), copied during the call. matrix_free = 1 keeps only the element
 * data (1/nu per element) and applies A element by element, the element sum
 * gathered per output node (3D meshes with n >= 4; DCG_ERR_UNSUPPORTED
 * otherwise); 0 stores BSR.
 * On success *out owns the device data; free with dcg_destroy. */
int dcg_assemble(const dcg_mesh* mesh, double dt, double nu, const double* nu_elem,
                 int matrix_free, dcg_problem** out, void* stream);

/* Build the inner hierarchy for `opts`: Z_J = V^T A V (read off the assembled
 * matrix, or probed from the matrix-free operator, and checked on the device
 * to be one constant stencil, the Q1 Laplacian / d), Galerkin coarse stencils
 * Z_{k-1} = P^T Z_k P (Algorithm 2 setup), RAS patch inverses (Section 4.2)
 * and the coarsest exact solver. May be called again with new options. */
int dcg_setup(dcg_problem* p, const dcg_options* opts, void* stream);

/* Solve A x = f to ||f - A x|| <= tol ||f|| (true residual, FP64): with
 * deflate = 1 the flexible deflated CG of Algorithm 2 (outer FCG of
 * Algorithm 1 or GMRES, stop rule of Section 4.1 on the recursive deflated
 * residual, reconstruction Eq. x_defl), with deflate = 0 plain CG (the CG
 * column of Table 2).
 * f_dev, x_dev: device arrays of N doubles; x_dev holds the initial guess on
 * entry and the solution on exit. A deflated pass that ends above tol (its
 * recursion converged, or stalled: see dcg_options.stall_window) is
 * reconstructed and the solve continues from its true residual
 * (stats.restarts counts these). Returns DCG_OK, DCG_ERR_NOT_CONVERGED or
 * DCG_ERR_BREAKDOWN (stats filled in all three cases), or an error. */
int dcg_solve(dcg_problem* p, const double* f_dev, double* x_dev, double tol,
              int max_it, dcg_stats* stats, void* stream);

/* Same as dcg_solve (Algorithm 2) with host arrays: copies f to the device,
 * solves from x0 = x_host, copies the solution back into x_host (all on
 * `stream`; the device staging vectors of 2 N doubles are allocated on the
 * first call and kept until dcg_destroy). */
int dcg_solve_host(dcg_problem* p, const double* f_host, double* x_host, double tol,
                   int max_it, dcg_stats* stats, void* stream);

/* Solve nprob problems, each with nrhs right-hand sides, in one call:
 * f_dev[p*nrhs + r], x_dev[p*nrhs + r] are device arrays of problem p's N
 * (x in: initial guess, out: solution). Problems may differ in dim, n, dt and
 * options; each must have been set up and may appear only once. The problems
 * are independent, so they run concurrently. When every problem's solve can
 * be captured (dcg_options.device_loop = 1, deflated CG with W-cycle inner
 * solves, no kernel-class timing) the whole batch is captured into one CUDA
 * graph, a branch per problem with its pairs in sequence, every pair stopping
 * at its own device-side convergence test, and launched once: no host read
 * inside the batch. The branches run on as many hardware queues as
 * CUDA_DEVICE_MAX_CONNECTIONS allows (8 unless set before the first CUDA
 * call; 32 lets a large batch overlap). Otherwise up to 16 host workers, each
 * with its own non-blocking stream, take problems from a shared counter and
 * solve that problem's right-hand sides in turn with the host-driven loop.
 * The work starts after what is already queued on `stream` and `stream`
 * waits for all of it; the call returns when every solve has ended. stats: nprob*nrhs entries, filled per pair. Returns
 * DCG_OK if every pair converged, else the first non-OK pair status, or the
 * first hard error (DCG_ERR_CUDA, ...) a worker met. */
int dcg_solve_batched(int nprob, dcg_problem* const* probs, int nrhs,
                      const double* const* f_dev, double* const* x_dev, double tol,
                      int max_it, dcg_stats* stats, void* stream);

/* Choose W-cycle options for this problem by measurement. The paper fixes
 * its options by hand (Section 5); this call is a library extension with no
 * counterpart there. Starting from `base`, every candidate that differs in
 * max_levels (2..4, as the mesh allows), (patch, overlap) in {(4,1), (8,1),
 * (8,2), (12,2)} (kept when 2*overlap <= patch and the RAS box has <= 256
 * nodes) and, in mixed precision, ras_inverse (FP32, BF16) is set up and
 * timed: `reps` inner solves (Algorithm 3, zero start, relative tolerance
 * inner_tol, at most base->inner_nmax cycles) of g = V^T f on `stream`.
 * The fastest candidate wins; candidates that fail to reach inner_tol are
 * skipped. On return the problem is set up with the winner, *best holds it
 * and *best_ms its time per inner solve. f_dev: device array of N (a
 * representative right-hand side). Temporary device memory: 2 n_nodes doubles.
 * On an error return the problem may be left set up with the candidate that
 * was being tried, or not set up (DCG_ERR_STATE on solve): set it up again. */
int dcg_autotune(dcg_problem* p, const dcg_options* base, const double* f_dev, double inner_tol,
                 int reps, dcg_options* best, double* best_ms, void* stream);

/* Frees everything dcg_assemble and dcg_setup allocated for the problem
 * (the operator of Section 3.1, the hierarchy of Algorithm 2's set-up, the
 * solver vectors, captured graphs); NULL is ignored. */
void dcg_destroy(dcg_problem* p);

/* ---- queries and test hooks (same kernels as the solver) --------------- */

/* Sizes: N unknowns, interior nodes, stored blocks, multigrid levels. */
int dcg_problem_info(const dcg_problem* p, long long* n_unknowns, long long* n_nodes,
                     long long* nnzb, int* levels);

/* Interior nodes of multigrid level `level` (1 = coarsest, levels = finest,
 * the inner system of Algorithm 2) after dcg_setup; DCG_ERR_STATE before. */
int dcg_level_nodes(const dcg_problem* p, int level, long long* nodes);

/* Copy the BSR pattern / values to host arrays of n_nodes+1, nnzb and
 * nnzb*b*b entries (synchronous). */
int dcg_export_pattern(const dcg_problem* p, int* row_ptr, int* col_idx);
int dcg_export_values(const dcg_problem* p, double* values);

/* y = A x with the assembled operator A = M_dev/dt + K_div (Section 3.1
 * block structure, the paper's A* = M + dt A divided by dt), FP64, device
 * arrays of N; or the matrix-free element-by-element product. */
int dcg_spmv(const dcg_problem* p, const double* x_dev, double* y_dev, void* stream);

/* y = A x with the arithmetic of `precision`: DCG_FP64, or DCG_MIXED for
 * FP32 arithmetic on FP64 arrays, which only the matrix-free operator has
 * (the sum over elements of Section 3.1's element blocks, regrouped per
 * output node); DCG_ERR_UNSUPPORTED for DCG_MIXED on an assembled problem.
 * Inside the deflated CG of a matrix-free problem set up with DCG_MIXED the
 * products of the outer iterations run in FP32, the right-hand side
 * projection, reconstruction and true residual in FP64. */
int dcg_spmv_prec(const dcg_problem* p, const double* x_dev, double* y_dev, int precision, void* stream);

/* Deflation space of Eq. Vmatrix, V = (1/sqrt d)(v kron I) with v the
 * indicator of the diagonal components: q = V^T y (N -> n_nodes) and
 * y = V q (n_nodes -> N), device arrays (pi(z) = V Multigrid(V^T z) in
 * Algorithm 2). */
int dcg_extract(const dcg_problem* p, const double* y_dev, double* q_dev, void* stream);
int dcg_embed(const dcg_problem* p, const double* q_dev, double* y_dev, void* stream);

/* Inner operator Z_J z (FP64 stencil of level J, n_nodes in and out). */
int dcg_inner_apply(const dcg_problem* p, const double* z_dev, double* y_dev, void* stream);

/* Algorithm 3 with a fixed cycle count: z <- z + W-cycle(g - Z_J z) repeated
 * `ncycles` times (z in/out, FP64, n_nodes), in the precision set up. */
int dcg_mg_cycles(dcg_problem* p, const double* g_dev, double* z_dev, int ncycles, void* stream);

/* Algorithm 3: cycles until ||g - Z_J z|| <= tol ||g|| or nmax; *ncycles out.
 * The residual is formed in FP64; with an FP32 cycle its norm (which only
 * feeds this test) is summed from the FP32 copy the cycle receives. */
int dcg_mg_solve(dcg_problem* p, const double* g_dev, double* z_dev, double tol, int nmax,
                 int* ncycles, void* stream);

/* One RAS smoothing step on level `level` (1 = coarsest, J = finest) in the
 * set-up precision: z <- z + S_k (f - Z_k z); FP64 arrays of that level's
 * node count. */
int dcg_ras_step(dcg_problem* p, int level, const double* f_dev, double* z_dev, void* stream);

/* Exact coarsest-level solve z = Z_1^-1 f (FP64 arrays of level-1 size). */
int dcg_coarse_solve(dcg_problem* p, const double* f_dev, double* z_dev, void* stream);

/* ---- time stepping and reconstruction (Section 2.3; Section 5.2) ------- */
#define DCG_IMPLICIT_EULER  0  /* theta-method with theta = 1: alpha = dt */
#define DCG_CRANK_NICOLSON  1  /* theta = 1/2: alpha = dt / 2 */
#define DCG_BDF2            2  /* alpha = 2 dt / 3; the first step takes sigma^-1 = sigma^0 */

/* alpha(dt) of a scheme (Eq. weak_IE: a step solves (M + alpha A) sigma^n =
 * F*_n, i.e. this library's A_alpha = M_dev / alpha + K_div): assemble the
 * problem with dt = dcg_scheme_alpha(scheme, dt) to step with `dt`.
 * Returns -1 for an unknown scheme. */
double dcg_scheme_alpha(int scheme, double dt);

/* y = K_div x, the divergence form alone (N doubles in and out, device), by
 * the constant 3^d stencil of the uniform Q1 mesh (Section 3.2.1, a_ij). */
int dcg_apply_div(const dcg_problem* p, const double* x, double* y, void* stream);

/* Right-hand side b^n of one step for a problem assembled with alpha =
 * dcg_scheme_alpha(scheme, dt), from the previous steps s1 = sigma^{n-1},
 * s2 = sigma^{n-2} (BDF2 only; NULL = s1) and the load vectors F1 = F^n,
 * F0 = F^{n-1} (Crank-Nicolson only) of the forcing:
 *   implicit Euler  b = (M_dev/alpha) s1 + F1
 *   Crank-Nicolson  b = (M_dev/alpha - K_div) s1 + F1 + F0
 *   BDF2            b = (M_dev/alpha)(4/3 s1 - 1/3 s2) + F1
 * (M_dev/alpha) w is formed as A_alpha w - K_div w. Device arrays of N
 * doubles; a scratch of 3 N doubles is allocated on `stream` for the call. */
int dcg_time_rhs(dcg_problem* p, int scheme, const double* s1, const double* s2, const double* F1,
                 const double* F0, double* rhs, void* stream);

/* Pressure p = -(1/d) tr(sigma) at every interior node (Section 5.2):
 * sigma N doubles in, pres n_nodes doubles out (device). */
int dcg_pressure(const dcg_problem* p, const double* sigma, double* pres, void* stream);

/* (div sigma)_k = sum_p d_p sigma_kp at every element centre, where it is
 * exact for the Q1 fields (the mean over the element's edges along p of the
 * difference quotients); elements lexicographic (x fastest), d values per
 * element: n^d * d doubles out (device). */
int dcg_divergence(const dcg_problem* p, const double* sigma, double* div_elem, void* stream);

/* nsteps steps of `scheme` with step dt (the problem assembled with alpha =
 * dcg_scheme_alpha(scheme, dt) and set up): F[0..nsteps] the load vectors
 * F^n of the forcing at t_n, sigma0 the initial stress, sigma_out[0..nsteps-1]
 * receive sigma^1..sigma^nsteps (each step solves to tol from the previous
 * step as initial guess; stats[k], if given, its statistics). u_elem (may be
 * NULL): element-centre velocity u = u_0 + int div(sigma) dt (Section 5.2),
 * n^d * d doubles in (u_0) and out, integrated by the scheme's own rule
 * (right endpoint for implicit Euler and BDF2, trapezoid for Crank-Nicolson).
 * Returns the first non-OK step status (later steps are not run). Scratch of
 * 4 N + 2 d n^d doubles is allocated for the call. */
int dcg_time_integrate(dcg_problem* p, int scheme, double dt, int nsteps, const double* sigma0,
                       const double* const* F, double* const* sigma_out, double* u_elem, double tol, int max_it,
                       dcg_stats* stats, void* stream);

/* ---- timing of kernel classes (CUDA events, off by default) ----------- */
#define DCG_PROF_SPMV        0  /* operator products (fused BSR variants, matrix-free) */
#define DCG_PROF_VEC         1  /* vector updates and reductions */
#define DCG_PROF_RAS_SOLVE   2  /* RAS residual + shared-inverse products */
#define DCG_PROF_RAS_UPDATE  3  /* RAS weighted combination */
#define DCG_PROF_TRANSFER    4  /* level residual, restriction, prolongation */
#define DCG_PROF_COARSE      5  /* coarsest exact solve */
#define DCG_PROF_INNER_RES   6  /* FP64 inner residual of Algorithm 3 */

/* Enable timing for the classes whose bits are set in `mask` (bit c for
 * class c; 0 disables) and reset the accumulators. Launches of those classes
 * are bracketed by CUDA events on their stream (inside the W-cycle graph as
 * event-record nodes); the graph is rebuilt when the mask changes. */
int dcg_profile_enable(dcg_problem* p, unsigned mask, void* stream);

/* Accumulated device time (ms), launch count and algorithmic flops / bytes
 * (the work the method requires, not hardware counters) of one class since
 * dcg_profile_enable. Synchronises `stream`. */
int dcg_profile_read(dcg_problem* p, int cls, double* ms, long long* launches, double* flops, double* bytes,
                     void* stream);

/* ---- allocation-free coarsest solve ------------------------------------ */
/* The paper has no counterpart of this entry point: it is a service for
 * callers that cannot allocate device memory when they need the solve (a
 * process whose device memory a caching allocator has already reserved, or a
 * latency-critical loop that must not take an allocation's implicit
 * synchronisation).
 *
 * dcg_coarse_solve_static computes z = Z_1^-1 f on the coarsest level like
 * dcg_coarse_solve, always in FP64, and allocates nothing: the intermediate
 * vector lives in a fixed array of DCG_STATIC_COARSE_MAX doubles (1 MiB)
 * compiled into the library, which every GPU that loads the library keeps
 * until the process exits. f_dev, z_dev: distinct device arrays of the
 * coarsest level's node count (layout as the scalar vectors above; the
 * caller owns them). A coarsest level with more than DCG_STATIC_COARSE_MAX
 * nodes is rejected with DCG_ERR_INVALID_ARG and a message. The first call on
 * a device looks the array's device address up (cudaGetSymbolAddress); make
 * it before any stream capture. All calls share the array: calls whose work
 * overlaps on the GPU race and must be serialised by the caller. */
#define DCG_STATIC_COARSE_MAX 131072
int dcg_coarse_solve_static(dcg_problem* p, const double* f_dev, double* z_dev, void* stream);

/* ---- diagnostics (no counterpart in the paper) -------------------------- */

/* Arithmetic rate of this GPU's FMA pipes as the library's kernels see
 * them, measured with independent FMA chains on all SMs (no memory
 * traffic): precision DCG_FP64 for FP64 FMAs, DCG_MIXED for FP32 FMAs.
 * *tflops = 2 x FMAs per second / 1e12, best of three timed launches
 * (about 20 ms of GPU time each; synchronises `stream`). It is the ALU peak
 * the rooflines of the FP64-bound kernels are quoted against. */
int dcg_measure_fma_rate(int precision, double* tflops, void* stream);

/* Self-test of the bounded mbarrier wait that every bulk-copy kernel uses:
 * one CTA waits, with a limit of max_polls polls, on an mbarrier that nothing
 * will complete (no copy is in flight), records that the wait gave up and
 * returns normally. *gave_up = 1 when the wait gave up as designed; the CUDA
 * context stays usable. Synchronises `stream`. */
int dcg_selftest_bounded_wait(unsigned max_polls, int* gave_up, void* stream);

/* Number of kernels this library has launched in the process so far (a
 * replay of the captured W-cycle graph counts each of its kernel nodes). */
long long dcg_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* DCG_H */
