/*
 * fa.h -- C ABI of the parareal matrix-function library (GB300, sm_103a).
 *
 * The library evaluates f(A) as the state of a matrix ODE dX/dt = Fl(X),
 * X(0) = X0, integrated by the classical parareal method (Algorithm 1 of
 * Chehab & Petcu, "Parallel Matrix Function Evaluation via Initial value ODE
 * modelling"):
 *
 *   FA_FLOW_INV   dX/dt = X (I - A) X, X(0) = I, X(1) = A^{-1}
 *                 (Section 2, Example 1, eq. eqQ);
 *   FA_FLOW_EXP   dX/dt = A X,         X(0) = I, X(1) = exp(A)
 *                 (Section 2, Example 2);
 *   FA_FLOW_SQRT  dX/dt = A - X^2,     X(0) = I, X(inf) = A^{1/2} for SPD A
 *                 (an instance of the steady-state framework, eq. "stat" of
 *                 the introduction and Section 4).
 *
 * The time interval [0, T] is cut into N uniform slices T_n = n T / N.  The
 * fine propagator F runs J classical RK4 steps per slice, the coarse
 * propagator G runs m forward-Euler substeps per slice, and each parareal
 * iteration is: F on all N slices at once (the parallel step of Algorithm 1),
 * then the sequential correction U_{n+1} = G(U^new_n) + F(U^old_n) - G(U^old_n)
 * (eq. eqStepk+1), then the convergence test
 * max_n ||U^{k+1}_n - U^k_n||_F / ||U^{k+1}_n||_F < tol.
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Matrices at the boundary are float64, row-major, n x n, contiguous
 *   (leading dimension n).  Arrays of matrices are batch-major [count][n][n].
 * - Pointers named d* are device pointers (any CUDA allocation of the current
 *   device, e.g. PyTorch tensors); pointers named h* are host pointers.  The
 *   caller owns all of them; the library never frees them.
 * - All work is enqueued on the plan's stream.  fa_parareal_solve* synchronise
 *   that stream (they read the convergence scalar every iteration);
 *   fa_fine_sweep, fa_coarse_sweep, fa_plan_set_matrix and fa_refine are
 *   asynchronous and report device-side failures on the next synchronising
 *   call.
 * - Nothing is thrown across the ABI.  Every call returns an fa_status; on
 *   failure, fa_last_error() (thread-local) holds a one-line explanation.
 * - A plan owns no device memory except the workspace that the caller binds
 *   with fa_plan_bind_workspace (the library calls no cudaMalloc).
 * - Mixed-precision forms (FA_BF16*) use BF16 tensor-core products with
 *   float32 accumulation, a double-float32 (hi + lo) RK4 state, and float64
 *   for the parareal correction and the coarse-state additions; the norm
 *   terms of the stopping test are summed in float32 over 32 columns of a row
 *   and in float64 beyond (about 1e-6 relative, enough for any tolerance the
 *   products can reach).
 */
#ifndef FA_H
#define FA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FA_OK = 0,
  FA_ERR_ARG = 1,            /* invalid argument (sizes, pointers, enum values) */
  FA_ERR_CUDA = 2,           /* a CUDA runtime/driver call failed */
  FA_ERR_WORKSPACE = 3,      /* no workspace bound, or the bound one is too small */
  FA_ERR_NONFINITE = 4,      /* a NaN/Inf appeared in the iterates or the inputs */
  FA_ERR_NOT_CONVERGED = 5,  /* max_iters reached; the output is still written */
  FA_ERR_TIMEOUT = 6,        /* a device-side wait gave up (error flag set by a kernel) */
  FA_ERR_UNSUPPORTED = 7     /* valid but not supported (e.g. device is not sm_103) */
} fa_status;

/* FA_FLOW_COS  cos(A) by Algorithm 5 (Section 3, Example 3): A0 = 2^-m A with the smallest m >= 0
 *              such that 2^-m ||A||_inf <= 1; the block linear flow dU/dt = B U of eq. eqB,
 *              B = [[0, A0], [-A0, 0]], from U(0) = (0; I) over [0, 1] (so U(1) = (sin A0; cos A0)),
 *              held as the second block column of an order-2n exponential-flow state
 *              (X(0) = diag(0, I)) and solved by the plan's method, schemes and dtypes; then
 *              C <- 2 C^2 - I, m times, in float64.  T must be 1; fine scheme RK4 or explicit
 *              Euler, forward-Euler G; fa_parareal_solve(_host) are its only compute calls. */
typedef enum { FA_FLOW_INV = 0, FA_FLOW_EXP = 1, FA_FLOW_SQRT = 2, FA_FLOW_COS = 3 } fa_flow;

/* Arithmetic of the fine and coarse propagators' matrix products.
 * FA_F64     float64 everywhere (SIMT FMA).
 * FA_BF16    one BF16 product per GEMM (operands rounded to BF16).
 * FA_BF16X3  operands split into BF16 terms x = x0 + x1 (+ ...); products
 *            x0y0 + x0y1 + x1y0.
 * FA_BF16X4  products x0y0 + x0y1 + x1y0 + x2y0 (left operand to three terms).
 * FA_BF16X6  every product xa yb with a + b <= 2.
 * All BF16 forms accumulate in float32 on the tensor cores (tcgen05); the multi-term forms
 * drain the main product x0y0 into float32 registers every 64-wide k-block (the accumulator
 * truncates), FA_BF16 keeps it in the accumulator over the whole k extent (its own rounding,
 * 2^-9, is far above that truncation: about 4e-6 relative at k = 4096).
 * FA_FP8E4M3 (fine propagator of the square-root flow only) the RK4 stage operands as E4M3 with
 *            one float32 scale per 128 x 128 tile (delayed scaling: 448 / (2 amax) of the same
 *            tile one stage earlier, saturating conversion), float32 accumulation per 128-wide
 *            k-block, rescaled by the two operand tiles' scales; the coarse propagator then runs
 *            in float64 or a BF16 form (coarse_dtype). */
typedef enum {
  FA_F64 = 0,
  FA_BF16 = 1,
  FA_BF16X3 = 2,
  FA_BF16X4 = 3,
  FA_BF16X6 = 4,
  FA_FP8E4M3 = 5
} fa_dtype;

typedef struct {
  int n;              /* matrix order, 1 <= n <= 16384 */
  int flow;           /* fa_flow */
  double T;           /* horizon, > 0 (Examples 1 and 2 use T = 1) */
  int N;              /* number of time slices, >= 1 */
  int coarse_steps;   /* m: forward-Euler substeps of G per slice, >= 1 */
  int fine_steps;     /* J: RK4 steps of F per slice, >= 1 */
  int max_iters;      /* K: maximum parareal iterations (fine sweeps after Step 0), >= 0 */
  double tol;         /* stop when max_n ||dU_n||_F / ||U_n||_F < tol (0 = run all K) */
  int fine_dtype;     /* fa_dtype of F */
  int coarse_dtype;   /* fa_dtype of G (FA_F64, or the same BF16 form as F; any BF16 form when F
                         is FA_FP8E4M3) */
  int refine_steps;   /* refinement steps on the result (inverse: float64 Newton-Schulz; square
                         root: Newton with the Sylvester equation, see fa_refine); 0 = none */
  int coarse_kind;    /* fa_coarse_kind of G (FA_COARSE_EULER = the paper's forward Euler) */
  int method;         /* fa_method (FA_METHOD_CLASSICAL = Algorithm 1) */
  double span_drop;   /* FA_METHOD_MODIFIED: a block joins the space when its norm after the
                         Gram-Schmidt sweeps exceeds span_drop times its norm (0 = the default:
                         1e-12 for float64 F, 1e-7 for the BF16 forms) */
  int max_basis;      /* FA_METHOD_MODIFIED: capacity of the space in blocks, <= 4096 (0 = the
                         default (N + 1) min(max_iters, 3)); blocks beyond it are left to G.
                         The workspace holds two float64 n x n matrices per block. */
  int fine_scheme;    /* fa_scheme of F's fine_steps steps per slice (0 = classical RK4) */
  int coarse_scheme;  /* fa_scheme of G's coarse_steps steps per slice (0 = forward Euler) */
} fa_problem_desc;

/* Time-stepping schemes of the propagators (Section 2: "any time marching scheme"; its
 * Examples 1 and 2 use explicit Euler and Crank-Nicolson propagators).
 * FA_SCHEME_DEFAULT  classical RK4 for F, forward Euler for G.
 * FA_SCHEME_RK4      classical RK4 (F only).
 * FA_SCHEME_EULER    explicit (forward) Euler, X <- X + h Fl(X).
 * FA_SCHEME_CN       Crank-Nicolson, exponential flow only: (I - h/2 A) X' = (I + h/2 A) X,
 *                    applied as X' = X + h M X with M = (I - h/2 A)^{-1} A formed once per
 *                    matrix by a float64 Gauss-Jordan solve on the GPU. */
typedef enum {
  FA_SCHEME_DEFAULT = 0,
  FA_SCHEME_RK4 = 1,
  FA_SCHEME_EULER = 2,
  FA_SCHEME_CN = 3
} fa_scheme;

/* Parareal method.
 * FA_METHOD_CLASSICAL  Algorithm 1 (Section 2).
 * FA_METHOD_MODIFIED   Algorithm 3 (Section 3), for linear homogeneous flows (the exponential
 *                      flow): every iteration enlarges a space S^k = Span(S^{k-1}, U^k_0 .. U^k_N)
 *                      with globalQR (Algorithm 2: Gram-Schmidt in the Frobenius inner product,
 *                      here two sweeps per block, a block removed when its reduced norm is below
 *                      span_drop times its norm), runs F on the new basis blocks only (all of
 *                      them at once, in the fine sweep's arithmetic), and updates sequentially
 *                      U_{n+1} = sum_i alpha_i F(Q_i) + G(U_n - sum_i alpha_i Q_i),
 *                      alpha_i = <U_n, Q_i>_F (F is linear, so the first term is F(P U_n)).  The
 *                      basis, its fine images and the update are float64. */
typedef enum { FA_METHOD_CLASSICAL = 0, FA_METHOD_MODIFIED = 1 } fa_method;

typedef struct {
  int iters;           /* fine sweeps performed */
  int converged;       /* 1 if the tolerance was reached */
  double last_dx;      /* max_n ||dU_n||_F / ||U_n||_F of the last iteration */
  double t_init_ms;    /* matrix set-up + Step 0 */
  double t_fine_ms;    /* all fine sweeps */
  double t_coarse_ms;  /* all coarse sweeps (with correction and norms) */
  double t_refine_ms;  /* refinement */
  double *dx_history;  /* caller-owned host array of max_iters doubles, or NULL */
  int g_fallback_iter; /* learned G: the iteration after which G was switched to forward Euler
                          because the convergence measure grew (0 = never) */
  int coef_fallbacks;  /* learned G: coarse steps whose network output was not finite (Euler used) */
  int records;         /* pair records written by the recorder (fa_plan_set_recorder) */
  int basis_dim;       /* FA_METHOD_MODIFIED: blocks in the final space */
  int double_angle_steps; /* FA_FLOW_COS: m of Algorithm 5 */
  int fine_blocks;     /* matrices propagated by F in all (classical: iterations x N) */
} fa_report;

/* Coarse propagator G.
 * FA_COARSE_EULER    m forward-Euler substeps per slice (Section 2, Example 1).
 * FA_COARSE_LEARNED  the learned polynomial step (below; not part of the paper's method):
 *                    G(X) = X + sum_{j=1..4} c_j dT^j X_[j], X_[j] the j-th Taylor coefficient
 *                    of the flow through X, c from a small network of cheap features of X.
 *                    Needs coarse_steps = 1 and the inverse or exponential flow. */
typedef enum { FA_COARSE_EULER = 0, FA_COARSE_LEARNED = 1 } fa_coarse_kind;

typedef struct fa_plan_s *fa_plan_t;

/* Create a plan for one problem shape.  Validates the descriptor (FA_ERR_ARG
 * on n < 1, N < 1, J < 1, m < 1, T <= 0, K < 0, unknown flow or dtype) and
 * checks that the current device is sm_103 (FA_ERR_UNSUPPORTED otherwise).
 * `stream` is a cudaStream_t (NULL = legacy default stream).  On success
 * *out receives the plan and *workspace_bytes the device workspace size the
 * plan needs; bind it before any compute call.  No device memory is
 * allocated. */
fa_status fa_plan(fa_plan_t *out, const fa_problem_desc *d, void *stream,
                  size_t *workspace_bytes);

/* Bind caller-allocated device memory (>= the size fa_plan returned, 256-byte
 * aligned) as the plan's workspace.  The memory must stay valid until the plan
 * is destroyed or another workspace is bound.  FA_ERR_WORKSPACE if too small
 * or misaligned. */
fa_status fa_plan_bind_workspace(fa_plan_t p, void *d_workspace, size_t bytes);

/* Load A (device, n x n row-major float64) into the plan: builds the operand
 * forms the propagators use (BF16 terms of A or of I - A, transposes).  Must
 * precede fa_fine_sweep / fa_coarse_sweep / fa_refine; fa_parareal_solve
 * calls it itself.  A may be freed afterwards. */
fa_status fa_plan_set_matrix(fa_plan_t p, const double *dA);

/* Fine propagator on every slice at once (the parallel step of Algorithm 1):
 * dF[b] = F(T_{b+1}, T_b, dU[b]) for b = 0..N-1, i.e. J RK4 steps of size
 * T/(N J) from dU[b].  dU and dF are [N][n][n] float64 device arrays; they
 * must not overlap. */
fa_status fa_fine_sweep(fa_plan_t p, const double *dU, double *dF);

/* Coarse sweep with correction (the sequential part of Algorithm 1):
 *   V_0 = dU0;  for n = 0..N-1:  G_n = G(V_n),  V_{n+1} = G_n + D_n,
 * with D_n = dD[n] (pass dD = NULL for Step 0, eq. eqStep0: V_{n+1} = G_n).
 * Writes dUnew[0..N] = V ([N+1][n][n]) and dGnew[0..N-1] = G_n ([N][n][n]).
 * If dNorms is not NULL, dUold ([N+1][n][n], the previous iterate; it may be
 * the same array as dUnew, read before overwritten) must be given and
 * dNorms[2n], dNorms[2n+1] (float64, device, [N][2]) receive
 * ||V_{n+1} - Uold_{n+1}||_F^2 and ||V_{n+1}||_F^2, summed in a fixed order
 * (bitwise reproducible; in the mixed forms each 32-column run of a row in
 * float32, the rest in float64). */
fa_status fa_coarse_sweep(fa_plan_t p, const double *dU0, const double *dD,
                          double *dUnew, double *dGnew, double *dNorms,
                          const double *dUold);

/* Refinement of dX in place, `refine_steps` steps (not part of the paper's method; the
 * mixed-precision forms use it to reach float64-level accuracy):
 *   inverse flow      Newton-Schulz X <- X (2I - A X), float64 products;
 *   square-root flow  Newton X <- sym(X) + E with X E + E X = A - X^2: R = A - X^2 in float64,
 *                     the Sylvester equation solved through the matrix sign function,
 *                     sign([[X, R], [0, -X]] / mu) = [[I, 2E], [0, -I]] (Roberts 1980, mu the
 *                     largest eigenvalue of X from a power iteration), by Newton-Schulz sign
 *                     steps with BF16x6 term products on the tensor cores, stopped two steps
 *                     after ||I - P^2||_F / sqrt(n) < 1e-6 (at most 60 steps).  Needs an SPD
 *                     A and an X near A^{1/2}; FA_ERR_NONFINITE if the iteration diverges.
 * FA_ERR_UNSUPPORTED for the exponential flow.  Synchronises the plan's stream (the sign
 * iteration reads its stopping measure every step). */
fa_status fa_refine(fa_plan_t p, double *dX);

/* Whole solve on device buffers: set A, Step 0, up to max_iters parareal
 * iterations, optional refinement; dXout (n x n) receives U_N.  dX0 = NULL
 * means X0 = I.  Returns FA_ERR_NOT_CONVERGED (with dXout written) when the
 * tolerance was not met.  `report` may be NULL. */
fa_status fa_parareal_solve(fa_plan_t p, const double *dA, const double *dX0,
                            double *dXout, fa_report *report);

/* The same solve on HOST buffers (pageable or pinned): copies hA (and hX0)
 * into the workspace, solves, and copies U_N back into hXout. */
fa_status fa_parareal_solve_host(fa_plan_t p, const double *hA, const double *hX0,
                                 double *hXout, fa_report *report);

/* Diagnostic: one matrix product dC = dL * dR (n x n, device, row-major
 * float64) through the plan's coarse arithmetic (the BF16 term products on
 * the tensor cores for FA_BF16* coarse dtypes, float64 otherwise), without
 * any epilogue arithmetic.  Mixed forms need a flow with an L-form operand
 * buffer (FA_FLOW_INV or FA_FLOW_SQRT); FA_ERR_UNSUPPORTED otherwise. */
fa_status fa_debug_product(fa_plan_t p, const double *dL, const double *dR, double *dC);

/* Allocation-free product dC = dL * dR for callers that cannot allocate device memory
 * (their device memory is budgeted before start-up, or they hold only their inputs and
 * outputs and cannot own a workspace).  The paper has no counterpart; this is a convenience
 * of the library.  dL, dR, dC: n x n row-major float64 device arrays, 1 <= n <= 1024;
 * dtype one of FA_BF16* (the tensor-core term products of the planned path, float32
 * accumulation as described for the dtypes above).  The BF16 operand terms
 * live in a fixed array inside the library (about 12 MB per GPU that loads it, held until
 * process exit); no cudaMalloc, cudaFree or allocating library call is made.  The first call
 * on a device looks the array up (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Calls share the array: calls that overlap on the GPU
 * (other streams, other host threads) race.  FA_ERR_ARG for n outside [1, 1024], a non-BF16
 * dtype or null pointers; FA_ERR_UNSUPPORTED on a device other than sm_103.  Asynchronous on
 * `stream` (a cudaStream_t, NULL = legacy default stream): the status covers the arguments and
 * the launches only.  A device-side wait of the product kernel that gives up (the bounded waits
 * that FA_ERR_TIMEOUT reports for planned calls) is not reported by this call; dC is then
 * partly written. */
fa_status fa_product_noalloc(int n, int dtype, const double *dL, const double *dR, double *dC,
                             void *stream);

/* Diagnostic: when d_counters (device, >= 16 unsigned 64-bit words, zeroed by the
 * caller) is not NULL, later tensor-core launches add per-role cycle counts to it:
 * [0] producer waiting for free slots, [1] MMA waiting for operand tiles, [2] MMA
 * waiting for a free main chunk, [3] MMA waiting for the correction buffer,
 * [4] drain waiting for a main chunk, [5] drain waiting for corrections, [6] drain
 * waiting for the finished-tile buffer, [7] epilogue waiting for a finished tile,
 * [8] epilogue busy, [9] drain busy, [10] kernel cycles per CTA, [11] tiles.
 * NULL switches it off. */
fa_status fa_debug_set_profile(unsigned long long *d_counters);

/* Diagnostic of the failure detection: later tensor-core launches (process-wide) give up any
 * device-side wait after `wait_cycles` SM cycles (0 = the default, about 2 s), and, when
 * skip_loads_cta >= 0, that CTA of each launch issues no operand loads, so its waits run out:
 * the kernel raises its abort flag, records FA_ERR_TIMEOUT in the plan's error word (reported
 * by the next synchronising call), waits briefly, releases its tensor memory and returns; no
 * copy is left in flight.  The other CTAs finish their tiles, so the output is partly written.
 * (0, -1) restores normal operation.  FA_ERR_ARG for wait_cycles < 0. */
fa_status fa_debug_set_wait_fault(long long wait_cycles, int skip_loads_cta);

/* ---- Batches: many independent problems of mixed order and flow -------------------------
 *
 * Every RK4 stage and every coarse step of all problems runs as one persistent tensor-core
 * launch over the union of their tiles (a ragged work list: each problem keeps its own order,
 * operands and epilogue); from the second iteration on, one parareal iteration of the whole
 * batch is replayed as a CUDA graph.  Problem i solves flow flows[i] on an ns[i] x ns[i]
 * matrix to horizon Ts[i] with coarse_steps[i] Euler substeps per slice; all share N,
 * fine_steps, max_iters, tol and the BF16 form `dtype`.  Convergence is per problem (its
 * own max_n ||dU_n||_F / ||U_n||_F); the batch iterates until every problem converged or
 * max_iters.  Same conventions as single plans: the caller binds one workspace. */
typedef struct fa_batch_s *fa_batch_t;

fa_status fa_batch_plan(fa_batch_t *out, int count, const int *ns, const int *flows,
                        const double *Ts, const int *coarse_steps, int N, int fine_steps,
                        int max_iters, double tol, int dtype, void *stream,
                        size_t *workspace_bytes);
fa_status fa_batch_bind_workspace(fa_batch_t b, void *d_workspace, size_t bytes);
/* dA[i] / dXout[i]: device pointers (host array of `count`), row-major float64 n_i x n_i.
 * A problem that meets tol leaves the batch: dXout[i] receives its U_N of that iteration, and
 * later launches no longer contain its tiles (the segment tables are rebuilt and the iteration
 * graph captured again), so each problem runs exactly the iterations a single solve of it runs.
 * iters[i] (host, optional): iteration at which problem i met tol (or the count run);
 * last_dx[i] (host, optional): its convergence measure at that iteration.  Returns
 * FA_ERR_NOT_CONVERGED (outputs written) if some problem missed tol. */
fa_status fa_batch_solve(fa_batch_t b, const double *const *dA, double *const *dXout, int *iters,
                         double *last_dx);
fa_status fa_batch_destroy(fa_batch_t b);

/* Autotune a batch's launch schedule (not part of the paper's method).  Knobs: per size bucket
 * of n (<= 64, 128, 256, 512, 1024, larger), whether the epilogue prefetches its tile's state
 * into L2 while the tile's products run, and the tile order inside a slice (M-tile or N-tile
 * fastest); per launch, the order of the problems in the ragged tile list (as given, or largest
 * n first).  Coordinate descent from the defaults, timing the batch's own fine-sweep stage
 * launch (CUDA events, 3 repetitions) on the matrices dA; a change is kept when it saves more
 * than 1 %.  None of the knobs changes any result bit (each tile's arithmetic and the order of
 * every reduction are fixed).  If `cache_path` names a file holding an entry for this batch
 * (its count, N, J, dtype and a signature of the problems' n, flow, T and m), that schedule is
 * used without timing; otherwise the tuned schedule is appended to the file.  NULL: no file.
 * Synchronises the batch's stream.  Call after fa_batch_bind_workspace (which resets the
 * schedule to the defaults). */
fa_status fa_batch_autotune(fa_batch_t b, const double *const *dA, const char *cache_path);
/* One-line account of the last fa_batch_autotune (choices and timings); "" before one. */
const char *fa_batch_tuning(fa_batch_t b);

/* The same for one plan: times its fine-sweep stage product(s) with each combination of the
 * epilogue prefetch and the tile order (the plan's matrix must be set) and keeps the fastest
 * (more than 1 % better than the first) for all its tensor-core launches.  No-op for float64
 * plans.  Results do not change.  fa_plan_tuning returns the account. */
fa_status fa_plan_autotune(fa_plan_t p);
const char *fa_plan_tuning(fa_plan_t p);

/* ---- Learned coarse propagator ----------------------------------------------------------
 *
 * Not part of the paper's method: a coarse propagator whose coefficients are learned from
 * fine-propagator trajectories.  For a state X at slice n (time T_n = n dT, dT = T / N):
 *
 *   Taylor terms  inverse flow:     X_[j] = X (B X)^j, B = I - A (the one-slice map is the
 *                                   Neumann series X (I - dT B X)^{-1});
 *                 exponential flow: X_[j] = A^j X / j!;
 *   features      f = [T_n / T, dT, Gershgorin lower and upper bounds of A,
 *                      h(A) / n, h(X) / n, ||Fl(X)||_F / sqrt(n), ||X||_F / sqrt(n)],
 *                 h(Y) = (1/8) sum_k z_k^T Y z_k (Hutchinson) over the Rademacher probes
 *                 z_k[j] = -1 if bit 63 of SplitMix64 output k n + j (seed FA_PROBE_SEED;
 *                 output c is mix(seed + (c + 1) 0x9E3779B97F4A7C15), Steele, Lea and Flood
 *                 2014) is set, else +1;
 *   network       c = W3 g(W2 g(W1 x + b1) + b2) + b3, x = (f - mu) / sd, g = GELU (exact,
 *                 x Phi(x)); W1: 128 x 8, W2: 128 x 128, W3: 4 x 128 used as BF16 (rounded to
 *                 nearest even from the float32 blob), everything else float32; float32
 *                 activations and accumulation;
 *   update        G(X) = X + sum_j c_j dT^j X_[j]; c = (1, 0, 0, 0) is forward Euler.
 *
 * Fallbacks to forward Euler: a slice whose c is not finite uses (1, 0, 0, 0)
 * (report.coef_fallbacks); if the convergence measure grows from one iteration to the next,
 * the rest of the solve uses Euler G (G of the current iterate is recomputed with Euler so that
 * the correction stays consistent; report.g_fallback_iter).
 *
 * Parameter blob: FA_MLP_PARAMS float32 values, in order mu[8], sd[8], W1[128][8], b1[128],
 * W2[128][128], b2[128], W3[4][128], b3[4] (row-major; W maps inputs to outputs as W x).
 *
 * Pair record (training data for the pair (X, Y = F(X)), FA_RECORD_DOUBLES float64 values):
 * [0..7] the features of X; [8..23] M (4 x 4 row-major), M_ab = <Z_a, Z_b>_F; [24..27]
 * v_a = <Z_a, D>_F; [28] dd = ||D||_F^2; [29..31] zero; with Z_a = dT^a X_[a], D = Y - X.  The
 * relative residual ||sum_a c_a Z_a - D||^2 / ||D||^2 = (c^T M c - 2 c^T v + dd) / dd is the
 * training loss of the pair. */
#define FA_MLP_FEATURES 8
#define FA_MLP_HIDDEN 128
#define FA_MLP_COEFS 4
#define FA_MLP_PARAMS 18196
#define FA_RECORD_DOUBLES 32
#define FA_PROBES 8
#define FA_PROBE_SEED 0x150507959ULL

/* Copy the network blob (device, FA_MLP_PARAMS float32) into the plan (asynchronous).  The plan
 * must have coarse_kind = FA_COARSE_LEARNED (FA_ERR_ARG otherwise); solves and coarse sweeps
 * of such a plan fail with FA_ERR_ARG until this has been called. */
fa_status fa_plan_set_learned(fa_plan_t p, const float *d_params);

/* Opt-in third fallback to Euler (off by default): with enable != 0, fa_parareal_solve on this
 * learned plan first runs Step 0 and one iteration with Euler G in the solve's own buffers (one
 * extra fine sweep, counted in report.t_init_ms), then the learned solve; if the learned solve's
 * first convergence measure exceeds Euler's, the rest of it uses Euler G (report.g_fallback_iter
 * = 1).  The first measure mixes the coarse trajectory's error into the comparison, so a G that
 * converges faster can still trip it: on the wide inverse family at n = 64, N = 8 the Taylor-4
 * step's first measure is 0.4458 against Euler's 0.4444.  FA_ERR_ARG unless the plan has
 * coarse_kind = FA_COARSE_LEARNED. */
fa_status fa_plan_set_learned_check(fa_plan_t p, int enable);

/* Coefficients c (device float32 [N][4]) that the plan's last coarse sweep used, per slice. */
fa_status fa_plan_learned_coefs(fa_plan_t p, float *d_coef);

/* Device scratch (bytes) that fa_learned_records and the recorder need for this plan: four
 * [N][n][n] float64 arrays plus the stats partials. */
fa_status fa_learned_records_scratch(fa_plan_t p, size_t *bytes);

/* Pair records of (dU[b], dF[b]) for b = 0..N-1 (device [N][n][n] float64; dF[b] is meant to be
 * F(dU[b]) from fa_fine_sweep) into d_records (device [N][FA_RECORD_DOUBLES]), feature time
 * T_b / T = b / N.  The Taylor terms are computed in the plan's fine arithmetic (BF16 term
 * products on the tensor cores for FA_BF16* fine dtypes, float64 otherwise); the plan's
 * matrix must be set.  FA_ERR_UNSUPPORTED for the square-root flow. */
fa_status fa_learned_records(fa_plan_t p, const double *dU, const double *dF, double *d_records,
                             void *d_scratch, size_t scratch_bytes);

/* Record training pairs during fa_parareal_solve: after every fine sweep, the records of
 * (U^k_n, F(U^k_n)) for n = 0..N-1 are appended to d_records (device, capacity_pairs records)
 * while they fit; report.records counts them.  d_scratch as for fa_learned_records.
 * d_records = NULL switches recording off. */
fa_status fa_plan_set_recorder(fa_plan_t p, double *d_records, int capacity_pairs,
                               void *d_scratch, size_t scratch_bytes);

/* Network forward pass: d_coef[b][0..3] (device float32) for `batch` feature rows d_feat
 * (device float64, row b at d_feat + b * feat_stride; feat_stride >= 8, e.g. FA_RECORD_DOUBLES
 * to read the features of records).  Non-finite outputs are replaced by (1, 0, 0, 0). */
fa_status fa_mlp_forward(const float *d_params, int batch, const double *d_feat, int feat_stride,
                         float *d_coef, void *stream);

/* Device scratch (bytes) of fa_mlp_loss_grad for a batch. */
fa_status fa_mlp_scratch_bytes(int batch, size_t *bytes);

/* Mean loss over `batch` pair records (device float64 [batch][FA_RECORD_DOUBLES]) into *d_loss
 * (device float64) and its gradient with respect to the blob into d_grad (device float32
 * [FA_MLP_PARAMS]; zero for mu and sd), taken at the BF16 weight values the network uses.  The
 * batch sums of the weight gradients are formed in float64 in sample order (bitwise
 * reproducible). */
fa_status fa_mlp_loss_grad(const float *d_params, int batch, const double *d_records,
                           float *d_grad, double *d_loss, void *d_scratch, size_t scratch_bytes,
                           void *stream);

/* One Adam step (Kingma and Ba 2015) on W1..b3 of the blob (mu and sd unchanged), float32:
 * m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2; p -= lr (m / (1 - b1^t)) /
 * (sqrt(v / (1 - b2^t)) + eps).  d_m, d_v: device float32 [FA_MLP_PARAMS], zero before step 1;
 * `step` = t >= 1. */
fa_status fa_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int step,
                      float lr, float beta1, float beta2, float eps, void *stream);

/* ---- Accelerated inverse-matrix approximation (Algorithm 8, Section 4) ------------------
 *
 * The steady state of dX/dt = I - A X is A^{-1} (e.g. for SPD A); Section 4 accelerates its
 * explicit time marching with a control u that starts at e = X~ - X0 (X~ an approximation of
 * A^{-1}, from a preconditioner) and decays as u' = -A u:
 *     X^(k+1) = X^(k) + dt (I - A X^(k) + u^(k)),   u^(k+1) = (I - dt A) u^(k).
 * Each step is one product A [X | u] (two slices sharing the left factor A) whose epilogue
 * writes both updates and the residual ||I - A X^(k)||_F.
 *
 * fa_aima_plan: a plan for order n with products in `dtype` (FA_F64 or a BF16 form; the state
 * stays float64); bind its workspace with fa_plan_bind_workspace.
 * fa_aima: `steps` iterations from dX0 with the initial error dE (device n x n float64
 * row-major); dXout receives X^(steps); h_res (host, steps + 1 doubles, or NULL) receives
 * ||I - A X^(k)||_F for k = 0..steps.  FA_ERR_ARG for dt <= 0, steps < 0 or steps >= n^2, or a
 * plan not made by fa_aima_plan.  Synchronises the plan's stream. */
fa_status fa_aima_plan(fa_plan_t *out, int n, int dtype, void *stream, size_t *workspace_bytes);
fa_status fa_aima(fa_plan_t p, const double *dA, const double *dX0, const double *dE, double dt,
                  int steps, double *dXout, double *h_res);

/* Release the plan (not the workspace, which the caller owns). */
fa_status fa_plan_destroy(fa_plan_t p);

/* Static description of a status code. */
const char *fa_status_string(fa_status s);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *fa_last_error(void);

/* Number of kernels the library launched on this thread since the last reset
 * (diagnostics for launch counting); fa_launch_count_reset sets it to 0. */
unsigned long long fa_launch_count(void);
void fa_launch_count_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* FA_H */
