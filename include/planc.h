/*
 * planc.h -- C ABI of libplanc.so, a GB300 (sm_103a) implementation of the
 * hot path of alternating-update non-negative CP decomposition (NNCP) as
 * described in "PLANC: Parallel Low-rank Approximation with Non-negativity
 * Constraints" (arXiv 1909.01149).
 *
 * The problem (Eq. nncp):  min_{H^(n) >= 0} || X - sum_r H^(1)(:,r) o ... o
 * H^(N)(:,r) ||^2, solved by the alternating updates of Alg. 1 with the
 * normalisation and error computation of Alg. 4.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns a planc_status_t; nothing throws or aborts across the
 *    ABI.  On failure planc_last_error(ctx) holds a one-line message.
 *  - X is an I_1 x ... x I_N dense tensor stored linearly with mode 1
 *    fastest (the paper's "natural mode-descending" order, Sec. 4.1.2).
 *    It lives in device memory, is BORROWED by planc_init and must stay
 *    alive and unchanged until planc_destroy.
 *  - A factor matrix H^(n) is I_n x R, ROW-MAJOR (the R entries of a row are
 *    contiguous), in device memory, of the context's factor dtype (F64 when X
 *    is F64, else F32).  "void* const* H" is a HOST array of N device
 *    pointers, one per mode.
 *  - MTTKRP results M^(n) have the same layout as H^(n).
 *  - Gram matrices G^(n) = H^(n)^T H^(n) and S^(n) are R x R row-major
 *    double (FP64) in device memory; "G" arrays hold N of them back to back.
 *  - lambda is a length-R double vector.
 *  - All device buffers passed in are caller-owned; the library owns only
 *    its workspace (partial-MTTKRP temporaries, split-K partials, reduction
 *    scratch), allocated in planc_init and freed in planc_destroy.
 *  - Calls are asynchronous on the context's CUDA stream, except those that
 *    return host scalars (planc_fit, planc_nncp_solve, planc_cp_grad), which
 *    synchronise that stream before returning.
 *  - Modes are 0-based at the ABI (mode n = paper's mode n+1).
 */
#ifndef PLANC_H
#define PLANC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PLANC_OK = 0,
  PLANC_E_INVALID = 1,        /* bad argument (NULL pointer, out-of-range n) */
  PLANC_E_SHAPE = 2,          /* N < 2, R < 1, a dimension < 1, size overflow */
  PLANC_E_DTYPE = 3,          /* unsupported dtype combination */
  PLANC_E_NOMEM = 4,          /* workspace allocation failed */
  PLANC_E_CUDA = 5,           /* a CUDA runtime/driver call failed */
  PLANC_E_NUMERIC = 6,        /* non-finite value or a non-positive pivot */
  PLANC_E_NOT_CONVERGED = 7,  /* reserved: NNLS caps are reported, not errors */
  PLANC_E_TIMEOUT = 8,        /* a bounded device-side wait gave up */
  PLANC_E_UNSUPPORTED = 9     /* valid request this build does not implement */
} planc_status_t;

typedef enum { PLANC_F64 = 0, PLANC_F32 = 1, PLANC_BF16 = 2, PLANC_F16 = 3 } planc_dtype_t;

/* NNLS-Update choices of Sec. 4.3 (MU, HALS, BPP, ADMM, NES) plus projected
 * gradient (PGD), the project's gradient-driven option, and UCP, the
 * unconstrained update of Sec. 6 (CP-ALS: H S = M solved exactly, no
 * non-negativity; a non-positive pivot while inverting S, i.e. S not
 * positive definite, reports PLANC_E_NUMERIC at the end of a solve).
 * NES is the Nesterov-type update of Sec. 4.3.5 (Eq. nesnls, Eq.
 * nesinnerupd): accelerated projected gradient on the proximal problem
 * 1/2 tr(H S H^T) - tr(M^T H) + lam_p/2 ||H - H*||^2 (H* the warm start),
 * with lam_p, the step 1/L and the momentum beta taken from the extreme
 * eigenvalues mu0, L0 of S: lam_p = max(0, (L0 - 100 mu0) / 99) (condition
 * number at most 100), L = L0 + lam_p, beta = (1 - sqrt(q)) / (1 + sqrt(q)),
 * q = (mu0 + lam_p) / L; it stops after the step where
 * max|X_{k+1} - Y_k| <= nes_tol max|X_{k+1}| over the whole factor, or after
 * nes_max_inner steps.  In planc_nncp_solve it adds the outer acceleration
 * of Eq. nesouterupd (see planc_solve_opts.nes_accel). */
typedef enum {
  PLANC_MU = 0, PLANC_HALS = 1, PLANC_BPP = 2, PLANC_ADMM = 3, PLANC_PGD = 4, PLANC_UCP = 5,
  PLANC_NES = 6
} planc_nls_t;

/* Tuning of the NNLS updates; planc_nls_opts_default() fills the values the
 * library's readings of Sec. 4.3 use. */
typedef struct {
  double mu_eps;        /* MU denominator guard (Eq. muupd): 1e-16 */
  int admm_max_inner;   /* ADMM inner steps cap (Sec. 4.3.4): 5 */
  double admm_tol;      /* ADMM primal/dual stopping ratio: 1e-2 */
  int bpp_max_iter;     /* BPP exchange cap; <= 0 means 10 * R */
  int pgd_steps;        /* projected-gradient steps per update: 1 */
  int nes_max_inner;    /* Nesterov inner steps cap (Sec. 4.3.5): 20, <= 64 */
  double nes_tol;       /* Nesterov stopping ratio: 1e-3 */
} planc_nls_opts;

/* Options of planc_nncp_solve. */
typedef struct {
  planc_nls_t alg;      /* NNLS-Update of Alg. 1 */
  int iters;            /* outer iterations to run (Sec. 6.1.2: fixed count) */
  double tol;           /* stop when rel. error <= tol; <= 0 runs all iters */
  planc_nls_opts nls;
  int use_graph;        /* 1: replay each outer iteration as a CUDA graph */
  int profile;          /* 1: time the partial-MTTKRP launches with events */
  int nes_accel;        /* alg NES: 1 (default) adds the outer acceleration of
                           Eq. nesouterupd after every outer iteration i >= 2:
                           F_new = [F_i + s_i (F_i - F_{i-1})]_+ for every
                           factor (lambda absorbed into the last mode),
                           s_i = i^(1/N), accepted iff its relative error
                           (one extra MTTKRP) is lower than iteration i's */
  int batch_persistent; /* planc_batch_solve only: 1 (default) runs the whole
                           solve as one persistent launch; 0 as one launch per
                           phase over all instances */
} planc_solve_opts;

/* Result record of planc_nncp_solve (host memory). */
typedef struct {
  int iters_done;
  double rel_err;       /* eps of the last outer iteration (Alg. 4) */
  double fit;           /* 1 - eps */
  double* rel_err_hist; /* optional host array, length >= opts.iters */
  int32_t* inner_hist;  /* optional host array, length >= opts.iters * N:
                           inner steps per NNLS call (ADMM or NES steps, max
                           BPP exchanges over rows, pgd_steps for PGD, 1 for
                           MU/HALS/UCP) */
  int bpp_unconverged;  /* rows whose BPP hit the exchange cap (summed) */
  float pm_ms;          /* profile: summed time of the partial MTTKRPs */
  int pm_launches;      /* profile: number of partial-MTTKRP launches timed */
  long long launches;   /* kernels this call launched (graph replays included) */
  int pm_tensor_cores;  /* bit 0 / bit 1: left / right partial MTTKRP ran on
                           the tcgen05 tensor-core path */
  int32_t* accel_hist;  /* optional host array, length >= opts.iters: 1 where
                           the outer acceleration was accepted (NES) */
  int accel_accepted;   /* number of accepted outer accelerations */
} planc_report;

typedef struct planc_ctx* planc_t;

/* ---- status and defaults ------------------------------------------------ */

/* Static string naming a status code. */
const char* planc_status_str(planc_status_t s);

/* Last error message of ctx (empty string if none); valid until the next
 * call on ctx.  planc_last_error(NULL) returns the last error of a failed
 * planc_init on the calling thread. */
const char* planc_last_error(planc_t ctx);

/* Default NNLS options (see planc_nls_opts). Never fails. */
planc_nls_opts planc_nls_opts_default(void);

/* Root split S of the dimension tree (Sec. 4.2.2) for dims[0..N-1], returned
 * 1-based in *split (1 <= S < N): the contiguous split whose two mode
 * products are nearest (minimal |log(prod_{k<S} I_k / prod_{k>=S} I_k)|),
 * ties to the larger S.  Host-only.  PLANC_E_SHAPE on N < 2 or dims < 1. */
planc_status_t planc_plan_split(int N, const int64_t* dims, int* split);

/* ---- context ------------------------------------------------------------ */

/* Create a context for the tensor X (Alg. 1 "Require").
 *   N, dims      order and mode sizes (2 <= N <= 16, dims[n] >= 1, prod < 2^40)
 *   R            CP rank (1 <= R <= 256)
 *   x_dtype, X   storage type and device pointer of X (borrowed, see above);
 *                F32/BF16/F16 data are accumulated in FP32, F64 in FP64
 *   f_dtype      factor dtype: F64 iff x_dtype is F64, else F32
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream)
 *   split        root split S, 1-based; -1 chooses planc_plan_split's S
 * The partial MTTKRPs run on the tcgen05 tensor cores when the shape allows
 * (BF16 or FP32 X, R <= 64, TMA-compatible strides, X 16-byte aligned; the
 * resident-operand kernel when its factor image fits in shared memory, the
 * streamed-operand kernel otherwise; BF16 X with R <= 32 and FP16 X with
 * R <= 32 as one GEMM against the split Khatri-Rao image, which needs the
 * row stride of X_(1:S) a multiple of 16 bytes) and on the CUDA-core
 * kernels otherwise (planc_pm_tensor_cores reports which).  PLANC_PM_KRP=0
 * (read at context creation and at each launch) turns the Khatri-Rao GEMM
 * form off (BF16 then uses the weighted-row kernels, FP16 the CUDA cores).
 * Environment switches: PLANC_PM_PATH=simt (read here) forces the CUDA-core
 * partial MTTKRPs; PLANC_FUSED_MODES=0 (read here) keeps the per-mode update
 * on the multi-launch path; PLANC_TC_STREAMED_KRP (set; read at each launch)
 * forces the streamed-operand tensor-core kernel; PLANC_PDL=0 (read once per
 * process) launches without programmatic dependent launch.  They select
 * among equivalent paths for tests and measurements; results agree within
 * the stated tolerances.
 * Allocates the workspace (dimension-tree temporaries, split-K partials,
 * reduction scratch).  Errors: PLANC_E_SHAPE, PLANC_E_DTYPE, PLANC_E_INVALID,
 * PLANC_E_NOMEM, PLANC_E_CUDA (no device / not sm_103). */
planc_status_t planc_init(planc_t* out, int N, const int64_t* dims, int R,
                          planc_dtype_t x_dtype, const void* X,
                          planc_dtype_t f_dtype, void* cuda_stream, int split);

/* Free the workspace and the context (NULL is a no-op). */
planc_status_t planc_destroy(planc_t ctx);

/* The split S (1-based) the context uses. */
int planc_get_split(planc_t ctx);

/* Which partial MTTKRPs run on the tcgen05 tensor cores: bit 0 the left
 * branch T^{1:S}, bit 1 the right branch T^{S+1:N} (0 = CUDA cores). */
int planc_pm_tensor_cores(planc_t ctx);

/* Text of the dimension tree used for dims[0..N-1] with root split `split`
 * (1-based; -1 = planc_plan_split's choice): the root line, then one line per
 * edge, "PM {1,...,N} -> {a,...,b}" for the two partial MTTKRPs and
 * "mTTV {c,...,b} -> {...}" for the multi-TTVs of Alg. 3 (below the root the
 * first mode of a node is split off, Fig. ourDT).  Host-only; writes at most
 * len bytes including the terminating NUL.  PLANC_E_INVALID if it does not
 * fit, PLANC_E_SHAPE on a bad N or split. */
planc_status_t planc_describe(int N, const int64_t* dims, int split, char* buf, size_t len);

/* ---- the steps of Alg. 1 ------------------------------------------------ */

/* alpha = ||X||^2 (Alg. 4, Norm-Squared), FP64 result written to the device
 * double *alpha.  Asynchronous. */
planc_status_t planc_sqnorm(planc_t ctx, double* alpha);

/* M^(n) = X_(n) (H^N kr ... kr H^(n+1) kr H^(n-1) kr ... kr H^1)
 * (Alg. 1 MTTKRP), computed through the dimension tree of Alg. 3: the
 * partial MTTKRP of the root branch that holds mode n followed by the
 * multi-TTV chain down to leaf n.  H[k] for k != n are read; H[n] is not.
 * M is a device I_n x R row-major buffer (caller-owned).  Asynchronous.
 * Errors: PLANC_E_INVALID (n out of range, NULL pointers). */
planc_status_t planc_mttkrp(planc_t ctx, void* const* H, int n, void* M);

/* M^(n) for every mode n at the same factors (the all-mode MTTKRP the
 * dimension tree of Alg. 3 is built for): each root partial MTTKRP runs once
 * (two passes over X for any N) and each branch's multi-TTV chain reuses its
 * nodes mode after mode.  M: host array of N device pointers, I_n x R
 * row-major (caller-owned).  Asynchronous.  Errors: PLANC_E_INVALID. */
planc_status_t planc_mttkrp_all(planc_t ctx, void* const* H, void* const* M);

/* Partial MTTKRP (Sec. 4.2.2) of one root branch:
 *   side 0: T^{1:S} = X_(1:S) K^{S+1:N}  ((prod_{k<S} I_k) x R)
 *   side 1: T^{S+1:N} = X_(1:S)^T K^{1:S}  ((prod_{k>=S} I_k) x R)
 * written column-major (R slowest) to the device buffer T.  The benchmark
 * and the tests use this to time and check the HBM-bound kernel alone.
 * Asynchronous.  Errors: PLANC_E_INVALID (side not 0 or 1, T NULL, or a NULL
 * factor among the modes of the other branch, which form K). */
planc_status_t planc_partial_mttkrp(planc_t ctx, void* const* H, int side,
                                    void* T);

/* S^(n) = G^(1) * ... * G^(n-1) * G^(n+1) * ... * G^(N) (the S step of Alg. 1).
 * G: device N*R*R doubles; S: device R*R doubles.  Asynchronous. */
planc_status_t planc_gram_hadamard(planc_t ctx, const double* G, int n,
                                   double* S);

/* G = H^T H (Alg. 1, local SYRK) for a rows x R row-major factor H (ctx
 * factor dtype), accumulated with FP64 across row blocks; G device R*R
 * doubles.  Asynchronous. */
planc_status_t planc_gram(planc_t ctx, int64_t rows, const void* H, double* G);

/* NNLS-Update (Alg. 1; Sec. 4.3): updates the rows x R row-major Hhat in
 * place, given S (device R*R doubles, symmetric positive semidefinite) and
 * M (device rows x R, ctx factor dtype).  On entry H is the warm start; on
 * exit the updated (unnormalised) factor.
 *   alg  MU (Eq. muupd, one step), HALS (Eq. halsupd, one sweep in column
 *        order), BPP (Eq. snls, exact NNLS per row, FP64 passive-set
 *        Cholesky), ADMM (Eq. admmupd, FP64 inverse of S + rho I by the
 *        symmetric sweep operator, U reset to zero), NES (see planc_nls_t;
 *        eigenvalues of S in the factor precision), PGD
 *        (projected gradient), UCP (H = M S^{-1}).
 *   opts may be NULL (defaults).
 *   aux  ADMM dual U (device rows x R) to use and return, or NULL for the
 *        library's zero-initialised scratch; ignored by other algorithms.
 *   inner_iters  device int32 or NULL: ADMM / NES steps taken / max BPP
 *        exchanges over rows (1 for MU, HALS, UCP; pgd_steps for PGD; 0 for
 *        NES when S = 0, which leaves H unchanged).
 * Asynchronous.  A BPP row that hits the exchange cap returns its current
 * clipped iterate (no error).  Errors: PLANC_E_INVALID, PLANC_E_SHAPE
 * (rows > the largest mode of the context), PLANC_E_UNSUPPORTED (R > 64). */
planc_status_t planc_nls_update(planc_t ctx, planc_nls_t alg,
                                const planc_nls_opts* opts, int64_t rows,
                                const double* S, const void* M, void* H,
                                void* aux, int32_t* inner_iters);

/* Column normalisation of Alg. 4: lambda_r = ||Hhat(:, r)||_2 (FP64
 * accumulation), H = Hhat diag(lambda)^{-1} in place (a zero column keeps
 * lambda_r = 0 and stays zero), and, if G is not NULL, G = H^T H of the
 * normalised H.  lambda: device R doubles.  Asynchronous.  Errors:
 * PLANC_E_INVALID, PLANC_E_SHAPE (rows > the largest mode), PLANC_E_UNSUPPORTED
 * (R > 64; planc_gram likewise). */
planc_status_t planc_normalize(planc_t ctx, int64_t rows, void* H,
                               double* lambda, double* G);

/* Relative error of the model [[lambda; H^(1..N)]] by the identity of
 * Sec. A.2 / Alg. 4: eps = sqrt(max(0, alpha - 2 beta + gamma) / alpha) with
 * alpha = ||X||^2, beta = <M^(N), H^(N) diag(lambda)>, gamma = lambda^T
 * (G^(1) * ... * G^(N)) lambda.  Runs an MTTKRP for the last mode.
 * lambda is a DEVICE double[R]; rel_err and fit are HOST doubles (fit =
 * 1 - eps; either may be NULL).  Synchronises the stream. */
planc_status_t planc_fit(planc_t ctx, void* const* H, const double* lambda,
                         double* rel_err, double* fit);

/* The whole of Alg. 1 + Alg. 4: alpha = ||X||^2, lambda = 1, G^(n) of the
 * initial factors, then opts->iters outer iterations of (dimension-tree
 * MTTKRP, S^(n), NNLS-Update with warm start H^(n) diag(lambda),
 * normalisation, G^(n)) for n = 1..N and the error identity after mode N.
 * H: host array of N device pointers, initial factors in, normalised
 * factors out.  lambda: HOST double[R] out.  report: optional host record.
 * Synchronises the stream.  Requirements: R <= 64, 0 <= opts->iters <=
 * 1024 - ceil(16 / N) (the per-iteration history is kept on the device).
 * Errors: PLANC_E_INVALID (NULL H, iters out of range, unknown alg),
 * PLANC_E_UNSUPPORTED (R > 64), PLANC_E_NUMERIC (UCP or ADMM: S not positive
 * definite), PLANC_E_TIMEOUT (a bounded wait in a kernel gave up),
 * PLANC_E_CUDA. */
planc_status_t planc_nncp_solve(planc_t ctx, const planc_solve_opts* opts,
                                void* const* H, double* lambda,
                                planc_report* report);

/* Default solve options: HALS, 10 iterations, tol 0, default NNLS options,
 * graph replay on, profiling off, NES outer acceleration on. */
planc_solve_opts planc_solve_opts_default(void);

/* CP reconstruction loss f = ||X - [[H^(1..N)]]||^2 (Eq. nncp objective,
 * lambda = 1) and its gradient df/dH^(n) = 2 (H^(n) S^(n) - M^(n)) for every
 * mode (the MTTKRP and Hadamard-of-Grams matrices of Alg. 1).  H and dH:
 * host arrays of N device pointers (dH row-major I_n x R in the factor dtype,
 * caller-owned, overwritten).  loss: HOST double, or NULL to skip the loss.
 * The two root partial MTTKRPs are each computed once from the given factors
 * (2 passes over X for any N) and the multi-TTV chains are recomputed per
 * mode; nothing else is stored.  The loss uses the identity
 * f = ||X||^2 - 2 <M^(N), H^(N)> + 1^T (G^(1) * ... * G^(N)) 1, evaluated in
 * FP64; ||X||^2 is computed on the context's first call with a loss and
 * reused (X is unchanged while the context lives).  Overwrites the context's
 * lambda buffer (the next solve resets it).
 * Asynchronous when loss is NULL; synchronises the stream otherwise.
 * Errors: PLANC_E_INVALID (NULL pointers), PLANC_E_UNSUPPORTED (R > 64). */
planc_status_t planc_cp_grad(planc_t ctx, void* const* H, void* const* dH,
                             double* loss);

/* ---- batched solve --------------------------------------------------------- */

/* One 3-way instance of planc_batch_solve.  X: device, I_1 x I_2 x I_3, mode 1
 * fastest, F32 or BF16, starting on a 16-byte boundary, borrowed.  H: three device F32 factors I_n x R
 * row-major (in: initial factors, out: the solution, columns normalised as in
 * planc_nncp_solve).  lambda: host R doubles or NULL (out).  rel_err_hist:
 * host opts.iters doubles or NULL (out, eps per outer iteration). */
typedef struct {
  int64_t dims[3];
  int R;
  planc_dtype_t x_dtype;
  const void* X;
  void* H[3];
  double* lambda;
  double* rel_err_hist;
  double rel_err;   /* out: eps after the last outer iteration */
} planc_batch_instance;

/* NNCP (Alg. 1 with the dimension tree of Alg. 3 and the normalisation and
 * error identity of Alg. 4) of `count` independent 3-way instances of
 * different sizes.  With opts.batch_persistent (the default) the whole solve
 * is one persistent launch: thread-block clusters of 8 CTAs, as many as fit
 * on the GPU at once, each solving whole instances in turn (every phase of
 * every outer iteration: alpha, the initial Grams, left partial MTTKRP over
 * the CTAs' row blocks, the multi-TTVs, right partial MTTKRP over the CTAs'
 * slabs, the fused per-mode update and the error identity, separated by
 * cluster barriers); the instances are dealt longest-first onto the
 * least-loaded cluster by an estimate of their work.  With batch_persistent
 * 0 each phase of an outer iteration is one launch over a work table of
 * every instance's tiles (the partial MTTKRPs as persistent grids, each CTA
 * a contiguous run of tiles holding an equal share of the elements).  With
 * opts.use_graph the launch sequence is captured and run as one CUDA graph.
 * The schedule (rank blocking of both partial MTTKRPs; per-phase launches
 * also their tile shapes) is chosen by timing candidates on the first call
 * for a batch of that signature (cached per process).  Requirements: each I_n in
 * 1..1024, R in 1..32, x_dtype F32 or BF16, opts.alg MU, HALS or PGD,
 * opts.tol ignored (fixed iterations).  Workspace is allocated and freed
 * inside the call.  cuda_stream NULL: a private stream is used.
 * Synchronises the stream.  Errors (message in planc_last_error(NULL)): PLANC_E_INVALID,
 * PLANC_E_SHAPE, PLANC_E_DTYPE, PLANC_E_UNSUPPORTED, PLANC_E_NOMEM,
 * PLANC_E_CUDA, PLANC_E_TIMEOUT (a bounded wait in a kernel gave up).  (The
 * paper solves one tensor at a time; batching is this library's extension.) */
planc_status_t planc_batch_solve(planc_batch_instance* inst, int count,
                                 const planc_solve_opts* opts, void* cuda_stream,
                                 planc_report* report);

/* How the persistent launch of planc_batch_solve deals `count` instances to
 * `nclusters` thread-block clusters (host-only; the device pointers in inst
 * are not read).  Each instance's estimated cost per outer iteration is its
 * partial-MTTKRP FMAs (elements times both ranks padded to the classes 8, 16
 * or 32) plus a fixed share for the latency of its phases; instances are
 * taken longest-first (ties in index order), each onto the least-loaded
 * cluster (lowest index on ties).  Out: clist (count ints) lists cluster q's
 * instances at clist[coff[q]] .. clist[coff[q + 1] - 1], in the order it
 * solves them; coff (nclusters + 1 ints); load (nclusters doubles, or NULL)
 * the clusters' summed costs.  planc_batch_solve uses the clusters that fit
 * on the GPU at once, at most count.  Errors: PLANC_E_INVALID (NULL
 * argument, count < 1, nclusters outside 1..count), PLANC_E_SHAPE (dims or
 * R below 1). */
planc_status_t planc_batch_plan(const planc_batch_instance* inst, int count, int nclusters,
                                int* clist, int* coff, double* load);

/* The schedule the most recent planc_batch_solve on the calling thread used
 * for its two partial MTTKRPs, as chosen by timing every candidate on the
 * first call for a batch signature: out[0] rows per left-branch work item
 * (128, 256, 512: two per thread), out[1] threads per right-branch item
 * (64, 128, 256),
 * out[2] / out[3] the rank blocking of the left / right kernel (0: every
 * instance padded to rank 32; 1: classes 16 and 32; 2: classes 8, 16 and
 * 32; an instance runs in the smallest class that holds its rank).  The
 * environment variable PLANC_BATCH_RANK_BLOCKING="l,r" (0..2 each) forces
 * the two rank blockings (tests compare them).  out: host int[4].
 * Host-only.  Errors: PLANC_E_INVALID (out NULL). */
planc_status_t planc_batch_schedule(int* out);

/* ---- allocation-free variant --------------------------------------------- */

/* alpha = ||X||^2 for a flat device buffer X of n elements of x_dtype, written
 * to the device double *alpha, on cuda_stream (NULL = legacy stream), without
 * a context and without allocating any device memory.  (The paper has no
 * counterpart; this is a library convenience.)
 *
 * For callers that cannot allocate device memory when they need the
 * reduction: work enqueued while a stream is being captured into a CUDA graph
 * (allocation is not allowed during capture), runtimes that own all device
 * memory through their own fixed pool, and latency-critical loops that must
 * stay out of the allocator.  The per-block partial sums live in a
 * statically sized device array inside the library (1024 doubles, 8 KiB per
 * device that loads the library, held until the process exits); the result
 * equals planc_sqnorm's.
 *
 * The first call on each device looks up that array's device address with
 * cudaGetSymbolAddress while the device is current (and looks it up again
 * when the device's CUDA context has been destroyed and created anew since);
 * make that first call outside any stream capture.  All calls share the one array, so calls whose
 * work overlaps on the GPU (different streams, no ordering between them) race
 * on it; calls ordered on one stream are safe.  Every call overwrites the
 * partials it reads, so nothing needs clearing between calls.
 * Errors: PLANC_E_INVALID (NULL pointer), PLANC_E_DTYPE, PLANC_E_SHAPE (n < 1,
 * n > 2^40, or a GPU whose reduction grid would need more than 1024
 * partials), PLANC_E_CUDA.  Asynchronous. */
planc_status_t planc_sqnorm_noalloc(planc_dtype_t x_dtype, const void* X, int64_t n,
                                    double* alpha, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PLANC_H */
