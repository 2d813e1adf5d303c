// Internal declarations of libplanc: the context, and the host launchers of
// every kernel (each launcher lives beside its kernels in a .cu file).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/planc.h"
#include "common.cuh"

namespace planc {

// Type-erased description of a partial Khatri-Rao product (see Krp<TF>).
struct KrpHost {
  int nm = 0;
  int64_t dim[PLANC_MAX_N] = {};
  const void* H[PLANC_MAX_N] = {};
};

// Count of kernels this library has launched (all contexts); the solve
// reports how many of its kernels ran.
void note_launches(int n);
// launches of the solve's hot kernels use programmatic dependent launch
// unless PLANC_PDL=0 (read once)
bool pdl_enabled();
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
}
long long launch_count();

inline size_t dtype_size(planc_dtype_t d) {
  return d == PLANC_F64 ? 8 : d == PLANC_F32 ? 4 : 2;
}

// ---- partial MTTKRP (root branches of the dimension tree, Sec. 4.2.2) -----
// SIMT path, any dtype/shape/rank.  Computes, for side "left",
//   out[m, r] = sum_{c<C} X[m + L c] * K[c, r]           (m < L)
// and for side "right"
//   out[m, r] = sum_{l<L} X[l + L m] * K[l, r]           (m < C)
// with K the partial Khatri-Rao product `krp`.  Output is R-slowest
// (out[m + Mdim r]) or row-major (out[m R + r]).  With nsplit > 1 the
// reduction dimension is split over CTAs into `part` (nsplit x Mdim x R)
// and summed in a fixed order by a second kernel.
int pm_simt_nsplit(bool left, int64_t L, int64_t C, int R, int sm_count);
cudaError_t launch_pm_simt(planc_dtype_t xdt, const void* X, int64_t L, int64_t C,
                           bool left, const KrpHost& krp, int R, void* out,
                           bool out_rowmajor, void* part, int nsplit, cudaStream_t st);

// tcgen05 path (FP32 X as 3xTF32, BF16/F16 X as kind::f16 with a two-term
// BF16 split of the Khatri-Rao operand).  Returns cudaErrorNotSupported when
// the shape/rank/dtype is not eligible; the caller then uses the SIMT path.
bool pm_tc_eligible(planc_dtype_t xdt, bool left, int64_t L, int64_t C, int R,
                    const KrpHost& krp_dims);
size_t pm_tc_workspace_bytes(planc_dtype_t xdt, bool left, int64_t L, int64_t C, int R,
                             const KrpHost& krp_dims, int sm_count);
cudaError_t launch_pm_tc(planc_dtype_t xdt, const void* X, int64_t L, int64_t C,
                         bool left, const KrpHost& krp, int R, void* out,
                         bool out_rowmajor, void* work, size_t work_bytes,
                         int* err_flag, int sm_count, cudaStream_t st);
// Partial MTTKRPs as one GEMM against the split Khatri-Rao image
// (kern_pm_krp.cu): BF16 X both root branches, FP32 X the right branch when
// the image is small next to X; launch_pm_tc takes it when eligible and the
// workspace holds it (PLANC_PM_KRP=0 turns it off)
bool pm_krp_eligible(planc_dtype_t xdt, bool left, int64_t L, int64_t C, int R,
                     const KrpHost& krp_dims);
size_t pm_krp_workspace_bytes(planc_dtype_t xdt, bool left, int64_t L, int64_t C, int R,
                              int sm_count);
cudaError_t launch_pm_krp(planc_dtype_t xdt, const void* X, int64_t L, int64_t C, bool left,
                          const KrpHost& krp, int R, void* out, bool out_rowmajor, void* work,
                          size_t work_bytes, int* err_flag, int sm_count, cudaStream_t st);

// ---- multi-TTV (Sec. 4.2.2) --------------------------------------------------
// T is the node tensor T^{a:b} viewed as T[p + P1 q + P1 Q r].
// contract_first: out[q, r] = sum_p T[p, q, r] h[p, r]  (h row-major P1 x R)
// contract_rest : out[p, r] = sum_q T[p, q, r] K[q, r]  (K partial KRP)
cudaError_t launch_contract_first(bool f64, const void* T, int64_t P1, int64_t Q, int R,
                                  const void* h, void* out, bool out_rowmajor,
                                  cudaStream_t st);
int contract_rest_qsplit(int64_t P1, int64_t Q, int R, int sm_count);
bool contract_rest_v4_ok(int64_t P1, const void* T);
cudaError_t launch_contract_rest(bool f64, const void* T, int64_t P1, int64_t Q, int R,
                                 const KrpHost& krp, void* out, void* part, int qsplit,
                                 cudaStream_t st);

// ---- reductions, Grams, normalisation, error ---------------------------------
int sqnorm_blocks(int64_t n, int sm_count);
cudaError_t launch_sqnorm(planc_dtype_t xdt, const void* X, int64_t n, double* part,
                          int nblk, double* alpha, cudaStream_t st);
cudaError_t launch_gram_hadamard(const double* G, int N, int n, int R, double* S,
                                 cudaStream_t st);
int rowblocks(int64_t rows);
// Column sums of squares of Hhat per row block (FP64 partials) and, if M is
// given, per-block partials of <M, Hhat>.
cudaError_t launch_colsq(bool f64, int64_t rows, int R, const void* Hhat, const void* M,
                         double* colsq_part, double* dot_part, int nblk, cudaStream_t st);
// lambda from the partials, H = Hhat / lambda in place, FP64 Gram partials.
cudaError_t launch_scale_gram(bool f64, int64_t rows, int R, void* H, const double* colsq_part,
                              int nblk, double* lambda, double* gram_part, bool scale,
                              cudaStream_t st);
// G = sum of the Gram partials (fixed order).
cudaError_t launch_gram_reduce(int R, const double* gram_part, int nblk, double* G, float* Gf,
                               cudaStream_t st);
// The error identity of Alg. 4: eps = sqrt(max(0, alpha - 2 beta + gamma) /
// alpha) with beta = sum of the dot partials and gamma = lambda^T (G^(1) *
// ... * G^(N)) lambda.  fit_out receives {eps, beta, gamma}.
cudaError_t launch_fit(int R, const double* Gall, int N, const double* lambda,
                       const double* dot_part, int dot_nblk, const double* alpha,
                       double* fit_out, cudaStream_t st);
// <M, H diag(lambda)> partials for planc_fit.
cudaError_t launch_dot_lambda(bool f64, int64_t rows, int R, const void* M, const void* H,
                              const double* lambda, double* dot_part, int nblk,
                              cudaStream_t st);
// dH^(n) = 2 (H^(n) S^(n) - M^(n)) for all N modes in one launch (S^(n) from
// the Grams: FP32 copies G32 for FP32 factors, G64 for FP64)
cudaError_t launch_cp_grad_all(bool f64, int N, const int64_t* rows, int R,
                               void* const* H, void* const* dH, const double* G64,
                               const float* G32, int sm_count, cudaStream_t st);
// G^(n) = H^(n)T H^(n) for all N modes in one launch (FP64 and the FP32
// copy; a loop over the rows per entry: for factors with few rows)
cudaError_t launch_gram_all(bool f64, int N, const int64_t* rows, int R, void* const* H,
                            double* G, float* Gf, cudaStream_t st);
cudaError_t launch_fill(double* p, double v, int64_t n, cudaStream_t st);

// outer acceleration of the Nesterov-type solve: every factor of the model,
// concatenated (element e of the whole belongs to mode n with
// off[n] <= e < off[n+1])
struct AccelModes {
  int N, R;
  int64_t off[PLANC_MAX_N + 1];
  void* H[PLANC_MAX_N];   // current iterate (normalised; lambda separate)
  void* Hp[PLANC_MAX_N];  // previous outer iterate
  void* Hc[PLANC_MAX_N];  // candidate
};
cudaError_t launch_accel_extrapolate(bool f64, const AccelModes& t, const double* lam,
                                     const double* lam_prev, const int* counter, cudaStream_t st);
cudaError_t launch_accel_finish(bool f64, const AccelModes& t, const double* nu, double* lam_c,
                                cudaStream_t st);
cudaError_t launch_accel_select(bool f64, const AccelModes& t, double* scal, const int* counter,
                                int32_t* hist, int cap, int* flags, double* lam, double* lam_prev,
                                const double* lam_c, double* G, float* Gf, const double* Gc,
                                cudaStream_t st);

// ---- NNLS updates (Sec. 4.3) ---------------------------------------------------
struct NlsArgs {
  planc_nls_t alg;
  planc_nls_opts opts;
  int64_t rows;
  int R;
  const double* S;        // R x R FP64
  const void* M;          // rows x R
  void* H;                // rows x R, in/out
  const double* lambda;   // warm-start column scale (NULL = none)
  void* U;                // ADMM dual / Nesterov Y (rows x R)
  void* V;                // Nesterov H* (rows x R)
  bool U_zero;            // ADMM: start from U = 0 (else read U)
  int32_t* inner;         // device int or NULL
  double* scratch;        // FP64 scratch (>= nls_scratch_doubles)
  int* flags;             // int scratch (>= 8 ints)
  bool f64;
  bool reset_inner = true;  // BPP: zero *inner first (false: the caller did)
};
size_t nls_scratch_doubles(int64_t rows, int R);
// p[0..n) = v (one small launch)
cudaError_t launch_set_int(int32_t* p, int v, int n, cudaStream_t st);
// (S + rho I)^{-1} into scr (rho = trace(S)/R, or 0 with ucp): [0] rho,
// [1] 1 if a pivot was not positive; the inverse (FP64) at scr + 8 and in the
// factor precision at scr + 8 + R^2
cudaError_t launch_inv_prep(bool f64, const double* S, int R, double* scr, int ucp,
                            cudaStream_t st);
// Nesterov-type update parameters from S into scr: [0] lam_p, [1] L,
// [2] beta, [3] 1/L, [4] lam_p/L, [5] 1 if S = 0; P in the factor precision
// at scr + 8 + R^2
cudaError_t launch_nes_prep(bool f64, const double* S, int R, double* scr, cudaStream_t st);
cudaError_t launch_nls(const NlsArgs& a, cudaStream_t st);

// ---- fused per-mode update (S, NNLS, normalisation, Gram, error) ------------------
// sets the message planc_last_error(NULL) returns on this thread
void set_thread_error(const char* msg);

// One instance of a batched 3-way solve, as the batched kernels read it
// (device copy of a table built by planc_batch_solve).
struct BatchInst {
  const void* X;      // I1 x I2 x I3, mode 1 fastest (F32 or BF16, see xbf16)
  int64_t I[3];
  int R;
  int xbf16;
  float* H[3];        // I_n x R row-major
  float* T;           // T^{1:2}: (I1 I2) x R, R slowest
  float* M;           // M^(n): max I_n x R row-major
  double* G;          // 3 x R x R
  float* Gf;          // the same in FP32
  double* lam;        // R
  double* alpha;      // ||X||^2
  double* hist;       // iters x (eps, beta, gamma)
  int32_t* inner;     // iters x 3
};
cudaError_t launch_mode_batch(const BatchInst* tab, int count, int n, int it, planc_nls_t alg,
                              const planc_nls_opts& o, int* err, cudaStream_t st);
int mode_batch_max_rows();
// The whole batched solve in one persistent launch (kern_mode.cu): nclusters
// thread-block clusters, cluster q solving the instances clist[coff[q]] ..
// clist[coff[q + 1] - 1] in turn (alg MU, HALS or PGD); mode 1 / 2 runs only
// the left / right partial MTTKRPs (schedule timing).  hmax: the longest
// second or third mode of the batch; h1max: the longest first mode when the
// right branch stages H1 in shared memory, else 0; sqpart: 8 doubles per
// instance.
cudaError_t launch_batch_persistent(const BatchInst* tab, const int* clist, const int* coff,
                                    int nclusters, int iters, planc_nls_t alg,
                                    const planc_nls_opts& o, int sched_l, int sched_r, int mode,
                                    int hmax, int h1max, double* sqpart, int* err,
                                    cudaStream_t st);
// clusters of the persistent launch that fit on the device at once (0 if none)
int batch_persistent_max_clusters(planc_nls_t alg, int hmax, int h1max);
constexpr int kBatchClusterCtas = 8;  // CTAs per cluster of the persistent launch
bool mode_fused_eligible(planc_nls_t alg, int64_t rows, int R, bool f64);
// the per-iteration history record (error triple and inner counts at index
// *counter, then ++*counter), done by the last mode's fused update when given
struct RecArgs {
  double* hist = nullptr;
  const int32_t* inner_now = nullptr;
  int32_t* inner_hist = nullptr;
  int* counter = nullptr;
  int N = 0, cap = 0;
};
// nes_scr: the prepared parameters when alg is NES (launch_nes_prep) or UCP
// (launch_inv_prep: the inverse of S); flags[1] counts singular S (UCP)
cudaError_t launch_mode_fused(bool f64, int64_t rows, int R, int N, int n, const double* G,
                              float* Gf, const void* M, void* H, double* lam, planc_nls_t alg,
                              const planc_nls_opts& o, int32_t* inner, const double* alpha,
                              double* fit_out, int* err, const double* nes_scr,
                              const RecArgs& rec, int* flags, cudaStream_t st);

// ---- PM-right / mTTV split reductions -------------------------------------------
cudaError_t launch_split_reduce(bool f64, const void* part, int nsplit, int64_t Mdim, int R,
                                void* out, bool out_rowmajor, cudaStream_t st);

}  // namespace planc

// ---- the context ------------------------------------------------------------------
struct planc_ctx {
  int N = 0, R = 0, S = 0;          // S: number of modes in the left branch
  int64_t dims[PLANC_MAX_N] = {};
  int64_t L = 1, C = 1, I = 1, max_dim = 1;
  planc_dtype_t xd = PLANC_F32, fd = PLANC_F32;
  const void* X = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0, sm_count = 148;
  std::string err;

  // workspace (one allocation, carved)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* T_side[2] = {nullptr, nullptr};  // root partials T^{1:S}, T^{S+1:N}
  void* node[2] = {nullptr, nullptr};    // internal-node ping-pong
  void* part = nullptr;                  // split-K / q-split partials
  size_t part_bytes = 0;
  void* tc_work = nullptr;               // tcgen05 path scratch
  size_t tc_bytes = 0;
  int* tc_err = nullptr;                 // tcgen05 bounded-wait error flag
  void* Mbuf = nullptr;                  // max_dim x R
  void* Ubuf = nullptr;                  // ADMM dual / Nesterov Y, max_dim x R
  void* Vbuf = nullptr;                  // Nesterov H*, max_dim x R
  // outer acceleration (Nesterov-type solve)
  void* Hprev[PLANC_MAX_N] = {};         // previous outer iterate
  void* Hcand[PLANC_MAX_N] = {};         // candidate
  double* lam_prev = nullptr;            // R
  double* lam_cand = nullptr;            // R
  double* nu = nullptr;                  // N x R candidate column norms
  double* Gc = nullptr;                  // N x R x R candidate Grams
  int32_t* accel_hist = nullptr;         // per outer iteration: accepted
  double* G = nullptr;                   // N x R x R
  float* Gf = nullptr;                   // the same Grams rounded to FP32
  double* Sm = nullptr;                  // R x R
  double* lam = nullptr;                 // R
  double* scal = nullptr;                // [0] alpha, [1..] scratch
  double grad_alpha = -1.0;              // ||X||^2 for planc_cp_grad's loss (< 0: not yet)
  double* hist = nullptr;                // per-iteration rel. error (device)
  int hist_cap = 0;
  double* red = nullptr;                 // reduction partials
  size_t red_doubles = 0;
  double* nls_scr = nullptr;             // NNLS scratch
  size_t nls_scr_doubles = 0;
  int32_t* inner = nullptr;              // per-call inner counts (device)
  int inner_cap = 0;
  int* flags = nullptr;

  // dimension-tree state during a solve
  int nsplit[2] = {1, 1};
  bool use_tc[2] = {false, false};
  bool fused_modes = true;
  size_t node_elems = 0;

  // side stream for work that overlaps the MTTKRP (fork / join events)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // profiling (partial-MTTKRP launches)
  bool profiling = false;
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
};
