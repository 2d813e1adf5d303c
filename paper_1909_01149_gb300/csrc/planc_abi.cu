// C ABI of libplanc (include/planc.h): argument checking, the workspace, the
// dimension-tree driver of Alg. 3 and the outer loop of Alg. 1 / Alg. 4.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

using namespace planc;

namespace planc {
static std::atomic<long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("PLANC_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}
}  // namespace planc

namespace {

thread_local std::string g_init_error;

planc_status_t fail(planc_t ctx, planc_status_t st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf; else g_init_error = buf;
  return st;
}

}  // namespace

// the calling thread's context-free error message (planc_last_error(NULL))
void planc::set_thread_error(const char* msg) { g_init_error = msg; }

namespace {

planc_status_t cuda_fail(planc_t ctx, cudaError_t e, const char* what) {
  return fail(ctx, PLANC_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

bool is_f64(planc_t ctx) { return ctx->fd == PLANC_F64; }
size_t fsize(planc_t ctx) { return dtype_size(ctx->fd); }

// modes [a, b] (0-based, inclusive) of a root branch: side 0 = {0..S-1},
// side 1 = {S..N-1}
int side_a(planc_t ctx, int s) { return s == 0 ? 0 : ctx->S; }
int side_b(planc_t ctx, int s) { return s == 0 ? ctx->S - 1 : ctx->N - 1; }
int side_of(planc_t ctx, int n) { return n < ctx->S ? 0 : 1; }

int64_t prod(planc_t ctx, int a, int b) {
  int64_t p = 1;
  for (int k = a; k <= b; ++k) p *= ctx->dims[k];
  return p;
}

KrpHost krp_of(planc_t ctx, void* const* H, int a, int b) {
  KrpHost k;
  k.nm = 0;
  for (int m = a; m <= b; ++m) {
    k.dim[k.nm] = ctx->dims[m];
    k.H[k.nm] = H[m];
    ++k.nm;
  }
  return k;
}

// ---- dimension tree pieces (Alg. 3) ---------------------------------------------

// Partial MTTKRP of a root branch; the result goes to `out` (R-slowest), or
// row-major when the branch holds a single mode (then it is M^(a) itself).
planc_status_t run_pm(planc_t ctx, void* const* H, int side, void* out, bool rowmajor) {
  const bool left = side == 0;
  KrpHost k = left ? krp_of(ctx, H, ctx->S, ctx->N - 1) : krp_of(ctx, H, 0, ctx->S - 1);
  cudaError_t e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ctx->profiling && ctx->ev_used + 2 <= (int)ctx->ev.size()) {
    e0 = ctx->ev[ctx->ev_used];
    e1 = ctx->ev[ctx->ev_used + 1];
    ctx->ev_used += 2;
    cudaEventRecord(e0, ctx->stream);
  }
  if (ctx->use_tc[side]) {
    e = launch_pm_tc(ctx->xd, ctx->X, ctx->L, ctx->C, left, k, ctx->R, out, rowmajor,
                     ctx->tc_work, ctx->tc_bytes, ctx->tc_err, ctx->sm_count, ctx->stream);
  } else {
    e = launch_pm_simt(ctx->xd, ctx->X, ctx->L, ctx->C, left, k, ctx->R, out, rowmajor,
                       ctx->part, ctx->nsplit[side], ctx->stream);
  }
  if (e1) cudaEventRecord(e1, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "partial MTTKRP launch");
  return PLANC_OK;
}

// T^{a+1:b} = contract mode a of T^{a:b} with H^(a) (internal node or leaf)
planc_status_t run_contract_first(planc_t ctx, const void* T, int a, int b, const void* Ha,
                                  void* out, bool rowmajor) {
  int64_t P1 = ctx->dims[a];
  int64_t Q = prod(ctx, a + 1, b);
  CK(launch_contract_first(is_f64(ctx), T, P1, Q, ctx->R, Ha, out, rowmajor, ctx->stream),
     "multi-TTV (node) launch");
  return PLANC_OK;
}

// M^(a) = T^{a:b} contracted over modes a+1..b with K^{a+1:b}
planc_status_t run_contract_rest(planc_t ctx, const void* T, int a, int b, void* const* H,
                                 void* M) {
  int64_t P1 = ctx->dims[a];
  int64_t Q = prod(ctx, a + 1, b);
  int qs = contract_rest_qsplit(P1, Q, ctx->R, ctx->sm_count);
  KrpHost k = krp_of(ctx, H, a + 1, b);
  CK(launch_contract_rest(is_f64(ctx), T, P1, Q, ctx->R, k, M, ctx->part, qs, ctx->stream),
     "multi-TTV (leaf) launch");
  return PLANC_OK;
}

// Dimension-tree walk for one mode.  `cur` holds the node T^{c:b} the walk
// starts from (c <= n) or nullptr to start with the branch's partial MTTKRP;
// on return it holds T^{n:b} (when n < b) so a later mode of the same branch
// can continue from it.
planc_status_t dt_mode(planc_t ctx, void* const* H, int n, void* M, const void** cur,
                       int* cur_first) {
  const int s = side_of(ctx, n);
  const int a = side_a(ctx, s), b = side_b(ctx, s);
  planc_status_t st;
  if (*cur == nullptr || *cur_first > n) {
    if (a == b) return run_pm(ctx, H, s, M, true);      // the branch is the leaf
    if ((st = run_pm(ctx, H, s, ctx->T_side[s], false)) != PLANC_OK) return st;
    *cur = ctx->T_side[s];
    *cur_first = a;
  }
  // walk down to T^{n:b}, or straight to the leaf M^(b)
  while (*cur_first < n) {
    const int c = *cur_first;
    if (c + 1 == b) {  // contracting mode c of T^{b-1:b} yields M^(b)
      st = run_contract_first(ctx, *cur, c, b, H[c], M, true);
      *cur = nullptr;
      *cur_first = b + 1;
      return st;
    }
    void* dst = (*cur == ctx->node[0]) ? ctx->node[1] : ctx->node[0];
    if ((st = run_contract_first(ctx, *cur, c, b, H[c], dst, false)) != PLANC_OK) return st;
    *cur = dst;
    *cur_first = c + 1;
  }
  return run_contract_rest(ctx, *cur, n, b, H, M);
}

void* carve(char*& p, size_t bytes) {
  void* r = p;
  p += (bytes + 255) / 256 * 256;
  return r;
}

}  // namespace

// ============================================================================
extern "C" {

const char* planc_status_str(planc_status_t s) {
  switch (s) {
    case PLANC_OK: return "ok";
    case PLANC_E_INVALID: return "invalid argument";
    case PLANC_E_SHAPE: return "invalid shape";
    case PLANC_E_DTYPE: return "unsupported dtype";
    case PLANC_E_NOMEM: return "out of device memory";
    case PLANC_E_CUDA: return "CUDA error";
    case PLANC_E_NUMERIC: return "numerical failure";
    case PLANC_E_NOT_CONVERGED: return "not converged";
    case PLANC_E_TIMEOUT: return "device wait timed out";
    case PLANC_E_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* planc_last_error(planc_t ctx) {
  return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

planc_nls_opts planc_nls_opts_default(void) {
  planc_nls_opts o;
  o.mu_eps = 1e-16;
  o.admm_max_inner = 5;
  o.admm_tol = 1e-2;
  o.bpp_max_iter = 0;
  o.pgd_steps = 1;
  o.nes_max_inner = 20;
  o.nes_tol = 1e-3;
  return o;
}

planc_solve_opts planc_solve_opts_default(void) {
  planc_solve_opts o;
  o.alg = PLANC_HALS;
  o.iters = 10;
  o.tol = 0.0;
  o.nls = planc_nls_opts_default();
  o.use_graph = 1;
  o.profile = 0;
  o.nes_accel = 1;
  o.batch_persistent = 1;
  return o;
}

planc_status_t planc_plan_split(int N, const int64_t* dims, int* split) {
  if (N < 2 || N > PLANC_MAX_N || !dims || !split)
    return fail(nullptr, PLANC_E_SHAPE, "N must be in [2, %d]", PLANC_MAX_N);
  for (int k = 0; k < N; ++k)
    if (dims[k] < 1) return fail(nullptr, PLANC_E_SHAPE, "dims[%d] < 1", k);
  double best = 0.0;
  int best_s = 1;
  for (int s = 1; s < N; ++s) {
    double l = 0.0, r = 0.0;
    for (int k = 0; k < s; ++k) l += std::log((double)dims[k]);
    for (int k = s; k < N; ++k) r += std::log((double)dims[k]);
    double score = std::fabs(l - r);
    if (s == 1 || score <= best + 1e-12) { best = score; best_s = s; }
  }
  *split = best_s;
  return PLANC_OK;
}

planc_status_t planc_init(planc_t* out, int N, const int64_t* dims, int R, planc_dtype_t x_dtype,
                          const void* X, planc_dtype_t f_dtype, void* cuda_stream, int split) {
  g_init_error.clear();
  if (!out) return fail(nullptr, PLANC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (N < 2 || N > PLANC_MAX_N) return fail(nullptr, PLANC_E_SHAPE, "N=%d not in [2, %d]", N, PLANC_MAX_N);
  if (!dims) return fail(nullptr, PLANC_E_INVALID, "dims is NULL");
  if (R < 1 || R > PLANC_MAX_R) return fail(nullptr, PLANC_E_SHAPE, "R=%d not in [1, %d]", R, PLANC_MAX_R);
  double logI = 0.0;
  for (int k = 0; k < N; ++k) {
    if (dims[k] < 1) return fail(nullptr, PLANC_E_SHAPE, "dims[%d]=%lld < 1", k, (long long)dims[k]);
    logI += std::log2((double)dims[k]);
  }
  if (logI > 40.0) return fail(nullptr, PLANC_E_SHAPE, "tensor has more than 2^40 entries");
  if ((int)x_dtype < 0 || (int)x_dtype > 3) return fail(nullptr, PLANC_E_DTYPE, "bad x_dtype");
  if ((x_dtype == PLANC_F64) != (f_dtype == PLANC_F64) || (f_dtype != PLANC_F64 && f_dtype != PLANC_F32))
    return fail(nullptr, PLANC_E_DTYPE, "factor dtype must be F64 for F64 X and F32 otherwise");
  if (!X) return fail(nullptr, PLANC_E_INVALID, "X is NULL");
  if (split == 0 || split >= N || split < -1)
    return fail(nullptr, PLANC_E_SHAPE, "split %d not in [1, N-1] (or -1)", split);

  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(nullptr, PLANC_E_CUDA, "no CUDA device: %s", cudaGetErrorString(ce));
  cudaDeviceProp prop;
  ce = cudaGetDeviceProperties(&prop, dev);
  if (ce != cudaSuccess) return fail(nullptr, PLANC_E_CUDA, "device query: %s", cudaGetErrorString(ce));
  if (prop.major != 10 || prop.minor != 3)
    return fail(nullptr, PLANC_E_CUDA, "device is sm_%d%d; this library is built for sm_103a",
                prop.major, prop.minor);

  planc_ctx* ctx = new (std::nothrow) planc_ctx();
  if (!ctx) return fail(nullptr, PLANC_E_NOMEM, "host allocation failed");
  ctx->N = N;
  ctx->R = R;
  for (int k = 0; k < N; ++k) ctx->dims[k] = dims[k];
  int S = split;
  if (S < 0) planc_plan_split(N, dims, &S);
  ctx->S = S;
  ctx->L = prod(ctx, 0, S - 1);
  ctx->C = prod(ctx, S, N - 1);
  ctx->I = ctx->L * ctx->C;
  ctx->max_dim = *std::max_element(dims, dims + N);
  ctx->xd = x_dtype;
  ctx->fd = f_dtype;
  ctx->X = X;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->device = dev;
  ctx->sm_count = prop.multiProcessorCount;

  // ---- workspace sizes
  const size_t fs = fsize(ctx);
  size_t part_elems = 0;
  // PLANC_PM_PATH=simt keeps the partial MTTKRPs on the CUDA-core kernels
  // (for A/B comparisons); by default eligible shapes use the tensor cores.
  const char* path = getenv("PLANC_PM_PATH");
  const bool allow_tc = !(path && strcmp(path, "simt") == 0);
  // PLANC_FUSED_MODES=0 keeps every mode update on the multi-kernel path
  const char* fm = getenv("PLANC_FUSED_MODES");
  ctx->fused_modes = !(fm && strcmp(fm, "0") == 0);
  for (int s = 0; s < 2; ++s) {
    const bool left = s == 0;
    KrpHost kd;  // dims of the branch's Khatri-Rao operand (pointers unused)
    for (int m = left ? S : 0; m < (left ? N : S); ++m) kd.dim[kd.nm++] = dims[m];
    ctx->use_tc[s] = allow_tc && ((uintptr_t)X & 15) == 0 &&
                     pm_tc_eligible(x_dtype, left, ctx->L, ctx->C, R, kd);
    if (!ctx->use_tc[s]) {
      ctx->nsplit[s] = pm_simt_nsplit(left, ctx->L, ctx->C, R, ctx->sm_count);
      if (ctx->nsplit[s] > 1)
        part_elems = std::max(part_elems, (size_t)ctx->nsplit[s] * (left ? ctx->L : ctx->C) * R);
    } else {
      ctx->tc_bytes = std::max(ctx->tc_bytes, pm_tc_workspace_bytes(x_dtype, left, ctx->L, ctx->C,
                                                                     R, kd, ctx->sm_count));
    }
  }
  // multi-TTV leaf partials, every (node, mode) pair the walks can meet
  size_t node_elems = 0;
  for (int s = 0; s < 2; ++s) {
    int a = side_a(ctx, s), b = side_b(ctx, s);
    for (int c = a; c < b; ++c) {
      int64_t P1 = dims[c], Q = prod(ctx, c + 1, b);
      int qs = contract_rest_qsplit(P1, Q, R, ctx->sm_count);
      if (qs > 1) part_elems = std::max(part_elems, (size_t)qs * P1 * R);
      if (c > a && b - c >= 1 && c < b) node_elems = std::max(node_elems, (size_t)P1 * Q * R);
    }
  }
  ctx->node_elems = node_elems;
  ctx->part_bytes = part_elems * fs;
  const int nblk = rowblocks(ctx->max_dim);
  ctx->red_doubles = (size_t)nblk * R + nblk + (size_t)nblk * R * R + 4 * ctx->sm_count + 64;
  ctx->nls_scr_doubles = nls_scratch_doubles(ctx->max_dim, R);
  ctx->hist_cap = 3 * 1024;
  ctx->inner_cap = 1024 * N;

  size_t bytes = 0;
  auto add = [&](size_t b) { bytes += (b + 255) / 256 * 256; };
  add(S > 1 ? (size_t)ctx->L * R * fs : 0);
  add(N - S > 1 ? (size_t)ctx->C * R * fs : 0);
  add(node_elems * fs);
  add(node_elems * fs);
  add(ctx->part_bytes);
  add(ctx->tc_bytes);
  add(64 * sizeof(int));                    // tc_err
  add((size_t)ctx->max_dim * R * fs);       // Mbuf
  add((size_t)ctx->max_dim * R * fs);       // Ubuf
  add((size_t)ctx->max_dim * R * fs);       // Vbuf
  for (int k = 0; k < N; ++k) {
    add((size_t)dims[k] * R * fs);          // Hprev[k]
    add((size_t)dims[k] * R * fs);          // Hcand[k]
  }
  add((size_t)R * 8);                       // lam_prev
  add((size_t)R * 8);                       // lam_cand
  add((size_t)N * R * 8);                   // nu
  add((size_t)N * R * R * 8);               // Gc
  add((size_t)(ctx->hist_cap / 3) * 4);     // accel_hist
  add((size_t)N * R * R * 8);               // G
  add((size_t)N * R * R * 4);               // G in FP32
  add((size_t)R * R * 8);                   // S
  add((size_t)R * 8);                       // lambda
  add(64 * 8);                              // scal
  add((size_t)ctx->hist_cap * 8);
  add(ctx->red_doubles * 8);
  add(ctx->nls_scr_doubles * 8);
  add((size_t)ctx->inner_cap * 4);
  add(16 * sizeof(int));                    // flags
  ce = cudaMalloc(&ctx->ws, bytes);
  if (ce != cudaSuccess) {
    delete ctx;
    cudaGetLastError();
    return fail(nullptr, PLANC_E_NOMEM, "workspace of %zu bytes: %s", bytes, cudaGetErrorString(ce));
  }
  ctx->ws_bytes = bytes;
  char* p = (char*)ctx->ws;
  ctx->T_side[0] = carve(p, S > 1 ? (size_t)ctx->L * R * fs : 0);
  ctx->T_side[1] = carve(p, N - S > 1 ? (size_t)ctx->C * R * fs : 0);
  ctx->node[0] = carve(p, node_elems * fs);
  ctx->node[1] = carve(p, node_elems * fs);
  ctx->part = carve(p, ctx->part_bytes);
  ctx->tc_work = carve(p, ctx->tc_bytes);
  ctx->tc_err = (int*)carve(p, 64 * sizeof(int));
  ctx->Mbuf = carve(p, (size_t)ctx->max_dim * R * fs);
  ctx->Ubuf = carve(p, (size_t)ctx->max_dim * R * fs);
  ctx->Vbuf = carve(p, (size_t)ctx->max_dim * R * fs);
  for (int k = 0; k < N; ++k) {
    ctx->Hprev[k] = carve(p, (size_t)dims[k] * R * fs);
    ctx->Hcand[k] = carve(p, (size_t)dims[k] * R * fs);
  }
  ctx->lam_prev = (double*)carve(p, (size_t)R * 8);
  ctx->lam_cand = (double*)carve(p, (size_t)R * 8);
  ctx->nu = (double*)carve(p, (size_t)N * R * 8);
  ctx->Gc = (double*)carve(p, (size_t)N * R * R * 8);
  ctx->accel_hist = (int32_t*)carve(p, (size_t)(ctx->hist_cap / 3) * 4);
  ctx->G = (double*)carve(p, (size_t)N * R * R * 8);
  ctx->Gf = (float*)carve(p, (size_t)N * R * R * 4);
  ctx->Sm = (double*)carve(p, (size_t)R * R * 8);
  ctx->lam = (double*)carve(p, (size_t)R * 8);
  ctx->scal = (double*)carve(p, 64 * 8);
  ctx->hist = (double*)carve(p, (size_t)ctx->hist_cap * 8);
  ctx->red = (double*)carve(p, ctx->red_doubles * 8);
  ctx->nls_scr = (double*)carve(p, ctx->nls_scr_doubles * 8);
  ctx->inner = (int32_t*)carve(p, (size_t)ctx->inner_cap * 4);
  ctx->flags = (int*)carve(p, 16 * sizeof(int));
  ce = cudaMemsetAsync(ctx->ws, 0, bytes, ctx->stream);
  if (ce != cudaSuccess) {
    cudaFree(ctx->ws);
    delete ctx;
    return fail(nullptr, PLANC_E_CUDA, "workspace clear: %s", cudaGetErrorString(ce));
  }
  *out = ctx;
  return PLANC_OK;
}

planc_status_t planc_destroy(planc_t ctx) {
  if (!ctx) return PLANC_OK;
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->ws) cudaFree(ctx->ws);
  delete ctx;
  return PLANC_OK;
}

int planc_get_split(planc_t ctx) { return ctx ? ctx->S : -1; }

int planc_pm_tensor_cores(planc_t ctx) {
  return ctx ? (ctx->use_tc[0] ? 1 : 0) | (ctx->use_tc[1] ? 2 : 0) : 0;
}

planc_status_t planc_describe(int N, const int64_t* dims, int split, char* buf, size_t len) {
  if (!buf || len == 0) return fail(nullptr, PLANC_E_INVALID, "buf is NULL");
  int S = split;
  if (S == -1) {
    planc_status_t st = planc_plan_split(N, dims, &S);
    if (st != PLANC_OK) return st;
  } else if (N < 2 || N > PLANC_MAX_N || S < 1 || S >= N) {
    return fail(nullptr, PLANC_E_SHAPE, "bad N or split");
  }
  std::string s;
  auto set = [&](int a, int b) {
    std::string t = "{";
    for (int k = a; k <= b; ++k) {
      t += std::to_string(k + 1);
      if (k < b) t += ",";
    }
    return t + "}";
  };
  char line[256];
  const std::string root = set(0, N - 1);
  snprintf(line, sizeof line, "root %s split S=%d\n", root.c_str(), S);
  s += line;
  for (int side = 0; side < 2; ++side) {
    int a = side == 0 ? 0 : S, b = side == 0 ? S - 1 : N - 1;
    snprintf(line, sizeof line, "PM %s -> %s\n", root.c_str(), set(a, b).c_str());
    s += line;
    for (int c = a; c < b; ++c) {
      snprintf(line, sizeof line, "mTTV %s -> %s\n", set(c, b).c_str(), set(c, c).c_str());
      s += line;
      snprintf(line, sizeof line, "mTTV %s -> %s\n", set(c, b).c_str(), set(c + 1, b).c_str());
      s += line;
    }
  }
  if (s.size() + 1 > len) return fail(nullptr, PLANC_E_INVALID, "buffer too small");
  snprintf(buf, len, "%s", s.c_str());
  return PLANC_OK;
}

planc_status_t planc_sqnorm(planc_t ctx, double* alpha) {
  if (!ctx) return PLANC_E_INVALID;
  if (!alpha) return fail(ctx, PLANC_E_INVALID, "alpha is NULL");
  int nb = sqnorm_blocks(ctx->I, ctx->sm_count);
  CK(launch_sqnorm(ctx->xd, ctx->X, ctx->I, ctx->red, nb, alpha, ctx->stream), "sqnorm launch");
  return PLANC_OK;
}

planc_status_t planc_mttkrp(planc_t ctx, void* const* H, int n, void* M) {
  if (!ctx) return PLANC_E_INVALID;
  if (!H || !M) return fail(ctx, PLANC_E_INVALID, "H or M is NULL");
  if (n < 0 || n >= ctx->N) return fail(ctx, PLANC_E_INVALID, "mode %d out of range", n);
  for (int k = 0; k < ctx->N; ++k)
    if (k != n && !H[k]) return fail(ctx, PLANC_E_INVALID, "H[%d] is NULL", k);
  const void* cur = nullptr;
  int cf = 0;
  return dt_mode(ctx, H, n, M, &cur, &cf);
}

planc_status_t planc_mttkrp_all(planc_t ctx, void* const* H, void* const* M) {
  if (!ctx) return PLANC_E_INVALID;
  if (!H || !M) return fail(ctx, PLANC_E_INVALID, "H or M is NULL");
  for (int k = 0; k < ctx->N; ++k)
    if (!H[k] || !M[k]) return fail(ctx, PLANC_E_INVALID, "NULL factor or output pointer");
  // one walk of the tree at fixed factors: each root partial MTTKRP once, the
  // multi-TTV chains of a branch reuse its nodes mode after mode
  const void* cur[2] = {nullptr, nullptr};
  int cf[2] = {0, 0};
  planc_status_t st;
  for (int n = 0; n < ctx->N; ++n) {
    const int s = side_of(ctx, n);
    if ((st = dt_mode(ctx, H, n, M[n], &cur[s], &cf[s])) != PLANC_OK) return st;
  }
  return PLANC_OK;
}

planc_status_t planc_partial_mttkrp(planc_t ctx, void* const* H, int side, void* T) {
  if (!ctx) return PLANC_E_INVALID;
  if (!H || !T || (side != 0 && side != 1)) return fail(ctx, PLANC_E_INVALID, "bad arguments");
  // the Khatri-Rao operand of a branch is built from the other branch's modes
  for (int k = side_a(ctx, 1 - side); k <= side_b(ctx, 1 - side); ++k)
    if (!H[k]) return fail(ctx, PLANC_E_INVALID, "H[%d] is NULL", k);
  return run_pm(ctx, H, side, T, false);
}

planc_status_t planc_gram_hadamard(planc_t ctx, const double* G, int n, double* S) {
  if (!ctx) return PLANC_E_INVALID;
  if (!G || !S || n < 0 || n >= ctx->N) return fail(ctx, PLANC_E_INVALID, "bad arguments");
  CK(launch_gram_hadamard(G, ctx->N, n, ctx->R, S, ctx->stream), "gram_hadamard launch");
  return PLANC_OK;
}

static planc_status_t gram_impl(planc_t ctx, int64_t rows, void* H, double* G, double* lambda,
                                bool scale, const void* M, double* dot_part_out) {
  const int R = ctx->R;
  const int nb = rowblocks(rows);
  double* colsq = ctx->red;
  double* dotp = colsq + (size_t)nb * R;
  double* gpart = dotp + nb;
  if (scale)
    CK(launch_colsq(is_f64(ctx), rows, R, H, M, colsq, dotp, nb, ctx->stream), "colsq launch");
  CK(launch_scale_gram(is_f64(ctx), rows, R, H, colsq, nb, lambda, gpart, scale, ctx->stream),
     "scale/gram launch");
  if (G) {
    // the solver's own Grams also keep their FP32 copy (read by the fused mode update)
    float* Gf = (G >= ctx->G && G < ctx->G + (size_t)ctx->N * R * R) ? ctx->Gf + (G - ctx->G)
                                                                        : nullptr;
    CK(launch_gram_reduce(R, gpart, nb, G, Gf, ctx->stream), "gram reduce launch");
  }
  (void)dot_part_out;
  return PLANC_OK;
}

planc_status_t planc_gram(planc_t ctx, int64_t rows, const void* H, double* G) {
  if (!ctx) return PLANC_E_INVALID;
  if (!H || !G || rows < 1) return fail(ctx, PLANC_E_INVALID, "bad arguments");
  if (ctx->R > PLANC_MAX_NLS_R) return fail(ctx, PLANC_E_UNSUPPORTED, "Gram needs R <= %d", PLANC_MAX_NLS_R);
  if (rows > ctx->max_dim) return fail(ctx, PLANC_E_SHAPE, "rows > largest mode");
  return gram_impl(ctx, rows, const_cast<void*>(H), G, nullptr, false, nullptr, nullptr);
}

planc_status_t planc_normalize(planc_t ctx, int64_t rows, void* H, double* lambda, double* G) {
  if (!ctx) return PLANC_E_INVALID;
  if (!H || !lambda || rows < 1) return fail(ctx, PLANC_E_INVALID, "bad arguments");
  if (ctx->R > PLANC_MAX_NLS_R) return fail(ctx, PLANC_E_UNSUPPORTED, "needs R <= %d", PLANC_MAX_NLS_R);
  if (rows > ctx->max_dim) return fail(ctx, PLANC_E_SHAPE, "rows > largest mode");
  return gram_impl(ctx, rows, H, G, lambda, true, nullptr, nullptr);
}

planc_status_t planc_nls_update(planc_t ctx, planc_nls_t alg, const planc_nls_opts* opts,
                                int64_t rows, const double* S, const void* M, void* H, void* aux,
                                int32_t* inner_iters) {
  if (!ctx) return PLANC_E_INVALID;
  if (!S || !M || !H || rows < 1) return fail(ctx, PLANC_E_INVALID, "bad arguments");
  if ((int)alg < 0 || (int)alg > 6) return fail(ctx, PLANC_E_INVALID, "unknown NNLS algorithm");
  if (ctx->R > PLANC_MAX_NLS_R) return fail(ctx, PLANC_E_UNSUPPORTED, "NNLS needs R <= %d", PLANC_MAX_NLS_R);
  if (rows > ctx->max_dim) return fail(ctx, PLANC_E_SHAPE, "rows > largest mode");
  NlsArgs a;
  a.alg = alg;
  a.opts = opts ? *opts : planc_nls_opts_default();
  a.rows = rows;
  a.R = ctx->R;
  a.S = S;
  a.M = M;
  a.H = H;
  a.lambda = nullptr;
  a.U = aux ? aux : ctx->Ubuf;
  a.U_zero = aux == nullptr;
  a.V = ctx->Vbuf;
  a.inner = inner_iters;
  a.scratch = ctx->nls_scr;
  a.flags = ctx->flags;
  a.f64 = is_f64(ctx);
  CK(launch_nls(a, ctx->stream), "NNLS launch");
  return PLANC_OK;
}

planc_status_t planc_fit(planc_t ctx, void* const* H, const double* lambda, double* rel_err,
                         double* fit) {
  if (!ctx) return PLANC_E_INVALID;
  if (!H || !lambda) return fail(ctx, PLANC_E_INVALID, "bad arguments");
  for (int k = 0; k < ctx->N; ++k)
    if (!H[k]) return fail(ctx, PLANC_E_INVALID, "H[%d] is NULL", k);
  if (ctx->R > PLANC_MAX_NLS_R) return fail(ctx, PLANC_E_UNSUPPORTED, "fit needs R <= %d", PLANC_MAX_NLS_R);
  const int N = ctx->N, R = ctx->R;
  planc_status_t st;
  if ((st = planc_sqnorm(ctx, ctx->scal)) != PLANC_OK) return st;
  if ((st = planc_mttkrp(ctx, H, N - 1, ctx->Mbuf)) != PLANC_OK) return st;
  for (int k = 0; k < N; ++k)
    if ((st = gram_impl(ctx, ctx->dims[k], H[k], ctx->G + (size_t)k * R * R, nullptr, false,
                        nullptr, nullptr)) != PLANC_OK)
      return st;
  const int64_t rows = ctx->dims[N - 1];
  const int nb = rowblocks(rows);
  double* dotp = ctx->red + (size_t)nb * R;
  CK(launch_dot_lambda(is_f64(ctx), rows, R, ctx->Mbuf, H[N - 1], lambda, dotp, nb, ctx->stream),
     "dot launch");
  CK(launch_fit(R, ctx->G, N, lambda, dotp, nb, ctx->scal, ctx->scal + 8, ctx->stream),
     "fit launch");
  double out[3];
  CK(cudaMemcpyAsync(out, ctx->scal + 8, sizeof out, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  if (rel_err) *rel_err = out[0];
  if (fit) *fit = 1.0 - out[0];
  return PLANC_OK;
}

}  // extern "C"

// ---- outer loop ---------------------------------------------------------------------
namespace {

__global__ void record_kernel(const double* __restrict__ fit3, double* __restrict__ hist,
                              const int32_t* __restrict__ inner_now, int32_t* __restrict__ inner_hist,
                              int N, int* __restrict__ counter, int cap_iters) {
  pdl_wait();
  int it = *counter;
  if (it < cap_iters) {
    hist[3 * it + 0] = fit3[0];
    hist[3 * it + 1] = fit3[1];
    hist[3 * it + 2] = fit3[2];
    for (int n = 0; n < N; ++n) inner_hist[it * N + n] = inner_now[n];
  }
  *counter = it + 1;
}

// Outer acceleration of the Nesterov-type solve (Sec. 4.3.5, Eq. nesouterupd),
// after the error of the iteration is in scal[8]: the candidate
// [F_i + s_i (F_i - F_{i-1})]_+ (lambda absorbed into the last mode), its
// normalisation (column norms multiplied into lambda_c) and Grams, one
// MTTKRP for its last mode, its error by the identity of Alg. 4 in
// scal[16], then the decision (never on the first iteration, which only
// stores the previous iterate) and the copy of the accepted iterate into
// H, lambda, G and the previous iterate.
planc_status_t accelerate(planc_t ctx, void* const* H, const int* counter) {
  const int N = ctx->N, R = ctx->R;
  const bool f64 = is_f64(ctx);
  AccelModes t;
  t.N = N;
  t.R = R;
  t.off[0] = 0;
  for (int k = 0; k < N; ++k) {
    t.off[k + 1] = t.off[k] + ctx->dims[k] * R;
    t.H[k] = H[k];
    t.Hp[k] = ctx->Hprev[k];
    t.Hc[k] = ctx->Hcand[k];
  }
  CK(launch_accel_extrapolate(f64, t, ctx->lam, ctx->lam_prev, counter, ctx->stream),
     "extrapolate launch");
  planc_status_t st;
  for (int k = 0; k < N; ++k)
    if ((st = gram_impl(ctx, ctx->dims[k], ctx->Hcand[k], ctx->Gc + (size_t)k * R * R,
                        ctx->nu + (size_t)k * R, true, nullptr, nullptr)) != PLANC_OK)
      return st;
  CK(launch_accel_finish(f64, t, ctx->nu, ctx->lam_cand, ctx->stream), "lambda launch");
  const void* cur = nullptr;
  int cf = 0;
  if ((st = dt_mode(ctx, ctx->Hcand, N - 1, ctx->Mbuf, &cur, &cf)) != PLANC_OK) return st;
  const int64_t rows = ctx->dims[N - 1];
  const int nb = rowblocks(rows);
  double* dotp = ctx->red + (size_t)nb * R;
  CK(launch_dot_lambda(f64, rows, R, ctx->Mbuf, ctx->Hcand[N - 1], ctx->lam_cand, dotp, nb,
                       ctx->stream), "dot launch");
  CK(launch_fit(R, ctx->Gc, N, ctx->lam_cand, dotp, nb, ctx->scal, ctx->scal + 16, ctx->stream),
     "fit launch");
  CK(launch_accel_select(f64, t, ctx->scal, counter, ctx->accel_hist, ctx->hist_cap / 3,
                         ctx->flags, ctx->lam, ctx->lam_prev, ctx->lam_cand, ctx->G, ctx->Gf,
                         ctx->Gc, ctx->stream), "select launch");
  return PLANC_OK;
}

// One outer iteration (Alg. 1 "for n = 1 to N" with Alg. 4's normalisation
// and error).  Every pointer it touches is fixed across iterations, so the
// whole sequence can be captured once as a CUDA graph and replayed.
planc_status_t outer_iteration(planc_t ctx, const planc_solve_opts& o, void* const* H) {
  const int N = ctx->N, R = ctx->R;
  const void* cur[2] = {nullptr, nullptr};
  int cf[2] = {0, 0};
  int* counter = ctx->flags + 4;
  int32_t* inner_now = ctx->inner + ctx->inner_cap - PLANC_MAX_N;
  planc_status_t st;
  const bool accel = o.alg == PLANC_NES && o.nes_accel;
  bool recorded = false;
  for (int n = 0; n < N; ++n) {
    const int s = side_of(ctx, n);
    const bool fused = ctx->fused_modes && mode_fused_eligible(o.alg, ctx->dims[n], R, is_f64(ctx));
    const bool prepared = o.alg == PLANC_NES || o.alg == PLANC_UCP || o.alg == PLANC_ADMM ||
                          o.alg == PLANC_BPP;
    const bool fork = fused && prepared && ctx->side;
    auto prep = [&](cudaStream_t sp) -> planc_status_t {
      CK(launch_gram_hadamard(ctx->G, N, n, R, ctx->Sm, sp), "gram_hadamard launch");
      if (o.alg == PLANC_NES)
        CK(launch_nes_prep(is_f64(ctx), ctx->Sm, R, ctx->nls_scr, sp), "NES prep launch");
      else if (o.alg == PLANC_BPP)  // the exchange count starts from zero
        CK(launch_set_int(inner_now + n, 0, 1, sp), "inner reset launch");
      else  // UCP: S^{-1}; ADMM: (S + rho I)^{-1}
        CK(launch_inv_prep(is_f64(ctx), ctx->Sm, R, ctx->nls_scr, o.alg == PLANC_UCP ? 1 : 0, sp),
           "inverse prep launch");
      return PLANC_OK;
    };
    if (fork) {
      // S^(n) and what the update prepares from it (the Nesterov parameters,
      // or S^{-1} for UCP) need only the Grams: they run on the side stream
      // while the MTTKRP of mode n runs
      CK(cudaEventRecord(ctx->ev_fork, ctx->stream), "fork record");
      CK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0), "fork wait");
      if ((st = prep(ctx->side)) != PLANC_OK) return st;
      CK(cudaEventRecord(ctx->ev_join, ctx->side), "join record");
    }
    if ((st = dt_mode(ctx, H, n, ctx->Mbuf, &cur[s], &cf[s])) != PLANC_OK) return st;
    const bool last = n == N - 1;
    if (fused) {
      if (prepared) {
        if (fork) {
          CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0), "join wait");
        } else if ((st = prep(ctx->stream)) != PLANC_OK) {
          return st;
        }
      }
      if (o.alg == PLANC_BPP) {
        // BPP solves the rows (one warp each; the passive systems through
        // S^{-1} or a factorisation); the cluster launch below then does the
        // rest of the mode
        NlsArgs a;
        a.alg = PLANC_BPP;
        a.opts = o.nls;
        a.rows = ctx->dims[n];
        a.R = R;
        a.S = ctx->Sm;
        a.M = ctx->Mbuf;
        a.H = H[n];
        a.lambda = ctx->lam;  // warm start H^(n) diag(lambda)
        a.inner = inner_now + n;
        a.reset_inner = false;
        a.scratch = ctx->nls_scr;
        a.flags = ctx->flags;
        a.f64 = is_f64(ctx);
        CK(launch_nls(a, ctx->stream), "NNLS launch");
      }
      // one launch: S^(n), NNLS, lambda, normalisation, G^(n) (+ error after
      // mode N, and then the history record unless an acceleration follows)
      RecArgs rec;
      if (last && !accel) {
        rec.hist = ctx->hist;
        rec.inner_now = inner_now;
        rec.inner_hist = ctx->inner;
        rec.counter = counter;
        rec.N = N;
        rec.cap = ctx->hist_cap / 3;
        recorded = true;
      }
      CK(launch_mode_fused(is_f64(ctx), ctx->dims[n], R, N, n, ctx->G, ctx->Gf, ctx->Mbuf, H[n],
                           ctx->lam, o.alg, o.nls, inner_now + n, ctx->scal,
                           last ? ctx->scal + 8 : nullptr, ctx->tc_err, ctx->nls_scr, rec,
                           ctx->flags, ctx->stream),
         "fused mode update launch");
      continue;
    }
    CK(launch_gram_hadamard(ctx->G, N, n, R, ctx->Sm, ctx->stream), "gram_hadamard launch");
    NlsArgs a;
    a.alg = o.alg;
    a.opts = o.nls;
    a.rows = ctx->dims[n];
    a.R = R;
    a.S = ctx->Sm;
    a.M = ctx->Mbuf;
    a.H = H[n];
    a.lambda = ctx->lam;  // warm start H^(n) diag(lambda)
    a.U = ctx->Ubuf;
    a.U_zero = true;
    a.V = ctx->Vbuf;
    a.inner = inner_now + n;
    a.scratch = ctx->nls_scr;
    a.flags = ctx->flags;
    a.f64 = is_f64(ctx);
    CK(launch_nls(a, ctx->stream), "NNLS launch");
    // normalise, lambda, G^(n); after the last mode the error identity
    const int64_t rows = ctx->dims[n];
    const int nb = rowblocks(rows);
    double* colsq = ctx->red;
    double* dotp = colsq + (size_t)nb * R;
    double* gpart = dotp + nb;
    CK(launch_colsq(is_f64(ctx), rows, R, H[n], last ? ctx->Mbuf : nullptr, colsq, dotp, nb,
                    ctx->stream), "colsq launch");
    CK(launch_scale_gram(is_f64(ctx), rows, R, H[n], colsq, nb, ctx->lam, gpart, true,
                         ctx->stream), "scale/gram launch");
    CK(launch_gram_reduce(R, gpart, nb, ctx->G + (size_t)n * R * R, ctx->Gf + (size_t)n * R * R,
                          ctx->stream),
       "gram reduce launch");
    if (last)
      CK(launch_fit(R, ctx->G, N, ctx->lam, dotp, nb, ctx->scal, ctx->scal + 8, ctx->stream),
         "fit launch");
  }
  if (accel && (st = accelerate(ctx, H, counter)) != PLANC_OK) return st;
  if (!recorded) {
    CK(launch_pdl(record_kernel, dim3(1), dim3(1), 0, ctx->stream, (const double*)(ctx->scal + 8),
                  ctx->hist, (const int32_t*)inner_now, ctx->inner, N, counter, ctx->hist_cap / 3),
       "record launch");
    note_launches(1);
  }
  return PLANC_OK;
}

}  // namespace

extern "C" {

planc_status_t planc_nncp_solve(planc_t ctx, const planc_solve_opts* opts, void* const* H,
                                double* lambda, planc_report* report) {
  if (!ctx) return PLANC_E_INVALID;
  planc_solve_opts o = opts ? *opts : planc_solve_opts_default();
  if (!H) return fail(ctx, PLANC_E_INVALID, "H is NULL");
  for (int k = 0; k < ctx->N; ++k)
    if (!H[k]) return fail(ctx, PLANC_E_INVALID, "H[%d] is NULL", k);
  if (o.iters < 0) return fail(ctx, PLANC_E_INVALID, "iters < 0");
  if ((int)o.alg < 0 || (int)o.alg > 6) return fail(ctx, PLANC_E_INVALID, "unknown NNLS algorithm");
  if (ctx->R > PLANC_MAX_NLS_R) return fail(ctx, PLANC_E_UNSUPPORTED, "solve needs R <= %d", PLANC_MAX_NLS_R);
  const int N = ctx->N, R = ctx->R;
  const int cap_iters = std::min(ctx->hist_cap / 3, (ctx->inner_cap - PLANC_MAX_N) / N);
  if (o.iters > cap_iters) return fail(ctx, PLANC_E_INVALID, "iters > %d", cap_iters);
  planc_status_t st;
  const long long c_start = launch_count();
  long long launches = 0;

  // initialise: alpha, lambda = 1, G^(n) of the initial factors (Alg. 4)
  if ((st = planc_sqnorm(ctx, ctx->scal)) != PLANC_OK) return st;
  CK(launch_fill(ctx->lam, 1.0, R, ctx->stream), "fill launch");
  for (int k = 0; k < N; ++k)
    if ((st = gram_impl(ctx, ctx->dims[k], H[k], ctx->G + (size_t)k * R * R, nullptr, false,
                        nullptr, nullptr)) != PLANC_OK)
      return st;
  CK(cudaMemsetAsync(ctx->flags, 0, 16 * sizeof(int), ctx->stream), "memset");
  CK(cudaMemsetAsync(ctx->hist, 0, (size_t)ctx->hist_cap * 8, ctx->stream), "memset");
  CK(cudaMemsetAsync(ctx->accel_hist, 0, (size_t)(ctx->hist_cap / 3) * 4, ctx->stream), "memset");

  if ((o.alg == PLANC_NES || o.alg == PLANC_UCP || o.alg == PLANC_ADMM) &&
      ctx->side == nullptr && ctx->stream != nullptr) {
    CK(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking), "side stream");
    CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming), "event create");
    CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming), "event create");
  }
  ctx->profiling = o.profile != 0;
  ctx->ev_used = 0;
  if (ctx->profiling) {
    size_t need = (size_t)4 * std::max(1, o.iters);
    while (ctx->ev.size() < need) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e), "event create");
      ctx->ev.push_back(e);
    }
  }
  const bool graph = o.use_graph && !ctx->profiling && o.tol <= 0.0 && o.iters > 1 &&
                     ctx->stream != nullptr;  // the legacy stream cannot be captured
  cudaGraphExec_t exec = nullptr;
  int done = 0;
  if (graph) {
    cudaGraph_t g = nullptr;
    const long long c0 = launch_count();
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    st = outer_iteration(ctx, o, H);
    cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
    launches = (c0 - c_start) + (launch_count() - c0) * (long long)o.iters;
    if (st != PLANC_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "end capture");
    ce = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "graph instantiate");
    for (int it = 0; it < o.iters; ++it) {
      ce = cudaGraphLaunch(exec, ctx->stream);
      if (ce != cudaSuccess) { cudaGraphExecDestroy(exec); return cuda_fail(ctx, ce, "graph launch"); }
    }
    done = o.iters;
    cudaGraphExecDestroy(exec);
  } else {
    for (int it = 0; it < o.iters; ++it) {
      if ((st = outer_iteration(ctx, o, H)) != PLANC_OK) { ctx->profiling = false; return st; }
      ++done;
      if (o.tol > 0.0) {
        double e3[3];
        CK(cudaMemcpyAsync(e3, ctx->scal + 8, sizeof e3, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
        CK(cudaStreamSynchronize(ctx->stream), "sync");
        if (e3[0] <= o.tol) break;
      }
    }
    launches = launch_count() - c_start;
  }
  ctx->profiling = false;

  // results
  std::vector<double> hist((size_t)3 * std::max(done, 1), 0.0);
  std::vector<int32_t> inner((size_t)N * std::max(done, 1), 0);
  std::vector<int32_t> accel((size_t)std::max(done, 1), 0);
  int flags[16];
  if (lambda) CK(cudaMemcpyAsync(lambda, ctx->lam, R * 8, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  if (done > 0) {
    CK(cudaMemcpyAsync(hist.data(), ctx->hist, (size_t)3 * done * 8, cudaMemcpyDeviceToHost,
                       ctx->stream), "D2H");
    CK(cudaMemcpyAsync(inner.data(), ctx->inner, (size_t)N * done * 4, cudaMemcpyDeviceToHost,
                       ctx->stream), "D2H");
    CK(cudaMemcpyAsync(accel.data(), ctx->accel_hist, (size_t)done * 4, cudaMemcpyDeviceToHost,
                       ctx->stream), "D2H");
  }
  int tc_err = 0;
  CK(cudaMemcpyAsync(flags, ctx->flags, sizeof flags, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  CK(cudaMemcpyAsync(&tc_err, ctx->tc_err, sizeof tc_err, cudaMemcpyDeviceToHost, ctx->stream),
     "D2H");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  if (report) {
    report->iters_done = done;
    report->rel_err = done > 0 ? hist[3 * (done - 1)] : 0.0;
    report->fit = 1.0 - report->rel_err;
    if (report->rel_err_hist)
      for (int i = 0; i < done; ++i) report->rel_err_hist[i] = hist[3 * i];
    if (report->inner_hist)
      for (int i = 0; i < done * N; ++i) report->inner_hist[i] = inner[i];
    report->bpp_unconverged = flags[0];
    report->accel_accepted = flags[6];
    if (report->accel_hist)
      for (int i = 0; i < done; ++i) report->accel_hist[i] = accel[i];
    report->launches = launches;
    report->pm_tensor_cores = (ctx->use_tc[0] ? 1 : 0) | (ctx->use_tc[1] ? 2 : 0);
    report->pm_ms = 0.f;
    report->pm_launches = 0;
    for (int i = 0; i + 1 < ctx->ev_used; i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]) == cudaSuccess) {
        report->pm_ms += ms;
        report->pm_launches += 1;
      }
    }
  }
  if (tc_err != 0)
    return fail(ctx, PLANC_E_TIMEOUT,
                "a pipeline wait gave up (code %d: 1-3, 21-31, 41-45 partial MTTKRP, 10 mode update)", tc_err);
  if (flags[1] != 0)
    return fail(ctx, PLANC_E_NUMERIC, "S is not positive definite: %d inversion(s) met a non-positive pivot", flags[1]);
  return PLANC_OK;
}

planc_status_t planc_cp_grad(planc_t ctx, void* const* H, void* const* dH, double* loss) {
  if (!ctx) return PLANC_E_INVALID;
  if (!H || !dH) return fail(ctx, PLANC_E_INVALID, "bad arguments");
  const int N = ctx->N, R = ctx->R;
  for (int k = 0; k < N; ++k)
    if (!H[k] || !dH[k]) return fail(ctx, PLANC_E_INVALID, "NULL factor or gradient pointer");
  if (R > PLANC_MAX_NLS_R) return fail(ctx, PLANC_E_UNSUPPORTED, "cp_grad needs R <= %d", PLANC_MAX_NLS_R);
  planc_status_t st;
  // M^(n) of the given factors into dH[n]: the root partial MTTKRPs run once
  // each and the multi-TTV chains are recomputed per mode (Alg. 3 with the
  // factors held fixed), so no node is kept beyond its branch
  if ((st = planc_mttkrp_all(ctx, H, dH)) != PLANC_OK) return st;
  if (ctx->max_dim <= 4096) {  // every Gram in one launch (a row loop per entry)
    CK(launch_gram_all(is_f64(ctx), N, ctx->dims, R, H, ctx->G, ctx->Gf, ctx->stream),
       "Gram launch");
  } else {
    for (int k = 0; k < N; ++k)
      if ((st = gram_impl(ctx, ctx->dims[k], H[k], ctx->G + (size_t)k * R * R, nullptr, false,
                          nullptr, nullptr)) != PLANC_OK)
        return st;
  }
  if (loss) {
    // f = ||X||^2 - 2 <M^(N), H^(N)> + 1^T (G^(1) * ... * G^(N)) 1  (lambda = 1);
    // ||X||^2 once per context (X is borrowed unchanged; the context's scalar
    // slot 0 only ever holds it)
    if (ctx->grad_alpha < 0.0 && (st = planc_sqnorm(ctx, ctx->scal)) != PLANC_OK) return st;
    CK(launch_fill(ctx->lam, 1.0, R, ctx->stream), "fill launch");
    const int64_t rows = ctx->dims[N - 1];
    const int nb = rowblocks(rows);
    double* dotp = ctx->red + (size_t)nb * R;
    CK(launch_dot_lambda(is_f64(ctx), rows, R, dH[N - 1], H[N - 1], ctx->lam, dotp, nb,
                         ctx->stream),
       "dot launch");
    CK(launch_fit(R, ctx->G, N, ctx->lam, dotp, nb, ctx->scal, ctx->scal + 8, ctx->stream),
       "fit launch");
  }
  // every mode's gradient rows in one launch (S^(n) formed per CTA)
  CK(launch_cp_grad_all(is_f64(ctx), N, ctx->dims, R, H, dH, ctx->G, ctx->Gf, ctx->sm_count,
                        ctx->stream),
     "gradient launch");
  if (loss) {
    double h[11] = {0};
    CK(cudaMemcpyAsync(h, ctx->scal, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
    CK(cudaStreamSynchronize(ctx->stream), "sync");
    ctx->grad_alpha = h[0];
    *loss = h[0] - 2.0 * h[9] + h[10];
  }
  return PLANC_OK;
}

}  // extern "C"
