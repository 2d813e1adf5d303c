// NNLS-Update kernels (Sec. 4.3): MU, HALS, ADMM, BPP, the Nesterov-type
// update, projected gradient and the unconstrained update, all in the row
// form of Eq. nls (rows of Hhat are independent, given S = K^T K and
// M = X_(n) K).
//
// MU, HALS, ADMM steps and PGD keep one row per thread with the row in
// registers (R padded to RP in {16, 32, 64}) and S (or the ADMM inverse) in
// shared memory, read as warp-wide broadcasts.  BPP gives each row a warp
// and does its passive-set Cholesky solves in FP64.  ADMM (and UCP) invert
// S + rho I once per call in FP64 and keep the explicit inverse for the row
// solves.
#include <algorithm>

#include "internal.h"

namespace planc {

namespace {

constexpr int ROWS_PER_CTA = 32;  // one warp per CTA: rows spread over many SMs

// Stage S (FP64, R x R) into shared memory as TA, zero-padded to RP x RP.
template <typename TA, int RP>
__device__ __forceinline__ void stage_S(TA* Ss, const double* __restrict__ S, int R) {
  for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
    int i = e / RP, j = e - i * RP;
    Ss[e] = (i < R && j < R) ? (TA)S[i * R + j] : TA(0);
  }
}

template <typename TA, int RP>
__device__ __forceinline__ void load_row(TA* v, const TA* __restrict__ src, int64_t row, int R,
                                         const double* __restrict__ lam) {
#pragma unroll
  for (int k = 0; k < RP; ++k) {
    TA x = TA(0);
    if (k < R) {
      x = src[row * R + k];
      if (lam) x = (TA)((double)x * lam[k]);
    }
    v[k] = x;
  }
}

// d = sum_k v[k] * Srow[k], four independent chains
template <typename TA, int RP>
__device__ __forceinline__ TA dot_row(const TA* v, const TA* Srow) {
  TA a0 = TA(0), a1 = TA(0), a2 = TA(0), a3 = TA(0);
#pragma unroll
  for (int k = 0; k < RP; k += 4) {
    a0 = fma(v[k + 0], Srow[k + 0], a0);
    a1 = fma(v[k + 1], Srow[k + 1], a1);
    a2 = fma(v[k + 2], Srow[k + 2], a2);
    a3 = fma(v[k + 3], Srow[k + 3], a3);
  }
  return (a0 + a1) + (a2 + a3);
}

// Per-thread row storage in shared memory: element k of the calling thread's
// row lives at v[k * ROWS_PER_CTA + lane] (each lane its own bank).
template <typename TA>
__device__ __forceinline__ TA& rowv(TA* v, int k) { return v[k * ROWS_PER_CTA + threadIdx.x]; }

// ---- MU (Eq. muupd): H <- H * M / (H S + eps) ---------------------------------------
template <typename TA, int RP>
__global__ void __launch_bounds__(ROWS_PER_CTA)
nls_mu_kernel(int64_t rows, int R, const double* __restrict__ S, const TA* __restrict__ M,
              TA* __restrict__ H, const double* __restrict__ lam, double eps) {
  __shared__ __align__(16) TA Ss[RP * RP];
  stage_S<TA, RP>(Ss, S, R);
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  TA h[RP];
  load_row<TA, RP>(h, H, i, R, lam);
#pragma unroll 1
  for (int r = 0; r < R; ++r) {
    TA d = dot_row<TA, RP>(h, Ss + r * RP);
    TA hr = H[i * R + r];
    if (lam) hr = (TA)((double)hr * lam[r]);
    H[i * R + r] = hr * M[i * R + r] / (d + (TA)eps);
  }
}

// ---- HALS (Eq. halsupd): one Gauss-Seidel sweep over the columns ----------------------
template <typename TA, int RP>
__global__ void __launch_bounds__(ROWS_PER_CTA)
nls_hals_kernel(int64_t rows, int R, const double* __restrict__ S, const TA* __restrict__ M,
                TA* __restrict__ H, const double* __restrict__ lam, double tiny) {
  __shared__ __align__(16) TA Ss[RP * RP];
  __shared__ TA hv[RP * ROWS_PER_CTA];
  stage_S<TA, RP>(Ss, S, R);
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < rows;
  for (int k = 0; k < RP; ++k) {
    TA x = TA(0);
    if (live && k < R) {
      x = H[i * R + k];
      if (lam) x = (TA)((double)x * lam[k]);
    }
    rowv(hv, k) = x;
  }
  __syncthreads();
  if (!live) return;
#pragma unroll 1
  for (int r = 0; r < R; ++r) {
    TA srr = Ss[r * RP + r];
    if (srr > (TA)tiny) {
      const TA* Sr = Ss + r * RP;
      TA a0 = TA(0), a1 = TA(0), a2 = TA(0), a3 = TA(0);
#pragma unroll
      for (int k = 0; k < RP; k += 4) {
        a0 = fma(rowv(hv, k + 0), Sr[k + 0], a0);
        a1 = fma(rowv(hv, k + 1), Sr[k + 1], a1);
        a2 = fma(rowv(hv, k + 2), Sr[k + 2], a2);
        a3 = fma(rowv(hv, k + 3), Sr[k + 3], a3);
      }
      TA d = (a0 + a1) + (a2 + a3);
      TA v = rowv(hv, r) + (M[i * R + r] - d) / srr;
      rowv(hv, r) = v > TA(0) ? v : TA(0);
    }
  }
  for (int r = 0; r < R; ++r) H[i * R + r] = rowv(hv, r);
}

// ---- projected gradient: H <- [H - eta (H S - M)]_+, eta = 1 / ||S||_F --------------
template <typename TA, int RP>
__global__ void __launch_bounds__(ROWS_PER_CTA)
nls_pgd_kernel(int64_t rows, int R, const double* __restrict__ S, const TA* __restrict__ M,
               TA* __restrict__ H, const double* __restrict__ lam, int steps) {
  __shared__ __align__(16) TA Ss[RP * RP];
  __shared__ TA hv[RP * ROWS_PER_CTA];
  stage_S<TA, RP>(Ss, S, R);
  // eta = 1 / ||S||_F; every lane holds the warp-wide sum (one warp per CTA)
  double f = 0.0;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) f += S[e] * S[e];
  f = warp_sum(f);
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const TA eta = (TA)(1.0 / fmax(sqrt(f), 1e-300));
  TA h[RP];
  load_row<TA, RP>(h, H, i, R, lam);
#pragma unroll
  for (int k = 0; k < RP; ++k) rowv(hv, k) = h[k];
  for (int st = 0; st < steps; ++st) {
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
      TA g = dot_row<TA, RP>(h, Ss + r * RP) - M[i * R + r];
      TA x = rowv(hv, r) - eta * g;
      rowv(hv, r) = x > TA(0) ? x : TA(0);
    }
#pragma unroll
    for (int k = 0; k < RP; ++k) h[k] = rowv(hv, k);
  }
  for (int r = 0; r < R; ++r) H[i * R + r] = rowv(hv, r);
}

// Projected gradient with one warp per row (R <= 64; used when the factor has
// few rows, so that one thread per row would leave the GPU idle): lane l owns
// columns l and l + 32; each step forms g = S h - m from the row's iterate,
// broadcast from shared memory, and column l of S (S is symmetric, so lanes
// read consecutive words), then h = max(0, h - eta g) with eta = 1 / ||S||_F.
constexpr int PGDW_WARPS = 8;

template <typename TA>
__global__ void __launch_bounds__(32 * PGDW_WARPS)
nls_pgd_warp_kernel(int64_t rows, int R, const double* __restrict__ S,
                    const TA* __restrict__ M, TA* __restrict__ H,
                    const double* __restrict__ lam, int steps) {
  constexpr int RP = 64;
  __shared__ __align__(16) TA Ss[RP * RP];
  __shared__ TA hw[PGDW_WARPS][RP];
  __shared__ double s_f[PGDW_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double f = 0.0;
  for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
    const int i = e / RP, j = e - i * RP;
    const double v = (i < R && j < R) ? S[i * R + j] : 0.0;
    Ss[e] = (TA)v;
    f = fma(v, v, f);
  }
  f = warp_sum(f);
  if (lane == 0) s_f[warp] = f;
  __syncthreads();
  f = 0.0;
#pragma unroll
  for (int w = 0; w < PGDW_WARPS; ++w) f += s_f[w];
  const int64_t row = (int64_t)blockIdx.x * PGDW_WARPS + warp;
  if (row >= rows) return;  // (no block-wide barrier follows)
  const TA eta = (TA)(1.0 / fmax(sqrt(f), 1e-300));
  const int c0 = lane, c1 = lane + 32;
  const bool v0 = c0 < R, v1 = c1 < R;
  TA h0 = v0 ? (TA)((double)H[row * R + c0] * (lam ? lam[c0] : 1.0)) : TA(0);
  TA h1 = v1 ? (TA)((double)H[row * R + c1] * (lam ? lam[c1] : 1.0)) : TA(0);
  const TA m0 = v0 ? M[row * R + c0] : TA(0), m1 = v1 ? M[row * R + c1] : TA(0);
  TA* hr = hw[warp];
  for (int st = 0; st < steps; ++st) {
    hr[c0] = h0;
    hr[c1] = h1;
    __syncwarp();
    TA g0a = TA(0), g0b = TA(0), g1a = TA(0), g1b = TA(0);
    int k = 0;
    for (; k + 2 <= R; k += 2) {
      const TA ha = hr[k], hb = hr[k + 1];
      g0a = fma(Ss[k * RP + c0], ha, g0a);
      g1a = fma(Ss[k * RP + c1], ha, g1a);
      g0b = fma(Ss[(k + 1) * RP + c0], hb, g0b);
      g1b = fma(Ss[(k + 1) * RP + c1], hb, g1b);
    }
    if (k < R) {
      const TA ha = hr[k];
      g0a = fma(Ss[k * RP + c0], ha, g0a);
      g1a = fma(Ss[k * RP + c1], ha, g1a);
    }
    __syncwarp();  // the iterate is read by every lane before it is overwritten
    const TA x0 = h0 - eta * ((g0a + g0b) - m0), x1 = h1 - eta * ((g1a + g1b) - m1);
    h0 = v0 && x0 > TA(0) ? x0 : TA(0);
    h1 = v1 && x1 > TA(0) ? x1 : TA(0);
  }
  if (v0) H[row * R + c0] = h0;
  if (v1) H[row * R + c1] = h1;
}

// ---- ADMM (Eq. admmupd) --------------------------------------------------------------
// Scratch layout (doubles): [0] rho, [1] 1 if a pivot was not positive, [8 ..) W = (S + rho I)^{-1}
// (R x R, FP64), then W as TA, then per-step per-block norm partials.
constexpr int ADMM_W = 8;

// ucp != 0: no shift (rho = 0), W = S^{-1} for the unconstrained update.
// W = (S + rho I)^{-1} by the symmetric sweep operator (Gauss-Jordan
// elimination in place, which needs no pivoting for a symmetric positive
// definite matrix): R steps, each a rank-1 update of the whole matrix spread
// over the CTA, instead of a Cholesky factorisation followed by a serial
// inverse per column.  Its pivots are those of the Cholesky factorisation, so
// a non-positive pivot flags the same matrices.
__global__ void __launch_bounds__(256)
admm_prep_kernel(const double* __restrict__ S, int R, double* __restrict__ scr, int wtf_f64,
                 int ucp) {
  extern __shared__ double sm[];
  const int LD = R + 1;        // padded leading dimension (no bank conflicts)
  double* A = sm;              // R x R (stride LD): S + rho I, swept in place
  double* col = sm + R * LD;   // R: column k before the step
  __shared__ double s_rho, s_inv;
  __shared__ int s_bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid < 32) {
    double tr = 0.0;
    for (int r = tid; r < R; r += 32) tr += S[r * R + r];
    tr = warp_sum(tr);
    if (tid == 0) {
      // reading: rho = trace(S) / R; an all-zero S (no information) uses rho = 1
      s_rho = ucp ? 0.0 : (tr > 0.0 ? tr / R : 1.0);
      s_bad = 0;
    }
  }
  __syncthreads();
  for (int e = tid; e < R * R; e += nt) {
    const int i = e / R, j = e - i * R;
    A[i * LD + j] = S[e] + (i == j ? s_rho : 0.0);
  }
  __syncthreads();
  for (int k = 0; k < R; ++k) {
    if (tid == 0) {
      double d = A[k * LD + k];
      if (!(d > 0.0)) { s_bad = 1; d = 1.0; }
      s_inv = 1.0 / d;
    }
    for (int i = tid; i < R; i += nt) col[i] = A[i * LD + k];
    __syncthreads();
    const double inv = s_inv;
    // A_ij -= A_ik A_kj / d for i, j != k (A symmetric: A_kj = A_jk = col[j])
    for (int e = tid; e < R * R; e += nt) {
      const int i = e / R, j = e - i * R;
      if (i != k && j != k) A[i * LD + j] = fma(-col[i] * inv, col[j], A[i * LD + j]);
    }
    __syncthreads();
    for (int i = tid; i < R; i += nt) {
      const double v = i == k ? -inv : col[i] * inv;
      A[i * LD + k] = v;
      A[k * LD + i] = v;
    }
    __syncthreads();
  }
  // after all R steps A = -(S + rho I)^{-1}
  double* W = scr + ADMM_W;
  for (int e = tid; e < R * R; e += nt) {
    const int i = e / R, j = e - i * R;
    const double w = -A[i * LD + j];
    W[e] = w;
    if (wtf_f64) ((double*)(W + R * R))[e] = w;
    else ((float*)(W + R * R))[e] = (float)w;
  }
  if (tid == 0) { scr[0] = s_rho; scr[1] = s_bad; }
}

// Stop test of an iterative update at the start of launch k (one warp per
// block; every block decides the same): flags[j] != 0 records that launch j
// stopped; otherwise the block partials of step k-1 decide.  Launch 0 clears
// the flags; a launch that stops sets its own, so later launches need only
// one read.  part_k1 points at step k-1's partials (stride words per block).
template <bool MAX>
__device__ __forceinline__ bool step_stop(int k, double* flags, const double* part_k1, int nblk,
                                          int stride, double tol, bool extra) {
  const int lane = threadIdx.x & 31;
  if (k == 0) {
    if (blockIdx.x == 0)
      for (int j = lane; j < 64; j += 32) flags[j] = 0.0;
    return false;
  }
  bool stop = extra || flags[k - 1] != 0.0;
  if (!stop) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int bl = lane; bl < nblk; bl += 32)
      for (int q = 0; q < stride; ++q)
        v[q] = MAX ? fmax(v[q], part_k1[bl * stride + q]) : v[q] + part_k1[bl * stride + q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double w = __shfl_xor_sync(0xffffffffu, v[q], o);
        v[q] = MAX ? fmax(v[q], w) : v[q] + w;
      }
    stop = MAX ? (v[0] <= tol * v[1]) : (v[0] < tol * v[1] && v[2] < tol * v[3]);
  }
  if (stop && blockIdx.x == 0 && lane == 0) flags[k] = 1.0;
  return stop;
}

// step k of at most kmax; part holds 4 norms per block per step
template <typename TA, int RP>
__global__ void __launch_bounds__(ROWS_PER_CTA)
admm_step_kernel(int64_t rows, int R, const TA* __restrict__ M, TA* __restrict__ H,
                 TA* __restrict__ U, const double* __restrict__ lam, const double* __restrict__ scr,
                 double* __restrict__ part, int nblk, int k, double tol, int u_zero,
                 int32_t* __restrict__ inner) {
  extern __shared__ __align__(16) unsigned char admm_smem[];
  TA* Ws = reinterpret_cast<TA*>(admm_smem);   // RP x RP
  TA* hv = Ws + RP * RP;                          // RP x ROWS_PER_CTA
  TA* uv = hv + RP * ROWS_PER_CTA;                // RP x ROWS_PER_CTA
  __shared__ double s_red[4][ROWS_PER_CTA];
  const int tid = threadIdx.x;
  const bool stop = step_stop<false>(k, part + (int64_t)PLANC_MAX_ADMM_STEPS * nblk * 4,
                                     part + (int64_t)(k > 0 ? k - 1 : 0) * nblk * 4, nblk, 4,
                                     tol, false);
  const TA* Wt = (const TA*)(scr + ADMM_W + R * R);
  for (int e = tid; e < RP * RP; e += blockDim.x) {
    int i = e / RP, j = e - i * RP;
    Ws[e] = (i < R && j < R) ? Wt[i * R + j] : TA(0);
  }
  __syncthreads();
  if (stop) return;
  const TA rho = (TA)scr[0];
  int64_t i = (int64_t)blockIdx.x * blockDim.x + tid;
  TA n_pr = TA(0), n_h = TA(0), n_du = TA(0), n_u = TA(0);
  if (i < rows) {
    TA rhs[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      TA h = TA(0), u = TA(0), m = TA(0);
      if (r < R) {
        h = H[i * R + r];
        if (k == 0 && lam) h = (TA)((double)h * lam[r]);
        if (!(u_zero && k == 0)) u = U[i * R + r];
        m = M[i * R + r];
      }
      rowv(hv, r) = h;
      rowv(uv, r) = u;
      rhs[r] = m + rho * (h + u);
    }
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
      TA ht = dot_row<TA, RP>(rhs, Ws + r * RP);  // W symmetric
      TA ur = rowv(uv, r), hr = rowv(hv, r);
      TA hn = ht - ur;
      hn = hn > TA(0) ? hn : TA(0);
      TA un = ur + hn - ht;
      H[i * R + r] = hn;
      U[i * R + r] = un;
      n_pr = fma(hn - ht, hn - ht, n_pr);
      n_h = fma(hn, hn, n_h);
      n_du = fma(hn - hr, hn - hr, n_du);
      n_u = fma(un, un, n_u);
    }
  }
  s_red[0][tid] = (double)n_pr;
  s_red[1][tid] = (double)n_h;
  s_red[2][tid] = (double)n_du;
  s_red[3][tid] = (double)n_u;
  __syncthreads();
  if (tid < 4) {
    double s = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) s += s_red[tid][t];
    part[((int64_t)k * nblk + blockIdx.x) * 4 + tid] = s;
  }
  if (tid == 0 && blockIdx.x == 0 && inner) *inner = k + 1;
}

// ---- BPP (Eq. snls; Kim-Park block principal pivoting) ---------------------------------
// One warp per row, R <= 64 (lane j holds indices j and j + 32), FP64; the
// passive-set Cholesky in shared memory with a padded leading dimension.
constexpr int BPP_WARPS = 4;

__device__ __forceinline__ uint64_t ballot64(bool lo, bool hi) {
  uint64_t a = __ballot_sync(0xffffffffu, lo);
  uint64_t b = __ballot_sync(0xffffffffu, hi);
  return a | (b << 32);
}

// RMAX > 0 (FP32 storage, R <= RMAX <= 32): the passive systems are inverted
// and solved in registers (lane p holds row p of S_FF and then of its
// inverse; pivot rows travel by warp shuffles), without a shared-memory
// round trip per elimination step.
template <typename TA, int RMAX>
__global__ void __launch_bounds__(32 * BPP_WARPS, 1)
nls_bpp_kernel(int64_t rows, int R, const double* __restrict__ S, const TA* __restrict__ M,
               TA* __restrict__ H, const double* __restrict__ lam, int max_iter,
               int32_t* __restrict__ inner, int* __restrict__ flags) {
  extern __shared__ double bsm[];
  // matrices with leading dimension LD = R + 1: a column read by the 32
  // lanes then spreads over the banks (stride R put every lane on one bank)
  const int LD = R + 1;
  double* Ss = bsm;                                   // R x R (stride LD)
  double* Ws = bsm + R * LD;                          // S^{-1} (stride LD; R <= 32)
  double* colk = Ws + R * LD;                         // 64: a column of the inversion
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* A = colk + 64 + (size_t)warp * (R * LD + 3 * 64);  // f x f (stride LD)
  double* xs = A + R * LD;                             // 64: passive solution / rhs
  double* zs = xs + 64;                                // 64: full x
  double* dinv = zs + 64;                              // 64: 1 / pivot
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    const int a = e / R, b = e - a * R;
    Ss[a * LD + b] = S[e];
    if (RMAX > 16) Ws[a * LD + b] = S[e];
  }
  // R <= 32: W = S^{-1} in place by Gauss-Jordan elimination (no pivoting: S
  // is symmetric positive definite; R steps of a rank-1 update spread over
  // the CTA, FP64, reciprocals from an FP32 seed and two Newton steps).  A
  // pivot that is not positive leaves W unused (every row then factors S_FF).
  // (R <= 16: the register factorisation of S_FF alone was faster on the
  // 4-way mouse-like workload; the inverse pays from R = 32)
  constexpr bool WPATH = RMAX > 16;
  __shared__ int s_wbad;
  if (threadIdx.x == 0) s_wbad = 0;
  if (WPATH) {
    for (int k = 0; k < R; ++k) {
      __syncthreads();
      const double p = Ws[k * LD + k];
      if (!(p > 0.0)) {
        if (threadIdx.x == 0) s_wbad = 1;
        break;  // uniform: every thread read the same pivot
      }
      double ip = (double)(1.0f / (float)p);
      ip = ip * (2.0 - p * ip);
      ip = ip * (2.0 - p * ip);
      for (int i = threadIdx.x; i < R; i += blockDim.x) colk[i] = Ws[i * LD + k];
      __syncthreads();
      // row k scaled (its pivot entry becomes 1 / p), then every other row
      for (int j = threadIdx.x; j < R; j += blockDim.x)
        Ws[k * LD + j] = (j == k ? 1.0 : Ws[k * LD + j]) * ip;
      __syncthreads();
      for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
        const int i = e / R, j = e - (e / R) * R;
        if (i != k) Ws[i * LD + j] = fma(-colk[i], Ws[k * LD + j], j == k ? 0.0 : Ws[i * LD + j]);
      }
    }
  }
  __syncthreads();
  const bool use_w = WPATH && s_wbad == 0;
  const int64_t row = (int64_t)blockIdx.x * BPP_WARPS + warp;
  if (row >= rows) return;

  const int j0 = lane, j1 = lane + 32;
  const bool v0 = j0 < R, v1 = j1 < R;
  double m0 = v0 ? (double)M[row * R + j0] : 0.0;
  double m1 = v1 ? (double)M[row * R + j1] : 0.0;
  double w0 = v0 ? (double)H[row * R + j0] * (lam ? lam[j0] : 1.0) : 0.0;
  double w1 = v1 ? (double)H[row * R + j1] * (lam ? lam[j1] : 1.0) : 0.0;
  uint64_t F = ballot64(v0 && w0 > 0.0, v1 && w1 > 0.0);  // passive set from the warm start
  double x0 = 0.0, x1 = 0.0, y0 = 0.0, y1 = 0.0;
  int bad = 0;

  // The passive system S_FF x_F = m_F is factored (register path: inverted)
  // in FP32 (this GPU's FP64 pipe is narrow, and the elimination is a chain
  // of dependent steps) and
  // x_F refined with FP64 residuals m_F - S_FF x_F until the correction is
  // below 1e-11 of x (mixed-precision iterative refinement: the result is the
  // FP64 solution to that accuracy; 1e-9 on the register path, whose results
  // are stored in FP32); a pivot that falls below 1e-5 of its diagonal
  // entry, or a refinement that does not settle in 6 steps, hands the system
  // to the FP64 factorisation.  FP64 storage uses the FP64 factorisation only.
  float* Af = reinterpret_cast<float*>(A);     // FP32 factor (stride LD)
  float* df = reinterpret_cast<float*>(dinv);  // [0, 64): 1 / pivot; [64, 128): diagonal, then rhs
  float* wf = df + 64;

  // S x for the full vector in zs: rows j0, j1
  // (four partial sums per row: a single chain of R dependent FP64 FMAs is
  // the latency of every refinement step on this GPU's narrow FP64 pipe)
  auto sx = [&](double& s0, double& s1) {
    double a[4] = {0.0, 0.0, 0.0, 0.0}, b[4] = {0.0, 0.0, 0.0, 0.0};
    int k = 0;
    for (; k + 4 <= R; k += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double xk = zs[k + u];
        if (v0) a[u] = fma(Ss[j0 * LD + k + u], xk, a[u]);
        if (v1) b[u] = fma(Ss[j1 * LD + k + u], xk, b[u]);
      }
    }
    for (; k < R; ++k) {
      const double xk = zs[k];
      if (v0) a[0] = fma(Ss[j0 * LD + k], xk, a[0]);
      if (v1) b[0] = fma(Ss[j1 * LD + k], xk, b[0]);
    }
    s0 = (a[0] + a[1]) + (a[2] + a[3]);
    s1 = (b[0] + b[1]) + (b[2] + b[3]);
  };
  // wf := (L L^T)^{-1} wf with the FP32 factor (positions 0..f-1)
  auto solve32 = [&](int f) {
    for (int c = 0; c < f; ++c) {
      const float zc = wf[c] * df[c];
      __syncwarp();
      for (int i = c + 1 + lane; i < f; i += 32) wf[i] = fmaf(-Af[i * LD + c], zc, wf[i]);
      if (lane == 0) wf[c] = zc;
      __syncwarp();
    }
    for (int c = f - 1; c >= 0; --c) {
      const float xc = wf[c] * df[c];
      __syncwarp();
      for (int i = lane; i < c; i += 32) wf[i] = fmaf(-Af[c * LD + i], xc, wf[i]);
      if (lane == 0) wf[c] = xc;
      __syncwarp();
    }
  };

  // Register path (RMAX > 0, so R <= 32 and every index j0 is one lane):
  // x_F into x0, true when the refinement settled (false: FP64 fallback).
  constexpr int RM = RMAX > 0 ? RMAX : 1;
  auto solve_reg = [&](int f, int p0, bool in0) -> bool {
    // position -> index table, zero past f
    int* tbl = reinterpret_cast<int*>(xs);
    if (in0) tbl[p0] = j0;
    if (lane >= f && lane < RM) tbl[lane] = 0;
    __syncwarp();
    const bool live = lane < f;
    const int myi = live ? tbl[lane] : 0;
    float a[RM];
#pragma unroll
    for (int q = 0; q < RM; ++q) a[q] = (live && q < f) ? (float)Ss[myi * LD + tbl[q]] : 0.f;
    const float d0 = (float)Ss[myi * LD + myi];
    __syncwarp();  // tbl read by all lanes before xs is reused
    // Gauss-Jordan inversion of S_FF in registers (symmetric positive
    // definite: no pivoting), lane p holding row p: step c scales row c by
    // the reciprocal of its pivot (the Schur complement's diagonal, the
    // square of the Cholesky pivot) and removes column c from every other
    // row.  Afterwards a[] holds row p of S_FF^{-1}, so a solve is one
    // matrix-vector product.  One chain of f steps (a Cholesky factor and
    // two triangular solves per refinement step were three); a pivot below
    // 1e-5 of its diagonal entry hands the system to the FP64 path as before.
    int good = 1;
#pragma unroll
    for (int c = 0; c < RM; ++c) {
      if (c < f) {
        const float fct = a[c];  // A[lane][c]; at lane c the pivot
        float ip = 1.f;
        if (lane == c) {
          float piv = fct;
          if (!(piv > 1e-5f * d0)) {
            good = 0;
            piv = 1.f;
          }
          ip = __frcp_rn(piv);
          a[c] = 1.f;
        }
#pragma unroll
        for (int q = 0; q < RM; ++q) a[q] *= ip;  // row c scaled (ip = 1 elsewhere)
        float rq[RM];
#pragma unroll
        for (int q = 0; q < RM; ++q) rq[q] = q < f ? __shfl_sync(0xffffffffu, a[q], c) : 0.f;
        if (lane != c) {
          a[c] = 0.f;
#pragma unroll
          for (int q = 0; q < RM; ++q) a[q] = fmaf(-fct, rq[q], a[q]);
        }
      }
    }
    if (!__all_sync(0xffffffffu, good)) return false;
    x0 = 0.0;
    double r0 = in0 ? m0 : 0.0;  // residual on F (x = 0)
    for (int st = 0; st <= 6; ++st) {
      // right-hand side to the position lanes, then d = S_FF^{-1} r
      float w = __shfl_sync(0xffffffffu, (float)r0, myi);
      if (!live) w = 0.f;
      float d4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < RM; ++j) {
        const float wj = __shfl_sync(0xffffffffu, w, j);
        d4[j & 3] = fmaf(a[j], wj, d4[j & 3]);  // a[j] = 0 for j >= f
      }
      w = live ? (d4[0] + d4[1]) + (d4[2] + d4[3]) : 0.f;
      const float dw = __shfl_sync(0xffffffffu, w, p0 & 31);
      const double d = in0 ? (double)dw : 0.0;
      x0 += d;
      if (st > 0) {  // (the first solve is never the last)
        // the stop test's maxima in FP32 (a ratio of 1e-9 is well inside its
        // range; FP64 shuffles cost twice as many and the FP64 pipe is narrow)
        float dm = fabsf((float)d), xm = fabsf((float)x0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
          xm = fmaxf(xm, __shfl_xor_sync(0xffffffffu, xm, o));
        }
        if (dm <= 1e-9f * xm) return true;
        if (st == 6) return false;
      }
      // FP64 residual m_F - S_FF x_F
      if (v0) zs[j0] = x0;
      __syncwarp();
      double s0, s1;
      sx(s0, s1);
      r0 = in0 ? m0 - s0 : 0.0;
      __syncwarp();
    }
    return false;
  };

  // S^{-1} path (R <= 32, the inverse given): with W = S^{-1}, the passive
  // solution is x_F = u_F - W_FG z, where u = W m_F (m taken as zero on the
  // inactive set G) and W_GG z = u_G: the inverse of a principal submatrix
  // from the Schur complement of W.  Only the g x g system of G is solved
  // (g <= 8, FP64 Gauss-Jordan with the rows on lanes, reciprocals from an
  // FP32 seed and two Newton steps); false (a non-positive pivot) hands the
  // system to the factorisation of S_FF.
  constexpr int GMAX = 8;
  auto recip = [](double d) {
    double y = (double)(1.0f / (float)d);
    y = y * (2.0 - d * y);
    return y * (2.0 - d * y);
  };
  auto solve_w = [&](int g, bool in0) -> bool {
    if (v0) zs[j0] = in0 ? m0 : 0.0;
    __syncwarp();
    double u = 0.0;
    if (v0)
      for (int k = 0; k < R; ++k) u = fma(Ws[j0 * LD + k], zs[k], u);
    __syncwarp();
    if (g == 0) {
      x0 = in0 ? u : 0.0;
      return true;
    }
    int* gl = reinterpret_cast<int*>(xs);  // the inactive indices in order
    const uint64_t Gm = ~F & ((1ull << R) - 1ull);
    if (v0 && !in0) gl[__popcll(Gm & ((1ull << j0) - 1ull))] = j0;
    __syncwarp();
    const bool rw = lane < g;
    const int gi = rw ? gl[lane] : 0;
    double a[GMAX];
#pragma unroll
    for (int k = 0; k < GMAX; ++k) a[k] = (rw && k < g) ? Ws[gi * LD + gl[k]] : 0.0;
    double b = __shfl_sync(0xffffffffu, u, gi);
    double dg = 1.0;
    bool good = true;
#pragma unroll
    for (int c = 0; c < GMAX; ++c) {
      if (c < g) {
        const double piv = __shfl_sync(0xffffffffu, a[c], c);
        if (!(piv > 0.0)) good = false;
        const double ip = recip(good ? piv : 1.0);
        const double bc = __shfl_sync(0xffffffffu, b, c);
        double ac[GMAX];
#pragma unroll
        for (int k = 0; k < GMAX; ++k) ac[k] = __shfl_sync(0xffffffffu, a[k], c);
        if (lane == c) {
          dg = piv;
        } else {
          const double fct = a[c] * ip;
#pragma unroll
          for (int k = 0; k < GMAX; ++k)
            if (k > c) a[k] = fma(-fct, ac[k], a[k]);
          b = fma(-fct, bc, b);
        }
      }
    }
    if (!good) {
      __syncwarp();
      return false;
    }
    const double z = rw ? b * recip(dg) : 0.0;
    double corr = 0.0;
    for (int i = 0; i < g; ++i) {
      const double zi = __shfl_sync(0xffffffffu, z, i);
      if (v0) corr = fma(Ws[j0 * LD + gl[i]], zi, corr);
    }
    __syncwarp();  // gl read by every lane before the scratch is reused
    x0 = in0 ? u - corr : 0.0;
    return true;
  };

  // x_F = S_FF^{-1} m_F, x_G = 0; y = S x - m on G, 0 on F
  auto solve = [&]() {
    const int f = __popcll(F);
    // position of j in F = popc(F & ((1 << j) - 1))
    const uint64_t below0 = (j0 == 0) ? 0ull : (F & ((1ull << j0) - 1ull));
    const uint64_t below1 = F & ((1ull << j1) - 1ull);
    const int p0 = __popcll(below0), p1 = __popcll(below1);
    const bool in0 = v0 && ((F >> j0) & 1ull), in1 = v1 && ((F >> j1) & 1ull);
    bool done = f == 0;
    x0 = 0.0;
    x1 = 0.0;
    if constexpr (RMAX > 0) {
      if (!done && use_w && R - f <= GMAX && R - f <= f) done = solve_w(R - f, in0);
      if (!done) done = solve_reg(f, p0, in0);
    }
    if (!done && RMAX == 0 && sizeof(TA) == 4) {
      // FP32 S_FF: each lane owns the columns of its indices, A[p_a][p_b] = S[a][b]
      for (int a = 0; a < R; ++a) {
        if (!((F >> a) & 1ull)) continue;
        const int pa = __popcll(a == 0 ? 0ull : (F & ((1ull << a) - 1ull)));
        if (in0) Af[pa * LD + p0] = (float)Ss[a * LD + j0];
        if (in1) Af[pa * LD + p1] = (float)Ss[a * LD + j1];
      }
      if (in0) wf[p0] = (float)Ss[j0 * LD + j0];
      if (in1) wf[p1] = (float)Ss[j1 * LD + j1];
      __syncwarp();
      // right-looking Cholesky (lower); lane 0 forms each pivot
      int good = 1;
      for (int c = 0; c < f; ++c) {
        if (lane == 0) {
          float d = Af[c * LD + c];
          if (!(d > 1e-5f * wf[c])) {
            good = 0;
            d = 1.f;
          }
          const float r = sqrtf(d);
          Af[c * LD + c] = r;
          df[c] = 1.f / r;
        }
        __syncwarp();
        const float ic = df[c];
        for (int i = c + 1 + lane; i < f; i += 32) Af[i * LD + c] *= ic;
        __syncwarp();
        for (int i = c + 1 + lane; i < f; i += 32) {
          const float aic = Af[i * LD + c];
          for (int j = c + 1; j <= i; ++j) Af[i * LD + j] = fmaf(-aic, Af[j * LD + c], Af[i * LD + j]);
        }
        __syncwarp();
      }
      good = __shfl_sync(0xffffffffu, good, 0);
      if (good) {
        double r0 = m0, r1 = m1;  // residual on F (x = 0)
        for (int st = 0; st <= 6; ++st) {
          if (in0) wf[p0] = (float)r0;
          if (in1) wf[p1] = (float)r1;
          __syncwarp();
          solve32(f);
          const double d0 = in0 ? (double)wf[p0] : 0.0, d1 = in1 ? (double)wf[p1] : 0.0;
          x0 += d0;
          x1 += d1;
          double dm = fmax(fabs(d0), fabs(d1)), xm = fmax(fabs(x0), fabs(x1));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
            xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
          }
          if (st > 0 && dm <= 1e-11 * xm) {
            done = true;
            break;
          }
          if (st == 6) break;
          // FP64 residual m_F - S_FF x_F
          if (v0) zs[j0] = x0;
          if (v1) zs[j1] = x1;
          __syncwarp();
          double s0, s1;
          sx(s0, s1);
          r0 = in0 ? m0 - s0 : 0.0;
          r1 = in1 ? m1 - s1 : 0.0;
          __syncwarp();
        }
      }
    }
    if (!done) {
      // FP64 factorisation: A = S_FF, rhs m_F
      for (int a = 0; a < R; ++a) {
        if (!((F >> a) & 1ull)) continue;
        const int pa = __popcll(a == 0 ? 0ull : (F & ((1ull << a) - 1ull)));
        if (in0) A[pa * LD + p0] = Ss[a * LD + j0];
        if (in1) A[pa * LD + p1] = Ss[a * LD + j1];
      }
      if (in0) xs[p0] = m0;
      if (in1) xs[p1] = m1;
      __syncwarp();
      // right-looking; the pivot's reciprocal is formed once and multiplied
      for (int c = 0; c < f; ++c) {
        if (lane == 0) {
          double d = A[c * LD + c];
          if (!(d > 0.0)) { bad = 1; d = 1e-300; }
          const double r = sqrt(d);
          A[c * LD + c] = r;
          dinv[c] = 1.0 / r;
        }
        __syncwarp();
        const double ic = dinv[c];
        for (int i = c + 1 + lane; i < f; i += 32) A[i * LD + c] *= ic;
        __syncwarp();
        for (int i = c + 1 + lane; i < f; i += 32) {
          const double aic = A[i * LD + c];
          for (int j = c + 1; j <= i; ++j) A[i * LD + j] = fma(-aic, A[j * LD + c], A[i * LD + j]);
        }
        __syncwarp();
      }
      for (int c = 0; c < f; ++c) {  // L z = m_F
        const double zc = xs[c] * dinv[c];
        __syncwarp();
        for (int i = c + 1 + lane; i < f; i += 32) xs[i] = fma(-A[i * LD + c], zc, xs[i]);
        if (lane == 0) xs[c] = zc;
        __syncwarp();
      }
      for (int c = f - 1; c >= 0; --c) {  // L^T x = z
        const double xc = xs[c] * dinv[c];
        __syncwarp();
        for (int i = lane; i < c; i += 32) xs[i] = fma(-A[c * LD + i], xc, xs[i]);
        if (lane == 0) xs[c] = xc;
        __syncwarp();
      }
      x0 = in0 ? xs[p0] : 0.0;
      x1 = in1 ? xs[p1] : 0.0;
    }
    if (v0) zs[j0] = x0;
    if (v1) zs[j1] = x1;
    __syncwarp();
    double s0, s1;
    sx(s0, s1);
    y0 = (v0 && !in0) ? s0 - m0 : 0.0;
    y1 = (v1 && !in1) ? s1 - m1 : 0.0;
    __syncwarp();
  };

  solve();
  int p = 3, ninf = R + 1, it = 0;
  bool converged = false;
  while (true) {
    bool f0 = v0 && ((F >> j0) & 1ull), f1 = v1 && ((F >> j1) & 1ull);
    bool i0 = v0 && (f0 ? x0 < 0.0 : y0 < 0.0);
    bool i1 = v1 && (f1 ? x1 < 0.0 : y1 < 0.0);
    uint64_t V = ballot64(i0, i1);
    int nv = __popcll(V);
    if (nv == 0) { converged = true; break; }
    if (it >= max_iter) break;
    uint64_t Vh;
    if (nv < ninf) { ninf = nv; p = 3; Vh = V; }
    else if (p >= 1) { --p; Vh = V; }
    else { Vh = 1ull << (63 - __clzll(V)); }
    F ^= Vh;
    solve();
    ++it;
  }
  if (v0) H[row * R + j0] = (TA)(x0 > 0.0 ? x0 : 0.0);
  if (v1) H[row * R + j1] = (TA)(x1 > 0.0 ? x1 : 0.0);
  if (lane == 0) {
    if (inner) atomicMax(inner, it);
    if (!converged) atomicAdd(flags + 0, 1);
    if (bad) atomicAdd(flags + 1, 1);
  }
}

__global__ void set_int_kernel(int32_t* p, int v, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

}  // namespace

cudaError_t launch_set_int(int32_t* p, int v, int n, cudaStream_t st) {
  set_int_kernel<<<(n + 255) / 256, 256, 0, st>>>(p, v, n);
  note_launches(1);
  return cudaGetLastError();
}

namespace {

// ---- UCP (unconstrained, Sec. 6): Hhat = M S^{-1}, one row per thread ----------------
template <typename TA, int RP>
__global__ void __launch_bounds__(ROWS_PER_CTA)
nls_ucp_kernel(int64_t rows, int R, const TA* __restrict__ M, TA* __restrict__ H,
               const double* __restrict__ scr, int* __restrict__ flags) {
  __shared__ TA Ws[RP * RP];
  const TA* Wt = (const TA*)(scr + ADMM_W + R * R);
  for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
    const int i = e / RP, j = e - i * RP;
    Ws[e] = (i < R && j < R) ? Wt[i * R + j] : TA(0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && scr[1] != 0.0 && flags) atomicAdd(flags + 1, 1);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  TA m[RP];
#pragma unroll
  for (int k = 0; k < RP; ++k) m[k] = k < R ? M[i * R + k] : TA(0);
  for (int r = 0; r < R; ++r) {
    TA acc = TA(0);
#pragma unroll
    for (int k = 0; k < RP; ++k) acc = fma(m[k], Ws[k * RP + r], acc);
    H[i * R + r] = acc;
  }
}

// ---- Nesterov-type update (Sec. 4.3.5, Eq. nesnls / Eq. nesinnerupd) ------------------
// Parameters from the extreme eigenvalues mu0, L0 of S (readings): the
// proximal weight lam_p = max(0, (L0 - kappa mu0) / (kappa - 1)) caps the
// condition number of f_p at kappa; L = L0 + lam_p, mu = mu0 + lam_p,
// beta = (1 - sqrt(mu/L)) / (1 + sqrt(mu/L)).  With P = I - (S + lam_p I)/L
// and b = (M + lam_p H*)/L one step is X_{k+1} = [Y_k P + b]_+ (the gradient
// step of f_p at Y_k), Y_{k+1} = X_{k+1} + beta (X_{k+1} - X_k).
// scr: [0] lam_p, [1] L, [2] beta, [3] 1/L, [4] lam_p/L, [5] 1 if L == 0;
// scr + ADMM_W + R^2: P in the factor precision; then the step partials.
constexpr double kNesKappa = 100.0;

// Precision traits of the parameter computation: FP64 for FP64 factors, FP32
// for FP32 factors (the FP64 pipe of this GPU makes the dependent chains of
// the reduction and of the Sturm counts ~50x slower than in FP32).
template <typename CT> struct NesCT;
template <> struct NesCT<double> {
  static constexpr int rounds = 13;        // 33^13 > 2^65
  static constexpr double tiny = 1e-300;
  static constexpr double big = 0x1p+400, small = 0x1p-400;
  static constexpr double pad = 1e-12;
};
template <> struct NesCT<float> {
  static constexpr int rounds = 6;         // 33^6 > 2^30
  static constexpr float tiny = 1e-30f;
  static constexpr float big = 0x1p+60f, small = 0x1p-60f;
  static constexpr float pad = 1e-5f;
};

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x, from the
// signs of its leading principal minors (Sturm sequence, division-free with
// power-of-two rescaling).
template <typename CT>
__device__ int sturm_below(const CT* d, const CT* e2, int n, CT x) {
  using T = NesCT<CT>;
  CT pm = CT(1), p = d[0] - x;
  int c = (p < CT(0)) ? 1 : 0;
  if (p == CT(0)) { c = 1; p = -T::tiny; }
  for (int i = 1; i < n; ++i) {
    CT q = fma(d[i] - x, p, -e2[i - 1] * pm);
    pm = p;
    p = q;
    const bool change = (p == CT(0)) ? true : ((p < CT(0)) != (pm < CT(0)));
    if (p == CT(0)) p = pm < CT(0) ? T::tiny : -T::tiny;
    c += change ? 1 : 0;
    const CT a = fabs(p);
    if (a > T::big) { p *= T::small; pm *= T::small; }
    else if (a < T::small && fabs(pm) < T::small) { p *= T::big; pm *= T::big; }
  }
  return c;
}

// One warp narrows [lo, hi] around the smallest (want_max = 0) or largest
// eigenvalue: 32 Sturm counts per round.
template <typename CT>
__device__ CT warp_extreme_eig(const CT* d, const CT* e2, int n, CT lo, CT hi, bool want_max) {
  const int lane = threadIdx.x & 31;
  for (int round = 0; round < NesCT<CT>::rounds; ++round) {
    const CT w = (hi - lo) / CT(33);
    const CT x = lo + w * CT(lane + 1);
    const int c = sturm_below<CT>(d, e2, n, x);
    const bool past = want_max ? (c >= n) : (c >= 1);
    const unsigned m = __ballot_sync(0xffffffffu, past);
    const CT xs = __shfl_sync(0xffffffffu, x, m ? (__ffs(m) - 1) : 0);
    const CT xp = __shfl_sync(0xffffffffu, x, m ? max(__ffs(m) - 2, 0) : 31);
    if (m == 0) {
      lo = xp;
    } else {
      if (__ffs(m) > 1) lo = xp;
      hi = xs;
    }
  }
  return CT(0.5) * (lo + hi);
}

// Two warps: warp 0 reduces S to tridiagonal form (Householder, lanes own
// rows for A v and columns for the rank-2 update, warp-synchronous: no
// block-wide barrier per column), then warps 0 and 1 find the smallest and
// the largest eigenvalue; thread 0 writes the step parameters and all 64
// threads P, in precision CT.
template <typename CT>
__global__ void __launch_bounds__(64)
nes_prep_kernel(const double* __restrict__ S, int R, double* __restrict__ scr, double kappa) {
  extern __shared__ __align__(16) unsigned char nes_prep_smem[];
  // R x R working copy of S with leading dimension R + 1: the lanes' row
  // and column reads fall in distinct banks
  const int LD = R + 1;
  CT* A = reinterpret_cast<CT*>(nes_prep_smem);
  CT* v = A + R * LD;       // Householder vector
  CT* w = v + 64;           // w = p - K v
  CT* d = w + 64;           // diagonal
  CT* e2 = d + 64;          // squared off-diagonal
  __shared__ double s_ev[2];
  __shared__ CT s_g;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int e = tid; e < R * R; e += 64) A[(e / R) * LD + e % R] = (CT)S[e];
  __syncthreads();
  if (tid < 32) {
    for (int k = 0; k + 2 < R; ++k) {
      const int m = R - k - 1;  // x = A[k+1.., k]
      CT ss = CT(0);
      for (int i = lane + 1; i < m; i += 32) {
        const CT x = A[(k + 1 + i) * LD + k];
        ss = fma(x, x, ss);
      }
      ss = warp_sum(ss);
      const CT x0 = A[(k + 1) * LD + k];
      if (ss == CT(0)) {  // already reduced
        if (lane == 0) e2[k] = x0 * x0;
        __syncwarp();
        continue;
      }
      const CT alpha = sqrt(fma(x0, x0, ss));
      const CT sig = x0 >= CT(0) ? -alpha : alpha;
      const CT v0 = x0 - sig;
      const CT tau = CT(2) / fma(v0, v0, ss);
      for (int i = lane; i < m; i += 32) v[i] = i == 0 ? v0 : A[(k + 1 + i) * LD + k];
      __syncwarp();
      // p = tau A_sub v: lane owns rows lane, lane + 32
      CT p0 = CT(0), p1 = CT(0);
      const int i0 = lane, i1 = lane + 32;
      const CT* r0 = A + (k + 1 + i0) * LD + k + 1;
      const CT* r1 = A + (k + 1 + i1) * LD + k + 1;
      for (int j = 0; j < m; ++j) {
        const CT vj = v[j];
        if (i0 < m) p0 = fma(r0[j], vj, p0);
        if (i1 < m) p1 = fma(r1[j], vj, p1);
      }
      p0 *= tau;
      p1 *= tau;
      CT vp = (i0 < m ? v[i0] * p0 : CT(0)) + (i1 < m ? v[i1] * p1 : CT(0));
      vp = warp_sum(vp);
      const CT K = CT(0.5) * tau * vp;
      if (i0 < m) w[i0] = fma(-K, v[i0], p0);
      if (i1 < m) w[i1] = fma(-K, v[i1], p1);
      __syncwarp();
      // A_sub -= v w^T + w v^T: lane owns columns lane, lane + 32
      const CT vc0 = i0 < m ? v[i0] : CT(0), wc0 = i0 < m ? w[i0] : CT(0);
      const CT vc1 = i1 < m ? v[i1] : CT(0), wc1 = i1 < m ? w[i1] : CT(0);
      for (int i = 0; i < m; ++i) {
        const CT vi = v[i], wi = w[i];
        CT* row = A + (k + 1 + i) * LD + k + 1;
        if (i0 < m) row[i0] = fma(-vi, wc0, fma(-wi, vc0, row[i0]));
        if (i1 < m) row[i1] = fma(-vi, wc1, fma(-wi, vc1, row[i1]));
      }
      if (lane == 0) e2[k] = sig * sig;
      __syncwarp();
    }
    for (int i = lane; i < R; i += 32) d[i] = A[i * LD + i];
    if (lane == 0 && R >= 2) {
      const CT x = A[(R - 1) * LD + R - 2];
      e2[R - 2] = x * x;
    }
    __syncwarp();
    // Gershgorin bound g; the tridiagonal is scaled by 1/g (so the Sturm
    // minors stay in range and the spectrum lies in [-1, 1])
    CT lo = CT(0), hi = CT(0);
    for (int i = lane; i < R; i += 32) {
      CT rad = CT(0);
      if (i > 0) rad += sqrt(e2[i - 1]);
      if (i + 1 < R) rad += sqrt(e2[i]);
      lo = i == lane ? d[i] - rad : fmin(lo, d[i] - rad);
      hi = i == lane ? d[i] + rad : fmax(hi, d[i] + rad);
    }
    CT g = lane < R ? fmax(fabs(lo), fabs(hi)) : CT(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
    __syncwarp();
    if (g > CT(0))
      for (int i = lane; i < R; i += 32) {
        d[i] /= g;
        if (i + 1 < R) e2[i] /= g * g;
      }
    if (lane == 0) s_g = g;
  }
  __syncthreads();
  const CT g = s_g;
  {
    double ev = 0.0;
    if (g > CT(0)) {
      const CT lim = CT(1) + NesCT<CT>::pad;
      ev = (double)g * (double)warp_extreme_eig<CT>(d, e2, R, -lim, lim, tid >= 32);
    }
    if (lane == 0) s_ev[tid >> 5] = ev;
  }
  __syncthreads();
  const double mu0 = fmax(s_ev[0], 0.0), L0 = fmax(s_ev[1], 0.0);
  const double lam_p = fmax(0.0, (L0 - kappa * mu0) / (kappa - 1.0));
  const double L = L0 + lam_p, mu = mu0 + lam_p;
  const bool skip = !(L > 0.0);
  if (tid == 0) {
    const double sq = skip ? 1.0 : sqrt(mu / L);
    scr[0] = lam_p;
    scr[1] = L;
    scr[2] = skip ? 0.0 : (1.0 - sq) / (1.0 + sq);
    scr[3] = skip ? 0.0 : 1.0 / L;
    scr[4] = skip ? 0.0 : lam_p / L;
    scr[5] = skip ? 1.0 : 0.0;
  }
  // P = I - (S + lam_p I) / L, kept in the factor precision after scr + ADMM_W + R^2
  const CT invL = skip ? CT(0) : (CT)(1.0 / L), lp = (CT)lam_p;
  CT* Pt = reinterpret_cast<CT*>(scr + ADMM_W + R * R);
  for (int e = tid; e < R * R; e += 64) {
    const int i = e / R, j = e - i * R;
    CT x = CT(0);
    if (!skip) x = (i == j ? CT(1) : CT(0)) - ((CT)S[e] + (i == j ? lp : CT(0))) * invL;
    Pt[e] = x;
  }
}

// Inner step k (0-based) of at most kmax.  H holds X_k (the warm start
// before step 0) and receives X_{k+1}; Y holds Y_k; Hs keeps
// H* = H diag(lam), written by step 0.  part: per block and step, the
// largest |X_{k+1} - Y_k| and the largest |X_{k+1}|; a step runs only if no
// earlier step met max|X_{j+1} - Y_j| <= tol max|X_{j+1}|.  A block (one
// warp) owns 32 consecutive rows: they are staged in shared memory with
// coalesced loads (stride-33 columns, no bank conflicts), each thread then
// updates its row, and the results leave with coalesced stores.
constexpr int NES_LD = ROWS_PER_CTA + 1;

template <typename TA, int RP>
__global__ void __launch_bounds__(ROWS_PER_CTA)
nes_step_kernel(int64_t rows, int R, const TA* __restrict__ M, TA* __restrict__ H,
                TA* __restrict__ Y, TA* __restrict__ Hs, const double* __restrict__ lam,
                const double* __restrict__ scr, double* __restrict__ part, int nblk, int k,
                double tol, int32_t* __restrict__ inner) {
  extern __shared__ __align__(16) unsigned char nes_smem[];
  TA* Ps = reinterpret_cast<TA*>(nes_smem);  // RP x RP
  TA* yv = Ps + RP * RP;                     // Y_k, then Y_{k+1}   (column r at r * NES_LD)
  TA* xv = yv + RP * NES_LD;                 // X_k, then X_{k+1}
  TA* bv = xv + RP * NES_LD;                 // b = (M + lam_p H*) / L
  const int tid = threadIdx.x;
  const bool skip = scr[5] != 0.0;
  const bool stop = step_stop<true>(k, part + (int64_t)PLANC_MAX_NES_STEPS * nblk * 2,
                                    part + (int64_t)(k > 0 ? k - 1 : 0) * nblk * 2, nblk, 2,
                                    tol, skip);
  const TA* Pt = (const TA*)(scr + ADMM_W + R * R);
  for (int e = tid; e < RP * RP; e += blockDim.x) {
    const int i = e / RP, j = e - i * RP;
    Ps[e] = (i < R && j < R) ? Pt[i * R + j] : TA(0);
  }
  __syncthreads();
  if (stop) return;
  const int64_t i0 = (int64_t)blockIdx.x * ROWS_PER_CTA;
  const int nr = (int)min((int64_t)ROWS_PER_CTA, rows - i0);
  const int64_t g0 = i0 * R;
  const int ne = nr * R;
  const TA invL = (TA)scr[3], lpL = (TA)scr[4], beta = (TA)scr[2];
  for (int e = tid; e < ne; e += ROWS_PER_CTA) {
    const int row = e / R, col = e - row * R;
    TA y, xo, hs;
    if (k == 0) {
      TA h = H[g0 + e];
      if (lam) h = (TA)((double)h * lam[col]);
      Hs[g0 + e] = h;
      y = xo = hs = h;
    } else {
      y = Y[g0 + e];
      xo = H[g0 + e];
      hs = Hs[g0 + e];
    }
    yv[col * NES_LD + row] = y;
    xv[col * NES_LD + row] = xo;
    bv[col * NES_LD + row] = fma(M[g0 + e], invL, hs * lpL);
  }
  __syncwarp();
  TA dmax = TA(0), xmax = TA(0);
  if (tid < nr && !skip) {
    TA y[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) y[r] = r < R ? yv[r * NES_LD + tid] : TA(0);
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
      TA xn = dot_row<TA, RP>(y, Ps + r * RP) + bv[r * NES_LD + tid];  // P symmetric
      xn = xn > TA(0) ? xn : TA(0);
      const TA xo = xv[r * NES_LD + tid];
      const TA yr = yv[r * NES_LD + tid];
      xv[r * NES_LD + tid] = xn;
      yv[r * NES_LD + tid] = fma(beta, xn - xo, xn);
      const TA dd = xn > yr ? xn - yr : yr - xn;
      dmax = dd > dmax ? dd : dmax;
      xmax = xn > xmax ? xn : xmax;
    }
  }
  __syncwarp();
  // S = 0 leaves H* (the staged X_0) in place
  for (int e = tid; e < ne; e += ROWS_PER_CTA) {
    const int row = e / R, col = e - row * R;
    H[g0 + e] = xv[col * NES_LD + row];
    if (!skip) Y[g0 + e] = yv[col * NES_LD + row];
  }
  double a = (double)dmax, b = (double)xmax;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  if (tid == 0) {
    part[((int64_t)k * nblk + blockIdx.x) * 2 + 0] = a;
    part[((int64_t)k * nblk + blockIdx.x) * 2 + 1] = b;
    if (blockIdx.x == 0 && inner) *inner = skip ? 0 : k + 1;
  }
}

template <typename TA, int RP>
cudaError_t run_rowwise(const NlsArgs& a, cudaStream_t st) {
  const int blocks = (int)((a.rows + ROWS_PER_CTA - 1) / ROWS_PER_CTA);
  const TA* M = (const TA*)a.M;
  TA* H = (TA*)a.H;
  switch (a.alg) {
    case PLANC_MU:
      nls_mu_kernel<TA, RP><<<blocks, ROWS_PER_CTA, 0, st>>>(a.rows, a.R, a.S, M, H, a.lambda,
                                                            a.opts.mu_eps);
      note_launches(1);
      break;
    case PLANC_HALS:
      nls_hals_kernel<TA, RP><<<blocks, ROWS_PER_CTA, 0, st>>>(
          a.rows, a.R, a.S, M, H, a.lambda, sizeof(TA) == 8 ? 1e-300 : 1e-30);
      note_launches(1);
      break;
    case PLANC_PGD:
      if (RP == 64 && a.rows <= 8192)  // few rows, wide rows: one warp per row
        nls_pgd_warp_kernel<TA><<<(unsigned)((a.rows + PGDW_WARPS - 1) / PGDW_WARPS),
                                  32 * PGDW_WARPS, 0, st>>>(a.rows, a.R, a.S, M, H, a.lambda,
                                                             std::max(1, a.opts.pgd_steps));
      else
        nls_pgd_kernel<TA, RP><<<blocks, ROWS_PER_CTA, 0, st>>>(a.rows, a.R, a.S, M, H, a.lambda,
                                                               std::max(1, a.opts.pgd_steps));
      note_launches(1);
      break;
    case PLANC_ADMM: {
      size_t smem = ((size_t)a.R * (a.R + 1) + a.R) * sizeof(double);
      cudaFuncSetAttribute(admm_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      admm_prep_kernel<<<1, 256, smem, st>>>(a.S, a.R, a.scratch, sizeof(TA) == 8, 0);
      note_launches(1);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      double* part = a.scratch + ADMM_W + 2 * (size_t)a.R * a.R;
      const int kmax = std::min(PLANC_MAX_ADMM_STEPS, std::max(1, a.opts.admm_max_inner));
      const size_t ssm = (size_t)(RP * RP + 2 * RP * ROWS_PER_CTA) * sizeof(TA);
      cudaFuncSetAttribute(admm_step_kernel<TA, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ssm);
      for (int k = 0; k < kmax; ++k) {
        admm_step_kernel<TA, RP><<<blocks, ROWS_PER_CTA, ssm, st>>>(
            a.rows, a.R, M, H, (TA*)a.U, a.lambda, a.scratch, part, blocks, k, a.opts.admm_tol,
            a.U_zero ? 1 : 0, a.inner);
        note_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
    case PLANC_NES: {
      cudaError_t e = launch_nes_prep(sizeof(TA) == 8, a.S, a.R, a.scratch, st);
      if (e != cudaSuccess) return e;
      double* part = a.scratch + ADMM_W + 2 * (size_t)a.R * a.R;
      const int kmax = std::min(PLANC_MAX_NES_STEPS, std::max(1, a.opts.nes_max_inner));
      const size_t ssm = (size_t)(RP * RP + 3 * RP * NES_LD) * sizeof(TA);
      cudaFuncSetAttribute(nes_step_kernel<TA, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ssm);
      for (int k = 0; k < kmax; ++k) {
        nes_step_kernel<TA, RP><<<blocks, ROWS_PER_CTA, ssm, st>>>(
            a.rows, a.R, M, H, (TA*)a.U, (TA*)a.V, a.lambda, a.scratch, part, blocks, k,
            a.opts.nes_tol, a.inner);
        note_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
    case PLANC_UCP: {
      size_t smem = ((size_t)a.R * (a.R + 1) + a.R) * sizeof(double);
      cudaFuncSetAttribute(admm_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      admm_prep_kernel<<<1, 256, smem, st>>>(a.S, a.R, a.scratch, sizeof(TA) == 8, 1);
      nls_ucp_kernel<TA, RP><<<blocks, ROWS_PER_CTA, 0, st>>>(a.rows, a.R, M, H, a.scratch,
                                                             a.flags);
      note_launches(2);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename TA>
cudaError_t run_nls_t(const NlsArgs& a, cudaStream_t st) {
  if (a.alg == PLANC_BPP) {
    const int blocks = (int)((a.rows + BPP_WARPS - 1) / BPP_WARPS);
    const size_t rl = (size_t)a.R * (a.R + 1);  // R x R with leading dimension R + 1
    size_t smem = (2 * rl + 64 + BPP_WARPS * (rl + 3 * 64)) * sizeof(double);
    cudaFuncSetAttribute(nls_bpp_kernel<TA, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if constexpr (sizeof(TA) == 4) {
      cudaFuncSetAttribute(nls_bpp_kernel<TA, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      cudaFuncSetAttribute(nls_bpp_kernel<TA, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    }
    if (a.inner && a.reset_inner) {
      set_int_kernel<<<1, 32, 0, st>>>(a.inner, 0, 1);
      note_launches(1);
    }
    int max_iter = a.opts.bpp_max_iter > 0 ? a.opts.bpp_max_iter : 10 * a.R;
    auto k = nls_bpp_kernel<TA, 0>;
    if constexpr (sizeof(TA) == 4) {
      if (a.R <= 16) k = nls_bpp_kernel<TA, 16>;
      else if (a.R <= 32) k = nls_bpp_kernel<TA, 32>;
    }
    k<<<blocks, 32 * BPP_WARPS, smem, st>>>(a.rows, a.R, a.S, (const TA*)a.M, (TA*)a.H, a.lambda,
                                           max_iter, a.inner, a.flags);
    note_launches(1);
    return cudaGetLastError();
  }
  if (a.inner && a.alg != PLANC_ADMM && a.alg != PLANC_NES) {
    int v = a.alg == PLANC_PGD ? std::max(1, a.opts.pgd_steps) : 1;
    set_int_kernel<<<1, 32, 0, st>>>(a.inner, v, 1);
    note_launches(1);
  }
  if (a.R <= 16) return run_rowwise<TA, 16>(a, st);
  if (a.R <= 32) return run_rowwise<TA, 32>(a, st);
  return run_rowwise<TA, 64>(a, st);
}

}  // namespace

cudaError_t launch_inv_prep(bool f64, const double* S, int R, double* scr, int ucp,
                            cudaStream_t st) {
  const size_t smem = ((size_t)R * (R + 1) + R) * sizeof(double);
  cudaFuncSetAttribute(admm_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  admm_prep_kernel<<<1, 256, smem, st>>>(S, R, scr, f64 ? 1 : 0, ucp);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_nes_prep(bool f64, const double* S, int R, double* scr, cudaStream_t st) {
  if (f64) {
    const size_t psm = ((size_t)R * (R + 1) + 4 * 64) * sizeof(double);
    cudaFuncSetAttribute(nes_prep_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)psm);
    nes_prep_kernel<double><<<1, 64, psm, st>>>(S, R, scr, kNesKappa);
  } else {
    const size_t psm = ((size_t)R * (R + 1) + 4 * 64) * sizeof(float);
    cudaFuncSetAttribute(nes_prep_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)psm);
    nes_prep_kernel<float><<<1, 64, psm, st>>>(S, R, scr, kNesKappa);
  }
  note_launches(1);
  return cudaGetLastError();
}

size_t nls_scratch_doubles(int64_t rows, int R) {
  int64_t blocks = (rows + ROWS_PER_CTA - 1) / ROWS_PER_CTA;
  const size_t per_block = std::max<size_t>((size_t)PLANC_MAX_ADMM_STEPS * 4,
                                             (size_t)PLANC_MAX_NES_STEPS * 2);
  return ADMM_W + 2 * (size_t)R * R + per_block * blocks + 64;
}

cudaError_t launch_nls(const NlsArgs& a, cudaStream_t st) {
  if (a.R > PLANC_MAX_NLS_R) return cudaErrorNotSupported;
  if (a.f64) return run_nls_t<double>(a, st);
  return run_nls_t<float>(a, st);
}

}  // namespace planc
