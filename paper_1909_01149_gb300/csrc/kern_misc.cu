// Reductions of Alg. 1 / Alg. 4: ||X||^2, Grams and their Hadamard product,
// column normalisation, and the relative-error identity.
//
// GB300's FP64 pipe is a small fraction of its FP32 rate, so FP64 is used
// where the paper's numerics need it (cross-block accumulation, the R x R
// products of the error identity) and FP32 partial sums over short runs feed
// it.  Every cross-block reduction sums partials in a fixed order, so
// results are bit-reproducible run to run.
#include <algorithm>

#include "internal.h"

namespace planc {

namespace {

// ---- alpha = ||X||^2 ---------------------------------------------------------
template <typename TX>
__global__ void __launch_bounds__(256)
sqnorm_kernel(const TX* __restrict__ X, int64_t n, double* __restrict__ part) {
  using TA = typename AccOf<TX>::type;
  constexpr int VEC = 16 / sizeof(TX);
  __shared__ double sred[8];
  double acc = 0.0;
  const int64_t nv = n / VEC;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool aligned = ((uintptr_t)X & 15) == 0;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (aligned) {
    const uint4* Xv = reinterpret_cast<const uint4*>(X);
    // four 16-byte vectors (up to 32 elements) per FP64 accumulation
    for (; i < nv; i += stride * 4) {
      TA s = TA(0);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int64_t j = i + stride * u;
        if (j < nv) {
          uint4 w = __ldg(Xv + j);
          const TX* e = reinterpret_cast<const TX*>(&w);
#pragma unroll
          for (int t = 0; t < VEC; ++t) { TA v = to_acc(e[t]); s = fma(v, v, s); }
        }
      }
      acc += (double)s;
    }
    // tail
    for (int64_t j = nv * VEC + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += stride) {
      double v = (double)to_acc(X[j]);
      acc += v * v;
    }
  } else {
    for (int64_t j = i; j < n; j += stride) {
      double v = (double)to_acc(X[j]);
      acc += v * v;
    }
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sred[w];
    part[blockIdx.x] = s;
  }
}

__global__ void sum_partials_kernel(const double* __restrict__ part, int n, double* out) {
  // one warp, fixed order: lane-strided sums then a shuffle tree
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) s += part[i];
  s = warp_sum(s);
  if (threadIdx.x == 0) *out = s;
}

// ---- S^(n) = Hadamard of the other Grams ----------------------------------------
__global__ void gram_hadamard_kernel(const double* __restrict__ G, int N, int n, int R,
                                     double* __restrict__ S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int RR = R * R;
  if (i >= RR) return;
  double s = 1.0;
  for (int k = 0; k < N; ++k)
    if (k != n) s *= G[(int64_t)k * RR + i];
  S[i] = s;
}

// ---- normalisation step 1: column sums of squares (+ <M, Hhat>) -------------------
template <typename TA>
__global__ void __launch_bounds__(256)
colsq_kernel(int64_t rows, int R, int64_t rb, const TA* __restrict__ Hh,
             const TA* __restrict__ M, double* __restrict__ colsq_part,
             double* __restrict__ dot_part) {
  __shared__ double s_col[256];
  __shared__ double s_dot[256];
  const int tid = threadIdx.x;
  const int nsub = 256 / R;                 // R <= 256
  const int r = tid % R, sub = tid / R;
  const bool active = sub < nsub;
  const int64_t i0 = (int64_t)blockIdx.x * rb;
  const int64_t i1 = min(rows, i0 + rb);
  TA a = TA(0), d = TA(0);
  if (active) {
    for (int64_t i = i0 + sub; i < i1; i += nsub) {
      TA v = Hh[i * R + r];
      a = fma(v, v, a);
      if (M) d = fma(M[i * R + r], v, d);
    }
  }
  s_col[tid] = active ? (double)a : 0.0;
  s_dot[tid] = active ? (double)d : 0.0;
  __syncthreads();
  if (tid < R) {
    double s = 0.0;
    for (int j = 0; j < nsub; ++j) s += s_col[tid + j * R];
    colsq_part[(int64_t)blockIdx.x * R + tid] = s;
  }
  if (M && tid == 0) {
    double s = 0.0;
    for (int j = 0; j < nsub * R; ++j) s += s_dot[j];
    dot_part[blockIdx.x] = s;
  }
}

// ---- normalisation step 2: lambda, scale, Gram partials ---------------------------
constexpr int SG_ROWS = 32;

template <typename TA>
__global__ void __launch_bounds__(256)
scale_gram_kernel(int64_t rows, int R, int64_t rb, TA* __restrict__ H,
                  const double* __restrict__ colsq_part, int nblk,
                  double* __restrict__ lambda, double* __restrict__ gram_part, int do_scale) {
  extern __shared__ unsigned char smem_raw[];
  double* s_lam = reinterpret_cast<double*>(smem_raw);               // R: 1 / lambda
  TA* s_rows = reinterpret_cast<TA*>(s_lam + R);                      // SG_ROWS x R
  const int tid = threadIdx.x;
  for (int r = tid; r < R; r += blockDim.x) {
    double s = 0.0;
    if (do_scale)
      for (int b = 0; b < nblk; ++b) s += colsq_part[(int64_t)b * R + r];
    double l = do_scale ? sqrt(s) : 1.0;
    s_lam[r] = l > 0.0 ? 1.0 / l : 0.0;  // one division per column, not per element
    if (blockIdx.x == 0 && lambda && do_scale) lambda[r] = l;
  }
  __syncthreads();
  const int64_t i0 = (int64_t)blockIdx.x * rb;
  const int64_t i1 = min(rows, i0 + rb);
  const int RR = R * R;
  // each thread owns (up to) ceil(R*R / 256) Gram entries
  constexpr int MAXE = (PLANC_MAX_NLS_R * PLANC_MAX_NLS_R + 255) / 256;
  TA g[MAXE];
  const int ne = (RR + 255) / 256;
  for (int e = 0; e < MAXE; ++e) g[e] = TA(0);
  for (int64_t c0 = i0; c0 < i1; c0 += SG_ROWS) {
    const int nr = (int)min((int64_t)SG_ROWS, i1 - c0);
    __syncthreads();
    for (int e = tid; e < nr * R; e += blockDim.x) {
      int lr = e / R, r = e - lr * R;
      int64_t gi = (c0 + lr) * R + r;
      const double il = s_lam[r];
      TA v = H[gi];
      if (do_scale) {
        v = (TA)((double)v * il);  // zero column (lambda 0): stays 0
        H[gi] = v;
      }
      s_rows[lr * R + r] = v;
    }
    __syncthreads();
    for (int e = 0; e < ne; ++e) {
      int idx = tid + 256 * e;
      if (idx < RR) {
        int r = idx / R, s = idx - r * R;
        TA acc = g[e];
        for (int lr = 0; lr < nr; ++lr) acc = fma(s_rows[lr * R + r], s_rows[lr * R + s], acc);
        g[e] = acc;
      }
    }
  }
  for (int e = 0; e < ne; ++e) {
    int idx = tid + 256 * e;
    if (idx < RR) gram_part[(int64_t)blockIdx.x * RR + idx] = (double)g[e];
  }
}

// ---- G = sum of Gram partials --------------------------------------------------------
__global__ void gram_reduce_kernel(int R, const double* __restrict__ gram_part, int nblk,
                                   double* __restrict__ G, float* __restrict__ Gf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int RR = R * R;
  if (i >= RR) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += gram_part[(int64_t)b * RR + i];
  G[i] = s;
  if (Gf) Gf[i] = (float)s;
}

// ---- error identity (Alg. 4) ---------------------------------------------------------
// gamma = lambda^T (G^(1) * ... * G^(N)) lambda, beta = sum of dot partials,
// eps = sqrt(max(0, alpha - 2 beta + gamma) / alpha).
__global__ void __launch_bounds__(256)
fit_kernel(int R, const double* __restrict__ Gall, int N, const double* __restrict__ lambda,
           const double* __restrict__ dot_part, int dot_nblk, const double* __restrict__ alpha,
           double* __restrict__ fit_out) {
  __shared__ double sred[8];
  const int RR = R * R;
  double gsum = 0.0;
  for (int i = threadIdx.x; i < RR; i += blockDim.x) {
    double p = 1.0;
    for (int k = 0; k < N; ++k) p *= Gall[(int64_t)k * RR + i];
    int r = i / R, s = i - r * R;
    gsum += lambda[r] * lambda[s] * p;
  }
  gsum = warp_sum(gsum);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = gsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double gamma = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) gamma += sred[w];
    double beta = 0.0;
    for (int b = 0; b < dot_nblk; ++b) beta += dot_part[b];
    double a = *alpha;
    double rad = a - 2.0 * beta + gamma;
    double eps = a > 0.0 ? sqrt(fmax(0.0, rad) / a) : 0.0;
    fit_out[0] = eps;
    fit_out[1] = beta;
    fit_out[2] = gamma;
  }
}

template <typename TA>
__global__ void __launch_bounds__(256)
dot_lambda_kernel(int64_t rows, int R, int64_t rb, const TA* __restrict__ M,
                  const TA* __restrict__ H, const double* __restrict__ lambda,
                  double* __restrict__ dot_part) {
  __shared__ double sred[8];
  const int64_t i0 = (int64_t)blockIdx.x * rb;
  const int64_t i1 = min(rows, i0 + rb);
  double acc = 0.0;
  for (int64_t e = i0 * R + threadIdx.x; e < i1 * R; e += blockDim.x) {
    int r = (int)(e % R);
    acc += (double)M[e] * (double)H[e] * lambda[r];
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sred[w];
    dot_part[blockIdx.x] = s;
  }
}

// G^(n) = H^(n)T H^(n) for every mode in one launch (blockIdx.y = n), one
// thread per entry looping over the rows: FP32 products over 32-row chunks,
// FP64 across chunks (the precision of the block-partial path), written in
// FP64 and as the FP32 copy.  For factors with few rows (the loop is per
// thread).
struct GramModes {
  int64_t rows[PLANC_MAX_N];
  const void* H[PLANC_MAX_N];
};

template <typename TA>
__global__ void gram_all_kernel(GramModes gm, int R, double* __restrict__ G,
                                float* __restrict__ Gf) {
  const int n = blockIdx.y;
  const int RR = R * R;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= RR) return;
  const int r = e / R, s = e - (e / R) * R;
  const TA* H = static_cast<const TA*>(gm.H[n]);
  const int64_t rows = gm.rows[n];
  double g = 0.0;
  for (int64_t i0 = 0; i0 < rows; i0 += 32) {
    TA a = TA(0);
    const int64_t i1 = min(rows, i0 + 32);
    for (int64_t i = i0; i < i1; ++i) a = fma(H[i * R + r], H[i * R + s], a);
    g += (double)a;
  }
  G[(size_t)n * RR + e] = g;
  if (Gf) Gf[(size_t)n * RR + e] = (float)g;
}

// ---- CP-loss gradient (Eq. nncp objective) -------------------------------------------
// dH^(n) = 2 (H^(n) S^(n) - M^(n)) for every mode in one launch (blockIdx.y =
// n): each CTA forms S^(n), the Hadamard product of the other modes' Grams
// (FP32 copies for FP32 factors, FP64 otherwise), in shared memory first.
struct GradModes {
  int64_t rows[PLANC_MAX_N];
  const void* H[PLANC_MAX_N];
  void* G[PLANC_MAX_N];  // in: M^(n); out: the gradient
};

template <typename TA>
__global__ void cp_grad_all_kernel(GradModes gm, int N, int R, const double* __restrict__ G64,
                                   const float* __restrict__ G32) {
  extern __shared__ __align__(16) unsigned char cg_smem[];
  TA* Ss = reinterpret_cast<TA*>(cg_smem);
  const int n = blockIdx.y;
  const int RR = R * R;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    TA v = TA(1);
    for (int k = 0; k < N; ++k)
      if (k != n) v *= sizeof(TA) == 4 ? (TA)G32[(size_t)k * RR + e] : (TA)G64[(size_t)k * RR + e];
    Ss[e] = v;
  }
  __syncthreads();
  const TA* H = static_cast<const TA*>(gm.H[n]);
  TA* Gd = static_cast<TA*>(gm.G[n]);
  const int64_t total = gm.rows[n] * (int64_t)R;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / R;
    const int r = (int)(e - i * R);
    const TA* h = H + i * R;
    TA acc = TA(0);
    for (int k = 0; k < R; ++k) acc = fma(h[k], Ss[k * R + r], acc);
    Gd[e] = TA(2) * (acc - Gd[e]);
  }
}

__global__ void fill_kernel(double* p, double v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

}  // namespace

int sqnorm_blocks(int64_t n, int sm_count) {
  int64_t b = (n + 256 * 64 - 1) / (256 * 64);
  b = std::min<int64_t>(b, 4LL * sm_count);
  return (int)std::max<int64_t>(b, 1);
}

cudaError_t launch_sqnorm(planc_dtype_t xdt, const void* X, int64_t n, double* part, int nblk,
                          double* alpha, cudaStream_t st) {
  switch (xdt) {
    case PLANC_F64: sqnorm_kernel<double><<<nblk, 256, 0, st>>>((const double*)X, n, part); break;
    case PLANC_F32: sqnorm_kernel<float><<<nblk, 256, 0, st>>>((const float*)X, n, part); break;
    case PLANC_BF16:
      sqnorm_kernel<__nv_bfloat16><<<nblk, 256, 0, st>>>((const __nv_bfloat16*)X, n, part);
      break;
    case PLANC_F16: sqnorm_kernel<__half><<<nblk, 256, 0, st>>>((const __half*)X, n, part); break;
  }
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_partials_kernel<<<1, 32, 0, st>>>(part, nblk, alpha);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gram_hadamard(const double* G, int N, int n, int R, double* S,
                                 cudaStream_t st) {
  int RR = R * R;
  gram_hadamard_kernel<<<(RR + 255) / 256, 256, 0, st>>>(G, N, n, R, S);
  note_launches(1);
  return cudaGetLastError();
}

// row blocks of the general-path normalisation / Gram kernels: 8 rows each up
// to 256 blocks (few-row factors still spread over many SMs)
int rowblocks(int64_t rows) {
  int64_t b = (rows + 7) / 8;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 256));
}

static int64_t rows_per_block(int64_t rows, int nblk) { return (rows + nblk - 1) / nblk; }

cudaError_t launch_colsq(bool f64, int64_t rows, int R, const void* Hhat, const void* M,
                         double* colsq_part, double* dot_part, int nblk, cudaStream_t st) {
  int64_t rb = rows_per_block(rows, nblk);
  if (f64)
    colsq_kernel<double><<<nblk, 256, 0, st>>>(rows, R, rb, (const double*)Hhat,
                                               (const double*)M, colsq_part, dot_part);
  else
    colsq_kernel<float><<<nblk, 256, 0, st>>>(rows, R, rb, (const float*)Hhat, (const float*)M,
                                              colsq_part, dot_part);
    note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scale_gram(bool f64, int64_t rows, int R, void* H, const double* colsq_part,
                              int nblk, double* lambda, double* gram_part, bool scale,
                              cudaStream_t st) {
  int64_t rb = rows_per_block(rows, nblk);
  size_t smem = R * sizeof(double) + (size_t)SG_ROWS * R * (f64 ? 8 : 4);
  if (f64) {
    cudaFuncSetAttribute(scale_gram_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    scale_gram_kernel<double><<<nblk, 256, smem, st>>>(rows, R, rb, (double*)H, colsq_part, nblk,
                                                       lambda, gram_part, scale ? 1 : 0);
    note_launches(1);
  } else {
    cudaFuncSetAttribute(scale_gram_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    scale_gram_kernel<float><<<nblk, 256, smem, st>>>(rows, R, rb, (float*)H, colsq_part, nblk,
                                                      lambda, gram_part, scale ? 1 : 0);
    note_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_gram_reduce(int R, const double* gram_part, int nblk, double* G, float* Gf,
                               cudaStream_t st) {
  int RR = R * R;
  gram_reduce_kernel<<<(RR + 255) / 256, 256, 0, st>>>(R, gram_part, nblk, G, Gf);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fit(int R, const double* Gall, int N, const double* lambda,
                       const double* dot_part, int dot_nblk, const double* alpha,
                       double* fit_out, cudaStream_t st) {
  fit_kernel<<<1, 256, 0, st>>>(R, Gall, N, lambda, dot_part, dot_nblk, alpha, fit_out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dot_lambda(bool f64, int64_t rows, int R, const void* M, const void* H,
                              const double* lambda, double* dot_part, int nblk,
                              cudaStream_t st) {
  int64_t rb = rows_per_block(rows, nblk);
  if (f64)
    dot_lambda_kernel<double><<<nblk, 256, 0, st>>>(rows, R, rb, (const double*)M,
                                                    (const double*)H, lambda, dot_part);
  else
    dot_lambda_kernel<float><<<nblk, 256, 0, st>>>(rows, R, rb, (const float*)M,
                                                   (const float*)H, lambda, dot_part);
    note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_cp_grad_all(bool f64, int N, const int64_t* rows, int R,
                               void* const* H, void* const* dH, const double* G64,
                               const float* G32, int sm_count, cudaStream_t st) {
  GradModes gm{};
  int64_t maxel = 1;
  for (int n = 0; n < N; ++n) {
    gm.rows[n] = rows[n];
    gm.H[n] = H[n];
    gm.G[n] = dH[n];
    maxel = std::max<int64_t>(maxel, rows[n] * R);
  }
  const int bx = (int)std::max<int64_t>(1, std::min<int64_t>((maxel + 255) / 256, 4LL * sm_count));
  const dim3 grid(bx, N);
  if (f64)
    cp_grad_all_kernel<double><<<grid, 256, (size_t)R * R * 8, st>>>(gm, N, R, G64, G32);
  else
    cp_grad_all_kernel<float><<<grid, 256, (size_t)R * R * 4, st>>>(gm, N, R, G64, G32);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gram_all(bool f64, int N, const int64_t* rows, int R, void* const* H,
                            double* G, float* Gf, cudaStream_t st) {
  GramModes gm{};
  for (int n = 0; n < N; ++n) {
    gm.rows[n] = rows[n];
    gm.H[n] = H[n];
  }
  const dim3 grid((unsigned)((R * R + 255) / 256), (unsigned)N);
  if (f64) gram_all_kernel<double><<<grid, 256, 0, st>>>(gm, R, G, Gf);
  else gram_all_kernel<float><<<grid, 256, 0, st>>>(gm, R, G, Gf);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* p, double v, int64_t n, cudaStream_t st) {
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1024));
  fill_kernel<<<blocks, 256, 0, st>>>(p, v, n);
  note_launches(1);
  return cudaGetLastError();
}

// ---- outer acceleration of the Nesterov-type solve (Sec. 4.3.5, Eq. nesouterupd) ----
namespace {

__device__ __forceinline__ int accel_mode(const AccelModes& t, int64_t e) {
  int n = 0;
  while (n + 1 < t.N && e >= t.off[n + 1]) ++n;
  return n;
}

// Hc^(n) = [F^(n) + s (F^(n) - F_prev^(n))]_+ with F^(N) = H^(N) diag(lam),
// s = i^(1/N), i = 1 + the number of completed outer iterations.
template <typename TA>
__global__ void __launch_bounds__(256)
accel_extrapolate_kernel(AccelModes t, const double* __restrict__ lam,
                         const double* __restrict__ lam_prev, const int* __restrict__ counter) {
  const double s = pow((double)(*counter + 1), 1.0 / t.N);
  const int64_t total = t.off[t.N];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int n = accel_mode(t, e);
    const int64_t idx = e - t.off[n];
    double F = (double)((const TA*)t.H[n])[idx];
    double Fp = (double)((const TA*)t.Hp[n])[idx];
    if (n == t.N - 1) {
      const int r = (int)(idx % t.R);
      F *= lam[r];
      Fp *= lam_prev[r];
    }
    const double c = fma(s, F - Fp, F);
    ((TA*)t.Hc[n])[idx] = (TA)(c > 0.0 ? c : 0.0);
  }
}

// lam_c[r] = prod_n nu^(n)_r (the candidate's column norms, mode order)
__global__ void accel_lam_kernel(const double* __restrict__ nu, int N, int R,
                                 double* __restrict__ lam_c) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double p = nu[r];
  for (int n = 1; n < N; ++n) p *= nu[(size_t)n * R + r];
  lam_c[r] = p;
}

// accept iff an earlier iterate exists and the candidate's error is lower
__global__ void accel_decide_kernel(double* __restrict__ scal, const int* __restrict__ counter,
                                    int32_t* __restrict__ hist, int cap, int* __restrict__ flags) {
  const int it = *counter;
  const bool acc = it >= 1 && scal[16] < scal[8];
  scal[24] = acc ? 1.0 : 0.0;
  if (it < cap) hist[it] = acc ? 1 : 0;
  if (acc) {
    flags[6] += 1;
    scal[8] = scal[16];
    scal[9] = scal[17];
    scal[10] = scal[18];
  }
}

// the accepted iterate becomes the current and the previous one
template <typename TA>
__global__ void __launch_bounds__(256)
accel_select_kernel(AccelModes t, double* __restrict__ lam, double* __restrict__ lam_prev,
                    const double* __restrict__ lam_c, double* __restrict__ G,
                    float* __restrict__ Gf, const double* __restrict__ Gc,
                    const double* __restrict__ scal) {
  const bool acc = scal[24] != 0.0;
  const int64_t total = t.off[t.N];
  const int64_t tid0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = tid0; e < total; e += stride) {
    const int n = accel_mode(t, e);
    const int64_t idx = e - t.off[n];
    TA v = acc ? ((const TA*)t.Hc[n])[idx] : ((const TA*)t.H[n])[idx];
    if (acc) ((TA*)t.H[n])[idx] = v;
    ((TA*)t.Hp[n])[idx] = v;
  }
  for (int64_t r = tid0; r < t.R; r += stride) {
    const double l = acc ? lam_c[r] : lam[r];
    lam[r] = l;
    lam_prev[r] = l;
  }
  if (acc)
    for (int64_t e = tid0; e < (int64_t)t.N * t.R * t.R; e += stride) {
      G[e] = Gc[e];
      Gf[e] = (float)Gc[e];
    }
}

int accel_blocks(const AccelModes& t) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((t.off[t.N] + 255) / 256, 592));
}

}  // namespace

cudaError_t launch_accel_extrapolate(bool f64, const AccelModes& t, const double* lam,
                                     const double* lam_prev, const int* counter, cudaStream_t st) {
  if (f64)
    accel_extrapolate_kernel<double><<<accel_blocks(t), 256, 0, st>>>(t, lam, lam_prev, counter);
  else
    accel_extrapolate_kernel<float><<<accel_blocks(t), 256, 0, st>>>(t, lam, lam_prev, counter);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_accel_finish(bool /*f64: lambda is FP64 either way*/, const AccelModes& t, const double* nu, double* lam_c,
                                cudaStream_t st) {
  accel_lam_kernel<<<(t.R + 63) / 64, 64, 0, st>>>(nu, t.N, t.R, lam_c);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_accel_select(bool f64, const AccelModes& t, double* scal, const int* counter,
                                int32_t* hist, int cap, int* flags, double* lam, double* lam_prev,
                                const double* lam_c, double* G, float* Gf, const double* Gc,
                                cudaStream_t st) {
  accel_decide_kernel<<<1, 1, 0, st>>>(scal, counter, hist, cap, flags);
  if (f64)
    accel_select_kernel<double><<<accel_blocks(t), 256, 0, st>>>(t, lam, lam_prev, lam_c, G, Gf,
                                                                 Gc, scal);
  else
    accel_select_kernel<float><<<accel_blocks(t), 256, 0, st>>>(t, lam, lam_prev, lam_c, G, Gf,
                                                                Gc, scal);
  note_launches(2);
  return cudaGetLastError();
}

}  // namespace planc
