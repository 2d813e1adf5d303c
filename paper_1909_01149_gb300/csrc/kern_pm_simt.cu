// Partial MTTKRP on CUDA cores (the general path): any dtype, shape and rank.
//
// The two root branches of the dimension tree (Sec. 4.2.2, Alg. 3) are
//   left : T^{1:S}   = X_(1:S)   K^{S+1:N}   (rows of X_(1:S) contiguous)
//   right: T^{S+1:N} = X_(1:S)^T K^{1:S}     (reduction over the contiguous dim)
// Both are GEMMs whose B operand is a partial Khatri-Rao product; here it is
// generated tile by tile in shared memory and never materialised in HBM.
// Register tiling: 128 x BN output tile per CTA, 4 x (BN/8) per thread,
// k-tiles of 16 staged in shared memory, two-level accumulation (the running
// sum is folded into a second accumulator every 128 k) to keep FP32 rounding
// growth at about sqrt of the tile count.
#include <algorithm>

#include "internal.h"

namespace planc {

namespace {

constexpr int BM = 128;
constexpr int BK = 16;
constexpr int FOLD = 8;  // fold the accumulator every FOLD k-tiles

template <typename TX, int BN, bool LEFT>
__global__ void __launch_bounds__(256)
pm_simt_kernel(const TX* __restrict__ X, int64_t L, Krp<typename AccOf<TX>::type> K, int R,
               int64_t Mdim, int64_t Kdim, int64_t kchunk,
               typename AccOf<TX>::type* __restrict__ out, int out_mode) {
  using TA = typename AccOf<TX>::type;
  constexpr int TN = BN / 8;
  __shared__ TA As[BK][BM + 1];
  __shared__ TA Bs[BK][BN];

  const int tid = threadIdx.x;
  const int mg = tid & 31;
  const int ng = tid >> 5;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int r0 = blockIdx.y * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = min(Kdim, kbeg + kchunk);

  TA acc[4][TN], acc2[4][TN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = acc2[i][j] = TA(0);

  int tile = 0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK, ++tile) {
    // A tile: As[kk][mm] = A[m0 + mm, k0 + kk]
#pragma unroll
    for (int i = 0; i < (BM * BK) / 256; ++i) {
      int e = tid + 256 * i;
      int kk, mm;
      if (LEFT) { kk = e >> 7; mm = e & 127; } else { kk = e & 15; mm = e >> 4; }
      int64_t gm = m0 + mm, gk = k0 + kk;
      TA v = TA(0);
      if (gm < Mdim && gk < kend)
        v = to_acc(LEFT ? X[gm + L * gk] : X[gk + L * gm]);
      As[kk][mm] = v;
    }
    // B tile: Bs[kk][nn] = K[k0 + kk, r0 + nn]
    for (int e = tid; e < BK * BN; e += 256) {
      int kk = e / BN, nn = e - kk * BN;
      int64_t gk = k0 + kk;
      int r = r0 + nn;
      Bs[kk][nn] = (gk < kend && r < R) ? krp_at(K, gk, r) : TA(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TA a[4], b[TN];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][mg + 32 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][ng * TN + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
    if ((tile + 1) % FOLD == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) { acc2[i][j] += acc[i][j]; acc[i][j] = TA(0); }
    }
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t m = m0 + mg + 32 * i;
    if (m >= Mdim) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int r = r0 + ng * TN + j;
      if (r >= R) continue;
      TA v = acc2[i][j] + acc[i][j];
      if (out_mode == 1) out[m * R + r] = v;
      else if (out_mode == 0) out[m + Mdim * r] = v;
      else out[(int64_t)blockIdx.z * Mdim * R + m + Mdim * r] = v;
    }
  }
}

template <typename TA>
__global__ void split_reduce_kernel(const TA* __restrict__ part, int nsplit, int64_t Mdim,
                                    int R, TA* __restrict__ out, int rowmajor) {
  pdl_wait();
  pdl_trigger();
  int64_t n = Mdim * R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    TA s = TA(0), c = TA(0);
    for (int z = 0; z < nsplit; ++z) neumaier_add(s, c, part[(int64_t)z * n + e]);
    int64_t m = e % Mdim;
    int r = (int)(e / Mdim);
    TA v = s + c;
    if (rowmajor) out[m * R + r] = v; else out[e] = v;
  }
}

template <typename TX, int BN, bool LEFT>
cudaError_t run_pm(const TX* X, int64_t L, int64_t C, const KrpHost& kh, int R, void* out,
                   bool rowmajor, void* part, int nsplit, cudaStream_t st) {
  using TA = typename AccOf<TX>::type;
  Krp<TA> K{};
  K.nm = kh.nm;
  K.R = R;
  for (int m = 0; m < kh.nm; ++m) { K.dim[m] = kh.dim[m]; K.H[m] = (const TA*)kh.H[m]; }
  int64_t Mdim = LEFT ? L : C, Kdim = LEFT ? C : L;
  int64_t kchunk = (Kdim + nsplit - 1) / nsplit;
  kchunk = (kchunk + BK - 1) / BK * BK;
  dim3 grid((unsigned)((Mdim + BM - 1) / BM), (unsigned)((R + BN - 1) / BN), (unsigned)nsplit);
  if (nsplit == 1) {
    pm_simt_kernel<TX, BN, LEFT><<<grid, 256, 0, st>>>(X, L, K, R, Mdim, Kdim, kchunk,
                                                       (TA*)out, rowmajor ? 1 : 0);
    note_launches(1);
    return cudaGetLastError();
  }
  pm_simt_kernel<TX, BN, LEFT><<<grid, 256, 0, st>>>(X, L, K, R, Mdim, Kdim, kchunk,
                                                     (TA*)part, 2);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_split_reduce(sizeof(TA) == 8, part, nsplit, Mdim, R, out, rowmajor, st);
}

template <typename TX, bool LEFT>
cudaError_t run_pm_bn(const TX* X, int64_t L, int64_t C, const KrpHost& kh, int R, void* out,
                      bool rowmajor, void* part, int nsplit, cudaStream_t st) {
  if (R <= 8) return run_pm<TX, 8, LEFT>(X, L, C, kh, R, out, rowmajor, part, nsplit, st);
  if (R <= 16) return run_pm<TX, 16, LEFT>(X, L, C, kh, R, out, rowmajor, part, nsplit, st);
  return run_pm<TX, 32, LEFT>(X, L, C, kh, R, out, rowmajor, part, nsplit, st);
}

template <typename TX>
cudaError_t run_pm_side(const TX* X, int64_t L, int64_t C, bool left, const KrpHost& kh,
                        int R, void* out, bool rowmajor, void* part, int nsplit,
                        cudaStream_t st) {
  if (left) return run_pm_bn<TX, true>(X, L, C, kh, R, out, rowmajor, part, nsplit, st);
  return run_pm_bn<TX, false>(X, L, C, kh, R, out, rowmajor, part, nsplit, st);
}

}  // namespace

int pm_simt_nsplit(bool left, int64_t L, int64_t C, int R, int sm_count) {
  int64_t Mdim = left ? L : C, Kdim = left ? C : L;
  int bn = R <= 8 ? 8 : R <= 16 ? 16 : 32;
  int64_t tiles = ((Mdim + BM - 1) / BM) * ((R + bn - 1) / bn);
  int64_t target = 4LL * sm_count;
  int64_t ns = (target + tiles - 1) / tiles;
  int64_t maxs = Kdim / (BK * FOLD);
  if (ns > maxs) ns = maxs;
  if (ns > 1024) ns = 1024;
  if (ns < 1) ns = 1;
  return (int)ns;
}

cudaError_t launch_pm_simt(planc_dtype_t xdt, const void* X, int64_t L, int64_t C, bool left,
                           const KrpHost& krp, int R, void* out, bool out_rowmajor, void* part,
                           int nsplit, cudaStream_t st) {
  switch (xdt) {
    case PLANC_F64:
      return run_pm_side((const double*)X, L, C, left, krp, R, out, out_rowmajor, part, nsplit, st);
    case PLANC_F32:
      return run_pm_side((const float*)X, L, C, left, krp, R, out, out_rowmajor, part, nsplit, st);
    case PLANC_BF16:
      return run_pm_side((const __nv_bfloat16*)X, L, C, left, krp, R, out, out_rowmajor, part,
                         nsplit, st);
    case PLANC_F16:
      return run_pm_side((const __half*)X, L, C, left, krp, R, out, out_rowmajor, part, nsplit, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_split_reduce(bool f64, const void* part, int nsplit, int64_t Mdim, int R,
                                void* out, bool out_rowmajor, cudaStream_t st) {
  int64_t n = Mdim * R;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  if (blocks < 1) blocks = 1;
  cudaError_t e;
  if (f64)
    e = launch_pdl(split_reduce_kernel<double>, dim3(blocks), dim3(256), 0, st,
                   (const double*)part, nsplit, Mdim, R, (double*)out, out_rowmajor ? 1 : 0);
  else
    e = launch_pdl(split_reduce_kernel<float>, dim3(blocks), dim3(256), 0, st,
                   (const float*)part, nsplit, Mdim, R, (float*)out, out_rowmajor ? 1 : 0);
  note_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace planc
