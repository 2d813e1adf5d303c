// Batched kernels for many small 3-way instances solved together: every
// launch covers all instances through a table of work items (instance, tile),
// and each CTA walks a contiguous run of items so that per-instance staging
// (a factor in shared memory) is redone only when the instance changes.
//
// Per outer iteration (Alg. 1 with the dimension tree of Alg. 3, N = 3, S = 2):
//   T^{1:2} = X_(1:2) H^(3)                 batch_pm_left   (first X pass)
//   M^(1)   = T^{1:2} x_2 H^(2)             batch_contract_rest
//   M^(2)   = T^{1:2} x_1 H^(1) (updated)    batch_contract_first
//   M^(3)   = X_(1:2)^T (H^(2) . H^(1))      batch_pm_right  (second X pass)
// with the fused per-mode update (kern_mode.cu) between them.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"

namespace planc {

namespace {

constexpr int BR = 32;  // widest rank class of the batched kernels (R <= 32)
constexpr int KU = 8;   // X loads a thread keeps in flight in the partial MTTKRPs

// Rank blocking: an instance's partial MTTKRPs run with its rank padded to
// the smallest class of the schedule that holds it (sched 0: 32; 1: 16, 32;
// 2: 8, 16, 32), so small ranks do not pay for 32 columns.
__device__ __forceinline__ int rank_class(int R, int sched) {
  if (sched >= 2 && R <= 8) return 8;
  if (sched >= 1 && R <= 16) return 16;
  return 32;
}

__device__ __forceinline__ float ldx(const BatchInst& b, int64_t e) {
  if (b.xbf16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(b.X)[e]);
  return __ldg(reinterpret_cast<const float*>(b.X) + e);
}

// first and one-past-last item of this CTA's contiguous run
__device__ __forceinline__ void item_run(int nitems, int& i0, int& i1) {
  const int per = (nitems + gridDim.x - 1) / gridDim.x;
  i0 = min(nitems, (int)blockIdx.x * per);
  i1 = min(nitems, i0 + per);
}

// rows f..f+nrow of a row-major nrow x R factor into shared memory with
// stride BRC (padding columns zero)
__device__ __forceinline__ void stage_factor(float* dst, const float* H, int nrow, int R,
                                             int BRC) {
  for (int e = threadIdx.x; e < nrow * BRC; e += blockDim.x) {
    const int i = e / BRC, r = e - (e / BRC) * BRC;
    dst[e] = r < R ? H[(int64_t)i * R + r] : 0.f;
  }
}

// ---- ||X||^2 per instance: items (b, chunk of 65536 elements) ----------------------
__global__ void __launch_bounds__(256)
batch_sqnorm_kernel(const BatchInst* __restrict__ tab, const int2* __restrict__ items,
                    int nitems, double* __restrict__ part) {
  __shared__ double sred[8];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchInst& b = tab[items[it].x];
    const int64_t n = b.I[0] * b.I[1] * b.I[2];
    const int64_t e0 = (int64_t)items[it].y * 65536, e1 = min(n, e0 + 65536);
    double acc = 0.0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const float x = ldx(b, e);
      acc += (double)(x * x);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += sred[w];
      part[it] = s;
    }
    __syncthreads();
  }
}

// alpha_b = sum of the partials of instance b (items of one instance are
// consecutive: first[b] .. first[b + 1] - 1)
__global__ void batch_sqnorm_finish_kernel(const BatchInst* __restrict__ tab, int count,
                                           const int* __restrict__ first,
                                           const double* __restrict__ part) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  double s = 0.0;
  for (int i = first[b]; i < first[b + 1]; ++i) s += part[i];
  *tab[b].alpha = s;
}

// ---- G^(n) = H^(n)T H^(n) of the initial factors, lambda = 1: items (b, n) -------
__global__ void __launch_bounds__(256)
batch_gram_kernel(const BatchInst* __restrict__ tab, int count) {
  const int b = blockIdx.x / 3, n = blockIdx.x - (blockIdx.x / 3) * 3;
  if (b >= count) return;
  const BatchInst& in = tab[b];
  const int R = in.R, rows = (int)in.I[n];
  const float* H = in.H[n];
  if (n == 0 && threadIdx.x < 32) in.lam[threadIdx.x] = 1.0;  // lambda starts at 1
  for (int pr = threadIdx.x; pr < R * R; pr += blockDim.x) {
    const int r = pr / R, s = pr - (pr / R) * R;
    double g = 0.0;
    for (int i0 = 0; i0 < rows; i0 += 32) {  // FP32 over 32 rows, FP64 across
      float a = 0.f;
      for (int i = i0; i < min(rows, i0 + 32); ++i)
        a = fmaf(H[(int64_t)i * R + r], H[(int64_t)i * R + s], a);
      g += (double)a;
    }
    in.G[(size_t)n * R * R + pr] = g;
    in.Gf[(size_t)n * R * R + pr] = (float)g;
  }
}

// ---- T^{1:2}[l, r] = sum_k X[l, k] H3[k, r]: items (b, block of 2 TL rows l) ----------
// Each thread computes two adjacent rows l0, l0 + 1 (l0 even): both share
// every read of H3's row k (staged in shared memory with stride BRC, the rank
// class, read as broadcast 16-byte loads), and when L is even the two X
// values arrive in one load (float2 / bf16x2).  KU k steps issue their X
// loads together.
template <bool BF16>
__device__ __forceinline__ void ldx2(const void* X, int64_t e, bool pair, bool live0,
                                     bool live1, float& a, float& b) {
  if (BF16) {
    const __nv_bfloat16* p = reinterpret_cast<const __nv_bfloat16*>(X) + e;
    if (pair && live1) {
      const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(p);
      a = __low2float(v);
      b = __high2float(v);
    } else {
      a = live0 ? __bfloat162float(p[0]) : 0.f;
      b = live1 ? __bfloat162float(p[1]) : 0.f;
    }
  } else {
    const float* p = reinterpret_cast<const float*>(X) + e;
    if (pair && live1) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(p));
      a = v.x;
      b = v.y;
    } else {
      a = live0 ? __ldg(p) : 0.f;
      b = live1 ? __ldg(p + 1) : 0.f;
    }
  }
}

template <int BRC, bool BF16>
__device__ __forceinline__ void left_rows2(const BatchInst& b, int64_t l0, int64_t L, int C,
                                           int R, const float* bsm) {
  const bool live0 = l0 < L, live1 = l0 + 1 < L;
  // l0 even: X[l0 + L k] starts an aligned pair for every k when L is even
  // and X itself is aligned to a pair
  const bool pair = (L & 1) == 0 &&
                    (reinterpret_cast<uintptr_t>(b.X) & (BF16 ? 3u : 7u)) == 0;
  float a0[BRC], a1[BRC];
#pragma unroll
  for (int r = 0; r < BRC; ++r) { a0[r] = 0.f; a1[r] = 0.f; }
  if (live0) {
    int k = 0;
    for (; k + KU <= C; k += KU) {
      float x0[KU], x1[KU];
#pragma unroll
      for (int u = 0; u < KU; ++u) ldx2<BF16>(b.X, l0 + L * (k + u), pair, live0, live1, x0[u], x1[u]);
#pragma unroll
      for (int u = 0; u < KU; ++u) {
        const float4* h = reinterpret_cast<const float4*>(bsm + (k + u) * BRC);
#pragma unroll
        for (int q = 0; q < BRC / 4; ++q) {
          const float4 hv = h[q];
          a0[4 * q + 0] = fmaf(x0[u], hv.x, a0[4 * q + 0]);
          a0[4 * q + 1] = fmaf(x0[u], hv.y, a0[4 * q + 1]);
          a0[4 * q + 2] = fmaf(x0[u], hv.z, a0[4 * q + 2]);
          a0[4 * q + 3] = fmaf(x0[u], hv.w, a0[4 * q + 3]);
          a1[4 * q + 0] = fmaf(x1[u], hv.x, a1[4 * q + 0]);
          a1[4 * q + 1] = fmaf(x1[u], hv.y, a1[4 * q + 1]);
          a1[4 * q + 2] = fmaf(x1[u], hv.z, a1[4 * q + 2]);
          a1[4 * q + 3] = fmaf(x1[u], hv.w, a1[4 * q + 3]);
        }
      }
    }
    for (; k < C; ++k) {
      float x0, x1;
      ldx2<BF16>(b.X, l0 + L * k, pair, live0, live1, x0, x1);
      const float4* h = reinterpret_cast<const float4*>(bsm + k * BRC);
#pragma unroll
      for (int q = 0; q < BRC / 4; ++q) {
        const float4 hv = h[q];
        a0[4 * q + 0] = fmaf(x0, hv.x, a0[4 * q + 0]);
        a0[4 * q + 1] = fmaf(x0, hv.y, a0[4 * q + 1]);
        a0[4 * q + 2] = fmaf(x0, hv.z, a0[4 * q + 2]);
        a0[4 * q + 3] = fmaf(x0, hv.w, a0[4 * q + 3]);
        a1[4 * q + 0] = fmaf(x1, hv.x, a1[4 * q + 0]);
        a1[4 * q + 1] = fmaf(x1, hv.y, a1[4 * q + 1]);
        a1[4 * q + 2] = fmaf(x1, hv.z, a1[4 * q + 2]);
        a1[4 * q + 3] = fmaf(x1, hv.w, a1[4 * q + 3]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < BRC; ++r)
    if (r < R) {
      if (live0) b.T[l0 + L * r] = a0[r];
      if (live1) b.T[l0 + 1 + L * r] = a1[r];
    }
}

template <int BRC>
__device__ __forceinline__ void left_rows2_dt(const BatchInst& b, int64_t l0, int64_t L, int C,
                                              int R, const float* bsm) {
  if (b.xbf16) left_rows2<BRC, true>(b, l0, L, C, R, bsm);
  else left_rows2<BRC, false>(b, l0, L, C, R, bsm);
}

template <int TL>
__global__ void __launch_bounds__(TL)
batch_pm_left_kernel(const BatchInst* __restrict__ tab, const int2* __restrict__ items,
                     int nitems, int sched) {
  extern __shared__ __align__(16) float bsm[];
  int i0, i1;
  item_run(nitems, i0, i1);
  int cur = -1;
  for (int it = i0; it < i1; ++it) {
    const int bi = items[it].x;
    const BatchInst& b = tab[bi];
    const int64_t L = b.I[0] * b.I[1];
    const int C = (int)b.I[2], R = b.R;
    const int cls = rank_class(R, sched);
    if (bi != cur) {
      __syncthreads();
      stage_factor(bsm, b.H[2], C, R, cls);
      __syncthreads();
      cur = bi;
    }
    const int64_t l0 = ((int64_t)items[it].y * TL + threadIdx.x) * 2;
    if (cls == 8) left_rows2_dt<8>(b, l0, L, C, R, bsm);
    else if (cls == 16) left_rows2_dt<16>(b, l0, L, C, R, bsm);
    else left_rows2_dt<32>(b, l0, L, C, R, bsm);
  }
}

// Sum over the warp of v[r] for r < 32, lane r returning the total of v[r].
__device__ __forceinline__ float reduce_scatter32(float* v, int lane) {
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool upper = (lane & w) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const float send = upper ? v[i] : v[i + w];
      const float keep = upper ? v[i + w] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return v[0];
}

// ---- M^(3)[c, r] = sum_{i1, i2} X[i1, i2, c] H1[i1, r] H2[i2, r]: items (b, c) ----------
// Threads own (i1, range of i2); for each the inner sum over i2 runs with H2
// from shared memory (stride BRC, the rank class) and is then weighted by
// H1[i1, r]; the CTA's per-thread sums are reduced through warp
// reduce-scatters and shared memory.
template <int NT, int BRC>
__device__ __forceinline__ void right_sums(const BatchInst& b, int64_t c, int I1, int I2,
                                           int64_t L, int R, const float* bsm, float* acc) {
  // units (i1, g): thread groups g = 0..ng-1 split the i2 range of each i1 so
  // that short modes (I1 < NT) still occupy every thread; consecutive threads
  // take consecutive i1 (coalesced X loads)
  const int ng = max(1, NT / I1);
  const int js = (I2 + ng - 1) / ng;  // i2 per group
  for (int u = threadIdx.x; u < I1 * ng; u += NT) {
    const int i = u % I1, g = u / I1;
    const int ja = g * js, jb = min(I2, ja + js);
    float in[BRC];
#pragma unroll
    for (int r = 0; r < BRC; ++r) in[r] = 0.f;
    const int64_t base = i + L * c;
    int j = ja;
    for (; j + KU <= jb; j += KU) {
      float x[KU];
#pragma unroll
      for (int v = 0; v < KU; ++v) x[v] = ldx(b, base + (int64_t)I1 * (j + v));
#pragma unroll
      for (int v = 0; v < KU; ++v) {
        const float4* h = reinterpret_cast<const float4*>(bsm + (j + v) * BRC);
#pragma unroll
        for (int q = 0; q < BRC / 4; ++q) {
          const float4 hv = h[q];
          in[4 * q + 0] = fmaf(x[v], hv.x, in[4 * q + 0]);
          in[4 * q + 1] = fmaf(x[v], hv.y, in[4 * q + 1]);
          in[4 * q + 2] = fmaf(x[v], hv.z, in[4 * q + 2]);
          in[4 * q + 3] = fmaf(x[v], hv.w, in[4 * q + 3]);
        }
      }
    }
    for (; j < jb; ++j) {
      const float x = ldx(b, base + (int64_t)I1 * j);
      const float4* h = reinterpret_cast<const float4*>(bsm + j * BRC);
#pragma unroll
      for (int q = 0; q < BRC / 4; ++q) {
        const float4 hv = h[q];
        in[4 * q + 0] = fmaf(x, hv.x, in[4 * q + 0]);
        in[4 * q + 1] = fmaf(x, hv.y, in[4 * q + 1]);
        in[4 * q + 2] = fmaf(x, hv.z, in[4 * q + 2]);
        in[4 * q + 3] = fmaf(x, hv.w, in[4 * q + 3]);
      }
    }
    const float* h1 = b.H[0] + (int64_t)i * R;
#pragma unroll
    for (int r = 0; r < BRC; ++r)
      if (r < R) acc[r] = fmaf(in[r], __ldg(h1 + r), acc[r]);
  }
}

template <int NT>
__global__ void __launch_bounds__(NT)
batch_pm_right_kernel(const BatchInst* __restrict__ tab, const int2* __restrict__ items,
                      int nitems, int sched) {
  extern __shared__ __align__(16) float bsm[];
  __shared__ float red[NT / 32][BR];
  int i0, i1;
  item_run(nitems, i0, i1);
  int cur = -1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = i0; it < i1; ++it) {
    const int bi = items[it].x;
    const BatchInst& b = tab[bi];
    const int I1 = (int)b.I[0], I2 = (int)b.I[1], R = b.R;
    const int64_t L = (int64_t)I1 * I2;
    const int64_t c = items[it].y;
    const int cls = rank_class(R, sched);
    if (bi != cur) {
      __syncthreads();
      stage_factor(bsm, b.H[1], I2, R, cls);
      __syncthreads();
      cur = bi;
    }
    float acc[BR];
#pragma unroll
    for (int r = 0; r < BR; ++r) acc[r] = 0.f;
    if (cls == 8) right_sums<NT, 8>(b, c, I1, I2, L, R, bsm, acc);
    else if (cls == 16) right_sums<NT, 16>(b, c, I1, I2, L, R, bsm, acc);
    else right_sums<NT, 32>(b, c, I1, I2, L, R, bsm, acc);
    const float v = reduce_scatter32(acc, lane);
    red[warp][lane] = v;
    __syncthreads();
    if (threadIdx.x < R) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < NT / 32; ++w) s += red[w][threadIdx.x];
      b.M[c * R + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// ---- M^(1)[i1, r] = sum_{i2} T[i1 + I1 i2, r] H2[i2, r]: items (b, r) -----------------
__global__ void __launch_bounds__(128)
batch_contract_rest_kernel(const BatchInst* __restrict__ tab, const int2* __restrict__ items,
                           int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchInst& b = tab[items[it].x];
    const int r = items[it].y;
    const int I1 = (int)b.I[0], I2 = (int)b.I[1], R = b.R;
    const float* Tr = b.T + (int64_t)I1 * I2 * r;
    for (int i = threadIdx.x; i < I1; i += blockDim.x) {
      float a0 = 0.f, a1 = 0.f;
      int j = 0;
      for (; j + 2 <= I2; j += 2) {
        a0 = fmaf(Tr[i + (int64_t)I1 * j], __ldg(b.H[1] + (int64_t)j * R + r), a0);
        a1 = fmaf(Tr[i + (int64_t)I1 * (j + 1)], __ldg(b.H[1] + (int64_t)(j + 1) * R + r), a1);
      }
      if (j < I2) a0 = fmaf(Tr[i + (int64_t)I1 * j], __ldg(b.H[1] + (int64_t)j * R + r), a0);
      b.M[(int64_t)i * R + r] = a0 + a1;
    }
  }
}

// ---- M^(2)[i2, r] = sum_{i1} T[i1 + I1 i2, r] H1[i1, r]: items (b, r) -----------------
// one warp per i2, lanes across i1
__global__ void __launch_bounds__(128)
batch_contract_first_kernel(const BatchInst* __restrict__ tab, const int2* __restrict__ items,
                            int nitems) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchInst& b = tab[items[it].x];
    const int r = items[it].y;
    const int I1 = (int)b.I[0], I2 = (int)b.I[1], R = b.R;
    const float* Tr = b.T + (int64_t)I1 * I2 * r;
    for (int j = warp; j < I2; j += blockDim.x / 32) {
      float a = 0.f;
      for (int i = lane; i < I1; i += 32)
        a = fmaf(Tr[i + (int64_t)I1 * j], __ldg(b.H[0] + (int64_t)i * R + r), a);
      a = warp_sum(a);
      if (lane == 0) b.M[(int64_t)j * R + r] = a;
    }
  }
}

}  // namespace

cudaError_t launch_batch_sqnorm(const BatchInst* tab, int count, const int2* items, int nitems,
                                const int* first, double* part, int sm_count, cudaStream_t st) {
  batch_sqnorm_kernel<<<std::min(nitems, 8 * sm_count), 256, 0, st>>>(tab, items, nitems, part);
  batch_sqnorm_finish_kernel<<<(count + 127) / 128, 128, 0, st>>>(tab, count, first, part);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_batch_gram(const BatchInst* tab, int count, cudaStream_t st) {
  batch_gram_kernel<<<3 * count, 256, 0, st>>>(tab, count);
  note_launches(1);
  return cudaGetLastError();
}

// tl: threads per item (64, 128 or 256; two rows each); smem_floats: max C x 32 over the batch;
// sched: rank-class schedule (see rank_class)
cudaError_t launch_batch_pm_left(const BatchInst* tab, const int2* items, int nitems, int tl,
                                 int grid, size_t smem_floats, int sched, cudaStream_t st) {
  const size_t smem = smem_floats * sizeof(float);
  cudaError_t e = cudaSuccess;
  switch (tl) {
    case 64:
      e = cudaFuncSetAttribute(batch_pm_left_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) batch_pm_left_kernel<64><<<grid, 64, smem, st>>>(tab, items, nitems, sched);
      break;
    case 128:
      e = cudaFuncSetAttribute(batch_pm_left_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) batch_pm_left_kernel<128><<<grid, 128, smem, st>>>(tab, items, nitems, sched);
      break;
    case 256:
      e = cudaFuncSetAttribute(batch_pm_left_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) batch_pm_left_kernel<256><<<grid, 256, smem, st>>>(tab, items, nitems, sched);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  note_launches(1);
  return cudaGetLastError();
}

// nt: threads per item (64, 128 or 256); smem_floats: max I2 x 32 over the batch;
// sched: rank-class schedule (see rank_class)
cudaError_t launch_batch_pm_right(const BatchInst* tab, const int2* items, int nitems, int nt,
                                  int grid, size_t smem_floats, int sched, cudaStream_t st) {
  const size_t smem = smem_floats * sizeof(float);
  cudaError_t e = cudaSuccess;
  switch (nt) {
    case 64:
      e = cudaFuncSetAttribute(batch_pm_right_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) batch_pm_right_kernel<64><<<grid, 64, smem, st>>>(tab, items, nitems, sched);
      break;
    case 128:
      e = cudaFuncSetAttribute(batch_pm_right_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) batch_pm_right_kernel<128><<<grid, 128, smem, st>>>(tab, items, nitems, sched);
      break;
    case 256:
      e = cudaFuncSetAttribute(batch_pm_right_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) batch_pm_right_kernel<256><<<grid, 256, smem, st>>>(tab, items, nitems, sched);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_contract(const BatchInst* tab, const int2* items, int nitems, bool rest,
                                  int sm_count, cudaStream_t st) {
  const int grid = std::min(nitems, 16 * sm_count);
  if (rest) batch_contract_rest_kernel<<<grid, 128, 0, st>>>(tab, items, nitems);
  else batch_contract_first_kernel<<<grid, 128, 0, st>>>(tab, items, nitems);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace planc
