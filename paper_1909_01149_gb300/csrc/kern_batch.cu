// Batched kernels for many small 3-way instances solved together, one launch
// per phase: every launch covers all instances through a table of work items
// (instance, tile).  The two partial MTTKRPs run as persistent grids: each CTA
// walks a contiguous run of items holding an equal share of the elements (so
// that per-instance staging, a factor in shared memory, is redone only when
// the instance changes) and streams X through a ring of shared-memory stages.
// The device code of every phase is in batch_dev.cuh (the single persistent
// launch of the whole solve, in kern_mode.cu, runs the same code).
//
// Per outer iteration (Alg. 1 with the dimension tree of Alg. 3, N = 3, S = 2):
//   T^{1:2} = X_(1:2) H^(3)                 batch_pm_left   (first X pass)
//   M^(1)   = T^{1:2} x_2 H^(2)             batch_contract_rest
//   M^(2)   = T^{1:2} x_1 H^(1) (updated)    batch_contract_first
//   M^(3)   = X_(1:2)^T (H^(2) . H^(1))      batch_pm_right  (second X pass)
// with the fused per-mode update (kern_mode.cu) between them.
#include <cuda_bf16.h>

#include <algorithm>

#include "batch_dev.cuh"
#include "internal.h"

namespace planc {

namespace {

using namespace bdev;

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
  if (n == 0 && threadIdx.x < 32) in.lam[threadIdx.x] = 1.0;  // lambda starts at 1
  for (int pr = threadIdx.x; pr < in.R * in.R; pr += blockDim.x) initial_gram_entry(in, n, pr);
}

// This CTA's run of items: contiguous, with about 1 / gridDim.x of the total
// work each (cumw: prefix sums of the items' element counts, nitems + 1 entries).
__device__ __forceinline__ int64_t lower_bound64(const int64_t* a, int n, int64_t v) {
  int lo = 0, hi = n;  // first index in [0, n) with a[i] >= v, else n
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ void work_run(const int64_t* cumw, int nitems, int& i0, int& i1) {
  const int64_t W = cumw[nitems];
  const int64_t s0 = W * blockIdx.x / gridDim.x, s1 = W * (blockIdx.x + 1) / gridDim.x;
  i0 = (int)lower_bound64(cumw, nitems, s0);
  i1 = blockIdx.x + 1 == gridDim.x ? nitems : (int)lower_bound64(cumw, nitems, s1);
}

// ---- T^{1:2} = X_(1:2) H^(3): items (b, block of 2 NT rows) -----------------------------
template <int NT>
__global__ void __launch_bounds__(NT)
batch_pm_left_kernel(const BatchInst* __restrict__ tab, const int2* __restrict__ items,
                     const int64_t* __restrict__ cumw, int nitems, int sched, int, int) {
  extern __shared__ __align__(16) unsigned char bsm[];
  int i0, i1;
  work_run(cumw, nitems, i0, i1);
  pm_left_run<NT>(tab, [items](int i) { return items[i]; }, i0, i1, sched, bsm);
}

// ---- M^(3) = X_(1:2)^T (H^(2) . H^(1)): items (b, c) -------------------------------------
// hcap: rows of the staged H2; h1cap: rows of the staged H1 (0: H1 is read
// from global memory)
template <int NT>
__global__ void __launch_bounds__(NT)
batch_pm_right_kernel(const BatchInst* __restrict__ tab, const int2* __restrict__ items,
                      const int64_t* __restrict__ cumw, int nitems, int sched, int hcap,
                      int h1cap) {
  extern __shared__ __align__(16) unsigned char bsm[];
  int i0, i1;
  work_run(cumw, nitems, i0, i1);
  pm_right_run<NT>(tab, [items](int i) { return items[i]; }, i0, i1, sched, bsm, hcap, h1cap);
}

// ---- M^(1) and M^(2) from T^{1:2}: items (b, r) ----------------------------------------
constexpr int CT = 256;  // threads of the contraction kernels

__global__ void __launch_bounds__(CT)
batch_contract_rest_kernel(const BatchInst* __restrict__ tab, const int2* __restrict__ items,
                           int nitems) {
  __shared__ float hcol[1024];
  __shared__ float part[CT];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x)
    contract_rest_item<CT>(tab[items[it].x], items[it].y, hcol, part);
}

__global__ void __launch_bounds__(CT)
batch_contract_first_kernel(const BatchInst* __restrict__ tab, const int2* __restrict__ items,
                            int nitems) {
  __shared__ float hcol[1024];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x)
    contract_first_item<CT>(tab[items[it].x], items[it].y, hcol);
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

size_t batch_pm_smem(int hmax, int h1max) { return pm_smem_bytes(hmax, h1max); }

namespace {
// a persistent grid: as many CTAs as fit on the device at once (at least one
// per SM), each walking its balanced run of items
template <typename K>
cudaError_t launch_staged(K kern, int nt, size_t smem, int sm_count, const BatchInst* tab,
                          const int2* items, const int64_t* cumw, int nitems, int sched,
                          int hcap, int h1cap, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // the whole unified L1 as shared memory, so that every CTA of the grid is
  // resident at once (the default carveout may hold fewer)
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(nitems, std::max(1, per_sm) * sm_count));
  kern<<<grid, nt, smem, st>>>(tab, items, cumw, nitems, sched, hcap, h1cap);
  note_launches(1);
  return cudaGetLastError();
}
}  // namespace

// tl: threads per CTA (64, 128 or 256; two rows each); hmax: longest third
// mode of the batch; sched: rank-class schedule (see rank_class)
cudaError_t launch_batch_pm_left(const BatchInst* tab, const int2* items, const int64_t* cumw,
                                 int nitems, int tl, int hmax, int sched, int sm_count,
                                 cudaStream_t st) {
  const size_t smem = batch_pm_smem(hmax, 0);
  switch (tl) {
    case 64: return launch_staged(batch_pm_left_kernel<64>, 64, smem, sm_count, tab, items, cumw, nitems, sched, hmax, 0, st);
    case 128: return launch_staged(batch_pm_left_kernel<128>, 128, smem, sm_count, tab, items, cumw, nitems, sched, hmax, 0, st);
    case 256: return launch_staged(batch_pm_left_kernel<256>, 256, smem, sm_count, tab, items, cumw, nitems, sched, hmax, 0, st);
    default: return cudaErrorInvalidValue;
  }
}

// nt: threads per CTA (64, 128 or 256); hmax: longest second mode of the
// batch; h1max: longest first mode when H1 is staged too, else 0; sched:
// rank-class schedule (see rank_class)
cudaError_t launch_batch_pm_right(const BatchInst* tab, const int2* items, const int64_t* cumw,
                                  int nitems, int nt, int hmax, int h1max, int sched, int sm_count,
                                  cudaStream_t st) {
  const size_t smem = batch_pm_smem(hmax, h1max);
  switch (nt) {
    case 64: return launch_staged(batch_pm_right_kernel<64>, 64, smem, sm_count, tab, items, cumw, nitems, sched, hmax, h1max, st);
    case 128: return launch_staged(batch_pm_right_kernel<128>, 128, smem, sm_count, tab, items, cumw, nitems, sched, hmax, h1max, st);
    case 256: return launch_staged(batch_pm_right_kernel<256>, 256, smem, sm_count, tab, items, cumw, nitems, sched, hmax, h1max, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch_contract(const BatchInst* tab, const int2* items, int nitems, bool rest,
                                  int sm_count, cudaStream_t st) {
  const int grid = std::min(nitems, 8 * sm_count);
  if (rest) batch_contract_rest_kernel<<<grid, CT, 0, st>>>(tab, items, nitems);
  else batch_contract_first_kernel<<<grid, CT, 0, st>>>(tab, items, nitems);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace planc
