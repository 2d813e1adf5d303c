// Shared device helpers of libplanc: element types, the on-the-fly partial
// Khatri-Rao product, and deterministic reduction utilities.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#define PLANC_MAX_N 16
#define PLANC_MAX_R 256
#define PLANC_MAX_NLS_R 64
#define PLANC_MAX_ADMM_STEPS 64
#define PLANC_MAX_NES_STEPS 64

namespace planc {

// ---- programmatic dependent launch: a kernel launched with the PDL
// attribute starts while its predecessor in the stream finishes; it runs its
// prologue (shared memory, barriers, TMEM), then waits here before touching
// global data (no-op for a kernel launched without the attribute), and lets
// its own successor launch early.  Every PDL kernel waits in every thread, so
// completion stays ordered along the stream.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }

// ---- element loads: every stored tensor type is widened to its accumulator
// type on load (F32/BF16/F16 -> float, F64 -> double).
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_acc(__half v) { return __half2float(v); }

template <typename TX> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

// ---- partial Khatri-Rao product K^{i:j} = H^j kr ... kr H^i (Alg. 3) -----
// Row index k enumerates the modes i..j with mode i fastest; the value in
// column r is prod_m H^(m)[k_m, r].  Factors are row-major I_m x R.
template <typename TF> struct Krp {
  int nm;                      // number of modes in the product (0 = all-ones)
  int R;                       // row stride of every factor
  int64_t dim[PLANC_MAX_N];    // mode sizes, fastest first
  const TF* H[PLANC_MAX_N];    // factor base pointers
};

// Decode row k of the product into per-mode row offsets (k_m * R).
template <typename TF>
__device__ __forceinline__ void krp_decode(const Krp<TF>& K, int64_t k, int64_t* off) {
  for (int m = 0; m < K.nm; ++m) {
    int64_t d = K.dim[m];
    int64_t q = k / d;
    off[m] = (k - q * d) * K.R;
    k = q;
  }
}

template <typename TF>
__device__ __forceinline__ TF krp_value(const Krp<TF>& K, const int64_t* off, int r) {
  TF v = TF(1);
  for (int m = 0; m < K.nm; ++m) v *= K.H[m][off[m] + r];
  return v;
}

template <typename TF>
__device__ __forceinline__ TF krp_at(const Krp<TF>& K, int64_t k, int r) {
  int64_t off[PLANC_MAX_N];
  krp_decode(K, k, off);
  return krp_value(K, off, r);
}

// ---- reductions ------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over a group of `width` consecutive lanes (width a power of two <= 32).
template <typename T>
__device__ __forceinline__ T group_sum(T v, int width) {
  for (int o = width >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, width);
  return v;
}

// Neumaier compensated accumulation: s + c is the running sum.
template <typename T>
__device__ __forceinline__ void neumaier_add(T& s, T& c, T x) {
  T t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
  s = t;
}

}  // namespace planc
