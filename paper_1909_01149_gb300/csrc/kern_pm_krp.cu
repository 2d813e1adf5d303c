// The partial MTTKRPs of both root branches for BF16 (and FP16) X as one
// tcgen05 GEMM each (Alg. 3: T^{1:S} = X_(1:S) K^{S+1:N} and T^{S+1:N} =
// X_(1:S)^T K^{1:S}):
//
//   right: D[c, r] = sum_k X[k + L c] K[k, r]   (k over the L leading entries)
//   left:  D[l, r] = sum_k X[l + L k] K[k, r]   (k over the C trailing entries)
//
// K (the Khatri-Rao product of the branch's other factors, first mode
// fastest) is formed once per call in FP32 and split into three BF16 terms
// hi + mid + lo (exact for FP32 values), stored K-major as the MMA's B
// operand: 3 R' rows of Kp = the reduction length rounded up to 64 (1.5 MB
// for a reduction of 16384 and R' = 16; it stays in L2).  A is X itself,
// loaded by TMA: K-major for the right branch (rows c, k contiguous),
// MN-major for the left (rows l contiguous).  Output rows lie on TMEM lanes,
// so the whole sum over k happens in the MMA: no per-row weighting or
// cross-row reduction in the epilogue, which only drains the accumulators
// every KR_SEG stages into FP32 registers (the tensor core truncates products
// to the running sum's exponent range, so chains are kept short: two
// alternating sub-accumulators of 8 MMAs each per drain, the chain length of
// the other partial-MTTKRP kernels).
//
// Work: units (128-row tile, 64-element k-step), split into equal contiguous
// ranges, one per CTA of a persistent grid (stream-K); each CTA writes one
// partial 128 x R' block per tile it touches, and krp_reduce_kernel sums a
// tile's partials in CTA order (fixed order: results do not depend on
// scheduling).
//
// FP16 X: the MMA takes both operands in one type, so the image is split into
// three FP16 terms instead.  FP16's exponent range is narrow (normal values
// from 6e-5): each column r of K is first scaled by 2^s_r, s_r chosen from
// the column's largest magnitude so that it lands in [2^14, 2^15) (a first
// kernel finds the maxima from the factors' column maxima), and the
// fixed-order reduction multiplies the
// column's sums by 2^-s_r (exact).  Terms far below a column's maximum lose
// their last split terms to FP16 subnormals; their error relative to the
// column's largest product stays near 2^-33.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "internal.h"
#include "tc_ptx.cuh"

namespace planc {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

namespace {

using namespace tc;

constexpr int KR_BM = 128;               // output rows (c) per tile
constexpr int KR_BK = 64;                // k per stage: 128 bytes of BF16, one swizzle row
constexpr int KR_UK = 16;                // k per MMA
constexpr int KR_SEG = 4;                // stages per accumulator drain (two chains of 8 MMAs)
constexpr int KR_THREADS = 192;          // TMA warp, MMA warp, 4 epilogue warps
constexpr int KR_MAX_STAGES = 8;
constexpr uint32_t KR_TMEM_COLS = 512;   // accumulator buffers: [even | odd k-steps] x N

struct KrpDev {
  int nm;
  int64_t dim[PLANC_MAX_N];
  const float* H[PLANC_MAX_N];
};

struct KrpParams {
  int64_t C;       // output rows
  int64_t U;       // units: m_tiles * ks
  int ks;          // k-steps per tile
  int R;
  int stages;
  int tmax;        // partial blocks per CTA
  float* part;     // [grid][tmax][128][RB]
  int* err;
};

// ---- B image: K^T split into hi | mid | lo, 3 RB rows of Kp 16-bit values --------------
// K[k, r] = H_0[i_0, r] * H_1[i_1, r] * ..., k = i_0 + dim_0 (i_1 + dim_1 (...)),
// zero for k >= L or r >= R
__device__ __forceinline__ float krp_entry(const KrpDev& kd, int R, int64_t k, int r) {
  int64_t rest = k;
  const int64_t i0 = rest % kd.dim[0];
  rest /= kd.dim[0];
  float v = kd.H[0][i0 * R + r];
  for (int m = 1; m < kd.nm; ++m) {
    const int64_t im = rest % kd.dim[m];
    rest /= kd.dim[m];
    v *= kd.H[m][im * R + r];
  }
  return v;
}

// FP16 image: the power-of-two exponent s_r of column r from its largest
// magnitude (bits of a non-negative float: integer order is float order)
__device__ __forceinline__ int f16_col_shift(unsigned maxbits) {
  const float mx = __uint_as_float(maxbits);
  if (!(mx > 0.f) || !(mx < 3.0e38f)) return 0;
  int e;
  frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1)
  return 15 - e;   // mx 2^s in [2^14, 2^15)
}

// cmax[r] = bits of max_k |K[k, r]| = prod_m max_i |H_m[i, r]| (the maximum
// of a product over independent indices; multiplied in the order
// krp_entry uses, so it equals the largest entry the image kernel forms):
// one block per column r < RB (zero past R)
__global__ void __launch_bounds__(256)
krp_colmax_kernel(KrpDev kd, int R, unsigned* __restrict__ cmax) {
  __shared__ float wmax[8];
  const int r = blockIdx.x, t = threadIdx.x;
  float prod = r < R ? 1.f : 0.f;
  for (int m = 0; m < kd.nm && r < R; ++m) {
    float mx = 0.f;
    for (int64_t i = t; i < kd.dim[m]; i += blockDim.x) mx = fmaxf(mx, fabsf(kd.H[m][i * R + r]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((t & 31) == 0) wmax[t >> 5] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, wmax[w]);
    __syncthreads();
    prod = m == 0 ? mx : prod * mx;
  }
  if (t == 0) cmax[r] = __float_as_uint(prod);
}

template <bool F16>
__global__ void krp_image_kernel(KrpDev kd, int R, int RB, int64_t L, int64_t Kp,
                                 void* __restrict__ Bt, const unsigned* __restrict__ cmax) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Kp * RB) return;
  const int64_t k = idx % Kp;
  const int r = (int)(idx / Kp);
  float v = 0.f;
  if (k < L && r < R) v = krp_entry(kd, R, k, r);
  if (F16) {
    v = ldexpf(v, f16_col_shift(cmax[r]));
    const __half hi = __float2half_rn(v);
    const float r1 = v - __half2float(hi);
    const __half mid = __float2half_rn(r1);
    const __half lo = __float2half_rn(r1 - __half2float(mid));
    __half* B = static_cast<__half*>(Bt);
    B[(int64_t)r * Kp + k] = hi;
    B[(int64_t)(RB + r) * Kp + k] = mid;
    B[(int64_t)(2 * RB + r) * Kp + k] = lo;
  } else {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
    __nv_bfloat16* B = static_cast<__nv_bfloat16*>(Bt);
    B[(int64_t)r * Kp + k] = hi;
    B[(int64_t)(RB + r) * Kp + k] = mid;
    B[(int64_t)(2 * RB + r) * Kp + k] = lo;
  }
}

// first unit of CTA g (of G) over U units
__host__ __device__ __forceinline__ int64_t unit0(int64_t U, int g, int G) {
  return U * g / G;
}

// ---- sum of a tile's partials over the CTAs that touched it, in CTA order ------------
// cmax (FP16 image): the column scales to undo, else NULL
__global__ void krp_reduce_kernel(const float* __restrict__ part, int64_t C, int R, int RB,
                                  int64_t U, int ks, int G, int tmax, float* __restrict__ out,
                                  int rowmajor, const unsigned* __restrict__ cmax) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= C * R) return;
  const int64_t c = idx / R;
  const int r = (int)(idx - c * R);
  const int64_t t = c / KR_BM;
  const int m = (int)(c - t * KR_BM);
  const int64_t ua = t * ks, ub = ua + ks;
  // the CTA whose range holds unit ua
  int g = (int)((ua * G) / U);
  while (g + 1 < G && unit0(U, g + 1, G) <= ua) ++g;
  while (g > 0 && unit0(U, g, G) > ua) --g;
  float s = 0.f;
  for (; g < G; ++g) {
    const int64_t u0 = unit0(U, g, G), u1 = unit0(U, g + 1, G);
    if (u0 >= ub) break;
    if (u1 <= ua || u1 <= u0) continue;  // no unit of this tile (or an empty range)
    const int64_t slot = t - u0 / ks;
    s += part[(((int64_t)g * tmax + slot) * KR_BM + m) * RB + r];
  }
  if (cmax) s = ldexpf(s, -f16_col_shift(cmax[r]));
  if (rowmajor) out[c * R + r] = s;
  else out[c + C * r] = s;
}

// ---- the GEMM: persistent, stream-K over (tile, k-step) units ------------------------
// F16: X and the image in FP16 (else BF16)
template <int RB, bool LEFT, bool F16 = false>
__global__ void __launch_bounds__(KR_THREADS, 1)
pm_krp_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
              const __grid_constant__ KrpParams p) {
  constexpr int N = 3 * RB;                           // [hi | mid | lo] columns
  constexpr uint32_t A_BYTES = KR_BM * KR_BK * 2;     // 16 KB
  constexpr uint32_t B_BYTES = N * KR_BK * 2;         // multiple of 1024
  constexpr uint32_t ST_BYTES = A_BYTES + B_BYTES;
  static_assert(B_BYTES % 1024 == 0 && N % 16 == 0 && N <= 128, "tile shape");
  // An accumulator buffer holds two sub-accumulators of N columns: the even
  // and the odd k-steps of a drain segment go to different ones, so each
  // FP32 accumulation chain is 8 MMAs long (the tensor core truncates
  // products to the running sum's exponent range: short chains keep the
  // bias at a few 1e-7) while drains, whose fixed cost showed in the launch
  // time, come every KR_SEG = 4 stages.
  constexpr uint32_t BSTRIDE = 2 * N <= 128 ? 128u : 256u;  // columns per buffer
  constexpr int KR_NACC = (int)(KR_TMEM_COLS / BSTRIDE);     // 4 or 2 buffers
  extern __shared__ uint8_t kr_raw[];
  const uint32_t raw = smem_u32(kr_raw);
  uint8_t* smem = kr_raw + (((raw + 1023u) & ~1023u) - raw);
  const int stages = p.stages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)stages * ST_BYTES);
  uint64_t* full = bars;                 // TMA -> MMA
  uint64_t* empty = full + stages;       // MMA -> TMA
  uint64_t* acc_full = empty + stages;   // MMA -> epilogue
  uint64_t* acc_empty = acc_full + KR_NACC;  // epilogue -> MMA
  uint64_t* drain = acc_empty + KR_NACC;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  {
    // the layout must fit the dynamic shared memory the launch provides
    uint32_t dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const uintptr_t end = reinterpret_cast<uintptr_t>(abort + 1);
    if (end - reinterpret_cast<uintptr_t>(kr_raw) > (uintptr_t)dyn) {
      if (threadIdx.x == 0) atomicExch(p.err, 41);
      return;  // uniform: no barrier, TMEM or memory access has happened yet
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < KR_NACC; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(drain, 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, KR_TMEM_COLS);
    tmem_relinquish();
  }
  pdl_wait();  // the B image (previous launch) is complete
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t u0 = unit0(p.U, blockIdx.x, gridDim.x);
  const int64_t u1 = unit0(p.U, blockIdx.x + 1, gridDim.x);
  const int ks = p.ks;
  // the end of the drain segment that starts at unit u
  auto seg_end = [&](int64_t u) {
    const int64_t tile_end = (u / ks + 1) * ks;
    return min(u1, min(tile_end, u + KR_SEG));
  };

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tA);
      prefetch_tmap(&tB);
      int s = 0;
      uint32_t ph = 0, armed = 0, armed_ph = 0;
      bool ok = true;
      for (int64_t u = u0; u < u1; ++u) {
        if (!mbar_wait(&empty[s], ph ^ 1, abort, p.err, 42)) { ok = false; break; }
        armed |= 1u << s;
        armed_ph = (armed_ph & ~(1u << s)) | (ph << s);
        mbar_arrive_expect_tx(&full[s], ST_BYTES);
        uint8_t* a = smem + (size_t)s * ST_BYTES;
        const int kx = (int)(u % ks) * KR_BK;
        const int m0 = (int)(u / ks) * KR_BM;
        if (LEFT) {  // MN-major: two boxes of 64 rows x 64 k (rows contiguous in X)
          tma_load_2d(a, &tA, &full[s], m0, kx);
          tma_load_2d(a + A_BYTES / 2, &tA, &full[s], m0 + 64, kx);
        } else {     // K-major: 128 rows x 64 k
          tma_load_2d(a, &tA, &full[s], kx, m0);
        }
        tma_load_2d(a + A_BYTES, &tB, &full[s], kx, 0);
        if (++s == stages) { s = 0; ph ^= 1; }
      }
      if (!ok) {
        // let the copies in flight land before the CTA exits
        for (int t = 0; t < stages; ++t) {
          if (!((armed >> t) & 1u)) continue;
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[t], (armed_ph >> t) & 1u) && clock64() - t0 < kWaitCycles / 16) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc(F16 ? 0u : 1u, LEFT, false, KR_BM, N);  // A, B: f16 / bf16
      int s = 0, buf = 0;
      uint32_t ph = 0, eph = 0;
      bool ok = true, issued = false;
      for (int64_t u = u0; u < u1 && ok;) {
        const int64_t ue = seg_end(u);
        if (!mbar_wait(&acc_empty[buf], ((eph >> buf) & 1u) ^ 1u, abort, p.err, 43)) break;
        eph ^= 1u << buf;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)buf * BSTRIDE;
        for (int i = 0; u < ue; ++u, ++i) {
          const uint32_t dsub = d + (uint32_t)(i & 1) * N;
          if (!mbar_wait(&full[s], ph, abort, p.err, 44)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_u32(smem + (size_t)s * ST_BYTES);
          const uint32_t b0 = a0 + A_BYTES;
#pragma unroll
          for (int kk = 0; kk < KR_BK / KR_UK; ++kk) {
            const uint64_t ad = LEFT ? smem_desc(a0 + kk * 2048, A_BYTES / 2, 1024, kLayoutSW128)
                                     : smem_desc(a0 + kk * 32, 16, 1024, kLayoutSW128);
            const uint64_t bd = smem_desc(b0 + kk * 32, 16, 1024, kLayoutSW128);
            mma_f16_ss(dsub, ad, bd, idesc, (i >= 2 || kk > 0) ? 1u : 0u);
          }
          mma_commit(&empty[s]);
          issued = true;
          if (++s == stages) { s = 0; ph ^= 1; }
        }
        if (!ok) break;
        mma_commit(&acc_full[buf]);
        buf = (buf + 1) % KR_NACC;
      }
      if (issued) {  // no MMA may be in flight when TMEM is freed
        mma_commit(drain);
        const long long t0 = clock64();
        while (!mbar_try_wait(drain, 0) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else {
    // epilogue: TMEM lane quarter q of the warp holds rows 32 q .. 32 q + 31
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    float sum[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) sum[r] = 0.f;
    const int64_t t_first = u0 / ks;
    int buf = 0;
    uint32_t fph = 0;
    for (int64_t u = u0; u < u1;) {
      const int64_t ue = seg_end(u);
      if (!mbar_wait(&acc_full[buf], (fph >> buf) & 1u, abort, p.err, 45)) break;
      fph ^= 1u << buf;
      tc_fence_after();
      const uint32_t taddr = tmem + (uint32_t)buf * BSTRIDE + lane_base;
      const bool two = ue - u >= 2;  // the odd sub-accumulator was written
#pragma unroll
      for (int c = 0; c < RB / 16; ++c) {
        float hi[16], mid[16], lo[16];
        tmem_ld16(taddr + c * 16, hi);
        tmem_ld16(taddr + RB + c * 16, mid);
        tmem_ld16(taddr + 2 * RB + c * 16, lo);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) sum[c * 16 + j] += hi[j] + (mid[j] + lo[j]);
        if (two) {
          tmem_ld16(taddr + N + c * 16, hi);
          tmem_ld16(taddr + N + RB + c * 16, mid);
          tmem_ld16(taddr + N + 2 * RB + c * 16, lo);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 16; ++j) sum[c * 16 + j] += hi[j] + (mid[j] + lo[j]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
      buf = (buf + 1) % KR_NACC;
      const int64_t t = (ue - 1) / ks;
      u = ue;
      if (u == u1 || u % ks == 0) {  // this CTA is done with tile t: its partial block
        float4* dst = reinterpret_cast<float4*>(
            p.part + (((int64_t)blockIdx.x * p.tmax + (t - t_first)) * KR_BM + row) * RB);
#pragma unroll
        for (int r4 = 0; r4 < RB / 4; ++r4) {
          dst[r4] = make_float4(sum[4 * r4], sum[4 * r4 + 1], sum[4 * r4 + 2], sum[4 * r4 + 3]);
          sum[4 * r4] = sum[4 * r4 + 1] = sum[4 * r4 + 2] = sum[4 * r4 + 3] = 0.f;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, KR_TMEM_COLS);
  }
}


// ---- FP32 X: the right branch with converter warps (3xTF32) ---------------------------
// The same GEMM for FP32 storage: converter warps split every X value of a
// stage into TF32 hi + lo in TMEM (the MMA's A operand), and two MMA warps
// issue x_hi [k_hi | k_lo] and x_lo k_hi (dropped x_lo k_lo below 2^-22), K
// carried in the image as TF32 hi and lo rows.  Rows are centred per drain
// segment as in the weighted-row kernel: the converters subtract the mean
// c_g of the row's values in the segment's first stage, so the tensor core's
// truncating accumulation sees small mixed-sign partial sums, and the
// epilogue adds c_g sum_{k in segment} K[k, r] back (the image kernel writes
// the column sums of K per 32-element k-step, TwoSum-compensated).
constexpr int K3_BK = 32;               // FP32 elements per stage (128 bytes)
constexpr int K3_UK = 8;                // per kind::tf32 MMA
constexpr int K3_THREADS = 352;         // TMA, MMA, 4 converters, 4 epilogue, second MMA
constexpr int K3_W_CONV0 = 2, K3_W_EPI0 = 6, K3_W_MMA2 = 10;
constexpr int K3_SEG = 8;               // stages per drain segment (centred)
constexpr int K3_MAX_STAGES = 6;

__device__ __forceinline__ float k3_tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// row `row` of a K-major 128-byte-swizzled tile of 32 fp32 per row
__device__ __forceinline__ void k3_lds_row(uint32_t x, int row, float* v) {
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const uint32_t a = x + row * 128 + (((jj ^ (row & 7)) & 7) << 4);
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v[4 * jj + 0]), "=f"(v[4 * jj + 1]), "=f"(v[4 * jj + 2]),
                   "=f"(v[4 * jj + 3])
                 : "r"(a)
                 : "memory");
  }
}

// mean of a row's 32 values (pairwise sum)
__device__ __forceinline__ float k3_mean32(const float* v) {
  float t[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) t[c] = v[2 * c] + v[2 * c + 1];
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
    for (int c = 0; c < w; ++c) t[c] += t[c + w];
  return t[0] * (1.f / 32.f);
}

// Image for FP32: Bt rows r (TF32 hi) and RB + r (TF32 lo) of Kp FP32 values,
// and cs[q RB + r] = sum of K[k, r] over the 32 k of k-step q (each warp
// covers one k-step of one r: Kp is a multiple of 32)
__global__ void krp32_image_kernel(KrpDev kd, int R, int RB, int64_t L, int64_t Kp,
                                   float* __restrict__ Bt, float* __restrict__ cs) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = idx < Kp * RB;  // whole warps are in or out (Kp * RB % 32 == 0)
  if (!__any_sync(0xffffffffu, in)) return;
  const int64_t k = in ? idx % Kp : 0;
  const int r = in ? (int)(idx / Kp) : 0;
  float v = 0.f;
  if (in && k < L && r < R) {
    int64_t rest = k;
    const int64_t i0 = rest % kd.dim[0];
    rest /= kd.dim[0];
    v = kd.H[0][i0 * R + r];
    for (int m = 1; m < kd.nm; ++m) {
      const int64_t im = rest % kd.dim[m];
      rest /= kd.dim[m];
      v *= kd.H[m][im * R + r];
    }
  }
  if (in) {
    const float hi = k3_tf32_rn(v);
    Bt[(int64_t)r * Kp + k] = hi;
    Bt[(int64_t)(RB + r) * Kp + k] = k3_tf32_rn(v - hi);
  }
  // column sum over the warp's 32 k, with the rounding errors carried (TwoSum)
  float s = v, e = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float t = __shfl_xor_sync(0xffffffffu, s, o);
    const float te = __shfl_xor_sync(0xffffffffu, e, o);
    const float sum = s + t;
    const float bb = sum - s;
    const float err = (s - (sum - bb)) + (t - bb);
    s = sum;
    e = e + te + err;
  }
  if (in && (threadIdx.x & 31) == 0) cs[(k / 32) * RB + r] = s + e;
}

// KrpParams with the FP32 extras
struct Krp32Params {
  int64_t C, U;
  int ks, R, stages, tmax, aslots;
  float* part;       // [grid][tmax][128][RB]
  const float* cs;   // column sums of K per k-step: [ks][RB]
  int* err;
};

template <int RB>
__global__ void __launch_bounds__(K3_THREADS, 1)
pm_krp32_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
                const __grid_constant__ Krp32Params p) {
  constexpr uint32_t A_BYTES = KR_BM * K3_BK * 4;   // 16 KB
  constexpr uint32_t B_BYTES = 2 * RB * K3_BK * 4;  // [hi | lo] rows
  constexpr uint32_t ST_BYTES = A_BYTES + B_BYTES;
  constexpr uint32_t ACC = 3 * RB;                  // [x_hi k_hi | x_hi k_lo | x_lo k_hi]
  static_assert(B_BYTES % 1024 == 0 && RB % 16 == 0 && RB <= 64, "tile shape");
  extern __shared__ uint8_t kr_raw[];
  const uint32_t raw = smem_u32(kr_raw);
  uint8_t* smem = kr_raw + (((raw + 1023u) & ~1023u) - raw);
  const int stages = p.stages, aslots = p.aslots;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)stages * ST_BYTES);
  uint64_t* full = bars;                  // TMA -> converters (A and B landed)
  uint64_t* x_empty = full + stages;      // converters (4) + MMA commits (2) -> TMA
  uint64_t* a_full = x_empty + stages;    // converters -> MMA warps
  uint64_t* a_empty = a_full + 4;         // MMA commits (2) -> converters
  uint64_t* acc_full = a_empty + 4;       // MMA commits (2) -> epilogue
  uint64_t* acc_empty = acc_full + 2;     // epilogue (4) -> MMA warps
  uint64_t* c_full = acc_empty + 2;       // converters (4) -> epilogue: centres
  uint64_t* c_empty = c_full + 4;         // epilogue (4) -> converters
  uint64_t* drain = c_empty + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* cring = reinterpret_cast<float*>(tmem_slot + 4);  // 4 slots x 128 rows
  float* segcs = cring + 4 * KR_BM;                         // 2 x RB: a segment's column sums
  {
    uint32_t dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const uintptr_t end = reinterpret_cast<uintptr_t>(segcs + 2 * RB);
    if (end - reinterpret_cast<uintptr_t>(kr_raw) > (uintptr_t)dyn || aslots < 1 || aslots > 4) {
      if (threadIdx.x == 0) atomicExch(p.err, 46);
      return;  // uniform: no barrier, TMEM or memory access has happened yet
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&x_empty[s], 6);
    }
    for (int a = 0; a < 4; ++a) {
      mbar_init(&a_full[a], 4);
      mbar_init(&a_empty[a], 2);
      mbar_init(&c_full[a], 4);
      mbar_init(&c_empty[a], 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 2);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(&drain[0], 1);
    mbar_init(&drain[1], 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  pdl_wait();  // the image (previous launch) is complete
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t acc0 = (uint32_t)aslots * 64u;  // accumulators after the A slots
  const int64_t u0 = unit0(p.U, blockIdx.x, gridDim.x);
  const int64_t u1 = unit0(p.U, blockIdx.x + 1, gridDim.x);
  const int ks = p.ks;
  auto seg_end = [&](int64_t u) {
    const int64_t tile_end = (u / ks + 1) * ks;
    return min(u1, min(tile_end, u + K3_SEG));
  };
  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tA);
      prefetch_tmap(&tB);
      int s = 0;
      uint32_t ph = 0, armed = 0, armed_ph = 0;
      bool ok = true;
      for (int64_t u = u0; u < u1; ++u) {
        if (!mbar_wait(&x_empty[s], ph ^ 1, abort, p.err, 47)) { ok = false; break; }
        armed |= 1u << s;
        armed_ph = (armed_ph & ~(1u << s)) | (ph << s);
        mbar_arrive_expect_tx(&full[s], ST_BYTES);
        uint8_t* a = smem + (size_t)s * ST_BYTES;
        const int kx = (int)(u % ks) * K3_BK;
        tma_load_2d(a, &tA, &full[s], kx, (int)(u / ks) * KR_BM);
        tma_load_2d(a + A_BYTES, &tB, &full[s], kx, 0);
        if (++s == stages) { s = 0; ph ^= 1; }
      }
      if (!ok) {
        for (int t = 0; t < stages; ++t) {
          if (!((armed >> t) & 1u)) continue;
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[t], (armed_ph >> t) & 1u) && clock64() - t0 < kWaitCycles / 16) {
          }
        }
      }
    }
  } else if (warp >= K3_W_CONV0 && warp < K3_W_EPI0) {
    // converters: row m of the tile (TMEM lane m) -> centred TF32 hi | lo
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    int s = 0, as = 0, cb = 0;
    uint32_t ph = 0, aph = 0, cph = 0;
    bool ok = true;
    for (int64_t u = u0; u < u1 && ok;) {
      const int64_t ue = seg_end(u);
      float cseg = 0.f;
      for (int i = 0; u < ue; ++u, ++i) {
        if (!mbar_wait(&full[s], ph, abort, p.err, 48)) { ok = false; break; }
        if (!mbar_wait(&a_empty[as], aph ^ 1, abort, p.err, 49)) { ok = false; break; }
        float v[K3_BK];
        k3_lds_row(smem_u32(smem + (size_t)s * ST_BYTES), row, v);
        __syncwarp();
        if (lane == 0) mbar_arrive(&x_empty[s]);
        tc_fence_after();
        if (i == 0) {
          // the segment's centre goes to a ring slot once the drain that last
          // read the slot (four segments back) has taken it
          if (!mbar_wait(&c_empty[cb], ((cph >> cb) & 1u) ^ 1u, abort, p.err, 50)) { ok = false; break; }
          cph ^= 1u << cb;
          cseg = k3_mean32(v);
          cring[cb * KR_BM + row] = cseg;
          __syncwarp();
          if (lane == 0) mbar_arrive(&c_full[cb]);
          cb = (cb + 1) & 3;
        }
        // hi = x' with the 13 low mantissa bits cleared (exact in TF32), lo =
        // x' - hi (exact in FP32; the MMA truncates it, unbiased on centred rows)
        uint32_t hi[K3_BK], lo[K3_BK];
#pragma unroll
        for (int c = 0; c < K3_BK; ++c) {
          const float x = v[c] - cseg;
          const uint32_t hb = __float_as_uint(x) & 0xffffe000u;
          hi[c] = hb;
          lo[c] = __float_as_uint(x - __uint_as_float(hb));
        }
        const uint32_t a = tmem + lane_base + (uint32_t)as * 64u;
        tmem_st16(a, hi);
        tmem_st16(a + 16, hi + 16);
        tmem_st16(a + 32, lo);
        tmem_st16(a + 48, lo + 16);
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&a_full[as]);
        if (++s == stages) { s = 0; ph ^= 1; }
        if (++as == aslots) { as = 0; aph ^= 1; }
      }
    }
  } else if (warp == 1 || warp == K3_W_MMA2) {
    if (lane == 0) {
      // warp 1: x_hi [k_hi | k_lo] (N = 2 RB); the second warp: x_lo k_hi (N = RB)
      const bool lo_warp = warp == K3_W_MMA2;
      const uint32_t idesc = lo_warp ? instr_desc(2u, false, false, KR_BM, RB)
                                     : instr_desc(2u, false, false, KR_BM, 2 * RB);
      int s = 0, as = 0, buf = 0;
      uint32_t aph = 0, eph = 0;
      bool ok = true, issued = false;
      for (int64_t u = u0; u < u1 && ok;) {
        const int64_t ue = seg_end(u);
        if (!mbar_wait(&acc_empty[buf], ((eph >> buf) & 1u) ^ 1u, abort, p.err, 51)) break;
        eph ^= 1u << buf;
        tc_fence_after();
        const uint32_t d = tmem + acc0 + (uint32_t)buf * ACC + (lo_warp ? 2u * RB : 0u);
        for (int i = 0; u < ue; ++u, ++i) {
          if (!mbar_wait(&a_full[as], aph, abort, p.err, 52)) { ok = false; break; }
          tc_fence_after();
          const uint32_t acol = tmem + (uint32_t)as * 64u + (lo_warp ? 32u : 0u);
          const uint32_t b0 = smem_u32(smem + (size_t)s * ST_BYTES + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < K3_BK / K3_UK; ++kk) {
            const uint64_t bd = smem_desc(b0 + kk * 32, 16, 1024, kLayoutSW128);
            mma_tf32_ts(d, acol + kk * K3_UK, bd, idesc, (i > 0 || kk > 0) ? 1u : 0u);
          }
          mma_commit(&a_empty[as]);
          mma_commit(&x_empty[s]);
          issued = true;
          if (++s == stages) s = 0;
          if (++as == aslots) { as = 0; aph ^= 1; }
        }
        if (!ok) break;
        mma_commit(&acc_full[buf]);
        buf ^= 1;
      }
      if (issued) {
        uint64_t* dr = &drain[lo_warp ? 1 : 0];
        mma_commit(dr);
        const long long t0 = clock64();
        while (!mbar_try_wait(dr, 0) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp >= K3_W_EPI0 && warp < K3_W_EPI0 + 4) {
    // epilogue: TMEM lane quarter q holds rows 32 q .. 32 q + 31
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    float sum[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) sum[r] = 0.f;
    const int64_t t_first = u0 / ks;
    int buf = 0, eb = 0;
    uint32_t fph = 0, ecph = 0;
    for (int64_t u = u0; u < u1;) {
      const int64_t ue = seg_end(u);
      // the segment's column sums of K: lane l holds columns l and 32 + l
      // (the segment's k-steps: u mod ks onwards; segments stay within a tile)
      float cs0 = 0.f, cs1 = 0.f;
      const int64_t q0 = u % ks;
      for (int64_t qq = q0; qq < q0 + (ue - u); ++qq) {
        if (lane < RB) cs0 += p.cs[qq * RB + lane];
        if (RB > 32 && lane + 32 < RB) cs1 += p.cs[qq * RB + 32 + lane];
      }
      if (!mbar_wait(&acc_full[buf], (fph >> buf) & 1u, abort, p.err, 53)) break;
      fph ^= 1u << buf;
      if (!mbar_wait(&c_full[eb], (ecph >> eb) & 1u, abort, p.err, 54)) break;
      ecph ^= 1u << eb;
      const float cseg = cring[eb * KR_BM + row];
      __syncwarp();
      if (lane == 0) mbar_arrive(&c_empty[eb]);
      eb = (eb + 1) & 3;
      tc_fence_after();
      const uint32_t taddr = tmem + acc0 + (uint32_t)buf * ACC + lane_base;
#pragma unroll
      for (int c = 0; c < RB / 16; ++c) {
        float a[16], b[16], e[16];
        tmem_ld16(taddr + c * 16, a);
        tmem_ld16(taddr + RB + c * 16, b);
        tmem_ld16(taddr + 2 * RB + c * 16, e);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = c * 16 + j;
          const float k = __shfl_sync(0xffffffffu, col < 32 ? cs0 : cs1, col & 31);
          sum[col] += fmaf(cseg, k, a[j] + (b[j] + e[j]));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
      buf ^= 1;
      const int64_t t = (ue - 1) / ks;
      u = ue;
      if (u == u1 || u % ks == 0) {
        float4* dst = reinterpret_cast<float4*>(
            p.part + (((int64_t)blockIdx.x * p.tmax + (t - t_first)) * KR_BM + row) * RB);
#pragma unroll
        for (int r4 = 0; r4 < RB / 4; ++r4) {
          dst[r4] = make_float4(sum[4 * r4], sum[4 * r4 + 1], sum[4 * r4 + 2], sum[4 * r4 + 3]);
          sum[4 * r4] = sum[4 * r4 + 1] = sum[4 * r4 + 2] = sum[4 * r4 + 3] = 0.f;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace

namespace {

struct KrpPlan {
  bool ok = false, f32 = false, f16 = false;
  int RB = 16;
  int64_t Kp = 0, U = 0;
  int ks = 0, grid = 0, tmax = 0, stages = 0, aslots = 4;
  size_t img_bytes = 0, cs_bytes = 0, part_bytes = 0, smem = 0;
};

// Mdim: output rows (C right, L left); Kdim: the reduction (L right, C left);
// f32: FP32 X (converter kernel; 32-element stages); f16: FP16 X (the image
// in FP16, with its column maxima after it)
KrpPlan krp_plan(int64_t Mdim, int64_t Kdim, int R, int sm_count, bool f32 = false,
                 bool f16 = false) {
  KrpPlan pl;
  pl.f32 = f32;
  pl.f16 = f16 && !f32;
  if (R < 1 || R > (f32 ? 64 : 32) || Mdim < 1 || Kdim < 1) return pl;
  pl.RB = R <= 16 ? 16 : R <= 32 ? 32 : 64;
  const int bk = f32 ? K3_BK : KR_BK;
  pl.Kp = (Kdim + 63) / 64 * 64;
  pl.ks = (int)(pl.Kp / bk);
  const int64_t m_tiles = (Mdim + KR_BM - 1) / KR_BM;
  pl.U = m_tiles * pl.ks;
  pl.grid = (int)std::max<int64_t>(1, std::min<int64_t>(pl.U, sm_count));
  int tmax = 1;
  for (int g = 0; g < pl.grid; ++g) {
    const int64_t u0 = unit0(pl.U, g, pl.grid), u1 = unit0(pl.U, g + 1, pl.grid);
    if (u1 > u0) tmax = std::max<int>(tmax, (int)((u1 - 1) / pl.ks - u0 / pl.ks + 1));
  }
  pl.tmax = tmax;
  pl.part_bytes = (size_t)pl.grid * tmax * KR_BM * pl.RB * 4;
  if (f32) {
    pl.aslots = pl.RB == 64 ? 2 : 4;  // TMEM: A slots of 64 columns + two accumulators of 3 RB
    pl.img_bytes = ((size_t)2 * pl.RB * pl.Kp * 4 + 255) / 256 * 256;
    pl.cs_bytes = ((size_t)pl.ks * pl.RB * 4 + 255) / 256 * 256;
    const size_t st_bytes = (size_t)KR_BM * K3_BK * 4 + (size_t)2 * pl.RB * K3_BK * 4;
    const size_t fixed = 1024 + 8 * (2 * K3_MAX_STAGES + 22) + 16 + 4 * (4 * KR_BM + 2 * 64);
    pl.stages = (int)std::min<size_t>(K3_MAX_STAGES, (227 * 1024 - fixed) / st_bytes);
    pl.smem = fixed + (size_t)pl.stages * st_bytes;
  } else {
    if (pl.RB > 32) return pl;
    pl.img_bytes = ((size_t)3 * pl.RB * pl.Kp * 2 + 255) / 256 * 256;
    if (pl.f16) pl.cs_bytes = 256;  // the column maxima (RB <= 32 words)
    const size_t st_bytes = (size_t)KR_BM * KR_BK * 2 + (size_t)3 * pl.RB * KR_BK * 2;
    const size_t fixed = 1024 + 8 * (2 * KR_MAX_STAGES + 2 * 4 + 1) + 16;
    pl.stages = (int)std::min<size_t>(KR_MAX_STAGES, (227 * 1024 - fixed) / st_bytes);
    pl.smem = fixed + (size_t)pl.stages * st_bytes;
  }
  pl.ok = pl.stages >= 3;
  return pl;
}

KrpPlan krp_plan_for(planc_dtype_t xdt, bool left, int64_t L, int64_t C, int R, int sm_count) {
  const bool f32 = xdt == PLANC_F32, f16 = xdt == PLANC_F16;
  return left ? krp_plan(L, C, R, sm_count, f32, f16) : krp_plan(C, L, R, sm_count, f32, f16);
}

// PLANC_PM_KRP=0 keeps both BF16 branches on the weighted-row kernels (read
// when a context is created and at every launch)
bool krp_enabled() {
  const char* v = getenv("PLANC_PM_KRP");
  return !(v && v[0] == '0');
}

}  // namespace

bool pm_krp_eligible(planc_dtype_t xdt, bool left, int64_t L, int64_t C, int R,
                     const KrpHost& kh) {
  if (!krp_enabled() || kh.nm < 1 || kh.nm > PLANC_MAX_N) return false;
  if (L >= (1LL << 31) || C >= (1LL << 31)) return false;
  if (xdt == PLANC_BF16 || xdt == PLANC_F16) {
    // TMA: the row stride of X (L 16-bit elements) a multiple of 16 bytes
    if (R < 1 || R > 32 || L % 8 != 0) return false;
  } else if (xdt == PLANC_F32) {
    // the right branch only (the left one's converters already set its pace),
    // and only where the FP32 image is small next to X (it is written and
    // read once per call: 2 R' x L x 4 bytes)
    if (left || R < 1 || R > 64 || L % 4 != 0) return false;
    const KrpPlan pl = krp_plan(C, L, R, 148, true);
    if (!pl.ok || (pl.img_bytes + pl.cs_bytes) * 16 > (size_t)L * C * 4) return false;
  } else {
    return false;
  }
  return tensor_map_encoder() != nullptr;
}

size_t pm_krp_workspace_bytes(planc_dtype_t xdt, bool left, int64_t L, int64_t C, int R,
                              int sm_count) {
  const KrpPlan pl = krp_plan_for(xdt, left, L, C, R, sm_count);
  return pl.ok ? pl.img_bytes + pl.cs_bytes + pl.part_bytes : 0;
}

cudaError_t launch_pm_krp(planc_dtype_t xdt, const void* X, int64_t L, int64_t C, bool left,
                          const KrpHost& kh, int R, void* out, bool out_rowmajor, void* work,
                          size_t work_bytes, int* err_flag, int sm_count, cudaStream_t st) {
  const bool f32 = xdt == PLANC_F32, f16 = xdt == PLANC_F16;
  if (f32 && left) return cudaErrorInvalidValue;
  const int64_t Mdim = left ? L : C, Kdim = left ? C : L;
  const KrpPlan pl = krp_plan(Mdim, Kdim, R, sm_count, f32, f16);
  if (!pl.ok || work_bytes < pl.img_bytes + pl.cs_bytes + pl.part_bytes) return cudaErrorInvalidValue;
  if (((uintptr_t)X & 15) != 0 || ((uintptr_t)work & 255) != 0) return cudaErrorInvalidValue;
  char* wb = static_cast<char*>(work);
  float* cs = reinterpret_cast<float*>(wb + pl.img_bytes);
  float* part = reinterpret_cast<float*>(wb + pl.img_bytes + pl.cs_bytes);
  // the split Khatri-Rao image
  KrpDev kd{};
  kd.nm = kh.nm;
  for (int m = 0; m < kh.nm; ++m) {
    kd.dim[m] = kh.dim[m];
    kd.H[m] = static_cast<const float*>(kh.H[m]);
  }
  {
    const int64_t n = pl.Kp * pl.RB;
    unsigned* cmax = reinterpret_cast<unsigned*>(cs);  // FP16: the column maxima
    if (f32) {
      krp32_image_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
          kd, R, pl.RB, Kdim, pl.Kp, reinterpret_cast<float*>(wb), cs);
    } else if (f16) {
      krp_colmax_kernel<<<(unsigned)pl.RB, 256, 0, st>>>(kd, R, cmax);
      krp_image_kernel<true><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(kd, R, pl.RB, Kdim,
                                                                          pl.Kp, wb, cmax);
      note_launches(1);
    } else {
      krp_image_kernel<false><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
          kd, R, pl.RB, Kdim, pl.Kp, wb, nullptr);
    }
    note_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // tensor maps: A = X as L x C (L contiguous; right: rows c, boxes of one
  // 128-byte row of k by 128 rows; left: rows l, two 64 x 64 boxes per
  // stage), B = the image, K-major
  const CUtensorMapDataType dt = f32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                       : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint64_t es = f32 ? 4 : 2;
  const cuuint32_t bk = f32 ? K3_BK : KR_BK;
  const int nrows_b = (f32 ? 2 : 3) * pl.RB;
  CUtensorMap tA, tB;
  cuuint32_t estr[2] = {1u, 1u};
  {
    cuuint64_t gdim[2] = {(cuuint64_t)L, (cuuint64_t)C};
    cuuint64_t gstride[1] = {(cuuint64_t)L * es};
    cuuint32_t box[2] = {bk, (cuuint32_t)(left ? 64 : KR_BM)};
    if (tensor_map_encoder()(&tA, dt, 2, const_cast<void*>(X), gdim, gstride, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    cuuint64_t gdim[2] = {(cuuint64_t)pl.Kp, (cuuint64_t)nrows_b};
    cuuint64_t gstride[1] = {(cuuint64_t)pl.Kp * es};
    cuuint32_t box[2] = {bk, (cuuint32_t)nrows_b};
    if (tensor_map_encoder()(&tB, dt, 2, wb, gdim, gstride, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  cudaError_t e;
  if (f32) {
    Krp32Params p{};
    p.C = Mdim;
    p.U = pl.U;
    p.ks = pl.ks;
    p.R = R;
    p.stages = pl.stages;
    p.tmax = pl.tmax;
    p.aslots = pl.aslots;
    p.part = part;
    p.cs = cs;
    p.err = err_flag;
    auto k = pl.RB == 16 ? pm_krp32_kernel<16> : pl.RB == 32 ? pm_krp32_kernel<32> : pm_krp32_kernel<64>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k, dim3(pl.grid), dim3(K3_THREADS), pl.smem, st, tA, tB, p);
  } else {
    KrpParams p{};
    p.C = Mdim;
    p.U = pl.U;
    p.ks = pl.ks;
    p.R = R;
    p.stages = pl.stages;
    p.tmax = pl.tmax;
    p.part = part;
    p.err = err_flag;
    auto k = f16 ? (pl.RB == 16 ? (left ? pm_krp_kernel<16, true, true> : pm_krp_kernel<16, false, true>)
                                : (left ? pm_krp_kernel<32, true, true> : pm_krp_kernel<32, false, true>))
                 : (pl.RB == 16 ? (left ? pm_krp_kernel<16, true> : pm_krp_kernel<16, false>)
                                : (left ? pm_krp_kernel<32, true> : pm_krp_kernel<32, false>));
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k, dim3(pl.grid), dim3(KR_THREADS), pl.smem, st, tA, tB, p);
  }
  if (e != cudaSuccess) return e;
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t n = Mdim * R;
  krp_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      part, Mdim, R, pl.RB, pl.U, pl.ks, pl.grid, pl.tmax, static_cast<float*>(out),
      out_rowmajor ? 1 : 0, f16 ? reinterpret_cast<const unsigned*>(cs) : nullptr);
  note_launches(1);
  return cudaGetLastError();
}
}  // namespace planc
