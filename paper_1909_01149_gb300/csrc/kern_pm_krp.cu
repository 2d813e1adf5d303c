// The partial MTTKRPs of both root branches for BF16 X as one tcgen05 GEMM
// each (Alg. 3: T^{1:S} = X_(1:S) K^{S+1:N} and T^{S+1:N} = X_(1:S)^T K^{1:S}):
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
#include <cuda.h>
#include <cuda_bf16.h>
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

// ---- B image: K^T split into hi | mid | lo, 3 RB rows of Kp BF16 ----------------------
// K[k, r] = H_0[i_0, r] * H_1[i_1, r] * ..., k = i_0 + dim_0 (i_1 + dim_1 (...)),
// zero for k >= L or r >= R
__global__ void krp_image_kernel(KrpDev kd, int R, int RB, int64_t L, int64_t Kp,
                                 __nv_bfloat16* __restrict__ Bt) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Kp * RB) return;
  const int64_t k = idx % Kp;
  const int r = (int)(idx / Kp);
  float v = 0.f;
  if (k < L && r < R) {
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
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(hi);
  const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
  const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
  Bt[(int64_t)r * Kp + k] = hi;
  Bt[(int64_t)(RB + r) * Kp + k] = mid;
  Bt[(int64_t)(2 * RB + r) * Kp + k] = lo;
}

// first unit of CTA g (of G) over U units
__host__ __device__ __forceinline__ int64_t unit0(int64_t U, int g, int G) {
  return U * g / G;
}

// ---- sum of a tile's partials over the CTAs that touched it, in CTA order ------------
__global__ void krp_reduce_kernel(const float* __restrict__ part, int64_t C, int R, int RB,
                                  int64_t U, int ks, int G, int tmax, float* __restrict__ out,
                                  int rowmajor) {
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
  if (rowmajor) out[c * R + r] = s;
  else out[c + C * r] = s;
}

// ---- the GEMM: persistent, stream-K over (tile, k-step) units ------------------------
template <int RB, bool LEFT>
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
      const uint32_t idesc = instr_desc(1u, LEFT, false, KR_BM, N);
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

}  // namespace

namespace {

struct KrpPlan {
  bool ok = false;
  int RB = 16;
  int64_t Kp = 0, U = 0;
  int ks = 0, grid = 0, tmax = 0, stages = 0;
  size_t img_bytes = 0, part_bytes = 0, smem = 0;
};

// Mdim: output rows (C right, L left); Kdim: the reduction (L right, C left)
KrpPlan krp_plan(int64_t Mdim, int64_t Kdim, int R, int sm_count) {
  KrpPlan pl;
  if (R < 1 || R > 32 || Mdim < 1 || Kdim < 1) return pl;
  pl.RB = R <= 16 ? 16 : 32;
  pl.Kp = (Kdim + KR_BK - 1) / KR_BK * KR_BK;
  pl.ks = (int)(pl.Kp / KR_BK);
  const int64_t m_tiles = (Mdim + KR_BM - 1) / KR_BM;
  pl.U = m_tiles * pl.ks;
  pl.grid = (int)std::max<int64_t>(1, std::min<int64_t>(pl.U, sm_count));
  int tmax = 1;
  for (int g = 0; g < pl.grid; ++g) {
    const int64_t u0 = unit0(pl.U, g, pl.grid), u1 = unit0(pl.U, g + 1, pl.grid);
    if (u1 > u0) tmax = std::max<int>(tmax, (int)((u1 - 1) / pl.ks - u0 / pl.ks + 1));
  }
  pl.tmax = tmax;
  pl.img_bytes = ((size_t)3 * pl.RB * pl.Kp * 2 + 255) / 256 * 256;
  pl.part_bytes = (size_t)pl.grid * tmax * KR_BM * pl.RB * 4;
  const size_t st_bytes = (size_t)KR_BM * KR_BK * 2 + (size_t)3 * pl.RB * KR_BK * 2;
  const size_t fixed = 1024 + 8 * (2 * KR_MAX_STAGES + 2 * 4 + 1) + 16;
  pl.stages = (int)std::min<size_t>(KR_MAX_STAGES, (227 * 1024 - fixed) / st_bytes);
  pl.smem = fixed + (size_t)pl.stages * st_bytes;
  pl.ok = pl.stages >= 3;
  return pl;
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
  (void)left;
  if (xdt != PLANC_BF16 || !krp_enabled()) return false;
  if (R < 1 || R > 32 || kh.nm < 1 || kh.nm > PLANC_MAX_N) return false;
  // TMA: the row stride of X (L BF16 elements) a multiple of 16 bytes
  if (L % 8 != 0 || L >= (1LL << 31) || C >= (1LL << 31)) return false;
  return tensor_map_encoder() != nullptr;
}

size_t pm_krp_workspace_bytes(bool left, int64_t L, int64_t C, int R, int sm_count) {
  const KrpPlan pl = left ? krp_plan(L, C, R, sm_count) : krp_plan(C, L, R, sm_count);
  return pl.ok ? pl.img_bytes + pl.part_bytes : 0;
}

cudaError_t launch_pm_krp(const void* X, int64_t L, int64_t C, bool left, const KrpHost& kh,
                          int R, void* out, bool out_rowmajor, void* work, size_t work_bytes,
                          int* err_flag, int sm_count, cudaStream_t st) {
  const int64_t Mdim = left ? L : C, Kdim = left ? C : L;
  const KrpPlan pl = krp_plan(Mdim, Kdim, R, sm_count);
  if (!pl.ok || work_bytes < pl.img_bytes + pl.part_bytes) return cudaErrorInvalidValue;
  if (((uintptr_t)X & 15) != 0 || ((uintptr_t)work & 255) != 0) return cudaErrorInvalidValue;
  __nv_bfloat16* img = static_cast<__nv_bfloat16*>(work);
  float* part = reinterpret_cast<float*>(static_cast<char*>(work) + pl.img_bytes);
  // the split Khatri-Rao image
  KrpDev kd{};
  kd.nm = kh.nm;
  for (int m = 0; m < kh.nm; ++m) {
    kd.dim[m] = kh.dim[m];
    kd.H[m] = static_cast<const float*>(kh.H[m]);
  }
  {
    const int64_t n = pl.Kp * pl.RB;
    krp_image_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(kd, R, pl.RB, Kdim, pl.Kp, img);
    note_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // tensor maps: A = X as L x C (L contiguous; right: rows c, 64 x 128 boxes
  // along L; left: rows l, two 64 x 64 boxes per stage), B = the image as
  // Kp x 3 RB
  CUtensorMap tA, tB;
  cuuint32_t estr[2] = {1u, 1u};
  {
    cuuint64_t gdim[2] = {(cuuint64_t)L, (cuuint64_t)C};
    cuuint64_t gstride[1] = {(cuuint64_t)L * 2};
    cuuint32_t box[2] = {(cuuint32_t)KR_BK, (cuuint32_t)(left ? 64 : KR_BM)};
    if (tensor_map_encoder()(&tA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(X), gdim, gstride,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    cuuint64_t gdim[2] = {(cuuint64_t)pl.Kp, (cuuint64_t)(3 * pl.RB)};
    cuuint64_t gstride[1] = {(cuuint64_t)pl.Kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)KR_BK, (cuuint32_t)(3 * pl.RB)};
    if (tensor_map_encoder()(&tB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, img, gdim, gstride, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  KrpParams p{};
  p.C = Mdim;
  p.U = pl.U;
  p.ks = pl.ks;
  p.R = R;
  p.stages = pl.stages;
  p.tmax = pl.tmax;
  p.part = part;
  p.err = err_flag;
  auto k = pl.RB == 16 ? (left ? pm_krp_kernel<16, true> : pm_krp_kernel<16, false>)
                       : (left ? pm_krp_kernel<32, true> : pm_krp_kernel<32, false>);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  e = launch_pdl(k, dim3(pl.grid), dim3(KR_THREADS), pl.smem, st, tA, tB, p);
  if (e != cudaSuccess) return e;
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t n = Mdim * R;
  krp_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      part, Mdim, R, pl.RB, pl.U, pl.ks, pl.grid, pl.tmax, static_cast<float*>(out),
      out_rowmajor ? 1 : 0);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace planc
