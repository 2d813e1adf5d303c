// Partial MTTKRP on the tcgen05 tensor cores (Sec. 4.2.2: the two root
// branches of the dimension tree are GEMMs with a Khatri-Rao operand).
//
//   left : T^{1:S}   (L x R) = X_(1:S)   (L x C) K^{S+1:N} (C x R)
//   right: T^{S+1:N} (C x R) = X_(1:S)^T (C x L) K^{1:S}   (L x R)
//
// X_(1:S) is column-major in memory (the tensor's own layout), so the left
// product reads X tiles "M-major" and the right product "K-major"; both are
// streamed by TMA in 128-byte-swizzled boxes straight into the MMA's shared
// memory operand.  The Khatri-Rao operand is generated on the fly by four
// producer warps (row-wise Hadamard products of factor rows, as the paper
// describes for its KRP) and split into three BF16 terms hi + mid + lo, so
// one kind::f16 MMA with N = 3 R' (R' = R rounded up to 16) accumulates
// X * K_hi, X * K_mid and X * K_lo side by side in TMEM; the epilogue adds
// the three column blocks.  X is exact in BF16, and the three-term split
// carries K to about 2^-26, so the product matches an FP32-operand GEMM.
//
// Roles (320 threads): warp 0 issues TMA, warp 1 issues MMAs and owns TMEM,
// warps 2-5 generate the Khatri-Rao operand, warps 6-9 drain the
// accumulators (double-buffered in TMEM so the epilogue of one tile overlaps
// the MMAs of the next).  The kernel is persistent: CTA b processes work
// items b, b + gridDim.x, ...  Every wait is bounded; a wait that gives up
// raises the error word and the CTA drains and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "tc_ptx.cuh"

namespace planc {

namespace {

using namespace tc;

constexpr int BM = 128;        // tile rows (M of the MMA)
constexpr int BK = 64;         // reduction elements per pipeline stage (128 B of bf16)
constexpr int UK = 16;         // reduction elements per kind::f16 MMA
constexpr int NTHREADS = 320;
constexpr int W_TMA = 0, W_MMA = 1, W_B0 = 2, W_EPI0 = 6;
constexpr int A_STAGE_BYTES = BM * BK * 2;   // 16 KB
constexpr uint32_t TMEM_COLS = 512;          // two accumulators at columns 0 and 256
constexpr int MAX_K_STAGES_PER_ITEM = 64;    // right side: bound the accumulation chain

struct TcParams {
  int64_t L, C;        // X_(1:S) is L x C, column-major
  int64_t Mdim, Kdim;  // rows of the product, reduction length
  int R, RB, N;        // rank, R rounded up to 16, MMA N = 3 RB
  int stages;
  int64_t items;       // work items = m_tiles x k-splits
  int64_t m_tiles;     // 128-row tiles over Mdim
  int64_t kspan;       // reduction elements per item (a multiple of BK)
  int out_mode;        // 0: out[m + Mdim r]; 1: out[m R + r]; 2: out[z Mdim R + m + Mdim r]
  float* out;
  int* err;
  Krp<float> K;
};

struct Item {
  int64_t m0, k0, k1;
  int64_t z;
};

template <bool LEFT>
__device__ __forceinline__ Item decode_item(const TcParams& p, int64_t it) {
  Item r;
  const int64_t mt = it % p.m_tiles;
  r.z = it / p.m_tiles;
  r.m0 = mt * BM;
  r.k0 = r.z * p.kspan;
  r.k1 = min(p.Kdim, r.k0 + p.kspan);
  return r;
}

// byte offset of element (row n, k) in a K-major 128-byte-swizzled operand
// tile whose rows hold 64 bf16 values
__device__ __forceinline__ uint32_t sw128_off(int n, int k) {
  return (uint32_t)((n >> 3) * 1024 + (n & 7) * 128 + ((((k >> 3) ^ (n & 7)) & 7) << 4) +
                    ((k & 7) << 1));
}

template <bool LEFT>
__global__ void __launch_bounds__(NTHREADS, 1)
pm_tc_bf16_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const int stages = p.stages;
  uint8_t* A = smem;
  uint8_t* B = A + (size_t)stages * A_STAGE_BYTES;
  const int b_stage_bytes = p.N * 128;
  uint64_t* bars = reinterpret_cast<uint64_t*>(B + (size_t)stages * b_stage_bytes);
  uint64_t* full_a = bars;
  uint64_t* full_b = full_a + stages;
  uint64_t* empty = full_b + stages;
  uint64_t* acc_full = empty + stages;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full_a[s], 1);
      mbar_init(&full_b[s], 4);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(drain, 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == W_MMA) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == W_TMA) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      prefetch_tmap(&tmap);
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      uint32_t armed = 0, armed_ph = 0;  // per stage: loads issued, parity of that phase
      for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
        const Item w = decode_item<LEFT>(p, it);
        for (int64_t k = w.k0; k < w.k1; k += BK) {
          if (!mbar_wait(&empty[s], ph ^ 1, abort, p.err, 1)) { ok = false; break; }
          armed |= 1u << s;
          armed_ph = (armed_ph & ~(1u << s)) | (ph << s);
          mbar_arrive_expect_tx(&full_a[s], A_STAGE_BYTES);
          uint8_t* a = A + (size_t)s * A_STAGE_BYTES;
          if (LEFT) {
            tma_load_2d(a, &tmap, &full_a[s], (int)w.m0, (int)k);
            tma_load_2d(a + A_STAGE_BYTES / 2, &tmap, &full_a[s], (int)(w.m0 + 64), (int)k);
          } else {
            tma_load_2d(a, &tmap, &full_a[s], (int)k, (int)w.m0);
          }
          if (++s == stages) { s = 0; ph ^= 1; }
        }
      }
      if (!ok) {
        // let the copies this thread issued land before the CTA exits
        for (int t = 0; t < stages; ++t) {
          if (!((armed >> t) & 1u)) continue;
          const uint32_t par = (armed_ph >> t) & 1u;
          const long long t0 = clock64();
          while (!mbar_try_wait(&full_a[t], par) && clock64() - t0 < kWaitCycles / 16) {
          }
        }
      }
    }
  } else if (warp == W_MMA) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = instr_desc(1u, LEFT, false, BM, p.N);
      int s = 0;
      uint32_t ph = 0;
      uint32_t eph[2] = {0, 0};
      int buf = 0;
      bool ok = true;
      bool issued = false;
      for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
        const Item w = decode_item<LEFT>(p, it);
        if (!mbar_wait(&acc_empty[buf], eph[buf] ^ 1, abort, p.err, 2)) { ok = false; break; }
        eph[buf] ^= 1;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)buf * 256u;
        uint32_t acc = 0;
        for (int64_t k = w.k0; k < w.k1; k += BK) {
          if (!mbar_wait(&full_a[s], ph, abort, p.err, 3)) { ok = false; break; }
          if (!mbar_wait(&full_b[s], ph, abort, p.err, 4)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_u32(A + (size_t)s * A_STAGE_BYTES);
          const uint32_t b0 = smem_u32(B + (size_t)s * b_stage_bytes);
#pragma unroll
          for (int kk = 0; kk < BK / UK; ++kk) {
            const uint64_t ad = LEFT ? smem_desc(a0 + kk * 2048, A_STAGE_BYTES / 2, 1024, kLayoutSW128)
                                     : smem_desc(a0 + kk * 32, 16, 1024, kLayoutSW128);
            const uint64_t bd = smem_desc(b0 + kk * 32, 16, 1024, kLayoutSW128);
            mma_f16_ss(d, ad, bd, idesc, acc);
            acc = 1;
          }
          issued = true;
          mma_commit(&empty[s]);
          if (++s == stages) { s = 0; ph ^= 1; }
        }
        if (!ok) break;
        mma_commit(&acc_full[buf]);
        buf ^= 1;
      }
      if (issued) {
        // every MMA of this thread has finished once this arrives
        mma_commit(drain);
        const long long t0 = clock64();
        while (!mbar_try_wait(drain, 0) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp < W_EPI0) {
    // ---------------------------------------------------------------- KRP producers
    const int t = threadIdx.x - W_B0 * 32;  // 0..127
    const int kk = t & 63;
    const int half = t >> 6;
    const int RB = p.RB;
    const int r_lo = half * (RB / 2), r_hi = r_lo + RB / 2;
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
      const Item w = decode_item<LEFT>(p, it);
      for (int64_t k = w.k0; k < w.k1; k += BK) {
        if (!mbar_wait(&empty[s], ph ^ 1, abort, p.err, 5)) { ok = false; break; }
        uint8_t* b = B + (size_t)s * b_stage_bytes;
        const int64_t kg = k + kk;
        const bool valid = kg < w.k1;
        int64_t off[PLANC_MAX_N];
        if (valid) krp_decode(p.K, kg, off);
        for (int r = r_lo; r < r_hi; ++r) {
          float v = (valid && r < p.R) ? krp_value(p.K, off, r) : 0.f;
          const __nv_bfloat16 hi = __float2bfloat16_rn(v);
          const float r1 = v - __bfloat162float(hi);
          const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
          const float r2 = r1 - __bfloat162float(mid);
          const __nv_bfloat16 lo = __float2bfloat16_rn(r2);
          *reinterpret_cast<__nv_bfloat16*>(b + sw128_off(r, kk)) = hi;
          *reinterpret_cast<__nv_bfloat16*>(b + sw128_off(RB + r, kk)) = mid;
          *reinterpret_cast<__nv_bfloat16*>(b + sw128_off(2 * RB + r, kk)) = lo;
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full_b[s]);
        if (++s == stages) { s = 0; ph ^= 1; }
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;
    uint32_t fph[2] = {0, 0};
    int buf = 0;
    for (int64_t it = blockIdx.x; it < p.items; it += gridDim.x) {
      const Item w = decode_item<LEFT>(p, it);
      if (!mbar_wait(&acc_full[buf], fph[buf], abort, p.err, 6)) break;
      fph[buf] ^= 1;
      tc_fence_after();
      const uint32_t taddr = tmem + (uint32_t)buf * 256u + ((uint32_t)(q * 32) << 16);
      const int64_t m = w.m0 + row;
      const bool live = m < p.Mdim;
      for (int r0 = 0; r0 < p.RB; r0 += 16) {
        float h[16], md[16], lo[16];
        tmem_ld16(taddr + r0, h);
        tmem_ld16(taddr + p.RB + r0, md);
        tmem_ld16(taddr + 2 * p.RB + r0, lo);
        tmem_ld_wait();
        if (live) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int r = r0 + j;
            if (r < p.R) {
              const float v = h[j] + (md[j] + lo[j]);
              if (p.out_mode == 0) p.out[m + p.Mdim * r] = v;
              else if (p.out_mode == 1) p.out[m * p.R + r] = v;
              else p.out[w.z * p.Mdim * p.R + m + p.Mdim * r] = v;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
      buf ^= 1;
    }
  }

  __syncthreads();
  if (warp == W_MMA) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ---- FP32 X: 3xTF32 with the X operand in TMEM ------------------------------------
//
// X (FP32) cannot be fed to the tensor cores exactly, so four converter warps
// read each TMA-staged X tile from shared memory, split every value into
// TF32 terms x = x_hi + x_lo (both rounded to nearest) and store them in
// TMEM, where tcgen05.mma reads its A operand (TMEM-resident A keeps the
// split off the shared-memory bandwidth).  The Khatri-Rao operand is split
// the same way (k = k_hi + k_lo) and laid out as B = [k_hi | k_lo].  Per MMA
// step:  D[:, 0:R')  += x_hi k_hi,   D[:, R':2R') += x_hi k_lo  (one MMA,
// N = 2R'),  D[:, R':2R') += x_lo k_hi  (N = R').  The epilogue adds the two
// column blocks; the dropped x_lo k_lo term is below 2^-22 relative.
//
// Roles (448 threads): warp 0 TMA, warp 1 MMA + TMEM owner, warps 2-5
// Khatri-Rao producers, warps 6-9 X converters, warps 10-13 epilogue.
constexpr int F_BK = 32;            // reduction elements per stage (128 B of fp32)
constexpr int F_UK = 8;             // reduction elements per kind::tf32 MMA
constexpr int F_NTHREADS = 448;
constexpr int F_W_CONV0 = 6, F_W_EPI0 = 10;
constexpr int F_X_STAGE_BYTES = BM * F_BK * 4;  // 16 KB
constexpr int F_A_SLOTS = 4;                    // TMEM slots of 64 columns (hi | lo)

__device__ __forceinline__ float tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// byte offset of fp32 element (row n, k) in a K-major 128-byte-swizzled tile
// whose rows hold 32 fp32 values
__device__ __forceinline__ uint32_t sw128_off32(int n, int k) {
  return (uint32_t)((n >> 3) * 1024 + (n & 7) * 128 + ((((k >> 2) ^ (n & 7)) & 7) << 4) +
                    ((k & 3) << 2));
}

template <bool LEFT>
__global__ void __launch_bounds__(F_NTHREADS, 1)
pm_tc_tf32_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const int stages = p.stages;
  const int RB = p.RB;
  uint8_t* Xs = smem;
  uint8_t* B = Xs + (size_t)stages * F_X_STAGE_BYTES;
  const int b_stage_bytes = 2 * RB * 128;
  uint64_t* bars = reinterpret_cast<uint64_t*>(B + (size_t)stages * b_stage_bytes);
  uint64_t* full_x = bars;
  uint64_t* x_empty = full_x + stages;
  uint64_t* full_b = x_empty + stages;
  uint64_t* b_empty = full_b + stages;
  uint64_t* a_full = b_empty + stages;
  uint64_t* a_empty = a_full + F_A_SLOTS;
  uint64_t* acc_full = a_empty + F_A_SLOTS;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full_x[s], 1);
      mbar_init(&x_empty[s], 4);
      mbar_init(&full_b[s], 4);
      mbar_init(&b_empty[s], 1);
    }
    for (int a = 0; a < F_A_SLOTS; ++a) {
      mbar_init(&a_full[a], 4);
      mbar_init(&a_empty[a], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(drain, 1);
    *abort = 0;
    fence_mbar_init();
  }
  if (warp == W_MMA) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t d_col0 = F_A_SLOTS * 64;  // accumulators after the A slots

  if (warp == W_TMA) {
    if (lane == 0) {
      prefetch_tmap(&tmap);
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      uint32_t armed = 0, armed_ph = 0;
      for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
        const Item w = decode_item<LEFT>(p, it);
        for (int64_t k = w.k0; k < w.k1; k += F_BK) {
          if (!mbar_wait(&x_empty[s], ph ^ 1, abort, p.err, 11)) { ok = false; break; }
          armed |= 1u << s;
          armed_ph = (armed_ph & ~(1u << s)) | (ph << s);
          mbar_arrive_expect_tx(&full_x[s], F_X_STAGE_BYTES);
          uint8_t* x = Xs + (size_t)s * F_X_STAGE_BYTES;
          if (LEFT) tma_load_2d(x, &tmap, &full_x[s], (int)w.m0, (int)k);
          else tma_load_2d(x, &tmap, &full_x[s], (int)k, (int)w.m0);
          if (++s == stages) { s = 0; ph ^= 1; }
        }
      }
      if (!ok) {
        for (int t = 0; t < stages; ++t) {
          if (!((armed >> t) & 1u)) continue;
          const uint32_t par = (armed_ph >> t) & 1u;
          const long long t0 = clock64();
          while (!mbar_try_wait(&full_x[t], par) && clock64() - t0 < kWaitCycles / 16) {
          }
        }
      }
    }
  } else if (warp == W_MMA) {
    if (lane == 0) {
      const uint32_t id_full = instr_desc(2u, false, false, BM, 2 * RB);
      const uint32_t id_half = instr_desc(2u, false, false, BM, RB);
      int s = 0, as = 0;
      uint32_t ph = 0, aph = 0;
      uint32_t eph[2] = {0, 0};
      int buf = 0;
      bool ok = true, issued = false;
      for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
        const Item w = decode_item<LEFT>(p, it);
        if (!mbar_wait(&acc_empty[buf], eph[buf] ^ 1, abort, p.err, 12)) { ok = false; break; }
        eph[buf] ^= 1;
        tc_fence_after();
        const uint32_t d = tmem + d_col0 + (uint32_t)buf * (uint32_t)(2 * RB);
        uint32_t acc = 0;
        for (int64_t k = w.k0; k < w.k1; k += F_BK) {
          if (!mbar_wait(&full_b[s], ph, abort, p.err, 13)) { ok = false; break; }
          if (!mbar_wait(&a_full[as], aph, abort, p.err, 14)) { ok = false; break; }
          tc_fence_after();
          const uint32_t b0 = smem_u32(B + (size_t)s * b_stage_bytes);
          const uint32_t a_hi = tmem + (uint32_t)as * 64u;
#pragma unroll
          for (int kk = 0; kk < F_BK / F_UK; ++kk) {
            const uint64_t bd = smem_desc(b0 + kk * 32, 16, 1024, kLayoutSW128);
            mma_tf32_ts(d, a_hi + kk * F_UK, bd, id_full, acc);
            mma_tf32_ts(d + RB, a_hi + 32 + kk * F_UK, bd, id_half, 1u);
            acc = 1;
          }
          issued = true;
          mma_commit(&b_empty[s]);
          mma_commit(&a_empty[as]);
          if (++s == stages) { s = 0; ph ^= 1; }
          if (++as == F_A_SLOTS) { as = 0; aph ^= 1; }
        }
        if (!ok) break;
        mma_commit(&acc_full[buf]);
        buf ^= 1;
      }
      if (issued) {
        mma_commit(drain);
        const long long t0 = clock64();
        while (!mbar_try_wait(drain, 0) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp < F_W_CONV0) {
    // Khatri-Rao producers: B = [k_hi | k_lo], 2 R' rows x 32 k, tf32
    const int t = threadIdx.x - W_B0 * 32;  // 0..127
    const int kk = t & 31;
    const int quarter = t >> 5;             // 4 groups of R'/4 columns
    const int r_lo = quarter * (RB / 4), r_hi = r_lo + RB / 4;
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
      const Item w = decode_item<LEFT>(p, it);
      for (int64_t k = w.k0; k < w.k1; k += F_BK) {
        if (!mbar_wait(&b_empty[s], ph ^ 1, abort, p.err, 15)) { ok = false; break; }
        uint8_t* b = B + (size_t)s * b_stage_bytes;
        const int64_t kg = k + kk;
        const bool valid = kg < w.k1;
        int64_t off[PLANC_MAX_N];
        if (valid) krp_decode(p.K, kg, off);
        for (int r = r_lo; r < r_hi; ++r) {
          const float v = (valid && r < p.R) ? krp_value(p.K, off, r) : 0.f;
          const float hi = tf32_rn(v);
          const float lo = tf32_rn(v - hi);
          *reinterpret_cast<float*>(b + sw128_off32(r, kk)) = hi;
          *reinterpret_cast<float*>(b + sw128_off32(RB + r, kk)) = lo;
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full_b[s]);
        if (++s == stages) { s = 0; ph ^= 1; }
      }
    }
  } else if (warp < F_W_EPI0) {
    // X converters: row m of the tile (TMEM lane m) -> tf32 hi | lo in TMEM
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    int s = 0, as = 0;
    uint32_t ph = 0, aph = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
      const Item w = decode_item<LEFT>(p, it);
      for (int64_t k = w.k0; k < w.k1; k += F_BK) {
        if (!mbar_wait(&full_x[s], ph, abort, p.err, 16)) { ok = false; break; }
        if (!mbar_wait(&a_empty[as], aph ^ 1, abort, p.err, 17)) { ok = false; break; }
        const uint8_t* x = Xs + (size_t)s * F_X_STAGE_BYTES;
        float v[F_BK];
        if (LEFT) {
          // tile stored [k][128 rows], 512 B per k (no swizzle)
#pragma unroll
          for (int c = 0; c < F_BK; ++c)
            v[c] = *reinterpret_cast<const float*>(x + c * 512 + row * 4);
        } else {
          // tile stored [128 rows][32 k], 128-byte swizzled
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 f = *reinterpret_cast<const float4*>(
                x + row * 128 + (((j ^ (row & 7)) & 7) << 4));
            v[4 * j + 0] = f.x; v[4 * j + 1] = f.y; v[4 * j + 2] = f.z; v[4 * j + 3] = f.w;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&x_empty[s]);  // the stage's smem is free again
        tc_fence_after();
        uint32_t hi[F_BK], lo[F_BK];
#pragma unroll
        for (int c = 0; c < F_BK; ++c) {
          const float h = tf32_rn(v[c]);
          hi[c] = __float_as_uint(h);
          lo[c] = __float_as_uint(tf32_rn(v[c] - h));
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
        if (++as == F_A_SLOTS) { as = 0; aph ^= 1; }
      }
    }
  } else {
    // epilogue
    const int q = warp & 3;
    const int row = q * 32 + lane;
    uint32_t fph[2] = {0, 0};
    int buf = 0;
    for (int64_t it = blockIdx.x; it < p.items; it += gridDim.x) {
      const Item w = decode_item<LEFT>(p, it);
      if (!mbar_wait(&acc_full[buf], fph[buf], abort, p.err, 18)) break;
      fph[buf] ^= 1;
      tc_fence_after();
      const uint32_t taddr =
          tmem + d_col0 + (uint32_t)buf * (uint32_t)(2 * RB) + ((uint32_t)(q * 32) << 16);
      const int64_t m = w.m0 + row;
      const bool live = m < p.Mdim;
      for (int r0 = 0; r0 < RB; r0 += 16) {
        float h[16], c[16];
        tmem_ld16(taddr + r0, h);
        tmem_ld16(taddr + RB + r0, c);
        tmem_ld_wait();
        if (live) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int r = r0 + j;
            if (r < p.R) {
              const float v = h[j] + c[j];
              if (p.out_mode == 0) p.out[m + p.Mdim * r] = v;
              else if (p.out_mode == 1) p.out[m * p.R + r] = v;
              else p.out[w.z * p.Mdim * p.R + m + p.Mdim * r] = v;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
      buf ^= 1;
    }
  }

  __syncthreads();
  if (warp == W_MMA) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ---- host side -------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

int stages_for(int N) {
  const int budget = 200 * 1024;
  int per = A_STAGE_BYTES + N * 128;
  int s = budget / per;
  return std::max(2, std::min(6, s));
}

int stages_for_f32(int RB) {
  const int budget = 200 * 1024;
  int per = F_X_STAGE_BYTES + 2 * RB * 128;
  return std::max(2, std::min(6, budget / per));
}

size_t smem_bytes_f32(int RB, int stages) {
  return 1024 + (size_t)stages * (F_X_STAGE_BYTES + 2 * RB * 128) +
         (4 * stages + 2 * F_A_SLOTS + 5) * 8 + 16;
}

size_t smem_bytes(int N, int stages) {
  return 1024 + (size_t)stages * (A_STAGE_BYTES + N * 128) + (3 * stages + 5) * 8 + 16;
}

// Reduction elements per work item (a multiple of the stage depth bk):
// enough items to fill the GPU twice over, and no item longer than max_k
// elements (this bounds the number of FP32 accumulations into one TMEM
// accumulator).
int64_t item_kspan(int64_t Mdim, int64_t Kdim, int sm_count, int bk, int64_t max_k) {
  const int64_t m_tiles = (Mdim + BM - 1) / BM;
  int64_t splits = std::max<int64_t>(1, (2 * sm_count + m_tiles - 1) / m_tiles);
  splits = std::max(splits, (Kdim + max_k - 1) / max_k);
  splits = std::min(splits, (Kdim + bk - 1) / bk);
  int64_t span = (Kdim + splits - 1) / splits;
  span = (span + bk - 1) / bk * bk;
  return std::max<int64_t>(span, bk);
}

int stage_bk(planc_dtype_t xdt) { return xdt == PLANC_F32 ? F_BK : BK; }
int64_t stage_max_k(planc_dtype_t xdt) { return xdt == PLANC_F32 ? 2048 : 4096; }

}  // namespace

bool pm_tc_eligible(planc_dtype_t xdt, bool left, int64_t L, int64_t C, int R) {
  (void)left;
  if (xdt != PLANC_BF16 && xdt != PLANC_F32) return false;
  if (R < 1 || R > 64) return false;
  // TMA: the row stride of X_(1:S) (L elements) must be a multiple of 16 bytes
  if ((L * (int64_t)dtype_size(xdt)) % 16 != 0) return false;
  if (L >= (1LL << 31) || C >= (1LL << 31)) return false;
  if (encode_fn() == nullptr) return false;
  return true;
}

size_t pm_tc_workspace_bytes(planc_dtype_t xdt, bool left, int64_t L, int64_t C, int R,
                             int sm_count) {
  if (!pm_tc_eligible(xdt, left, L, C, R)) return 0;
  const int64_t Mdim = left ? L : C, Kdim = left ? C : L;
  const int64_t span = item_kspan(Mdim, Kdim, sm_count, stage_bk(xdt), stage_max_k(xdt));
  const int64_t splits = (Kdim + span - 1) / span;
  return splits > 1 ? (size_t)splits * Mdim * R * sizeof(float) : 0;
}

cudaError_t launch_pm_tc(planc_dtype_t xdt, const void* X, int64_t L, int64_t C, bool left,
                         const KrpHost& kh, int R, void* out, bool out_rowmajor, void* work,
                         size_t work_bytes, int* err_flag, int sm_count, cudaStream_t st) {
  if (!pm_tc_eligible(xdt, left, L, C, R)) return cudaErrorNotSupported;
  if (((uintptr_t)X & 15) != 0) return cudaErrorNotSupported;
  TcParams p{};
  p.L = L;
  p.C = C;
  p.R = R;
  const bool f32 = xdt == PLANC_F32;
  p.RB = round_up(R, 16);
  p.N = f32 ? 2 * p.RB : 3 * p.RB;
  p.stages = f32 ? stages_for_f32(p.RB) : stages_for(p.N);
  p.err = err_flag;
  p.K.nm = kh.nm;
  p.K.R = R;
  for (int m = 0; m < kh.nm; ++m) {
    p.K.dim[m] = kh.dim[m];
    p.K.H[m] = (const float*)kh.H[m];
  }
  p.Mdim = left ? L : C;
  p.Kdim = left ? C : L;
  p.m_tiles = (p.Mdim + BM - 1) / BM;
  p.kspan = item_kspan(p.Mdim, p.Kdim, sm_count, stage_bk(xdt), stage_max_k(xdt));
  const int64_t splits = (p.Kdim + p.kspan - 1) / p.kspan;
  p.items = p.m_tiles * splits;
  if (splits > 1) {
    if (work_bytes < (size_t)splits * p.Mdim * R * sizeof(float)) return cudaErrorInvalidValue;
    p.out_mode = 2;
    p.out = (float*)work;
  } else {
    p.out_mode = out_rowmajor ? 1 : 0;
    p.out = (float*)out;
  }

  CUtensorMap tmap;
  cuuint64_t gdim[2] = {(cuuint64_t)L, (cuuint64_t)C};
  cuuint64_t gstride[1] = {(cuuint64_t)L * dtype_size(xdt)};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult cr;
  if (f32) {
    // left: [32 k][128 rows] unswizzled (512-byte rows); right: [128 rows][32 k] swizzled
    cuuint32_t box[2] = {left ? 128u : 32u, left ? 32u : 128u};
    cr = encode_fn()(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(X), gdim,
                     gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     left ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    cuuint32_t box[2] = {64u, left ? 64u : 128u};
    cr = encode_fn()(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(X), gdim,
                     gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;

  const size_t smem = f32 ? smem_bytes_f32(p.RB, p.stages) : smem_bytes(p.N, p.stages);
  const int grid = (int)std::min<int64_t>(p.items, sm_count);
  cudaError_t e;
  if (f32) {
    auto k = left ? pm_tc_tf32_kernel<true> : pm_tc_tf32_kernel<false>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, F_NTHREADS, smem, st>>>(tmap, p);
  } else {
    auto k = left ? pm_tc_bf16_kernel<true> : pm_tc_bf16_kernel<false>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NTHREADS, smem, st>>>(tmap, p);
  }
  note_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  return launch_split_reduce(false, work, (int)splits, p.Mdim, R, out, out_rowmajor, st);
}

}  // namespace planc
