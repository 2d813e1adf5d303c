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
#include <cstdlib>
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
  int h0_smem;         // 1: the first Khatri-Rao factor is staged in shared memory
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


// Modes a tensor-core Khatri-Rao operand may combine (loops over modes are
// unrolled to this bound so the per-mode indices stay in registers).
constexpr int TC_MAXM = 6;
// Stages accumulated into one TMEM accumulator before the epilogue drains it
// into FP32 registers.  The tensor core's FP32 accumulation truncates each
// product to the running sum's exponent range, so a chain of positive
// accumulations drifts low in proportion to its length (measured on the
// 512^3 workload: 1.4e-6 relative at 8 stages of 4 MMAs, 5.9e-7 at 4, 2.4e-7
// at 2); 8 stages bound it below the 1e-5 entry tolerance, and the right
// branch removes it by centring its rows (pm_tcr_kernel).
constexpr int SEG_STAGES = 8;

// Row k of the Khatri-Rao operand as per-mode row indices (mode 0 fastest).
__device__ __forceinline__ void kw_set(const TcParams& p, int64_t k64, int* idx) {
  uint32_t k = (uint32_t)k64;
#pragma unroll
  for (int m = 0; m < TC_MAXM; ++m) {
    if (m < p.K.nm) {
      const uint32_t d = (uint32_t)p.K.dim[m];
      const uint32_t q = k / d;
      idx[m] = (int)(k - q * d);
      k = q;
    } else {
      idx[m] = 0;
    }
  }
}

// Product of the factor rows of modes 1.. (all but the fastest mode) for
// columns r = lane and lane + 32: it changes only when the fastest index wraps.
__device__ __forceinline__ void kw_tail(const TcParams& p, const int* idx, int lane, float* P) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = lane + 32 * h;
    float v = 1.f;
    if (r < p.R) {
#pragma unroll
      for (int m = 1; m < TC_MAXM; ++m)
        if (m < p.K.nm) v *= __ldg(p.K.H[m] + (int64_t)idx[m] * p.K.R + r);
    }
    P[h] = v;
  }
}
// next row: step the fastest index; on a wrap carry into the higher modes
// and recompute the tail product
__device__ __forceinline__ void kw_next(const TcParams& p, int* idx, int lane, float* P) {
  if (++idx[0] < (int)p.K.dim[0]) return;
  idx[0] = 0;
  bool carry = true;
#pragma unroll
  for (int m = 1; m < TC_MAXM; ++m) {
    if (carry && m < p.K.nm) {
      if (++idx[m] < (int)p.K.dim[m]) carry = false;
      else idx[m] = 0;
    }
  }
  kw_tail(p, idx, lane, P);
}



__device__ __forceinline__ float lds_f32(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}

// Values of Khatri-Rao rows kk and kk + 1 (the cursor idx/P points at kk and
// is advanced past kk + 1) for columns r = lane and lane + 32.  SH: the first
// factor is read from its shared-memory copy at h0_s, else from global h0_g.
template <bool SH>
__device__ __forceinline__ void kw_pair(const TcParams& p, uint32_t h0_s, const float* h0_g,
                                        int* idx, float* P, int lane, int kk, int64_t nvalid,
                                        float v[2][2]) {
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const bool kv = kk + t < nvalid;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = lane + 32 * h;
      float x = 0.f;
      if (kv && r < p.R) {
        const int e = idx[0] * p.R + r;
        x = (SH ? lds_f32(h0_s + 4u * (uint32_t)e) : __ldg(h0_g + e)) * P[h];
      }
      v[t][h] = x;
    }
    kw_next(p, idx, lane, P);
  }
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
  float* sH0 = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(drain) + 16);

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
      uint32_t eph = 0;  // bit b: phase of acc_empty[b]
      int buf = 0;
      bool ok = true;
      bool issued = false;
      for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
        const Item w = decode_item<LEFT>(p, it);
        for (int64_t k = w.k0; k < w.k1 && ok; ) {
          // one accumulation segment of at most SEG_STAGES stages
          if (!mbar_wait(&acc_empty[buf], ((eph >> buf) & 1u) ^ 1u, abort, p.err, 2)) { ok = false; break; }
          eph ^= 1u << buf;
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)buf * 256u;
          uint32_t acc = 0;
          for (int st = 0; st < SEG_STAGES && k < w.k1; ++st, k += BK) {
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
    // The first Khatri-Rao factor is staged in shared memory once; warp wi
    // then builds rows [16 wi, 16 wi + 16) of every stage, two rows at a
    // time (lane = column r), so each of the three terms of a row pair is one
    // 32-bit store into the swizzled tile.
    const int wi = warp - W_B0;
    const int RB = p.RB;
    const bool h0_shared = p.h0_smem != 0;
    const uint32_t h0_s = smem_u32(sH0);
    if (h0_shared) {
      const int64_t n0 = p.K.dim[0] * (int64_t)p.R;
      for (int64_t e = threadIdx.x - W_B0 * 32; e < n0; e += 128) sH0[e] = __ldg(p.K.H[0] + e);
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
    constexpr int ROWS = BK / 4;
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
      const Item w = decode_item<LEFT>(p, it);
      for (int64_t k = w.k0; k < w.k1; k += BK) {
        if (!mbar_wait(&empty[s], ph ^ 1, abort, p.err, 5)) { ok = false; break; }
        uint8_t* b = B + (size_t)s * b_stage_bytes;
        const int kb = wi * ROWS;
        int idx[TC_MAXM];
        float P[2];
        kw_set(p, k + kb, idx);
        kw_tail(p, idx, lane, P);
        const int64_t nvalid = w.k1 - k;
#pragma unroll 4
        for (int kk = kb; kk < kb + ROWS; kk += 2) {
          float v[2][2];
          if (h0_shared) kw_pair<true>(p, h0_s, p.K.H[0], idx, P, lane, kk, nvalid, v);
          else kw_pair<false>(p, h0_s, p.K.H[0], idx, P, lane, kk, nvalid, v);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = lane + 32 * h;
            if (r < RB) {
              const __nv_bfloat162 hi = __floats2bfloat162_rn(v[0][h], v[1][h]);
              const float2 h2 = __bfloat1622float2(hi);
              const float a0 = v[0][h] - h2.x, a1 = v[1][h] - h2.y;
              const __nv_bfloat162 mid = __floats2bfloat162_rn(a0, a1);
              const float2 m2 = __bfloat1622float2(mid);
              const __nv_bfloat162 lo = __floats2bfloat162_rn(a0 - m2.x, a1 - m2.y);
              // rows r, RB + r, 2 RB + r share (row & 7) since RB % 8 == 0
              const uint32_t in_row = ((((uint32_t)kk >> 3) ^ ((uint32_t)r & 7u)) << 4) +
                                      (((uint32_t)kk & 7u) << 1);
              const uint32_t r0 = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128);
              const uint32_t rstride = (uint32_t)RB * 128u;  // RB rows further down
              *reinterpret_cast<__nv_bfloat162*>(b + r0 + in_row) = hi;
              *reinterpret_cast<__nv_bfloat162*>(b + r0 + rstride + in_row) = mid;
              *reinterpret_cast<__nv_bfloat162*>(b + r0 + 2 * rstride + in_row) = lo;
            }
          }
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
    uint32_t fph = 0;  // bit b: phase of acc_full[b]
    int buf = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
      const Item w = decode_item<LEFT>(p, it);
      float sum[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) sum[j] = 0.f;
      for (int64_t k = w.k0; k < w.k1; k += (int64_t)SEG_STAGES * BK) {
        if (!mbar_wait(&acc_full[buf], (fph >> buf) & 1u, abort, p.err, 6)) { ok = false; break; }
        fph ^= 1u << buf;
        tc_fence_after();
        const uint32_t taddr = tmem + (uint32_t)buf * 256u + ((uint32_t)(q * 32) << 16);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (c * 16 < p.RB) {
            float h[16], md[16], lo[16];
            tmem_ld16(taddr + c * 16, h);
            tmem_ld16(taddr + p.RB + c * 16, md);
            tmem_ld16(taddr + 2 * p.RB + c * 16, lo);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 16; ++j) sum[c * 16 + j] += h[j] + (md[j] + lo[j]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
        buf ^= 1;
      }
      if (!ok) break;
      const int64_t m = w.m0 + row;
      if (m < p.Mdim) {
#pragma unroll
        for (int r = 0; r < 64; ++r) {
          if (r < p.R) {
            if (p.out_mode == 0) p.out[m + p.Mdim * r] = sum[r];
            else if (p.out_mode == 1) p.out[m * p.R + r] = sum[r];
            else p.out[w.z * p.Mdim * p.R + m + p.Mdim * r] = sum[r];
          }
        }
      }
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
  float* sH0 = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(drain) + 16);

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
      uint32_t eph = 0;  // bit b: phase of acc_empty[b]
      int buf = 0;
      bool ok = true, issued = false;
      for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
        const Item w = decode_item<LEFT>(p, it);
        for (int64_t k = w.k0; k < w.k1 && ok; ) {
          if (!mbar_wait(&acc_empty[buf], ((eph >> buf) & 1u) ^ 1u, abort, p.err, 12)) { ok = false; break; }
          eph ^= 1u << buf;
          tc_fence_after();
          const uint32_t d = tmem + d_col0 + (uint32_t)buf * (uint32_t)(2 * RB);
          uint32_t acc = 0;
          for (int st = 0; st < SEG_STAGES && k < w.k1; ++st, k += F_BK) {
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
      }
      if (issued) {
        mma_commit(drain);
        const long long t0 = clock64();
        while (!mbar_try_wait(drain, 0) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp < F_W_CONV0) {
    // Khatri-Rao producers: B = [k_hi | k_lo], 2 R' rows x 32 k, tf32.  The
    // first factor is staged in shared memory; warp wi builds rows
    // [8 wi, 8 wi + 8) of each stage in pairs (lane = column r).
    const int wi = warp - W_B0;
    const bool h0_shared = p.h0_smem != 0;
    const uint32_t h0_s = smem_u32(sH0);
    if (h0_shared) {
      const int64_t n0 = p.K.dim[0] * (int64_t)p.R;
      for (int64_t e = threadIdx.x - W_B0 * 32; e < n0; e += 128) sH0[e] = __ldg(p.K.H[0] + e);
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
    constexpr int ROWS = F_BK / 4;
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
      const Item w = decode_item<LEFT>(p, it);
      for (int64_t k = w.k0; k < w.k1; k += F_BK) {
        if (!mbar_wait(&b_empty[s], ph ^ 1, abort, p.err, 15)) { ok = false; break; }
        uint8_t* b = B + (size_t)s * b_stage_bytes;
        const int kb = wi * ROWS;
        int idx[TC_MAXM];
        float P[2];
        kw_set(p, k + kb, idx);
        kw_tail(p, idx, lane, P);
        const int64_t nvalid = w.k1 - k;
#pragma unroll
        for (int kk = kb; kk < kb + ROWS; kk += 2) {
          float v[2][2];
          if (h0_shared) kw_pair<true>(p, h0_s, p.K.H[0], idx, P, lane, kk, nvalid, v);
          else kw_pair<false>(p, h0_s, p.K.H[0], idx, P, lane, kk, nvalid, v);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = lane + 32 * h;
            if (r < RB) {
              const float h0v = tf32_rn(v[0][h]), h1v = tf32_rn(v[1][h]);
              const uint32_t in_row = ((((uint32_t)kk >> 2) ^ ((uint32_t)r & 7u)) << 4) +
                                      (((uint32_t)kk & 3u) << 2);
              const uint32_t r0 = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128);
              *reinterpret_cast<float2*>(b + r0 + in_row) = make_float2(h0v, h1v);
              *reinterpret_cast<float2*>(b + r0 + (uint32_t)RB * 128u + in_row) =
                  make_float2(tf32_rn(v[0][h] - h0v), tf32_rn(v[1][h] - h1v));
            }
          }
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
        const uint32_t x = smem_u32(Xs + (size_t)s * F_X_STAGE_BYTES);
        float v[F_BK];
        if (LEFT) {
          // tile stored [k][128 rows], 512 B per k (no swizzle)
#pragma unroll
          for (int c = 0; c < F_BK; ++c) v[c] = lds_f32(x + c * 512 + row * 4);
        } else {
          // tile stored [128 rows][32 k], 128-byte swizzled
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint32_t a = x + row * 128 + (((j ^ (row & 7)) & 7) << 4);
            asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                         : "=f"(v[4 * j + 0]), "=f"(v[4 * j + 1]), "=f"(v[4 * j + 2]),
                           "=f"(v[4 * j + 3])
                         : "r"(a)
                         : "memory");
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
    // epilogue: drain each accumulation segment into FP32 registers
    const int q = warp & 3;
    const int row = q * 32 + lane;
    uint32_t fph = 0;  // bit b: phase of acc_full[b]
    int buf = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
      const Item w = decode_item<LEFT>(p, it);
      float sum[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) sum[j] = 0.f;
      for (int64_t k = w.k0; k < w.k1; k += (int64_t)SEG_STAGES * F_BK) {
        if (!mbar_wait(&acc_full[buf], (fph >> buf) & 1u, abort, p.err, 18)) { ok = false; break; }
        fph ^= 1u << buf;
        tc_fence_after();
        const uint32_t taddr =
            tmem + d_col0 + (uint32_t)buf * (uint32_t)(2 * RB) + ((uint32_t)(q * 32) << 16);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (c * 16 < RB) {
            float h[16], cr[16];
            tmem_ld16(taddr + c * 16, h);
            tmem_ld16(taddr + RB + c * 16, cr);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 16; ++j) sum[c * 16 + j] += h[j] + cr[j];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
        buf ^= 1;
      }
      if (!ok) break;
      const int64_t m = w.m0 + row;
      if (m < p.Mdim) {
#pragma unroll
        for (int r = 0; r < 64; ++r) {
          if (r < p.R) {
            if (p.out_mode == 0) p.out[m + p.Mdim * r] = sum[r];
            else if (p.out_mode == 1) p.out[m * p.R + r] = sum[r];
            else p.out[w.z * p.Mdim * p.R + m + p.Mdim * r] = sum[r];
          }
        }
      }
    }
  }

  __syncthreads();
  if (warp == W_MMA) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// Row r of a 128 x 32 FP32 X stage stored [rows][32 k] with the 128-byte swizzle.
__device__ __forceinline__ void lds_row_sw128(uint32_t x, int row, float* v) {
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

// The mean of a row's 32 values in one stage (pairwise sum over 32).
__device__ __forceinline__ float stage_mean(const float* v) {
  float t[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) t[c] = v[2 * c] + v[2 * c + 1];
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
    for (int c = 0; c < w; ++c) t[c] += t[c + w];
  return t[0] * (1.f / 32.f);
}

// ---- resident Khatri-Rao operand ------------------------------------------------------
//
// The Khatri-Rao operand factors row-wise as K[k, r] = H_in[k_in, r] * W[k_out, r]:
// one factor ("inner", the fastest mode of the operand) times the product of
// the others.  Here the split and swizzled H_in is built once per CTA and
// stays resident in shared memory as the MMA's B operand, so the pipeline
// carries only X; the outer weights W are applied when the epilogue drains
// the TMEM accumulators:
//
//   left : T(l, r)    = sum_{o} W[o, r] * sum_{c} X[l, c, o] H_in[c, r]
//          (X_(1:S) seen as L x d_in x n_out; one drain per outer index o)
//   right: T(c, r)    = sum_{j} W[j, r] * sum_{l} X[l, j, c] H_in[l, r]
//          (rows (j, c) of X seen as d_in x (L/d_in * C); the epilogue
//          weights every row by W[j] and sums the 128 rows of a tile, which
//          all belong to one c because L/d_in is a multiple of 128)
//
// FP32 X keeps the TMEM-resident 3xTF32 split of the converters; BF16 X is
// read by the MMA straight from the TMA tile.
struct TcrParams {
  int64_t L, C;
  int64_t rows;         // A rows: left L, right (L / d_in) * C
  int R, RB, N;         // rank, rank rounded to 16, MMA N of the widest block
  int d_in;             // rows of the resident factor
  int nst;              // stages per inner pass: ceil(d_in / bk)
  int stages;           // X pipeline depth
  int64_t n_out;        // left: outer indices C / d_in
  int64_t o_span;       // left: outer indices per work item
  int64_t m_tiles;      // left: 128-row tiles of A
  int64_t items;
  int tpc;              // right: 128-row tiles per output row c (= jdim / 128)
  int tpi;              // right: tiles per work item (divides tpc)
  int nsplit;           // right: work items per output row c (= tpc / tpi)
  int64_t jdim;         // right: L / d_in
  int out_mode;         // 0: out[m + Mdim r]; 1: out[m R + r]; 2: partial slice z
  int64_t Mdim;         // rows of the final output (left L, right C)
  int aslots;           // FP32: TMEM slots for the converted X tiles (<= F_A_SLOTS)
  int blockmode;        // right branch with L / d_in a multiple of 32 but not of 128:
                        // items are runs of tpi tiles; each 32-row block (one c)
                        // writes its weighted row sum to out[block * R + r]
  int64_t nblocks;      // blockmode: rows / 32
  int seg;              // stages accumulated into one TMEM accumulator per drain
  int center;           // FP32 X, right branch, RB <= 32: rows centred per stage (see kernel)
  float* out;
  int* err;
  const float* Hin;     // resident factor, d_in x R row-major
  Krp<float> W;         // the other factors (outer weights)
};

// weights W[o, r] = prod_m Hw_m[o_m, r] for r < R (o enumerates the weight
// modes, fastest first)
// Rows of the weight factors for outer index o (o enumerates the weight
// modes, fastest first): W[o, r] = prod_m row_m[r].
__device__ __forceinline__ void tcr_rows(const TcrParams& p, int64_t o, const float** row) {
  uint32_t k = (uint32_t)o;
#pragma unroll
  for (int m = 0; m < TC_MAXM; ++m) {
    if (m < p.W.nm) {
      const uint32_t d = (uint32_t)p.W.dim[m];
      const uint32_t q = k / d;
      row[m] = p.W.H[m] + (int64_t)(k - q * d) * p.R;
      k = q;
    } else {
      row[m] = nullptr;
    }
  }
}

// weights of columns col .. col + 3 (1 past R)
__device__ __forceinline__ float4 tcr_w4(const TcrParams& p, const float* const* row, int col) {
  float4 v = make_float4(1.f, 1.f, 1.f, 1.f);
  if (col < p.R) {
#pragma unroll
    for (int m = 0; m < TC_MAXM; ++m) {
      if (m < p.W.nm) {
        const float* rr = row[m] + col;
        if ((p.R & 3) == 0) {
          const float4 h = __ldg(reinterpret_cast<const float4*>(rr));
          v.x *= h.x; v.y *= h.y; v.z *= h.z; v.w *= h.w;
        } else {
          v.x *= __ldg(rr);
          if (col + 1 < p.R) v.y *= __ldg(rr + 1);
          if (col + 2 < p.R) v.z *= __ldg(rr + 2);
          if (col + 3 < p.R) v.w *= __ldg(rr + 3);
        }
      }
    }
  }
  return v;
}

// weights of columns 16 c .. 16 c + 15
__device__ __forceinline__ void tcr_w16(const TcrParams& p, const float* const* row, int c,
                                        float* w) {
#pragma unroll
  for (int r4 = 0; r4 < 4; ++r4) {
    const float4 v = tcr_w4(p, row, 16 * c + 4 * r4);
    w[4 * r4 + 0] = v.x; w[4 * r4 + 1] = v.y; w[4 * r4 + 2] = v.z; w[4 * r4 + 3] = v.w;
  }
}

// Sum of v[r] over the 32 lanes of the warp for r < 32: a recursive-halving
// reduce-scatter; lane r returns the warp-wide sum of v[r].
__device__ __forceinline__ float warp_reduce_scatter32(float* v, int lane) {
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

// RBX: 32 or 64, the register arrays of the epilogue hold RBX columns (RB <= RBX);
// CEN: the right branch with FP32 X and RB <= 32 centres its rows (see below)
template <bool LEFT, bool F32, int RBX, bool CEN = false>
__global__ void __launch_bounds__(F32 ? 352 : 192, 1)
pm_tcr_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TcrParams p) {
  constexpr int BKX = F32 ? F_BK : BK;             // reduction elements per stage
  constexpr int UKX = F32 ? F_UK : UK;
  constexpr int XST = BM * BKX * (F32 ? 4 : 2);    // X stage bytes (16 KB)
  constexpr int W_EPI = F32 ? 6 : 2;               // epilogue warps (F32: converters 2..5)
  // FP32: a second MMA warp issues the x_lo k_hi products into their own
  // accumulator (a tcgen05.mma costs its issuing thread a fixed ~80 cycles
  // for N <= 128, so two issuers double the MMA rate)
  constexpr int W_MMA2 = 10;
  // two MMA warps for FP32 X: R <= 32 with four TMEM A slots; R <= 64 in the
  // left branch with two (the accumulators of 3 RB columns fill the rest; the
  // right branch's epilogue, already its limit there, would read a third
  // accumulator: slower in A/B)
  constexpr bool DUAL = F32 && (RBX == 32 || LEFT);
  // Row centring (FP32 X, right branch, RB <= 32).  The tensor core's FP32
  // accumulation truncates every product to the running sum's exponent
  // range, so a chain of all-positive accumulations loses a little on every
  // MMA and comes out low (about 1.4e-6 relative after the 32 MMAs of an
  // 8-stage segment, nearly the same in every entry).  The right branch
  // yields the last mode's MTTKRP, whose inner product with the updated
  // factor is the error identity's beta, so there the converters feed the
  // MMA x' = x - c_g for every stage of a drain segment g, with c_g the
  // mean of the row's 32 values in the segment's first stage: the partial
  // sums stay small and change sign, and the truncation errors cancel.  The
  // converters hand c_g to the epilogue through a ring of four slots of 128
  // floats (c_full / c_empty); the epilogue adds back c_g colsum_g(H_in)[r]
  // when it drains segment g (any c_g is exact here, as long as both sides
  // use the same value).  A per-segment c keeps the converters' added work
  // to one subtraction per element (the converters set the pace of this
  // kernel).  (A uniform bias in the left branch only rescales lambda, which
  // the normalisation after each update absorbs.)
  static_assert(!CEN || (F32 && RBX == 32 && !LEFT), "centring: FP32 right branch, RB <= 32");
  constexpr bool CENTER = CEN;
  constexpr bool cen = CEN;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const int stages = p.stages;
  const int RB = p.RB;
  const int bstage = (F32 ? 2 : 3) * RB * 128;     // bytes of one B stage image
  uint8_t* Xs = smem;
  uint8_t* Bimg = Xs + (size_t)stages * XST;
  uint64_t* bars = reinterpret_cast<uint64_t*>(Bimg + (size_t)p.nst * bstage);
  uint64_t* full_x = bars;                    // TMA -> consumer (MMA or converters)
  uint64_t* x_empty = full_x + stages;        // consumer -> TMA
  uint64_t* a_full = x_empty + stages;        // F32: converters -> MMA
  uint64_t* a_empty = a_full + F_A_SLOTS;     // F32: MMA -> converters
  uint64_t* acc_full = a_empty + F_A_SLOTS;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* red = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(drain) + 16);  // 4 x 64
  // H_in (d_in x R, row-major FP32) arrives by one bulk copy into the X stage
  // area (idle until the pipeline starts) when aligned and small enough; the
  // image below is then built from shared memory
  uint64_t* hbar = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(red) + 1024);
  // centring: c_full[4] (converters -> epilogue), c_empty[4] (back), the
  // ring cring[slot * BM + row], and the column sums of H_in over each drain
  // segment, ksg[g * RB + r] = sum_{k in segment g} H_in[k, r]
  const int nsegs = (p.nst + p.seg - 1) / p.seg;
  uint64_t* c_full = hbar + 1;
  uint64_t* c_empty = c_full + 4;
  float* cring = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(c_empty + 4) + 15) & ~static_cast<uintptr_t>(15));
  float* ksg = cring + (cen ? 4 * BM : 0);
  {
    // the layout must fit the dynamic shared memory the launch provides
    uint32_t dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const uintptr_t end = reinterpret_cast<uintptr_t>(ksg + (cen ? nsegs * RB : 0));
    if (end - reinterpret_cast<uintptr_t>(smem_raw) > (uintptr_t)dyn) {
      if (threadIdx.x == 0) atomicExch(p.err, 31);
      return;  // uniform: no barrier, TMEM or memory access has happened yet
    }
  }

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full_x[s], 1);
      mbar_init(&x_empty[s], F32 ? 4 : 1);
    }
    for (int a = 0; a < F_A_SLOTS; ++a) {
      mbar_init(&a_full[a], 4);
      mbar_init(&a_empty[a], DUAL ? 2 : 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], DUAL ? 2 : 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(drain, DUAL ? 2 : 1);
    if (cen) {
      for (int b = 0; b < 4; ++b) {
        mbar_init(&c_full[b], 4);   // the converter warps
        mbar_init(&c_empty[b], 4);  // the epilogue warps
      }
    }
    *abort = 0;
    fence_mbar_init();
  }
  pdl_wait();  // the factors of the previous mode update are complete
  pdl_trigger();
  const uint32_t hbytes = (uint32_t)((int64_t)p.d_in * p.R * 4);
  const bool hbulk = (hbytes & 15u) == 0 && (reinterpret_cast<uintptr_t>(p.Hin) & 15u) == 0 &&
                     (size_t)hbytes <= (size_t)stages * XST;
  if (hbulk && threadIdx.x == 0) {
    mbar_init(hbar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(hbar, hbytes);
    bulk_g2s(Xs, p.Hin, hbytes, hbar);
  }
  if (warp == W_MMA) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  // the resident B image: stage j holds rows j*BKX .. j*BKX+BKX-1 of H_in
  // as split terms, K-major, 128-byte swizzled
  {
    const float* hsrc = p.Hin;
    if (hbulk) {
      __syncthreads();  // hbar initialised
      mbar_wait(hbar, 0, abort, p.err, 28);
      hsrc = reinterpret_cast<const float*>(Xs);
    }
    const int total = p.nst * BKX * RB;
    constexpr int BATCH = 8;  // loads issued together (global fallback)
    for (int e0 = threadIdx.x; e0 < total; e0 += BATCH * (int)blockDim.x) {
      float v[BATCH];
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int e = e0 + u * (int)blockDim.x;
        const int k = e / RB, r = e - (e / RB) * RB;
        v[u] = (e < total && k < p.d_in && r < p.R) ? hsrc[k * p.R + r] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int e = e0 + u * (int)blockDim.x;
        if (e >= total) break;
        const int k = e / RB, r = e - (e / RB) * RB;
        const int j = k / BKX, kk = k - j * BKX;
        uint8_t* bb = Bimg + (size_t)j * bstage;
        if (F32) {
          const float hi = tf32_rn(v[u]);
          *reinterpret_cast<float*>(bb + sw128_off32(r, kk)) = hi;
          *reinterpret_cast<float*>(bb + sw128_off32(RB + r, kk)) = tf32_rn(v[u] - hi);
        } else {
          const __nv_bfloat16 hi = __float2bfloat16_rn(v[u]);
          const float r1 = v[u] - __bfloat162float(hi);
          const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
          *reinterpret_cast<__nv_bfloat16*>(bb + sw128_off(r, kk)) = hi;
          *reinterpret_cast<__nv_bfloat16*>(bb + sw128_off(RB + r, kk)) = mid;
          *reinterpret_cast<__nv_bfloat16*>(bb + sw128_off(2 * RB + r, kk)) =
              __float2bfloat16_rn(r1 - __bfloat162float(mid));
        }
      }
    }
    if (cen) {
      // one warp per column sum: the lanes split the segment's rows and the
      // partial sums are combined with their rounding errors (Knuth's
      // TwoSum), so the sum is exact to about one FP32 rounding
      const int kseg = p.seg * BKX;
      const int nw = (int)blockDim.x >> 5;
      for (int e = warp; e < nsegs * RB; e += nw) {
        const int g = e / RB, r = e - (e / RB) * RB;
        float sm = 0.f, cm = 0.f;
        if (r < p.R) {
          const int k1 = min(p.d_in, (g + 1) * kseg);
          for (int k = g * kseg + lane; k < k1; k += 32) {
            const float x = hsrc[k * p.R + r];
            const float t = sm + x, z = t - sm;
            cm += (sm - (t - z)) + (x - z);
            sm = t;
          }
        }
#pragma unroll
        for (int w = 16; w >= 1; w >>= 1) {
          const float so = __shfl_xor_sync(0xffffffffu, sm, w);
          const float co = __shfl_xor_sync(0xffffffffu, cm, w);
          const float t = sm + so, z = t - sm;
          cm += co + ((sm - (t - z)) + (so - z));
          sm = t;
        }
        if (lane == 0) ksg[e] = sm + cm;
      }
    }
    fence_proxy_async_smem();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // FP32: p.aslots TMEM slots of 64 columns (x hi | x lo), then two
  // accumulator buffers; BF16: buffers of 256 columns [hi | mid | lo].
  const int aslots = F32 ? p.aslots : 1;
  const uint32_t d_col0 = F32 ? (uint32_t)aslots * 64u : 0u;
  // FP32 buffer: [hi: x_hi k_hi | x_hi k_lo (2 RB)] then, with two MMA warps
  // (DUAL), [lo: x_lo k_hi (RB)]; with one, x_lo k_hi adds onto x_hi k_lo
  const uint32_t d_stride = F32 ? (uint32_t)((DUAL ? 3 : 2) * RB) : 256u;

  // Work item layout.  Left: item = (128-row tile of L, range of outer
  // indices).  Right: item = (output row c, slice of its tpc row tiles).
  const int nsub = LEFT ? 1 : p.tpi;
  auto tile_m0 = [&](int64_t it, int u) -> int64_t {
    if (LEFT) return (it % p.m_tiles) * BM;
    if (p.blockmode) return (it * p.tpi + u) * BM;
    const int64_t c = it / p.nsplit, z = it % p.nsplit;
    return ((c * p.tpc) + z * p.tpi + u) * BM;
  };
  auto item_o0 = [&](int64_t it) { return LEFT ? (it / p.m_tiles) * p.o_span : (int64_t)0; };
  auto item_o1 = [&](int64_t it) {
    return LEFT ? min(p.n_out, (it / p.m_tiles) * p.o_span + p.o_span) : (int64_t)1;
  };

  if (warp == W_TMA) {
    if (lane == 0) {
      prefetch_tmap(&tmap);
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      uint32_t armed = 0, armed_ph = 0;
      for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
        for (int u = 0; u < nsub && ok; ++u) {
          const int64_t m0 = tile_m0(it, u);
          for (int64_t o = item_o0(it); o < item_o1(it) && ok; ++o) {
            for (int j = 0; j < p.nst; ++j) {
              if (!mbar_wait(&x_empty[s], ph ^ 1, abort, p.err, 21)) { ok = false; break; }
              armed |= 1u << s;
              armed_ph = (armed_ph & ~(1u << s)) | (ph << s);
              mbar_arrive_expect_tx(&full_x[s], XST);
              uint8_t* x = Xs + (size_t)s * XST;
              if (LEFT) {
                tma_load_3d(x, &tmap, &full_x[s], (int)m0, j * BKX, (int)o);
                if (!F32) tma_load_3d(x + XST / 2, &tmap, &full_x[s], (int)m0 + 64, j * BKX, (int)o);
              } else {
                tma_load_2d(x, &tmap, &full_x[s], j * BKX, (int)m0);
              }
              if (++s == stages) { s = 0; ph ^= 1; }
            }
          }
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
  } else if (warp == W_MMA || (F32 && warp == W_MMA2)) {
    if (lane == 0 && (warp == W_MMA || DUAL)) {
      const bool lo_warp = F32 && warp == W_MMA2;
      const uint32_t id_a = F32 ? instr_desc(2u, false, false, BM, 2 * RB)
                                : instr_desc(1u, LEFT, false, BM, 3 * RB);
      const uint32_t id_b = instr_desc(2u, false, false, BM, RB);
      int s = 0, as = 0;
      uint32_t ph = 0, aph = 0, eph = 0;
      int buf = 0;
      bool ok = true, issued = false;
      const uint32_t b_base = smem_u32(Bimg);
      for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
        for (int u = 0; u < nsub && ok; ++u) {
          for (int64_t o = item_o0(it); o < item_o1(it) && ok; ++o) {
            for (int g0 = 0; g0 < p.nst && ok; g0 += p.seg) {
              if (!mbar_wait(&acc_empty[buf], ((eph >> buf) & 1u) ^ 1u, abort, p.err, 22)) {
                ok = false;
                break;
              }
              eph ^= 1u << buf;
              tc_fence_after();
              const uint32_t d =
                  tmem + d_col0 + (uint32_t)buf * d_stride + (lo_warp ? (uint32_t)(2 * RB) : 0u);
              uint32_t acc = 0;
              const int g1 = min(p.nst, g0 + p.seg);
              for (int j = g0; j < g1; ++j) {
                // FP32: the converters consume X and hand over TMEM slots;
                // BF16: the MMA reads the X tile itself
                if (F32) {
                  if (!mbar_wait(&a_full[as], aph, abort, p.err, 24)) { ok = false; break; }
                } else {
                  if (!mbar_wait(&full_x[s], ph, abort, p.err, 23)) { ok = false; break; }
                }
                tc_fence_after();
                const uint32_t b0 = b_base + (uint32_t)(j * bstage);
                if (F32) {
                  const uint32_t a_hi = tmem + (uint32_t)as * 64u;
                  if (lo_warp) {
#pragma unroll
                    for (int kk = 0; kk < BKX / UKX; ++kk) {
                      const uint64_t bd = smem_desc(b0 + kk * 32, 16, 1024, kLayoutSW128);
                      mma_tf32_ts(d, a_hi + 32 + kk * UKX, bd, id_b, acc);
                      acc = 1;
                    }
                  } else {
#pragma unroll
                    for (int kk = 0; kk < BKX / UKX; ++kk) {
                      const uint64_t bd = smem_desc(b0 + kk * 32, 16, 1024, kLayoutSW128);
                      mma_tf32_ts(d, a_hi + kk * UKX, bd, id_a, acc);
                      if constexpr (!DUAL) mma_tf32_ts(d + RB, a_hi + 32 + kk * UKX, bd, id_b, 1u);
                      acc = 1;
                    }
                  }
                  mma_commit(&a_empty[as]);
                  if (++as == aslots) { as = 0; aph ^= 1; }
                } else {
                  const uint32_t a0 = smem_u32(Xs + (size_t)s * XST);
#pragma unroll
                  for (int kk = 0; kk < BKX / UKX; ++kk) {
                    const uint64_t ad = LEFT ? smem_desc(a0 + kk * 2048, XST / 2, 1024, kLayoutSW128)
                                             : smem_desc(a0 + kk * 32, 16, 1024, kLayoutSW128);
                    const uint64_t bd = smem_desc(b0 + kk * 32, 16, 1024, kLayoutSW128);
                    mma_f16_ss(d, ad, bd, id_a, acc);
                    acc = 1;
                  }
                  mma_commit(&x_empty[s]);
                  if (++s == stages) { s = 0; ph ^= 1; }
                }
                issued = true;
              }
              if (!ok) break;
              mma_commit(&acc_full[buf]);
              buf ^= 1;
            }
          }
        }
      }
      if (issued) {
        mma_commit(drain);
        const long long t0 = clock64();
        while (!mbar_try_wait(drain, 0) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (F32 && warp < W_EPI) {
    // X converters: row m of the tile (TMEM lane m) -> tf32 hi | lo in TMEM
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    int s = 0, as = 0;
    uint32_t ph = 0, aph = 0;
    bool ok = true;
    // centring: this segment's c, the stage's place in its segment, and the
    // ring slot with the slot phases
    float cseg = 0.f;
    int jseg = 0, cb = 0;
    uint32_t cph = 0;
    for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x) {
      for (int u = 0; u < nsub && ok; ++u) {
        for (int64_t o = item_o0(it); o < item_o1(it) && ok; ++o) {
          for (int j = 0; j < p.nst; ++j) {
            {
              if (!mbar_wait(&full_x[s], ph, abort, p.err, 25)) { ok = false; break; }
              if (!mbar_wait(&a_empty[as], aph ^ 1, abort, p.err, 26)) { ok = false; break; }
              const uint32_t x = smem_u32(Xs + (size_t)s * XST);
              float v[F_BK];
              if (LEFT) {
#pragma unroll
                for (int c = 0; c < F_BK; ++c) v[c] = lds_f32(x + c * 512 + row * 4);
              } else {
                lds_row_sw128(x, row, v);
              }
              __syncwarp();
              if (lane == 0) mbar_arrive(&x_empty[s]);
              tc_fence_after();
              if constexpr (CENTER) {
                if (cen) {
                  if (j == 0) jseg = 0;
                  if (jseg == 0) {
                    // first stage of a segment: its c goes to a ring slot once
                    // the drain that last read the slot (four segments back)
                    // has taken it
                    if (!mbar_wait(&c_empty[cb], ((cph >> cb) & 1u) ^ 1u, abort, p.err, 29)) {
                      ok = false;
                      break;
                    }
                    cph ^= 1u << cb;
                    cseg = stage_mean(v);
                    cring[cb * BM + row] = cseg;
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&c_full[cb]);
                    cb = (cb + 1) & 3;
                  }
#pragma unroll
                  for (int c = 0; c < F_BK; ++c) v[c] -= cseg;
                  if (++jseg == p.seg) jseg = 0;
                }
              }
              // 3xTF32 split: hi = x with the 13 low mantissa bits cleared
              // (exact in TF32), lo = x - hi (exact in FP32).  The MMA reads
              // lo by dropping its own low bits, a truncation toward zero:
              // centred rows have both signs and the errors cancel; otherwise
              // lo is rounded to TF32 first so that the split stays unbiased.
              uint32_t hi[F_BK], lo[F_BK];
#pragma unroll
              for (int c = 0; c < F_BK; ++c) {
                const uint32_t hb = __float_as_uint(v[c]) & 0xffffe000u;
                hi[c] = hb;
                const float l = v[c] - __uint_as_float(hb);
                lo[c] = cen ? __float_as_uint(l) : __float_as_uint(tf32_rn(l));
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
            }
            if (++s == stages) { s = 0; ph ^= 1; }
            if (++as == aslots) { as = 0; aph ^= 1; }
          }
        }
      }
    }
  } else if (warp >= W_EPI && warp < W_EPI + 4) {
    // epilogue: drain each group into registers and apply the outer weights
    const int q = warp & 3;
    const int row = q * 32 + lane;
    uint32_t fph = 0;
    int buf = 0;
    int eb = 0;         // centring: ring slot of the segment being drained
    uint32_t ecph = 0;  // and the phases of c_full
    bool ok = true;
    // Right branch, BF16 X, R <= 16: two consecutive items of this CTA (two output
    // rows) accumulate into the two halves of the 32 columns of sum[], and one
    // warp reduce-scatter and one round of the epilogue barriers write both.
    // (BF16 X: its right-branch epilogue is this kernel's limit there)
    constexpr bool PAIRABLE = !F32 && !LEFT && RBX == 32;
    const bool pair = PAIRABLE && RB <= 16 && !p.blockmode;
    float sum[RBX];
    int li = 0;  // items this CTA has started
    for (int64_t it = blockIdx.x; it < p.items && ok; it += gridDim.x, ++li) {
      const int half = pair ? (li & 1) : 0;
      if (half == 0) {
#pragma unroll
        for (int r = 0; r < RBX; ++r) sum[r] = 0.f;
      }
      for (int u = 0; u < nsub && ok; ++u) {
        if (!LEFT && p.blockmode) {
#pragma unroll
          for (int r = 0; r < RBX; ++r) sum[r] = 0.f;
        }
        // Weights.  Left: W[o] is the same for every row of the tile; one warp
        // stages it in shared memory before the accumulator wait.  Right: row
        // (j, c) carries W[j]; held in registers for BF16 X with RBX = 32,
        // read per 16-column chunk otherwise (register budget).
        const float* wrow[TC_MAXM];
        constexpr bool WREG = !F32 && RBX == 32;
        float wreg[WREG ? 32 : 1];
        const bool weighted = p.W.nm > 0;
        if (!LEFT && weighted) {
          const int64_t jrow = (tile_m0(it, u) + row) % p.jdim;
          tcr_rows(p, jrow, wrow);
          if constexpr (WREG) {
            tcr_w16(p, wrow, 0, wreg);
            tcr_w16(p, wrow, 1, wreg + 16);
          }
        }
        for (int64_t o = item_o0(it); o < item_o1(it) && ok; ++o) {
          float* ws = red + (o & 1) * 64;
          if (LEFT && weighted) {
            if (warp == W_EPI && lane < RBX / 4) {
              tcr_rows(p, o, wrow);
              *reinterpret_cast<float4*>(ws + 4 * lane) = tcr_w4(p, wrow, 4 * lane);
            }
            asm volatile("bar.sync 2, 128;" ::: "memory");
          }
          for (int g0 = 0; g0 < p.nst; g0 += p.seg) {
            if (!mbar_wait(&acc_full[buf], (fph >> buf) & 1u, abort, p.err, 27)) { ok = false; break; }
            // centring: this row's c of the segment (the slot goes back to the
            // converters once it is in a register)
            float cseg = 0.f;
            if (CENTER && cen) {
              if (!mbar_wait(&c_full[eb], (ecph >> eb) & 1u, abort, p.err, 30)) { ok = false; break; }
              ecph ^= 1u << eb;
              cseg = cring[eb * BM + row];
              __syncwarp();
              if (lane == 0) mbar_arrive(&c_empty[eb]);
              eb = (eb + 1) & 3;
            }
            fph ^= 1u << buf;
            tc_fence_after();
            const uint32_t taddr =
                tmem + d_col0 + (uint32_t)buf * d_stride + ((uint32_t)(q * 32) << 16);
#pragma unroll
            for (int c = 0; c < RBX / 16; ++c) {
              if (c * 16 < RB) {
                // FP32: x_hi k_hi + (x_hi k_lo + x_lo k_hi) [+ centring
                // correction]; BF16: hi + (mid + lo)
                float v[16], t1[16], t2[16];
                tmem_ld16(taddr + c * 16, v);
                tmem_ld16(taddr + RB + c * 16, t1);
                if (!F32 || DUAL) tmem_ld16(taddr + 2 * RB + c * 16, t2);
                tmem_ld_wait();
                if (!F32 || DUAL) {
#pragma unroll
                  for (int jj = 0; jj < 16; ++jj) t1[jj] += t2[jj];
                }
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) v[jj] += t1[jj];
                if (CENTER && cen) {
                  // + c_g colsum_g(H_in)[16 c + jj]
                  const float* kg = ksg + (g0 / p.seg) * RB + c * 16;
#pragma unroll
                  for (int q4 = 0; q4 < 4; ++q4) {
                    const float4 k4 = *reinterpret_cast<const float4*>(kg + 4 * q4);
                    v[4 * q4 + 0] = fmaf(cseg, k4.x, v[4 * q4 + 0]);
                    v[4 * q4 + 1] = fmaf(cseg, k4.y, v[4 * q4 + 1]);
                    v[4 * q4 + 2] = fmaf(cseg, k4.z, v[4 * q4 + 2]);
                    v[4 * q4 + 3] = fmaf(cseg, k4.w, v[4 * q4 + 3]);
                  }
                }
                if (weighted) {
                  float w[16];
                  if (LEFT) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) w[jj] = ws[c * 16 + jj];
                  } else if constexpr (WREG) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) w[jj] = wreg[c * 16 + jj];
                  } else {
                    tcr_w16(p, wrow, c, w);
                  }
                  if (RBX == 32 && half) {  // (pair: c == 0, the upper half)
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj)
                      sum[(16 + jj) % RBX] = fmaf(v[jj], w[jj], sum[(16 + jj) % RBX]);
                  } else {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) sum[c * 16 + jj] = fmaf(v[jj], w[jj], sum[c * 16 + jj]);
                  }
                } else if (RBX == 32 && half) {
#pragma unroll
                  for (int jj = 0; jj < 16; ++jj) sum[(16 + jj) % RBX] += v[jj];
                } else {
#pragma unroll
                  for (int jj = 0; jj < 16; ++jj) sum[c * 16 + jj] += v[jj];
                }
              }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
            buf ^= 1;
          }
        }
        if (!LEFT && p.blockmode && ok) {
          // this warp's 32 rows lie in one c: reduce-scatter them (lane r
          // ends with column r) and write the block's partial row
          const int64_t blk = (tile_m0(it, u) + q * 32) / 32;
#pragma unroll
          for (int h = 0; h < RBX / 32; ++h) {
            if (32 * h < p.R) {
              const float v = warp_reduce_scatter32(sum + 32 * h, lane);
              if (blk < p.nblocks && 32 * h + lane < p.R) p.out[blk * p.R + 32 * h + lane] = v;
            }
          }
        }
      }
      if (!ok) break;
      if (LEFT) {
        const int64_t m = tile_m0(it, 0) + row;
        if (m < p.rows) {
          float* base;
          int64_t stride;
          if (p.out_mode == 1) {
            base = p.out + m * p.R;
            stride = 1;
          } else {
            base = p.out + (p.out_mode == 2 ? (it / p.m_tiles) * p.Mdim * p.R : 0) + m;
            stride = p.Mdim;
          }
#pragma unroll
          for (int r = 0; r < RBX; ++r)
            if (r < p.R) base[r * stride] = sum[r];
        }
      } else if (!p.blockmode && !(pair && half == 0 && it + gridDim.x < p.items)) {
        // sum the item's rows (one output row c; paired: two items, one per
        // half of the columns): reduce-scatter within the warp (lane r ends
        // with column r), then across the four warps
#pragma unroll
        for (int h = 0; h < RBX / 32; ++h) {
          if (32 * h < p.R || pair) {
            const float v = warp_reduce_scatter32(sum + 32 * h, lane);
            red[q * 64 + 32 * h + lane] = v;
          }
        }
        asm volatile("bar.sync 2, 128;" ::: "memory");
        const int tid = threadIdx.x - W_EPI * 32;
        // paired: columns 16.. belong to this item, 0..15 to the one before
        const int col = pair ? (tid & 15) : tid;
        const int64_t iw = (pair && tid < 16 && half) ? it - gridDim.x : it;
        const bool valid = pair ? (tid < 16 ? col < p.R : (tid < 32 && half && col < p.R))
                                : tid < p.R;
        if (valid) {
          const float v = (red[tid] + red[64 + tid]) + (red[128 + tid] + red[192 + tid]);
          const int64_t c = iw / p.nsplit, z = iw % p.nsplit;
          if (p.out_mode == 0) p.out[c + p.Mdim * col] = v;
          else if (p.out_mode == 1) p.out[c * p.R + col] = v;
          else p.out[z * p.Mdim * p.R + c + p.Mdim * col] = v;
        }
        asm volatile("bar.sync 2, 128;" ::: "memory");
      }
    }
  }

  __syncthreads();
  if (warp == W_MMA) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// out[c, r] = sum over the bpc consecutive 32-row blocks of c of part[b, r]
// (fixed order, FP64 accumulation)
__global__ void block_reduce_kernel(const float* __restrict__ part, int64_t bpc, int64_t C, int R,
                                    float* __restrict__ out, int rowmajor) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= C * R) return;
  const int64_t c = e / R;
  const int r = (int)(e - c * R);
  double s = 0.0;
  for (int64_t b = 0; b < bpc; ++b) s += (double)part[(c * bpc + b) * R + r];
  if (rowmajor) out[c * R + r] = (float)s;
  else out[c + C * r] = (float)s;
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

cudaError_t launch_block_reduce(const void* part, int64_t bpc, int64_t C, int R, void* out,
                                bool rowmajor, cudaStream_t st) {
  const int64_t n = C * R;
  block_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      (const float*)part, bpc, C, R, (float*)out, rowmajor ? 1 : 0);
  note_launches(1);
  return cudaGetLastError();
}

// Shared-memory plan: pipeline depth and whether the first Khatri-Rao
// factor (h0_bytes) is staged in shared memory (kept only if at least four
// stages still fit).
struct SmemPlan {
  int stages;
  int h0_smem;
  size_t bytes;
};

SmemPlan plan_smem(bool f32, int RB, int N, int64_t h0_bytes) {
  const size_t budget = 227 * 1024 - 256;
  const size_t per = f32 ? (size_t)F_X_STAGE_BYTES + 2 * RB * 128 : (size_t)A_STAGE_BYTES + N * 128;
  auto bars = [&](int st) -> size_t {
    return (f32 ? (4 * st + 2 * F_A_SLOTS + 5) : (3 * st + 5)) * 8 + 16;
  };
  auto total = [&](int st, size_t h0) { return 1024 + st * per + bars(st) + h0; };
  SmemPlan pl{2, 0, 0};
  for (int st = 6; st >= 4; --st) {
    if (h0_bytes <= 64 * 1024 && total(st, (size_t)h0_bytes) <= budget) {
      pl.stages = st;
      pl.h0_smem = 1;
      pl.bytes = total(st, (size_t)h0_bytes);
      return pl;
    }
  }
  for (int st = 6; st >= 2; --st) {
    if (total(st, 0) <= budget) {
      pl.stages = st;
      pl.bytes = total(st, 0);
      return pl;
    }
  }
  pl.bytes = total(2, 0);
  return pl;
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
int64_t stage_max_k(planc_dtype_t) { return 1LL << 30; }


// ---- resident-operand plan ----------------------------------------------------------
struct TcrPlan {
  bool ok = false;
  int RB = 16, nst = 1, stages = 2;
  int64_t d_in = 0, n_out = 1, jdim = 1, rows = 0, m_tiles = 0, o_span = 1, items = 0;
  int tpc = 1, nsplit = 1;
  int64_t splits = 1;   // partial slices summed afterwards (left: outer splits, right: nsplit)
  bool blockmode = false;
  int64_t nblocks = 0;  // blockmode: 32-row blocks (partial rows in the workspace)
  size_t smem = 0;
};

TcrPlan tcr_plan(planc_dtype_t xdt, bool left, int64_t L, int64_t C, int R, const KrpHost& kh,
                 int sm_count) {
  TcrPlan pl;
  if (xdt != PLANC_BF16 && xdt != PLANC_F32) return pl;
  if (R < 1 || R > 64 || kh.nm < 1 || kh.nm - 1 > TC_MAXM) return pl;
  const bool f32 = xdt == PLANC_F32;
  const int64_t e = f32 ? 4 : 2;
  const int bk = f32 ? F_BK : BK;
  pl.RB = round_up(R, 16);
  pl.d_in = kh.dim[0];
  pl.nst = (int)((pl.d_in + bk - 1) / bk);
  const size_t bstage = (size_t)(f32 ? 2 : 3) * pl.RB * 128;
  const size_t bimg = (size_t)pl.nst * bstage;
  if (bimg > 136 * 1024) return pl;
  if (L >= (1LL << 31) || C >= (1LL << 31)) return pl;
  if (left) {
    if ((L * e) % 16 != 0) return pl;
    pl.n_out = C / pl.d_in;
    pl.rows = L;
    pl.m_tiles = (L + BM - 1) / BM;
    int64_t osplit = 1;
    if (pl.m_tiles < 2 * sm_count)
      osplit = std::min<int64_t>(pl.n_out, (2 * sm_count + pl.m_tiles - 1) / pl.m_tiles);
    pl.o_span = (pl.n_out + osplit - 1) / osplit;
    pl.splits = (pl.n_out + pl.o_span - 1) / pl.o_span;
    pl.items = pl.m_tiles * pl.splits;
  } else {
    if ((pl.d_in * e) % 16 != 0) return pl;
    pl.jdim = L / pl.d_in;
    pl.rows = pl.jdim * C;
    if (pl.rows >= (1LL << 31)) return pl;
    if (pl.jdim % BM != 0) {
      // block mode: every 32-row block lies in one output row c
      if (pl.jdim % 32 != 0) return pl;
      pl.blockmode = true;
      pl.m_tiles = (pl.rows + BM - 1) / BM;
      pl.nblocks = pl.rows / 32;
      const int64_t target = std::max<int64_t>(1, pl.m_tiles / (4LL * sm_count));
      int64_t tpi = 1;
      for (int64_t d = 1; d <= target; ++d)
        if (pl.m_tiles % d == 0) tpi = d;
      pl.tpc = (int)tpi;
      pl.nsplit = 1;
      pl.splits = 1;
      pl.items = pl.m_tiles / tpi;
    } else {
    pl.m_tiles = pl.rows / BM;
    pl.tpc = (int)(pl.jdim / BM);
    // items per output row c: enough items for ~4 per SM, dividing tpc
    int ns = 1;
    while (ns < pl.tpc && C * ns < 4LL * sm_count) ns *= 2;
    while (pl.tpc % ns != 0) --ns;
    pl.nsplit = ns;
    pl.splits = ns;
    pl.items = C * ns;
    }
  }
  const size_t xst = (size_t)BM * bk * e;
  const size_t budget = 227 * 1024 - 256;
  for (int st = 6; st >= 3; --st) {
    // ... barriers, TMEM slot, reduction area, H_in barrier, column sums
    const size_t total = 1024 + st * xst + bimg + (2 * st + 2 * F_A_SLOTS + 5) * 8 + 16 + 1024 +
                         16 + 64 + 16 + 4 * BM * 4 + (size_t)pl.nst * pl.RB * 4;
    if (total <= budget) {
      pl.stages = st;
      pl.smem = total;
      pl.ok = true;
      return pl;
    }
  }
  return pl;
}

}  // namespace

// the driver's tensor-map encoder (NULL if the driver lacks it), for the other
// tensor-core kernels
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn(); }

bool pm_tc_eligible(planc_dtype_t xdt, bool left, int64_t L, int64_t C, int R,
                    const KrpHost& kh) {
  // FP16 X: only the Khatri-Rao GEMM form (an FP16 image; the other
  // tensor-core kernels take BF16 or FP32)
  if (xdt == PLANC_F16) return pm_krp_eligible(xdt, left, L, C, R, kh);
  if (xdt != PLANC_BF16 && xdt != PLANC_F32) return false;
  if (R < 1 || R > 64) return false;
  if (kh.nm < 1 || kh.nm > TC_MAXM) return false;
  // TMA: the row stride of X_(1:S) (L elements) must be a multiple of 16 bytes
  if ((L * (int64_t)dtype_size(xdt)) % 16 != 0 &&
      !tcr_plan(xdt, left, L, C, R, kh, 148).ok)
    return false;
  if (L >= (1LL << 31) || C >= (1LL << 31)) return false;
  if (encode_fn() == nullptr) return false;
  return true;
}

size_t pm_tc_workspace_bytes(planc_dtype_t xdt, bool left, int64_t L, int64_t C, int R,
                             const KrpHost& kh, int sm_count) {
  if (!pm_tc_eligible(xdt, left, L, C, R, kh)) return 0;
  if (pm_krp_eligible(xdt, left, L, C, R, kh))
    return pm_krp_workspace_bytes(xdt, left, L, C, R, sm_count);
  const TcrPlan pl = tcr_plan(xdt, left, L, C, R, kh, sm_count);
  if (pl.ok) {
    if (pl.blockmode) return (size_t)pl.nblocks * R * sizeof(float);
    return pl.splits > 1 ? (size_t)pl.splits * (left ? L : C) * R * sizeof(float) : 0;
  }
  const int64_t Mdim = left ? L : C, Kdim = left ? C : L;
  const int64_t span = item_kspan(Mdim, Kdim, sm_count, stage_bk(xdt), stage_max_k(xdt));
  const int64_t splits = (Kdim + span - 1) / span;
  return splits > 1 ? (size_t)splits * Mdim * R * sizeof(float) : 0;
}

namespace {

// FP32 row centring in the tensor-core partial MTTKRP (PLANC_PM_CENTER=0 turns it off)
bool tcr_center() {
  static const bool on = [] {
    const char* v = getenv("PLANC_PM_CENTER");
    return !(v && v[0] == '0');
  }();
  return on;
}

// stages per accumulator drain (PLANC_PM_SEG overrides; 1..64)
int tcr_seg_stages(bool f32) {
  static const int env = [] {
    const char* v = getenv("PLANC_PM_SEG");
    return v ? atoi(v) : 0;
  }();
  (void)f32;
  return (env >= 1 && env <= 64) ? env : SEG_STAGES;
}

cudaError_t launch_tcr(planc_dtype_t xdt, const void* X, int64_t L, int64_t C, bool left,
                       const KrpHost& kh, int R, void* out, bool out_rowmajor, void* work,
                       size_t work_bytes, int* err_flag, const TcrPlan& pl, cudaStream_t st) {
  const bool f32 = xdt == PLANC_F32;
  TcrParams p{};
  p.L = L;
  p.C = C;
  p.rows = pl.rows;
  p.R = R;
  p.RB = pl.RB;
  p.N = (f32 ? 2 : 3) * pl.RB;
  p.d_in = (int)pl.d_in;
  p.nst = pl.nst;
  p.stages = pl.stages;
  p.n_out = pl.n_out;
  p.o_span = pl.o_span;
  p.m_tiles = pl.m_tiles;
  p.items = pl.items;
  p.tpc = pl.tpc;
  p.nsplit = pl.nsplit;
  p.tpi = pl.tpc / pl.nsplit;
  p.jdim = pl.jdim;
  p.Mdim = left ? L : C;
  // TMEM: A slots of 64 columns + 2 accumulator buffers <= 512 columns:
  // FP32 with two MMA warps (buffers of 3 RB): 4 slots for RB <= 32, 2 for
  // RB <= 64 (left branch); one MMA warp (2 RB): 4 slots; BF16: buffers of 256
  p.aslots = (f32 && pl.RB > 32 && left) ? 2 : 4;
  p.err = err_flag;
  p.Hin = (const float*)kh.H[0];
  p.W.nm = kh.nm - 1;
  p.W.R = R;
  for (int m = 1; m < kh.nm; ++m) {
    p.W.dim[m - 1] = kh.dim[m];
    p.W.H[m - 1] = (const float*)kh.H[m];
  }
  p.blockmode = pl.blockmode ? 1 : 0;
  p.nblocks = pl.nblocks;
  p.seg = tcr_seg_stages(f32);
  p.center = (f32 && !left && pl.RB <= 32 && tcr_center()) ? 1 : 0;
  if (pl.blockmode) {
    if (work_bytes < (size_t)pl.nblocks * R * sizeof(float)) return cudaErrorInvalidValue;
    p.out_mode = 3;
    p.out = (float*)work;
  } else if (pl.splits > 1) {
    if (work_bytes < (size_t)pl.splits * p.Mdim * R * sizeof(float)) return cudaErrorInvalidValue;
    p.out_mode = 2;
    p.out = (float*)work;
  } else {
    p.out_mode = out_rowmajor ? 1 : 0;
    p.out = (float*)out;
  }
  const cuuint64_t e = f32 ? 4 : 2;
  CUtensorMap tmap;
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult cr;
  const CUtensorMapDataType dt = f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (left) {
    // X as L x d_in x n_out
    cuuint64_t gdim[3] = {(cuuint64_t)L, (cuuint64_t)pl.d_in, (cuuint64_t)pl.n_out};
    cuuint64_t gstride[2] = {(cuuint64_t)L * e, (cuuint64_t)L * pl.d_in * e};
    cuuint32_t box[3] = {f32 ? 128u : 64u, (cuuint32_t)(f32 ? F_BK : BK), 1u};
    cr = encode_fn()(&tmap, dt, 3, const_cast<void*>(X), gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE,
                     f32 ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    // X as d_in x rows (rows = (L / d_in) * C)
    cuuint64_t gdim[2] = {(cuuint64_t)pl.d_in, (cuuint64_t)pl.rows};
    cuuint64_t gstride[1] = {(cuuint64_t)pl.d_in * e};
    cuuint32_t box[2] = {(cuuint32_t)(f32 ? F_BK : BK), 128u};
    cr = encode_fn()(&tmap, dt, 2, const_cast<void*>(X), gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const int threads = f32 ? 352 : 192;
  cudaError_t err;
  auto k = pl.RB <= 32
               ? (left ? (f32 ? pm_tcr_kernel<true, true, 32> : pm_tcr_kernel<true, false, 32>)
                       : (f32 ? (p.center ? pm_tcr_kernel<false, true, 32, true>
                                          : pm_tcr_kernel<false, true, 32>)
                              : pm_tcr_kernel<false, false, 32>))
               : (left ? (f32 ? pm_tcr_kernel<true, true, 64> : pm_tcr_kernel<true, false, 64>)
                       : (f32 ? pm_tcr_kernel<false, true, 64> : pm_tcr_kernel<false, false, 64>));
  err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<int64_t>(pl.items, sms);
  err = launch_pdl(k, dim3(grid), dim3(threads), pl.smem, st, tmap, p);
  if (err != cudaSuccess) return err;
  note_launches(1);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  if (pl.blockmode)
    return launch_block_reduce(work, pl.jdim / 32, C, R, out, out_rowmajor, st);
  if (pl.splits == 1) return err;
  return launch_split_reduce(false, work, (int)pl.splits, p.Mdim, R, out, out_rowmajor, st);
}

}  // namespace

cudaError_t launch_pm_tc(planc_dtype_t xdt, const void* X, int64_t L, int64_t C, bool left,
                         const KrpHost& kh, int R, void* out, bool out_rowmajor, void* work,
                         size_t work_bytes, int* err_flag, int sm_count, cudaStream_t st) {
  if (!pm_tc_eligible(xdt, left, L, C, R, kh)) return cudaErrorNotSupported;
  if (pm_krp_eligible(xdt, left, L, C, R, kh) &&
      work_bytes >= pm_krp_workspace_bytes(xdt, left, L, C, R, sm_count))
    return launch_pm_krp(xdt, X, L, C, left, kh, R, out, out_rowmajor, work, work_bytes,
                         err_flag, sm_count, st);
  if (xdt == PLANC_F16) return cudaErrorNotSupported;
  {
    const TcrPlan pl = tcr_plan(xdt, left, L, C, R, kh, sm_count);
    if (pl.ok && getenv("PLANC_TC_STREAMED_KRP") == nullptr)
      return launch_tcr(xdt, X, L, C, left, kh, R, out, out_rowmajor, work, work_bytes, err_flag,
                        pl, st);
  }
  if ((L * (int64_t)dtype_size(xdt)) % 16 != 0) return cudaErrorNotSupported;
  if (((uintptr_t)X & 15) != 0) return cudaErrorNotSupported;
  TcParams p{};
  p.L = L;
  p.C = C;
  p.R = R;
  const bool f32 = xdt == PLANC_F32;
  p.RB = round_up(R, 16);
  p.N = f32 ? 2 * p.RB : 3 * p.RB;
  const SmemPlan sp = plan_smem(f32, p.RB, p.N, kh.dim[0] * (int64_t)R * 4);
  p.stages = sp.stages;
  p.h0_smem = sp.h0_smem;
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

  const size_t smem = sp.bytes;
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
