// Device code of the batched solve of many small 3-way instances (Alg. 1 with
// the dimension tree of Alg. 3, N = 3, S = 2), shared by the per-phase
// kernels (kern_batch.cu: every launch covers all instances) and the single
// persistent launch (kern_mode.cu: one thread-block cluster works through
// whole instances):
//   T^{1:2} = X_(1:2) H^(3)                 pm_left_run     (first X pass)
//   M^(1)   = T^{1:2} x_2 H^(2)             contract_rest_item
//   M^(2)   = T^{1:2} x_1 H^(1) (updated)    contract_first_item
//   M^(3)   = X_(1:2)^T (H^(2) . H^(1))      pm_right_run    (second X pass)
// Factors, T and M are written inside the persistent launch by other CTAs,
// so every read of them here goes through L2 (__ldcg: never the read-only
// path, whose cache is not kept coherent with writes made during a launch).
#pragma once

#include <cuda_bf16.h>

#include "internal.h"

namespace planc {
namespace bdev {

constexpr int BR = 32;  // widest rank class of the batched kernels (R <= 32)

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
  return reinterpret_cast<const float*>(b.X)[e];
}

// a row-major nrow x R factor into shared memory with stride BRC (padding
// columns zero)
__device__ __forceinline__ void stage_factor(float* dst, const float* H, int nrow, int R,
                                             int BRC) {
  for (int e = threadIdx.x; e < nrow * BRC; e += blockDim.x) {
    const int i = e / BRC, r = e - (e / BRC) * BRC;
    dst[e] = r < R ? __ldcg(H + (int64_t)i * R + r) : 0.f;
  }
}

// ---- staged X: asynchronous 16-byte copies into a ring of shared-memory stages -----
// The two partial MTTKRPs stream X through NSTG stages of SW words each: while
// one stage is consumed, the copies of the next NSTG - 1 chunks are in flight
// (the kernels are otherwise bound by the latency of their X loads).  A
// contiguous byte range [byte0, byte1) of X is copied as the 16-byte-aligned
// range that starts at or before it (X itself starts on 16 bytes), so any
// dims and either storage type work: the range's first element sits `shift`
// elements into the copy, and bytes at or past byte1 are zero-filled without
// being read.
constexpr int SW = 4096;  // 32-bit words per stage
constexpr int NSTG = 2;   // stages (more gained nothing: the kernels are latency-bound in their FMA loop)

__device__ __forceinline__ void cp_async16(uint32_t sdst, const void* gsrc, uint32_t nbytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sdst), "l"(gsrc), "r"(nbytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// bytes [byte0 & ~15, byte1) of X into shared memory at sdst (16-byte aligned)
__device__ __forceinline__ void stage_range(uint32_t sdst, const char* xb, int64_t byte0,
                                            int64_t byte1, int tid, int nt) {
  const int64_t a0 = byte0 & ~(int64_t)15;
  const char* src = xb + a0;
  const int lim = (int)(byte1 - a0);  // at most one stage
  for (int off = tid * 16; off < lim; off += nt * 16) {
    const int left = lim - off;
    cp_async16(sdst + (uint32_t)off, src + off, left >= 16 ? 16u : (uint32_t)left);
  }
}

// shared-memory bytes of the two partial MTTKRPs: the X ring, a staged factor
// of at most hmax rows, and (right branch, h1max > 0) the staged H1 of at
// most h1max rows, transposed (stage_factor_t)
__host__ __device__ constexpr size_t pm_smem_bytes(int hmax, int h1max = 0) {
  return (size_t)NSTG * SW * 4 + ((size_t)hmax + (h1max > 0 ? (size_t)h1max + 1 : 0)) * BR * 4;
}

// a row-major nrow x R factor into shared memory transposed: column r at
// dst + r * ld, ld = nrow rounded up to even (rows nrow .. ld - 1 and columns
// R .. BRC - 1 zero), so that lanes reading consecutive row pairs of one
// column use distinct banks with 8-byte loads
__device__ __forceinline__ void stage_factor_t(float* dst, const float* H, int nrow, int R,
                                               int BRC) {
  const int ld = nrow + (nrow & 1);
  for (int e = threadIdx.x; e < ld * BRC; e += blockDim.x) {
    const int r = e / ld, i = e - (e / ld) * ld;
    dst[e] = (r < R && i < nrow) ? __ldcg(H + (int64_t)i * R + r) : 0.f;
  }
}

// The left branch's chunk: nk columns k0 .. k0 + nk - 1 of the item's row
// block, column kk the nb bytes from element l0 + L (k0 + kk), each copied as
// its 16-byte-aligned range into slot kk (SB bytes).  The CTA's threads take
// the chunk's 16-byte pieces in turn (piece idx: column idx / CPC, offset
// idx % CPC), so that no thread loops over columns it copies nothing of.
template <int ES, int RB, int NT>
__device__ __forceinline__ void left_copies(uint32_t dst, const char* xb, int64_t l0, int64_t L,
                                            int k0, int nk, int nb, int tid) {
  constexpr int SB = RB * ES + 16;
  constexpr int CPC = SB / 16;  // pieces per column (RB * ES is a multiple of 16)
  const int total = nk * CPC;
  for (int idx = tid; idx < total; idx += NT) {
    const int kk = idx / CPC, off = (idx - kk * CPC) * 16;
    const int64_t byte0 = (int64_t)ES * (l0 + L * (k0 + kk));
    const int64_t a0 = byte0 & ~(int64_t)15;
    const int lim = (int)(byte0 + nb - a0);
    if (off < lim)
      cp_async16(dst + (uint32_t)(kk * SB + off), xb + a0 + off,
                 lim - off >= 16 ? 16u : (uint32_t)(lim - off));
  }
}

// ---- T^{1:2}[l, r] = sum_k X[l, k] H3[k, r]: items (b, block of 2 NT rows l) ------------
// A chunk is KC columns k of the item's row block, each column a run of
// 2 NT elements of X at stride L, copied into a slot of SB bytes.  Each thread
// owns two adjacent rows and keeps both rows' R sums in registers across the
// item's chunks; every read of H3's row k (staged in shared memory with stride
// BRC, the rank class, as broadcast 16-byte loads) feeds both.
template <int NT>
struct LeftGeom {
  static constexpr int RB = 2 * NT;
  __device__ __forceinline__ static int sb(int es) { return RB * es + 16; }
  __device__ __forceinline__ static int kc(int es) { return min(32, 4 * SW / sb(es)); }
};

// nk columns of a staged chunk into the thread's two rows: column kk's first
// element sits sh_kk elements into its copy, sh_0 = sh0 and sh_{kk+1} =
// (sh_kk + Lm) mod (16 / ES) with Lm = L mod (16 / ES) (consecutive columns
// start L elements apart); H3's row k0 + kk is read as broadcast 16-byte loads
template <int NT, int BRC, bool BF16>
__device__ __forceinline__ void left_chunk(const unsigned char* stage, const float* hs, int sh0,
                                           int Lm, int k0, int nk, float* a0, float* a1) {
  constexpr int ES = BF16 ? 2 : 4;
  constexpr int SB = LeftGeom<NT>::RB * ES + 16;
  constexpr int MASK = 16 / ES - 1;
  const unsigned char* xs = stage + 2 * (int)threadIdx.x * ES;
  const float4* h = reinterpret_cast<const float4*>(hs + k0 * BRC);
  int sh = sh0;
#pragma unroll 4
  for (int kk = 0; kk < nk; ++kk, xs += SB, h += BRC / 4) {
    float x0, x1;
    if (BF16) {
      const __nv_bfloat16* p = reinterpret_cast<const __nv_bfloat16*>(xs) + sh;
      x0 = __bfloat162float(p[0]);
      x1 = __bfloat162float(p[1]);
    } else {
      const float* p = reinterpret_cast<const float*>(xs) + sh;
      x0 = p[0];
      x1 = p[1];
    }
    sh = (sh + Lm) & MASK;
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

// The CTA's contiguous run of left items i0 .. i1 - 1; item(i) gives
// (instance, row block).  bsm: the X ring followed by the staged H3 (16-byte
// aligned, pm_smem_bytes).  Every thread of the CTA (NT) takes part.
template <int NT, typename ItemFn>
__device__ __forceinline__ void pm_left_run(const BatchInst* __restrict__ tab, ItemFn item, int i0,
                                            int i1, int sched, unsigned char* bsm) {
  using G = LeftGeom<NT>;
  float* hs = reinterpret_cast<float*>(bsm + (size_t)NSTG * SW * 4);
  const uint32_t stg = (uint32_t)__cvta_generic_to_shared(bsm);
  const int tid = threadIdx.x;

  int pit = i0, pk = 0;  // next chunk to copy: item, first column
  auto issue = [&](int slot) {
    if (pit < i1) {
      const int2 itm = item(pit);
      const BatchInst& b = tab[itm.x];
      const int64_t L = b.I[0] * b.I[1];
      const int C = (int)b.I[2];
      const int es = b.xbf16 ? 2 : 4;
      const int64_t l0 = (int64_t)itm.y * G::RB;
      const int64_t nb = (int64_t)es * min((int64_t)G::RB, L - l0);
      const int nk = min(G::kc(es), C - pk);
      const char* xb = reinterpret_cast<const char*>(b.X);
      const uint32_t dst = stg + (uint32_t)(slot * SW * 4);
      if (es == 4) left_copies<4, G::RB, NT>(dst, xb, l0, L, pk, nk, (int)nb, tid);
      else left_copies<2, G::RB, NT>(dst, xb, l0, L, pk, nk, (int)nb, tid);
      pk += nk;
      if (pk >= C) {
        ++pit;
        pk = 0;
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int s = 0; s < NSTG - 1; ++s) issue(s);

  float a0[BR], a1[BR];
  int cur = -1, ck = 0, cls = 32;
  for (int it = i0, k = 0; it < i1; ++k) {
    cp_async_wait<NSTG - 2>();
    __syncthreads();  // chunk k visible; chunk k - 1 consumed by every thread
    issue((k + NSTG - 1) % NSTG);
    const int2 itm = item(it);
    const int bi = itm.x;
    const BatchInst& b = tab[bi];
    const int64_t L = b.I[0] * b.I[1];
    const int C = (int)b.I[2], R = b.R;
    const bool bf = b.xbf16 != 0;
    const int64_t l0 = (int64_t)itm.y * G::RB;
    const int nk = min(G::kc(bf ? 2 : 4), C - ck);
    if (ck == 0) {
      if (bi != cur) {  // H3 of a new instance (the old one is no longer read)
        cls = rank_class(R, sched);
        stage_factor(hs, b.H[2], C, R, cls);
        __syncthreads();
        cur = bi;
      }
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        a0[r] = 0.f;
        a1[r] = 0.f;
      }
    }
    const unsigned char* stage = bsm + (size_t)(k % NSTG) * SW * 4;
    // the chunk's first element within its copy (X starts on 16 bytes)
    const int mask = bf ? 7 : 3;
    const int sh0 = (int)((l0 + L * ck) & mask), Lm = (int)(L & mask);
    if (cls == 8) {
      if (bf) left_chunk<NT, 8, true>(stage, hs, sh0, Lm, ck, nk, a0, a1);
      else left_chunk<NT, 8, false>(stage, hs, sh0, Lm, ck, nk, a0, a1);
    } else if (cls == 16) {
      if (bf) left_chunk<NT, 16, true>(stage, hs, sh0, Lm, ck, nk, a0, a1);
      else left_chunk<NT, 16, false>(stage, hs, sh0, Lm, ck, nk, a0, a1);
    } else {
      if (bf) left_chunk<NT, 32, true>(stage, hs, sh0, Lm, ck, nk, a0, a1);
      else left_chunk<NT, 32, false>(stage, hs, sh0, Lm, ck, nk, a0, a1);
    }
    ck += nk;
    if (ck >= C) {  // the item's rows are complete
      const int64_t l = l0 + 2 * tid;
      const bool live0 = l < L, live1 = l + 1 < L;
      float* T = b.T;
#pragma unroll
      for (int r = 0; r < BR; ++r)
        if (r < R) {
          if (live0) T[l + L * r] = a0[r];
          if (live1) T[l + 1 + L * r] = a1[r];
        }
      ++it;
      ck = 0;
    }
  }
  cp_async_wait<0>();
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
// A chunk is KC columns i2 of the slab X[:, :, c] (one contiguous range).
// Units (pair of rows i1, i1 + 1; group g) cover the slab, the groups
// splitting each chunk's columns so that short first modes still occupy every
// thread.  When the units fit the CTA (I1 <= 2 NT) each thread keeps its
// unit's inner sums over i2 (H2 staged in shared memory, stride BRC) in
// registers across the item's chunks and weights them by H1[i1, r] once, at
// the item's end; longer first modes take one row per unit, looped over the
// CTA in every chunk, and weight per chunk.  The CTA then reduces the
// weighted sums (warp reduce-scatter, then shared memory).
__device__ __forceinline__ int right_kc(int I1, int es) {
  return max(1, (4 * SW - 16) / (es * I1));
}

template <bool BF16>
__device__ __forceinline__ float ldstage(const unsigned char* stage, int q) {
  if (BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(stage)[q]);
  return reinterpret_cast<const float*>(stage)[q];
}

// inner sums of the unit (rows i, i + 1 when live1; columns jj = g, g + ng,
// ... below nj of the chunk whose first column is j0) into in0, in1.  Row
// i + 1 is read even when it is not live (it stays inside the stage) and
// weighted by zero.
template <int BRC, bool BF16>
__device__ __forceinline__ void right_sums(const unsigned char* stage, int sh, const float* hs,
                                           int I1, int i, bool live1, int g, int ng, int j0,
                                           int nj, float* in0, float* in1) {
  int q = sh + g * I1 + i;
  const int qs = ng * I1;
  const float4* h = reinterpret_cast<const float4*>(hs + (j0 + g) * BRC);
  const int hs4 = ng * (BRC / 4);
#pragma unroll 4
  for (int jj = g; jj < nj; jj += ng, q += qs, h += hs4) {
    const float x0 = ldstage<BF16>(stage, q);
    const float v1 = ldstage<BF16>(stage, q + 1);
    const float x1 = live1 ? v1 : 0.f;
#pragma unroll
    for (int qq = 0; qq < BRC / 4; ++qq) {
      const float4 hv = h[qq];
      in0[4 * qq + 0] = fmaf(x0, hv.x, in0[4 * qq + 0]);
      in0[4 * qq + 1] = fmaf(x0, hv.y, in0[4 * qq + 1]);
      in0[4 * qq + 2] = fmaf(x0, hv.z, in0[4 * qq + 2]);
      in0[4 * qq + 3] = fmaf(x0, hv.w, in0[4 * qq + 3]);
      in1[4 * qq + 0] = fmaf(x1, hv.x, in1[4 * qq + 0]);
      in1[4 * qq + 1] = fmaf(x1, hv.y, in1[4 * qq + 1]);
      in1[4 * qq + 2] = fmaf(x1, hv.z, in1[4 * qq + 2]);
      in1[4 * qq + 3] = fmaf(x1, hv.w, in1[4 * qq + 3]);
    }
  }
}

// one row per unit (first modes longer than 2 NT): every row of the chunk,
// weighted by H1[i, r] into acc
template <int NT, int BRC, bool BF16>
__device__ __forceinline__ void right_rows(const unsigned char* stage, int sh, const float* hs,
                                           const float* H1, const float* h1s, int I1, int R,
                                           int j0, int nj, float* acc) {
  for (int i = threadIdx.x; i < I1; i += NT) {
    float t[BRC];
#pragma unroll
    for (int r = 0; r < BRC; ++r) t[r] = 0.f;
#pragma unroll 2
    for (int jj = 0; jj < nj; ++jj) {
      const float x = ldstage<BF16>(stage, sh + jj * I1 + i);
      const float4* h = reinterpret_cast<const float4*>(hs + (j0 + jj) * BRC);
#pragma unroll
      for (int qq = 0; qq < BRC / 4; ++qq) {
        const float4 hv = h[qq];
        t[4 * qq + 0] = fmaf(x, hv.x, t[4 * qq + 0]);
        t[4 * qq + 1] = fmaf(x, hv.y, t[4 * qq + 1]);
        t[4 * qq + 2] = fmaf(x, hv.z, t[4 * qq + 2]);
        t[4 * qq + 3] = fmaf(x, hv.w, t[4 * qq + 3]);
      }
    }
    if (h1s) {  // H1 staged in shared memory, transposed (column stride I1 rounded to even)
      const int ld = I1 + (I1 & 1);
#pragma unroll
      for (int r = 0; r < BRC; ++r) acc[r] = fmaf(t[r], h1s[r * ld + i], acc[r]);
    } else {
      const float* h1 = H1 + (int64_t)i * R;
#pragma unroll
      for (int r = 0; r < BRC; ++r)
        if (r < R) acc[r] = fmaf(t[r], __ldcg(h1 + r), acc[r]);
    }
  }
}

// one chunk of the item: the unit's sums (persistent units) or the rows'
// weighted sums (long first modes)
template <int NT, int BRC, bool BF16>
__device__ __forceinline__ void right_chunk(const unsigned char* stage, int sh, const float* hs,
                                            const float* H1, const float* h1s, int I1, int R,
                                            int j0, int nj, float* in0, float* in1) {
  const int P = (I1 + 1) >> 1;
  if (P <= NT) {
    const int ng = NT / P;
    const int u = threadIdx.x;
    if (u < P * ng) {
      const int i = 2 * (u % P);
      right_sums<BRC, BF16>(stage, sh, hs, I1, i, i + 1 < I1, u / P, ng, j0, nj, in0, in1);
    }
  } else {
    right_rows<NT, BRC, BF16>(stage, sh, hs, H1, h1s, I1, R, j0, nj, in0);
  }
}

// The CTA's contiguous run of right items i0 .. i1 - 1; item(i) gives
// (instance, slab c).  bsm: the X ring, the staged H2 (room for hcap rows)
// and, for instances with I1 <= h1cap, the staged H1 (pm_smem_bytes(hcap,
// h1cap)); H1 is read from global memory otherwise.
template <int NT, typename ItemFn>
__device__ __forceinline__ void pm_right_run(const BatchInst* __restrict__ tab, ItemFn item,
                                             int i0, int i1, int sched, unsigned char* bsm,
                                             int hcap, int h1cap) {
  __shared__ float red[NT / 32][BR];
  float* hs = reinterpret_cast<float*>(bsm + (size_t)NSTG * SW * 4);
  float* hs1 = hs + (size_t)hcap * BR;
  const float* h1s = nullptr;
  const uint32_t stg = (uint32_t)__cvta_generic_to_shared(bsm);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  int pit = i0, pj = 0;  // next chunk to copy: item, first column i2
  auto issue = [&](int slot) {
    if (pit < i1) {
      const int2 itm = item(pit);
      const BatchInst& b = tab[itm.x];
      const int I1 = (int)b.I[0], I2 = (int)b.I[1];
      const int64_t L = (int64_t)I1 * I2;
      const int es = b.xbf16 ? 2 : 4;
      const int nj = min(right_kc(I1, es), I2 - pj);
      const int64_t byte0 = (int64_t)es * (L * itm.y + (int64_t)I1 * pj);
      stage_range(stg + (uint32_t)(slot * SW * 4), reinterpret_cast<const char*>(b.X), byte0,
                  byte0 + (int64_t)es * I1 * nj, tid, NT);
      pj += nj;
      if (pj >= I2) {
        ++pit;
        pj = 0;
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int s = 0; s < NSTG - 1; ++s) issue(s);

  // persistent units: the unit's row sums; long first modes: the thread's
  // weighted sums (in0) only
  float in0[BR], in1[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) {
    in0[r] = 0.f;
    in1[r] = 0.f;
  }
  int cur = -1, cj = 0, cls = 32;
  for (int it = i0, k = 0; it < i1; ++k) {
    cp_async_wait<NSTG - 2>();
    __syncthreads();  // chunk k visible; chunk k - 1 consumed by every thread
    issue((k + NSTG - 1) % NSTG);
    const int2 itm = item(it);
    const int bi = itm.x;
    const BatchInst& b = tab[bi];
    const int I1 = (int)b.I[0], I2 = (int)b.I[1], R = b.R;
    const int64_t L = (int64_t)I1 * I2;
    const bool bf = b.xbf16 != 0;
    const int es = bf ? 2 : 4;
    const int nj = min(right_kc(I1, es), I2 - cj);
    if (cj == 0 && bi != cur) {  // H2 (and H1) of a new instance (the old ones are no longer read)
      cls = rank_class(R, sched);
      stage_factor(hs, b.H[1], I2, R, cls);
      h1s = I1 <= h1cap ? hs1 : nullptr;
      if (h1s) stage_factor_t(hs1, b.H[0], I1, R, cls);
      __syncthreads();
      cur = bi;
    }
    // the chunk's first element within its copy (X starts on 16 bytes)
    const int sh = (int)((L * itm.y + (int64_t)I1 * cj) & (16 / es - 1));
    const unsigned char* stage = bsm + (size_t)(k % NSTG) * SW * 4;
    if (cls == 8) {
      if (bf) right_chunk<NT, 8, true>(stage, sh, hs, b.H[0], h1s, I1, R, cj, nj, in0, in1);
      else right_chunk<NT, 8, false>(stage, sh, hs, b.H[0], h1s, I1, R, cj, nj, in0, in1);
    } else if (cls == 16) {
      if (bf) right_chunk<NT, 16, true>(stage, sh, hs, b.H[0], h1s, I1, R, cj, nj, in0, in1);
      else right_chunk<NT, 16, false>(stage, sh, hs, b.H[0], h1s, I1, R, cj, nj, in0, in1);
    } else {
      if (bf) right_chunk<NT, 32, true>(stage, sh, hs, b.H[0], h1s, I1, R, cj, nj, in0, in1);
      else right_chunk<NT, 32, false>(stage, sh, hs, b.H[0], h1s, I1, R, cj, nj, in0, in1);
    }
    cj += nj;
    if (cj >= I2) {  // the item's sums are complete
      const int P = (I1 + 1) >> 1;
      if (P <= NT) {  // weight the unit's sums by H1 (once per item)
        const int ng = NT / P;
        const int i = 2 * (tid % P);
        const bool live = tid < P * ng, live1 = live && i + 1 < I1;
        if (h1s) {  // staged rows i, i + 1 of every column (transposed; padding is zero)
          const int ld = I1 + (I1 & 1);
#pragma unroll
          for (int r = 0; r < BR; ++r) {
            float v = 0.f;
            if (live && r < cls) {
              const float2 w = *reinterpret_cast<const float2*>(h1s + r * ld + i);
              v = in0[r] * w.x;
              if (live1) v = fmaf(in1[r], w.y, v);
            }
            in0[r] = v;
          }
        } else {
          const float* h1 = b.H[0] + (int64_t)i * R;
#pragma unroll
          for (int r = 0; r < BR; ++r) {
            float v = 0.f;
            if (live && r < R) v = in0[r] * __ldcg(h1 + r);
            if (live1 && r < R) v = fmaf(in1[r], __ldcg(h1 + R + r), v);
            in0[r] = v;
          }
        }
      }
      const float v = reduce_scatter32(in0, lane);
      red[warp][lane] = v;
      __syncthreads();
      if (tid < R) {
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) sum += red[w][tid];
        b.M[(int64_t)itm.y * R + tid] = sum;
      }
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        in0[r] = 0.f;
        in1[r] = 0.f;
      }
      ++it;
      cj = 0;
    }
  }
  cp_async_wait<0>();
  __syncthreads();  // red and the ring are free for whatever the CTA runs next
}

// ---- M^(1)[i1, r] = sum_{i2} T[i1 + I1 i2, r] H2[i2, r] for one (b, r) ----------------
// Units (i1, group of i2): groups split the i2 range when I1 is short; the
// column H2[:, r] is staged in shared memory (hcol, >= I2 floats; part, NT
// floats); eight loads in flight per unit.  Every thread of the CTA (NT)
// takes part; the item starts and ends with a CTA barrier.
template <int NT>
__device__ __forceinline__ void contract_rest_item(const BatchInst& b, int r, float* hcol,
                                                   float* part) {
  const int tid = threadIdx.x;
  const int I1 = (int)b.I[0], I2 = (int)b.I[1], R = b.R;
  const float* Tr = b.T + (int64_t)I1 * I2 * r;
  __syncthreads();  // the previous item's reads of hcol and part are done
  for (int j = tid; j < I2; j += NT) hcol[j] = __ldcg(b.H[1] + (int64_t)j * R + r);
  __syncthreads();
  const int ng = I1 >= NT ? 1 : NT / I1;
  const int js = (I2 + ng - 1) / ng;
  for (int u = tid; u < I1 * ng; u += NT) {
    const int i = u % I1, g = u / I1;
    const int ja = g * js, jb = min(I2, ja + js);
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    int j = ja;
    for (; j + 8 <= jb; j += 8) {
      float x[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) x[v] = __ldcg(Tr + i + (int64_t)I1 * (j + v));
#pragma unroll
      for (int v = 0; v < 8; ++v) a[v & 3] = fmaf(x[v], hcol[j + v], a[v & 3]);
    }
    for (; j < jb; ++j) a[0] = fmaf(__ldcg(Tr + i + (int64_t)I1 * j), hcol[j], a[0]);
    const float s = (a[0] + a[1]) + (a[2] + a[3]);
    if (ng == 1) b.M[(int64_t)i * R + r] = s;
    else part[u] = s;
  }
  if (ng > 1) {
    __syncthreads();
    for (int i = tid; i < I1; i += NT) {
      float s = 0.f;
      for (int g = 0; g < ng; ++g) s += part[i + I1 * g];
      b.M[(int64_t)i * R + r] = s;
    }
  }
  __syncthreads();
}

// ---- M^(2)[i2, r] = sum_{i1} T[i1 + I1 i2, r] H1[i1, r] for one (b, r) ----------------
// a warp per four i2 (lanes across i1, four columns' loads in flight
// together); the column H1[:, r] is staged in shared memory (hcol, >= I1
// floats); the item starts and ends with a CTA barrier
template <int NT>
__device__ __forceinline__ void contract_first_item(const BatchInst& b, int r, float* hcol) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  const int I1 = (int)b.I[0], I2 = (int)b.I[1], R = b.R;
  const float* Tr = b.T + (int64_t)I1 * I2 * r;
  __syncthreads();  // the previous item's reads of hcol are done
  for (int i = tid; i < I1; i += NT) hcol[i] = __ldcg(b.H[0] + (int64_t)i * R + r);
  __syncthreads();
  for (int j0 = 4 * warp; j0 < I2; j0 += 4 * NW) {
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i = lane; i < I1; i += 32) {
      const float h = hcol[i];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (j0 + q < I2) a[q] = fmaf(__ldcg(Tr + i + (int64_t)I1 * (j0 + q)), h, a[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] = warp_sum(a[q]);
    if (lane < 4 && j0 + lane < I2) {
      const float v = lane == 0 ? a[0] : lane == 1 ? a[1] : lane == 2 ? a[2] : a[3];
      b.M[(int64_t)(j0 + lane) * R + r] = v;
    }
  }
  __syncthreads();
}

// ---- G^(n) = H^(n)T H^(n) of the initial factors, entry (r, s) ------------------------
// FP32 over blocks of 32 rows, FP64 across blocks
__device__ __forceinline__ void initial_gram_entry(const BatchInst& b, int n, int pr) {
  const int R = b.R, rows = (int)b.I[n];
  const int r = pr / R, s = pr - (pr / R) * R;
  const float* H = b.H[n];
  double g = 0.0;
  for (int i0 = 0; i0 < rows; i0 += 32) {
    float a = 0.f;
    for (int i = i0; i < min(rows, i0 + 32); ++i)
      a = fmaf(__ldcg(H + (int64_t)i * R + r), __ldcg(H + (int64_t)i * R + s), a);
    g += (double)a;
  }
  b.G[(size_t)n * R * R + pr] = g;
  b.Gf[(size_t)n * R * R + pr] = (float)g;
}

}  // namespace bdev
}  // namespace planc
