// Multi-TTV kernels of the dimension tree (Sec. 4.2.2, Alg. 3).
//
// A node tensor T^{a:b} is I_a x ... x I_b x R with R slowest, viewed here
// as T[p + P1 q + P1 Q r] with P1 = I_a (its first mode) and Q the product
// of its other modes.  Each multi-TTV is R independent matrix-vector
// products on the contiguous blocks T[r] (the paper's R GEMV calls); both
// kernels below do all R at once and are HBM-bandwidth bound.
//
//   contract_first: T^{a+1:b}(:, r) = T_(1)^{a:b}[r]^T H^(a)(:, r)
//                   (internal node, or the leaf M^(b) when a + 1 == b)
//   contract_rest : M^(a)(:, r)     = T_(1)^{a:b}[r] K^{a+1:b}(:, r)
//                   with K^{a+1:b} the partial Khatri-Rao product of the
//                   node's other factors, generated in shared memory.
#include <algorithm>

#include "internal.h"

namespace planc {

namespace {

constexpr int CF_THREADS = 256;
constexpr int CF_Q_PER_GROUP = 4;
constexpr int CF_SMEM_H = 4096;  // h column staged in shared memory up to this length

template <typename TA>
__global__ void __launch_bounds__(CF_THREADS)
contract_first_kernel(const TA* __restrict__ T, int64_t P1, int64_t Q, int R,
                      const TA* __restrict__ h, TA* __restrict__ out, int rowmajor,
                      int gw /* lanes per dot product, power of two <= 32 */) {
  __shared__ TA sh[CF_SMEM_H];
  const int r = blockIdx.y;
  const bool staged = P1 <= CF_SMEM_H;
  if (staged) {
    for (int64_t p = threadIdx.x; p < P1; p += CF_THREADS) sh[p] = h[p * R + r];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int gl = lane & (gw - 1);                       // lane inside the group
  const int group = threadIdx.x / gw;                   // group index in the CTA
  const int groups = CF_THREADS / gw;
  const int64_t qbase = (int64_t)blockIdx.x * groups * CF_Q_PER_GROUP;
  const TA* Tr = T + P1 * Q * (int64_t)r;
  for (int it = 0; it < CF_Q_PER_GROUP; ++it) {
    int64_t q = qbase + (int64_t)it * groups + group;
    TA s = TA(0);
    if (q < Q) {
      const TA* col = Tr + P1 * q;
      if (staged) {
        for (int64_t p = gl; p < P1; p += gw) s = fma(col[p], sh[p], s);
      } else {
        for (int64_t p = gl; p < P1; p += gw) s = fma(col[p], h[p * R + r], s);
      }
    }
    s = group_sum(s, gw);
    if (q < Q && gl == 0) {
      if (rowmajor) out[q * R + r] = s; else out[q + Q * (int64_t)r] = s;
    }
  }
}

constexpr int CR_THREADS = 256;
constexpr int CR_QCH = 1024;

template <typename TA>
__global__ void __launch_bounds__(CR_THREADS)
contract_rest_kernel(const TA* __restrict__ T, int64_t P1, int64_t Q, int R, Krp<TA> K,
                     int64_t qchunk, TA* __restrict__ out, int to_part) {
  __shared__ TA Ks[CR_QCH];
  __shared__ TA red[CR_THREADS];
  const int r = blockIdx.y;
  const int z = blockIdx.z;
  const int tid = threadIdx.x;
  const int64_t P1b = P1 >= CR_THREADS ? CR_THREADS : P1;
  const int nql = (int)(CR_THREADS / P1b);
  const bool active = tid < P1b * nql;
  const int pl = (int)(tid % P1b);
  const int ql = (int)(tid / P1b);
  const int64_t p = (int64_t)blockIdx.x * P1b + pl;
  const int64_t qbeg = (int64_t)z * qchunk;
  const int64_t qend = min(Q, qbeg + qchunk);
  const TA* Tr = T + P1 * Q * (int64_t)r;
  TA acc = TA(0), acc2 = TA(0);
  int cnt = 0;
  for (int64_t qc = qbeg; qc < qend; qc += CR_QCH) {
    const int64_t nq = min((int64_t)CR_QCH, qend - qc);
    __syncthreads();
    for (int64_t e = tid; e < nq; e += CR_THREADS) Ks[e] = krp_at(K, qc + e, r);
    __syncthreads();
    if (active && p < P1) {
      for (int64_t e = ql; e < nq; e += nql) {
        acc = fma(Tr[p + P1 * (qc + e)], Ks[e], acc);
        if (++cnt == 128) { acc2 += acc; acc = TA(0); cnt = 0; }
      }
    }
  }
  red[tid] = acc2 + acc;
  __syncthreads();
  if (active && ql == 0 && p < P1) {
    TA s = TA(0);
    for (int j = 0; j < nql; ++j) s += red[pl + P1b * j];
    if (to_part) out[(int64_t)z * P1 * R + p + P1 * (int64_t)r] = s;
    else out[p * R + r] = s;
  }
}


// ---- vectorised variants (FP32, P1 % 4 == 0, 16-byte aligned T) ---------------------
// contract_rest: each thread owns four consecutive p and streams float4 loads
// of T over its q-range, sixteen in flight; the Khatri-Rao values of the range
// are staged in shared memory.
constexpr int CR4_THREADS = 128;
constexpr int CR4_P = CR4_THREADS * 4;
// float4 loads a thread keeps in flight: the grid is small (P1 / 512 x R x
// qsplit CTAs), so each thread must cover more of the HBM latency
constexpr int CR4_INFLIGHT = 16;

__global__ void __launch_bounds__(CR4_THREADS)
contract_rest_v4_kernel(const float* __restrict__ T, int64_t P1, int64_t Q, int R, Krp<float> K,
                        int64_t qchunk, float* __restrict__ out, int to_part) {
  pdl_wait();
  pdl_trigger();
  __shared__ float Ks[CR_QCH];
  const int r = blockIdx.y;
  const int z = blockIdx.z;
  const int64_t p = (int64_t)blockIdx.x * CR4_P + 4 * threadIdx.x;
  const int64_t qbeg = (int64_t)z * qchunk;
  const int64_t qend = min(Q, qbeg + qchunk);
  const float* Tr = T + P1 * Q * (int64_t)r;
  const bool live = p < P1;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t qc = qbeg; qc < qend; qc += CR_QCH) {
    const int nq = (int)min((int64_t)CR_QCH, qend - qc);
    __syncthreads();
    for (int e = threadIdx.x; e < nq; e += CR4_THREADS) Ks[e] = krp_at(K, qc + e, r);
    __syncthreads();
    if (live) {
      const float4* base = reinterpret_cast<const float4*>(Tr + p + P1 * qc);
      const int64_t step = P1 / 4;
      int e = 0;
      for (; e + CR4_INFLIGHT <= nq; e += CR4_INFLIGHT) {
        float4 v[CR4_INFLIGHT];
#pragma unroll
        for (int u = 0; u < CR4_INFLIGHT; ++u) v[u] = __ldg(base + step * (e + u));
#pragma unroll
        for (int u = 0; u < CR4_INFLIGHT; ++u) {
          const float k = Ks[e + u];
          acc.x = fmaf(v[u].x, k, acc.x);
          acc.y = fmaf(v[u].y, k, acc.y);
          acc.z = fmaf(v[u].z, k, acc.z);
          acc.w = fmaf(v[u].w, k, acc.w);
        }
      }
      for (; e < nq; ++e) {
        const float4 v = __ldg(base + step * e);
        const float k = Ks[e];
        acc.x = fmaf(v.x, k, acc.x);
        acc.y = fmaf(v.y, k, acc.y);
        acc.z = fmaf(v.z, k, acc.z);
        acc.w = fmaf(v.w, k, acc.w);
      }
    }
  }
  if (!live) return;
  const float a[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (to_part) out[(int64_t)z * P1 * R + (p + u) + P1 * (int64_t)r] = a[u];
    else out[(p + u) * R + r] = a[u];
  }
}

// contract_first: each warp computes four outputs q at once (dot products of
// contiguous columns with h(:, r) staged in shared memory), lanes reading
// float4, so each lane keeps 4 * P1/128 loads in flight.
constexpr int CF4_THREADS = 256;
constexpr int CF4_QW = 4;  // outputs per warp

__global__ void __launch_bounds__(CF4_THREADS)
contract_first_v4_kernel(const float* __restrict__ T, int64_t P1, int64_t Q, int R,
                         const float* __restrict__ h, float* __restrict__ out, int rowmajor) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ float4 sh4[];  // P1 / 4
  const int r = blockIdx.y;
  for (int64_t e = threadIdx.x; e < P1 / 4; e += CF4_THREADS) {
    float4 v;
    v.x = h[(4 * e + 0) * R + r];
    v.y = h[(4 * e + 1) * R + r];
    v.z = h[(4 * e + 2) * R + r];
    v.w = h[(4 * e + 3) * R + r];
    sh4[e] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t q0 = ((int64_t)blockIdx.x * (CF4_THREADS / 32) + warp) * CF4_QW;
  const float* Tr = T + P1 * Q * (int64_t)r;
  const int64_t n4 = P1 / 4;
  float s[CF4_QW] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int64_t e = lane; e < n4; e += 32) {
    const float4 hv = sh4[e];
#pragma unroll
    for (int u = 0; u < CF4_QW; ++u) {
      if (q0 + u < Q) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(Tr + P1 * (q0 + u)) + e);
        s[u] = fmaf(v.x, hv.x, fmaf(v.y, hv.y, fmaf(v.z, hv.z, fmaf(v.w, hv.w, s[u]))));
      }
    }
  }
#pragma unroll
  for (int u = 0; u < CF4_QW; ++u) {
    const float v = warp_sum(s[u]);
    const int64_t q = q0 + u;
    if (lane == 0 && q < Q) {
      if (rowmajor) out[q * R + r] = v; else out[q + Q * (int64_t)r] = v;
    }
  }
}

template <typename TA>
Krp<TA> make_krp(const KrpHost& kh, int R) {
  Krp<TA> K{};
  K.nm = kh.nm;
  K.R = R;
  for (int m = 0; m < kh.nm; ++m) { K.dim[m] = kh.dim[m]; K.H[m] = (const TA*)kh.H[m]; }
  return K;
}

}  // namespace

cudaError_t launch_contract_first(bool f64, const void* T, int64_t P1, int64_t Q, int R,
                                  const void* h, void* out, bool out_rowmajor, cudaStream_t st) {
  if (!f64 && P1 % 4 == 0 && P1 >= 128 && P1 <= 16384 && ((uintptr_t)T & 15) == 0) {
    const int64_t qpb = (CF4_THREADS / 32) * CF4_QW;
    dim3 grid((unsigned)((Q + qpb - 1) / qpb), (unsigned)R);
    const size_t smem = (size_t)P1 * sizeof(float);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(contract_first_v4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    const cudaError_t e =
        launch_pdl(contract_first_v4_kernel, dim3(grid), dim3(CF4_THREADS), smem, st,
                   (const float*)T, P1, Q, R, (const float*)h, (float*)out, out_rowmajor ? 1 : 0);
    note_launches(1);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  int gw = 1;
  while (gw < 32 && gw < P1) gw <<= 1;
  int groups = CF_THREADS / gw;
  int64_t qpb = (int64_t)groups * CF_Q_PER_GROUP;
  dim3 grid((unsigned)((Q + qpb - 1) / qpb), (unsigned)R);
  if (f64)
    contract_first_kernel<double><<<grid, CF_THREADS, 0, st>>>(
        (const double*)T, P1, Q, R, (const double*)h, (double*)out, out_rowmajor ? 1 : 0, gw);
  else
    contract_first_kernel<float><<<grid, CF_THREADS, 0, st>>>(
        (const float*)T, P1, Q, R, (const float*)h, (float*)out, out_rowmajor ? 1 : 0, gw);
    note_launches(1);
  return cudaGetLastError();
}

bool contract_rest_v4_ok(int64_t P1, const void* T) {
  return P1 % 4 == 0 && P1 >= 64 && ((uintptr_t)T & 15) == 0;
}

int contract_rest_qsplit(int64_t P1, int64_t Q, int R, int sm_count) {
  if (P1 % 4 == 0 && P1 >= 64) {
    // vectorised kernel: CR4_P rows of p per CTA, aim for ~4 CTAs per SM
    const int64_t tiles = ((P1 + CR4_P - 1) / CR4_P) * R;
    int64_t qs = (4LL * sm_count + tiles - 1) / tiles;
    qs = std::min<int64_t>(qs, std::max<int64_t>(1, Q / 16));
    return (int)std::max<int64_t>(1, std::min<int64_t>(qs, 256));
  }
  int64_t P1b = std::min<int64_t>(P1, CR_THREADS);
  int64_t nql = CR_THREADS / P1b;
  int64_t tiles = ((P1 + P1b - 1) / P1b) * R;
  int64_t target = 4LL * sm_count;
  int64_t qs = (target + tiles - 1) / tiles;
  int64_t maxs = Q / (nql * 32);
  if (qs > maxs) qs = maxs;
  if (qs > 256) qs = 256;
  if (qs < 1) qs = 1;
  return (int)qs;
}

cudaError_t launch_contract_rest(bool f64, const void* T, int64_t P1, int64_t Q, int R,
                                 const KrpHost& krp, void* out, void* part, int qsplit,
                                 cudaStream_t st) {
  if (!f64 && contract_rest_v4_ok(P1, T)) {
    const int64_t qchunk = (Q + qsplit - 1) / qsplit;
    dim3 grid((unsigned)((P1 + CR4_P - 1) / CR4_P), (unsigned)R, (unsigned)qsplit);
    void* dst = qsplit > 1 ? part : out;
    cudaError_t e = launch_pdl(contract_rest_v4_kernel, grid, dim3(CR4_THREADS), 0, st,
                               (const float*)T, P1, Q, R, make_krp<float>(krp, R), qchunk,
                               (float*)dst, (int)(qsplit > 1));
    note_launches(1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess || qsplit == 1) return e;
    return launch_split_reduce(false, part, qsplit, P1, R, out, true, st);
  }
  int64_t P1b = std::min<int64_t>(P1, CR_THREADS);
  int64_t qchunk = (Q + qsplit - 1) / qsplit;
  dim3 grid((unsigned)((P1 + P1b - 1) / P1b), (unsigned)R, (unsigned)qsplit);
  void* dst = qsplit > 1 ? part : out;
  if (f64)
    contract_rest_kernel<double><<<grid, CR_THREADS, 0, st>>>(
        (const double*)T, P1, Q, R, make_krp<double>(krp, R), qchunk, (double*)dst, qsplit > 1);
  else
    contract_rest_kernel<float><<<grid, CR_THREADS, 0, st>>>(
        (const float*)T, P1, Q, R, make_krp<float>(krp, R), qchunk, (float*)dst, qsplit > 1);
    note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || qsplit == 1) return e;
  return launch_split_reduce(f64, part, qsplit, P1, R, out, true, st);
}

}  // namespace planc
