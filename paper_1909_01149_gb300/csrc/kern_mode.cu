// Fused per-mode update for small factor matrices: everything of Alg. 1 /
// Alg. 4 that follows the MTTKRP for mode n,
//   S^(n) = Hadamard of the other Grams,
//   Hhat  = NNLS-Update(S^(n), M^(n)) with warm start H^(n) diag(lambda)
//           (MU, Eq. muupd; HALS, Eq. halsupd; projected gradient; the
//           Nesterov-type steps of Eq. nesinnerupd, with the per-step stop
//           test reduced over the cluster; ADMM, Eq. admmupd, likewise;
//           UCP, H = M S^{-1}; BPP: the rows arrive solved by the BPP
//           kernel, and this launch does the rest),
//   lambda_r = ||Hhat(:, r)||, H^(n) = Hhat diag(lambda)^{-1}, G^(n) = H^T H,
//   and after the last mode the error identity of Sec. A.2,
// in a single launch of one thread-block cluster.
//
// The factor's rows are split over the cluster's CTAs (at most MC_RPC rows
// each, one thread per row with the row in registers for the NNLS sweep).
// The cross-CTA reductions (column norms, <M, Hhat>, the Gram, gamma) are
// pushed into the owning CTA's shared memory with distributed-shared-memory
// stores and read after a cluster barrier; every sum runs in a fixed order, so
// the result does not depend on scheduling.  Used when the factor has at most
// MC_CS * MC_RPC rows and R <= 32; larger factors and BPP / ADMM use the
// multi-kernel path.
#include <algorithm>

#include "batch_dev.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace planc {

namespace {

constexpr int MC_CS = 8;     // CTAs per cluster
constexpr int MC_NT = 128;   // threads per CTA
constexpr int MC_RPC = 128;  // rows per CTA at most (one per thread)

// ---- cluster / distributed shared memory ----------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// store v into the shared-memory word `local` of CTA `rank` of the cluster
__device__ __forceinline__ void st_cluster(const double* local, uint32_t rank, double v) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(local), d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(rank));
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(d), "d"(v) : "memory");
}

__device__ __forceinline__ void st_cluster_t(const double* local, uint32_t rank, double v) {
  st_cluster(local, rank, v);
}
__device__ __forceinline__ void st_cluster_t(const float* local, uint32_t rank, float v) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(local), d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(rank));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(d), "f"(v) : "memory");
}

// a load of data that, with COH, another CTA may have written earlier in the
// same launch: through L2 (__ldcg), never the read-only path
template <bool COH, typename T>
__device__ __forceinline__ T ldc(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// d = sum_k h[k] * S[r][k] with S row r read by explicit vector shared-memory
// loads at the point of use (keeps the compiler from holding all of S in
// registers when the column loop is unrolled).
template <int RP>
__device__ __forceinline__ float srow_dot(const float* h, uint32_t srow) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
  for (int k = 0; k < RP; k += 4) {
    float s0, s1, s2, s3;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(s0), "=f"(s1), "=f"(s2), "=f"(s3) : "r"(srow + 4u * k));
    a0 = fmaf(h[k + 0], s0, a0);
    a1 = fmaf(h[k + 1], s1, a1);
    a2 = fmaf(h[k + 2], s2, a2);
    a3 = fmaf(h[k + 3], s3, a3);
  }
  return (a0 + a1) + (a2 + a3);
}
template <int RP>
__device__ __forceinline__ double srow_dot(const double* h, uint32_t srow) {
  double a0 = 0.0, a1 = 0.0;
#pragma unroll
  for (int k = 0; k < RP; k += 2) {
    double s0, s1;
    asm volatile("ld.shared.v2.f64 {%0,%1}, [%2];" : "=d"(s0), "=d"(s1) : "r"(srow + 8u * k));
    a0 = fma(h[k + 0], s0, a0);
    a1 = fma(h[k + 1], s1, a1);
  }
  return a0 + a1;
}

// l = sqrt(s) and il = 1 / l in FP64 (0 and 0 for s <= 0): an FP32
// reciprocal-square-root seed (relative error below 2^-21) refined by one
// Newton-Raphson step y <- y (3 - s y^2) / 2, which squares the relative
// error (below 1e-12 after it); FP64 sqrt and division are avoided because
// this GPU's FP64 pipe is narrow.
__device__ __forceinline__ void sqrt_and_inv(double s, double& l, double& il) {
  if (!(s > 0.0)) {
    l = 0.0;
    il = 0.0;
    return;
  }
  if (s < 1e-30 || s > 1e30) {  // keep the FP32 seed well inside its range
    l = sqrt(s);
    il = 1.0 / l;
    return;
  }
  double y = (double)rsqrtf((float)s);
  y = y * (1.5 - 0.5 * s * y * y);
  l = s * y;
  il = y;
}

// sum over the cluster's CTAs of slot[src * stride], as a fixed pairwise tree
__device__ __forceinline__ double slot_sum(const double* slot, int stride) {
  double v[MC_CS];
#pragma unroll
  for (int i = 0; i < MC_CS; ++i) v[i] = slot[i * stride];
#pragma unroll
  for (int w = 1; w < MC_CS; w *= 2)
#pragma unroll
    for (int i = 0; i + w < MC_CS; i += 2 * w) v[i] += v[i + w];
  return v[0];
}

// x / y for the MU ratio: the FP32 fast division (within 2 ulp for the
// positive, moderate denominators MU produces) and exact division in FP64
__device__ __forceinline__ float mu_div(float x, float y) { return __fdividef(x, y); }
__device__ __forceinline__ double mu_div(double x, double y) { return x / y; }

// Row-swizzled layout of the CTA's factor rows in shared memory: row i holds
// its 16-byte groups in the order g ^ f(i), so that a warp reading one row
// per lane with 16-byte loads, and a warp reading one row across lanes, are
// both free of bank conflicts.
template <typename TA, int RP>
struct Swz {
  static constexpr int VPG = 16 / (int)sizeof(TA);  // elements per 16-byte group
  static constexpr int GR = RP / VPG;               // groups per row (4, 8 or 16)
  __device__ __forceinline__ static int f(int i) { return GR >= 8 ? (i & 7) : ((i >> 1) & 3); }
  __device__ __forceinline__ static int idx(int i, int k) {
    return i * RP + (((k / VPG) ^ f(i)) * VPG) + (k % VPG);
  }
  __device__ __forceinline__ static int gidx(int i, int g) { return i * RP + ((g ^ f(i)) * VPG); }
};

// four consecutive columns k0..k0+3 (k0 % 4 == 0) of row i
template <typename TA, int RP>
__device__ __forceinline__ void load4(const TA* Hs, int i, int k0, TA* v) {
  using S = Swz<TA, RP>;
  if constexpr (sizeof(TA) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(Hs + S::gidx(i, k0 / 4));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(Hs + S::gidx(i, k0 / 2));
    const double2 b = *reinterpret_cast<const double2*>(Hs + S::gidx(i, k0 / 2 + 1));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}

// upper-triangle enumeration (row-major, diagonal included) of an n x n grid
__device__ __forceinline__ int tri_index(int r, int s, int n) {  // r <= s
  return r * n - r * (r - 1) / 2 + (s - r);
}
// inverse of tri_index: the row from the quadratic formula (exact enough in
// FP32 for n <= 32 that one correction step suffices), then the column
__device__ __forceinline__ void tri_unpack(int p, int n, int& r, int& s) {
  const float b = 2.f * n + 1.f;
  int rr = (int)((b - sqrtf(b * b - 8.f * p)) * 0.5f);
  rr = max(0, min(n - 1, rr));
  if (tri_index(rr, rr, n) > p)
    --rr;
  else if (rr + 1 < n && tri_index(rr + 1, rr + 1, n) <= p)
    ++rr;
  r = rr;
  s = rr + (p - tri_index(rr, rr, n));
}

// LIN: with the landing area of the rows' bulk copies (the persistent batched
// solve loads the rows directly and has no use for it)
template <typename TA, int RP, bool LIN = true>
struct McLayout {
  static constexpr int NB = RP / 4;                     // 4-column blocks
  static constexpr int NBLK = NB * (NB + 1) / 2;        // upper-triangle 4x4 tiles
  static constexpr int RCN = MC_NT / NBLK;              // row chunks of the Gram
  static constexpr int NP = RP * (RP + 1) / 2;          // packed pairs r <= s
  static constexpr int NPO = (NP + MC_CS - 1) / MC_CS;  // pairs owned per CTA
  static constexpr int RED = 16;                        // warp sums (beta / gamma; ADMM 4 x 4)
  // byte offsets
  static constexpr size_t oSs = 0;
  static constexpr size_t oHs = oSs + sizeof(TA) * RP * RP;
  static constexpr size_t oMs = oHs + sizeof(TA) * MC_RPC * RP;
  static constexpr size_t oLin = oMs + sizeof(TA) * MC_RPC * RP;  // bulk-copy landing area
  static constexpr size_t oTp = oLin + (LIN ? sizeof(TA) * 2 * MC_RPC * RP : 0);
  static constexpr size_t oCs = oTp + sizeof(TA) * RCN * NBLK * 16;
  static constexpr size_t oGs = oCs + sizeof(double) * MC_CS * RP;
  static constexpr size_t oBeta = oGs + sizeof(double) * MC_CS * NPO;
  static constexpr size_t oGam = oBeta + sizeof(double) * MC_CS;
  static constexpr size_t oRed = oGam + sizeof(double) * MC_CS;
  static constexpr size_t oNes = oRed + sizeof(double) * RED;  // [parity][src CTA][<= 4]
  static constexpr size_t bytes = oNes + sizeof(double) * 2 * MC_CS * 4;
  static_assert(MC_NT % RP == 0 && MC_NT == MC_RPC && NPO <= MC_NT, "one row / pair per thread");
};

// G: the N Grams (FP64, R x R each), Gf: the same in FP32.  Mode n's entries
// of both are overwritten with G^(n) of the updated factor.  err: set to 10
// if the wait for the bulk copies of M and H gives up.
// ALG >= 0 fixes the update at compile time (the kernel then carries only
// that update's code: the launch is short and runs its code cold, so code
// size shows up as instruction-fetch stalls); ALG < 0 dispatches on alg.
// COH: M, H, the Grams, lambda and alpha were written earlier in the same
// launch (the persistent batched solve), so they are read through L2 and the
// rows are loaded directly (no bulk copies).
template <typename TA, int RP, int ALG = -1, bool COH = false>
__device__ __forceinline__ void mode_update_body(
    int rows, int R, int N, int n, double* __restrict__ G, float* __restrict__ Gf,
    const TA* __restrict__ M, TA* __restrict__ H, double* __restrict__ lam, int alg_rt,
    double mu_eps, int pgd_steps, double tiny, int32_t* __restrict__ inner,
    const double* __restrict__ alpha, double* __restrict__ fit_out, int* __restrict__ err,
    const double* __restrict__ nes_scr, int nes_kmax, double nes_tol,
    const RecArgs& rec = RecArgs(), int* __restrict__ nflags = nullptr) {
  using L = McLayout<TA, RP, !COH>;
  using S = Swz<TA, RP>;
  const int alg = ALG >= 0 ? ALG : alg_rt;
  extern __shared__ __align__(16) unsigned char mc_smem[];
  TA* Ss = reinterpret_cast<TA*>(mc_smem + L::oSs);                 // S^(n), RP x RP
  TA* Hs = reinterpret_cast<TA*>(mc_smem + L::oHs);                 // this CTA's rows
  TA* Ms = reinterpret_cast<TA*>(mc_smem + L::oMs);                 // its rows of M
  TA* Lin = reinterpret_cast<TA*>(mc_smem + L::oLin);               // M, H as copied
  TA* tp = reinterpret_cast<TA*>(mc_smem + L::oTp);                 // Gram tile partials
  double* cs_slot = reinterpret_cast<double*>(mc_smem + L::oCs);    // [src CTA][r]: Ghat(r, r)
  double* g_slot = reinterpret_cast<double*>(mc_smem + L::oGs);     // [src CTA][owned pair]
  double* beta_slot = reinterpret_cast<double*>(mc_smem + L::oBeta);  // [src CTA] (CTA 0)
  double* gam_slot = reinterpret_cast<double*>(mc_smem + L::oGam);    // [src CTA] (CTA 0)
  double* red = reinterpret_cast<double*>(mc_smem + L::oRed);
  double* nes_slot = reinterpret_cast<double*>(mc_smem + L::oNes);
  __shared__ double s_lam[RP], s_il[RP];
  __shared__ TA s_lamt[RP], s_inv[RP];
  __shared__ TA s_rinv[RP];  // 1 / S(r, r), or 0 where S(r, r) <= tiny (column kept)
  __shared__ TA s_eta;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_abort;
  const int t = threadIdx.x;
  const int RR = R * R;
  const uint32_t c = cluster_rank();
  const int per = (rows + MC_CS - 1) / MC_CS;  // rows per CTA (<= MC_RPC)
  const int row0 = (int)c * per;
  const int nrow = max(0, min(per, rows - row0));
  const int nel = nrow * R;
  // element e = t + j * MC_NT of a row-major block with R columns is at
  // (row a, column k); stepping j advances by (q_step, k_step) with a carry
  const int q_step = MC_NT / R, k_step = MC_NT - (MC_NT / R) * R;
  const int a_0 = t / R, k_0 = t - (t / R) * R;
  const TA* Mrow = M + (size_t)row0 * R;
  TA* Hrow = H + (size_t)row0 * R;
  // this CTA's rows of M and H arrive by two bulk copies when both ranges
  // start on 16 bytes and span a multiple of 16 bytes
  const uint32_t cbytes = (uint32_t)(nel * sizeof(TA));
  const bool bulk = !COH && nel > 0 && (cbytes & 15u) == 0 &&
                    ((reinterpret_cast<uintptr_t>(Mrow) | reinterpret_cast<uintptr_t>(Hrow)) & 15u) == 0;

  pdl_wait();  // the MTTKRP and the previous mode's Grams are complete
  pdl_trigger();
  // every CTA of the cluster must be running before any remote store
  cluster_arrive_relaxed();
  constexpr int EPT = RP * RP / MC_NT;      // entries of S per thread

  const double lam_t = t < R ? ldc<COH>(lam + t) : 0.0;
  // owned pair of this thread (for G^(n) and gamma): p = t * MC_CS + c
  const int p_own = t * MC_CS + (int)c;
  int r_own = 0, s_own = 0;
  if (t < L::NPO && p_own < L::NP) tri_unpack(p_own, RP, r_own, s_own);
  const bool owns = t < L::NPO && p_own < L::NP && s_own < R;
  // FP64 entries of the other Grams at the owned pair, for the entry S(r, s)
  // of gamma after the last mode (held in registers until then; more than
  // four other modes are read at that point instead)
  constexpr int QPRE = 4;
  double gq[QPRE];
  const bool pre = fit_out && owns && N - 1 <= QPRE;
#pragma unroll
  for (int qi = 0; qi < QPRE; ++qi)
    gq[qi] = (pre && qi + 1 < N) ? ldc<COH>(G + (size_t)(qi < n ? qi : qi + 1) * RR + r_own * R + s_own) : 1.0;
  // S^(n) = Hadamard of the other Grams, in TA (from the FP32 copies when TA
  // is FP32); entry (i, k) of S for e = t + j * MC_NT.  With at most QPRE
  // other modes all entries are loaded before the row copies are issued and
  // multiplied after.
  TA v[EPT];
  int off[EPT];
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int e = t + j * MC_NT, i = e / RP, k = e % RP;
    const bool in = i < R && k < R;
    v[j] = in ? TA(1) : TA(0);
    off[j] = in ? i * R + k : 0;
  }
  constexpr int QS = sizeof(TA) == 4 ? QPRE : 1;  // (FP64: loaded when used)
  const bool sfast = sizeof(TA) == 4 && N - 1 <= QPRE;
  TA gl[QS][EPT];
#pragma unroll
  for (int qi = 0; qi < QS; ++qi) {
    const size_t q = (size_t)(qi < n ? qi : qi + 1);
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      TA x = TA(1);
      if (sfast && qi + 1 < N) {
        if constexpr (sizeof(TA) == 4) x = ldc<COH>(Gf + q * RR + off[j]);
        else x = ldc<COH>(G + q * RR + off[j]);
      }
      gl[qi][j] = x;
    }
  }
  constexpr int LPT = MC_RPC * RP / MC_NT;  // staged elements per thread
  TA mv[LPT], hv[LPT];
  if (bulk) {
    if (t == 0) {
      s_abort = 0;
      tc::mbar_init(&s_bar, 1);
      tc::fence_mbar_init();
      tc::mbar_arrive_expect_tx(&s_bar, 2 * cbytes);
      tc::bulk_g2s(Lin, Mrow, cbytes, &s_bar);
      tc::bulk_g2s(Lin + MC_RPC * RP, Hrow, cbytes, &s_bar);
    }
  } else {
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
      const int e = t + j * MC_NT;
      mv[j] = e < nel ? ldc<COH>(Mrow + e) : TA(0);
      hv[j] = e < nel ? ldc<COH>(Hrow + e) : TA(0);
    }
  }
  if (sfast) {
#pragma unroll
    for (int qi = 0; qi < QS; ++qi)
#pragma unroll
      for (int j = 0; j < EPT; ++j) v[j] *= gl[qi][j];
  } else {
    for (int qi = 0; qi + 1 < N; ++qi) {
      const size_t q = (size_t)(qi < n ? qi : qi + 1);
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        if constexpr (sizeof(TA) == 4) v[j] *= ldc<COH>(Gf + q * RR + off[j]);
        else v[j] *= ldc<COH>(G + q * RR + off[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int e = t + j * MC_NT, i = e / RP;
    Ss[e] = v[j];
    if (e == i * RP + i) s_rinv[i] = v[j] > (TA)tiny ? TA(1) / v[j] : TA(0);
  }
  if (t < RP) {
    s_lam[t] = lam_t;
    s_lamt[t] = (TA)lam_t;
  }
  if (!bulk) {  // staged rows; padding rows are zero (mv = hv = 0 past nel)
    int a = a_0, k = k_0;
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
      if (a < MC_RPC) {
        Ms[S::idx(a, k)] = mv[j];
        Hs[S::idx(a, k)] = hv[j];
      }
      a += q_step;
      k += k_step;
      if (k >= R) {
        k -= R;
        ++a;
      }
    }
  }
  for (int k = R; k < RP; ++k) {  // padding columns of row t
    Ms[S::idx(t, k)] = TA(0);
    Hs[S::idx(t, k)] = TA(0);
  }
  __syncthreads();
  if (bulk) {
    // every thread waits for the copies (bounded); on a timeout the error
    // word is set and the kernel runs to the end on whatever arrived
    tc::mbar_wait(&s_bar, 0, &s_abort, err, 10);
    const TA* Lm = Lin;
    const TA* Lh = Lin + MC_RPC * RP;
    int a = a_0, k = k_0;
#pragma unroll 4
    for (int e = t; e < MC_RPC * R; e += MC_NT) {
      const bool in = e < nel;
      Ms[S::idx(a, k)] = in ? Lm[e] : TA(0);
      Hs[S::idx(a, k)] = in ? Lh[e] : TA(0);
      a += q_step;
      k += k_step;
      if (k >= R) {
        k -= R;
        ++a;
      }
    }
    __syncthreads();
  }
  if (alg == PLANC_PGD && t < 32) {
    TA f = TA(0);
    for (int e = t; e < RP * RP; e += 32) f = fma(Ss[e], Ss[e], f);
    const double fs = warp_sum((double)f);
    if (t == 0) s_eta = (TA)(1.0 / fmax(sqrt(fs), 1e-300));
  }
  const bool live = t < nrow;
  TA h[RP], m[RP];
#pragma unroll
  for (int g = 0; g < S::GR; ++g) {
    const TA* ms = Ms + S::gidx(t, g);
    const TA* hs = Hs + S::gidx(t, g);
#pragma unroll
    for (int u = 0; u < S::VPG; ++u) {
      m[g * S::VPG + u] = ms[u];
      // warm start H diag(lambda); BPP: the solved row Hhat as it is
      h[g * S::VPG + u] = alg == PLANC_BPP ? hs[u] : hs[u] * s_lamt[g * S::VPG + u];
    }
  }

  // ---- NNLS update of row t (row in registers)
  const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(Ss);
  if (live) {
    if (alg == PLANC_HALS) {
      // a column with S(r, r) <= tiny (and every padding column) has
      // s_rinv = 0 and keeps its non-negative value
#pragma unroll
      for (int r = 0; r < RP; ++r) {
        const TA d = srow_dot<RP>(h, s_base + (uint32_t)(r * RP * sizeof(TA)));
        const TA x = h[r] + (m[r] - d) * s_rinv[r];
        h[r] = x > TA(0) ? x : TA(0);
      }
    } else if (alg == PLANC_MU) {
      // Jacobi: every column uses the old row
      TA nh[RP];
#pragma unroll
      for (int r = 0; r < RP; ++r) {
        const TA d = srow_dot<RP>(h, s_base + (uint32_t)(r * RP * sizeof(TA)));
        nh[r] = r < R ? mu_div(h[r] * m[r], d + (TA)mu_eps) : TA(0);
      }
#pragma unroll
      for (int r = 0; r < RP; ++r) h[r] = nh[r];
    }
  }
  if (alg == PLANC_PGD) {
    __syncthreads();  // s_eta
    if (live) {
      const TA eta = s_eta;
      for (int st = 0; st < pgd_steps; ++st) {
        TA nh[RP];
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          const TA d = srow_dot<RP>(h, s_base + (uint32_t)(r * RP * sizeof(TA)));
          const TA x = h[r] - eta * (d - m[r]);
          nh[r] = (r < R && x > TA(0)) ? x : TA(0);
        }
#pragma unroll
        for (int r = 0; r < RP; ++r) h[r] = nh[r];
      }
    }
  }
  if (ALG == PLANC_UCP || (ALG < 0 && alg == PLANC_UCP)) {
    // H = M W with W = S^{-1} (prepared in FP64, stored in the factor
    // precision after scr + 8 + R^2); W replaces S in shared memory
    __syncthreads();
    const TA* Wt = reinterpret_cast<const TA*>(nes_scr + 8 + RR);
    for (int e = t; e < RP * RP; e += MC_NT) {
      const int i = e / RP, k = e - i * RP;
      Ss[e] = (i < R && k < R) ? Wt[i * R + k] : TA(0);
    }
    if (c == 0 && t == 0 && nflags && nes_scr[1] != 0.0) atomicAdd(nflags + 1, 1);
    __syncthreads();
    if (live) {
      TA nh[RP];
#pragma unroll
      for (int r = 0; r < RP; ++r)
        nh[r] = r < R ? srow_dot<RP>(m, s_base + (uint32_t)(r * RP * sizeof(TA))) : TA(0);
#pragma unroll
      for (int r = 0; r < RP; ++r) h[r] = nh[r];  // W symmetric: row r is column r
    }
  }
  int admm_steps = 0;
  // ADMM (Eq. admmupd): W = (S + rho I)^{-1} prepared in FP64 (stored in the
  // factor precision after scr + 8 + R^2), U = 0; each step
  //   Htil = (M + rho (H + U)) W,  H = [Htil - U]_+,  U = U + H - Htil,
  // then the four stop norms are summed over the cluster (compiled where the
  // fused path takes ADMM: FP32, or FP64 with R <= 16)
  constexpr bool kAdmm = (ALG == PLANC_ADMM || ALG < 0) && (sizeof(TA) == 4 || RP <= 16);
  if (kAdmm && alg == PLANC_ADMM) {
    __syncthreads();
    const TA* Wt = reinterpret_cast<const TA*>(nes_scr + 8 + RR);
    for (int e = t; e < RP * RP; e += MC_NT) {
      const int i = e / RP, k = e - i * RP;
      Ss[e] = (i < R && k < R) ? Wt[i * R + k] : TA(0);
    }
    const TA rho = (TA)nes_scr[0];
    if (c == 0 && t == 0 && nflags && nes_scr[1] != 0.0) atomicAdd(nflags + 1, 1);
    __syncthreads();
    TA u[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) u[r] = TA(0);
    cluster_wait();  // pairs with the arrive at kernel start: every CTA is running
    for (int k = 0; k < nes_kmax; ++k) {
      TA rhs[RP];
#pragma unroll
      for (int r = 0; r < RP; ++r) rhs[r] = fma(rho, h[r] + u[r], m[r]);
      TA npr = TA(0), nh = TA(0), ndu = TA(0), nu = TA(0);
      if (live) {
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          const TA ht = srow_dot<RP>(rhs, s_base + (uint32_t)(r * RP * sizeof(TA)));  // W symmetric
          TA hn = ht - u[r];
          hn = hn > TA(0) ? hn : TA(0);
          const TA un = u[r] + hn - ht;
          npr = fma(hn - ht, hn - ht, npr);
          nh = fma(hn, hn, nh);
          ndu = fma(hn - h[r], hn - h[r], ndu);
          nu = fma(un, un, nu);
          h[r] = hn;
          u[r] = un;
        }
      }
      double q4[4] = {(double)npr, (double)nh, (double)ndu, (double)nu};
#pragma unroll
      for (int q = 0; q < 4; ++q) q4[q] = warp_sum(q4[q]);
      if ((t & 31) == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[(t >> 5) + 4 * q] = q4[q];
      __syncthreads();
      double* sl = nes_slot + (k & 1) * MC_CS * 4;
      if (t < MC_CS) {  // thread d pushes this CTA's four sums to CTA d
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          double v = 0.0;
          for (int w = 0; w < MC_NT / 32; ++w) v += red[w + 4 * q];
          st_cluster(sl + c * 4 + q, (uint32_t)t, v);
        }
      }
      cluster_arrive();
      cluster_wait();
      double a4[4];  // the same slots in the same order in every CTA
#pragma unroll
      for (int q = 0; q < 4; ++q) a4[q] = slot_sum(sl + q, 4);
      ++admm_steps;
      if (a4[0] < nes_tol * a4[1] && a4[2] < nes_tol * a4[3]) break;
    }
    cluster_arrive_relaxed();  // re-pairs with the wait before the Gram exchange
  }
  int nes_steps = 0;
  // (compiled only where the fused path takes NES: FP32, or FP64 with R <= 16)
  constexpr bool kNes = sizeof(TA) == 4 || RP <= 16;
  if (kNes && alg == PLANC_NES) {
    // P = I - (S + lam_p I) / L over Ss (S is not read again); parameters
    // from the extreme eigenvalues of S (written to nes_scr beforehand)
    const bool skip = nes_scr[5] != 0.0;
    const TA lp = (TA)nes_scr[0], invL = (TA)nes_scr[3], lpL = (TA)nes_scr[4];
    const TA nbeta = (TA)nes_scr[2];
    for (int e = t; e < RP * RP; e += MC_NT) {
      const int i = e / RP, k = e - i * RP;
      TA pv = TA(0);
      if (i < R && k < R) pv = (i == k ? TA(1) : TA(0)) - (Ss[e] + (i == k ? lp : TA(0))) * invL;
      Ss[e] = pv;
    }
    __syncthreads();
    // X_0 = Y_0 = H* (the warm start), b = (M + lam_p H*) / L; padding
    // columns and rows stay zero throughout
    TA y[RP], x[RP], b[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      x[r] = h[r];
      y[r] = h[r];
      b[r] = fma(m[r], invL, h[r] * lpL);
    }
    cluster_wait();  // pairs with the arrive at kernel start: every CTA is running
    if (!skip) {
      for (int k = 0; k < nes_kmax; ++k) {
        TA nx[RP];
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          const TA z = srow_dot<RP>(y, s_base + (uint32_t)(r * RP * sizeof(TA))) + b[r];
          nx[r] = z > TA(0) ? z : TA(0);  // P symmetric: row r is column r
        }
        TA dmax = TA(0), xmax = TA(0);
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          const TA dd = nx[r] > y[r] ? nx[r] - y[r] : y[r] - nx[r];
          dmax = dd > dmax ? dd : dmax;
          xmax = nx[r] > xmax ? nx[r] : xmax;
          y[r] = fma(nbeta, nx[r] - x[r], nx[r]);
          x[r] = nx[r];
        }
        // maxima in the factor precision (max is exact: no FP64 work per
        // step for FP32 factors); only the final test in FP64
        TA da = dmax, xa = xmax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const TA u = __shfl_xor_sync(0xffffffffu, da, o), v = __shfl_xor_sync(0xffffffffu, xa, o);
          da = u > da ? u : da;
          xa = v > xa ? v : xa;
        }
        TA* redt = reinterpret_cast<TA*>(red);
        if ((t & 31) == 0) {
          redt[(t >> 5) * 2 + 0] = da;
          redt[(t >> 5) * 2 + 1] = xa;
        }
        __syncthreads();
        TA* sl = reinterpret_cast<TA*>(nes_slot) + (k & 1) * MC_CS * 2;
        if (t < MC_CS) {  // thread d pushes this CTA's maxima to CTA d
          TA a = redt[0], bx = redt[1];
          for (int w = 1; w < MC_NT / 32; ++w) {
            a = redt[w * 2 + 0] > a ? redt[w * 2 + 0] : a;
            bx = redt[w * 2 + 1] > bx ? redt[w * 2 + 1] : bx;
          }
          st_cluster_t(sl + c * 2 + 0, (uint32_t)t, a);
          st_cluster_t(sl + c * 2 + 1, (uint32_t)t, bx);
        }
        cluster_arrive();
        cluster_wait();
        TA a = TA(0), bx = TA(0);  // the same slots in the same order in every CTA
#pragma unroll
        for (int src = 0; src < MC_CS; ++src) {
          a = sl[src * 2 + 0] > a ? sl[src * 2 + 0] : a;
          bx = sl[src * 2 + 1] > bx ? sl[src * 2 + 1] : bx;
        }
        ++nes_steps;
        if ((double)a <= nes_tol * (double)bx) break;
      }
    }
    cluster_arrive_relaxed();  // re-pairs with the wait before the Gram exchange
#pragma unroll
    for (int r = 0; r < RP; ++r) h[r] = x[r];
#pragma unroll
    for (int g = 0; g < S::GR; ++g) {  // M again from shared memory (for <M, Hhat>)
      const TA* ms = Ms + S::gidx(t, g);
#pragma unroll
      for (int u = 0; u < S::VPG; ++u) m[g * S::VPG + u] = ms[u];
    }
  }
  // Hhat row into shared memory (padding rows stay zero); <M, Hhat> partial
  TA beta_t = TA(0);
#pragma unroll
  for (int g = 0; g < S::GR; ++g) {
    TA* dst = Hs + S::gidx(t, g);
#pragma unroll
    for (int u = 0; u < S::VPG; ++u) {
      const TA x = live ? h[g * S::VPG + u] : TA(0);
      dst[u] = x;
      beta_t = fma(m[g * S::VPG + u], x, beta_t);
    }
  }
  const double bw = warp_sum((double)beta_t);
  if ((t & 31) == 0) red[t >> 5] = bw;
  __syncthreads();

  // ---- Ghat = Hhat^T Hhat over this CTA's rows: 4x4 tiles (rb <= sb) x row
  // chunks, in TA.  Its diagonal gives lambda, and G^(n) = Ghat / (lambda lambda^T).
  if (t < L::RCN * L::NBLK) {
    const int blk = t % L::NBLK, ch = t / L::NBLK;
    int rb, sb;
    tri_unpack(blk, L::NB, rb, sb);
    const int rpc = (nrow + L::RCN - 1) / L::RCN;
    const int i0 = ch * rpc, i1 = min(nrow, i0 + rpc);
    TA acc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e] = TA(0);
    for (int i = i0; i < i1; ++i) {
      TA x[4], y[4];
      load4<TA, RP>(Hs, i, rb * 4, x);
      load4<TA, RP>(Hs, i, sb * 4, y);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u * 4 + w] = fma(x[u], y[w], acc[u * 4 + w]);
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) tp[(ch * L::NBLK + blk) * 16 + e] = acc[e];
  }
  __syncthreads();
  cluster_wait();  // pairs with the arrive at kernel start: every CTA is running
  // combine the chunks in FP64; the diagonal goes to every CTA (lambda), the
  // other pairs to their owner (p % MC_CS); beta to CTA 0.  (Each chunk is an
  // FP32 sum over at most 43 rows; fully compensated sums were measured to
  // cost 4% of the outer iteration with no change in the error against the
  // FP64 oracle.)
  for (int p = t; p < L::NP; p += MC_NT) {
    int r, s;
    tri_unpack(p, RP, r, s);
    const int blk = tri_index(r / 4, s / 4, L::NB), e = (r % 4) * 4 + (s % 4);
    double ga = 0.0;
    for (int ch = 0; ch < L::RCN; ++ch) ga += (double)tp[(ch * L::NBLK + blk) * 16 + e];
    if (r == s) {
      for (uint32_t dst = 0; dst < MC_CS; ++dst) st_cluster(cs_slot + c * RP + r, dst, (double)ga);
    } else {
      st_cluster(g_slot + c * L::NPO + p / MC_CS, (uint32_t)(p % MC_CS), (double)ga);
    }
  }
  if (t == 0) {
    double b = 0.0;
    for (int w = 0; w < MC_NT / 32; ++w) b += red[w];
    st_cluster(beta_slot + c, 0, b);
  }
  cluster_arrive();
  cluster_wait();

  // ---- lambda (identical in every CTA: same slots, same order)
  if (t < RP) {
    const double s = slot_sum(cs_slot + t, RP);
    double l = 0.0, il = 0.0;  // a zero column keeps lambda = 0 and stays zero
    if (t < R) sqrt_and_inv(s, l, il);
    s_lam[t] = l;
    s_il[t] = il;
    s_inv[t] = (TA)il;
    if (c == 0 && t < R) lam[t] = l;
  }
  __syncthreads();
  // ---- H = Hhat diag(lambda)^-1 for this CTA's rows (coalesced write)
  {
    int a = a_0, k = k_0;
#pragma unroll 4
    for (int e = t; e < nel; e += MC_NT) {
      Hrow[e] = Hs[S::idx(a, k)] * s_inv[k];
      a += q_step;
      k += k_step;
      if (k >= R) {
        k -= R;
        ++a;
      }
    }
  }
  // ---- owned pair: G^(n)(r, s) = Ghat(r, s) / (lambda_r lambda_s); gamma
  // partial lambda^T (S * G^(n)) lambda = sum S(r, s) Ghat(r, s)
  double gam = 0.0;
  if (owns) {
    const int r = r_own, s = s_own;
    double gh = 0.0;
    gh = r == s ? slot_sum(cs_slot + r, RP) : slot_sum(g_slot + t, L::NPO);
    const double g = gh * s_il[r] * s_il[s];
    double* Gn = G + (size_t)n * RR;
    float* Gnf = Gf + (size_t)n * RR;
    Gn[r * R + s] = g;
    Gn[s * R + r] = g;
    Gnf[r * R + s] = (float)g;
    Gnf[s * R + r] = (float)g;
    if (fit_out) {
      double sv = 1.0;
      if (pre) {
#pragma unroll
        for (int qi = 0; qi < QPRE; ++qi) sv *= gq[qi];
      } else {
        for (int q = 0; q < N; ++q)
          if (q != n) sv *= ldc<COH>(G + (size_t)q * RR + r * R + s);
      }
      gam = (r == s ? 1.0 : 2.0) * sv * gh;
    }
  }
  if (c == 0 && t == 0 && inner && alg != PLANC_BPP)  // (BPP: its kernel counts)
    *inner = alg == PLANC_PGD ? pgd_steps
             : alg == PLANC_NES ? (nes_scr[5] != 0.0 ? 0 : nes_steps)
             : alg == PLANC_ADMM ? admm_steps : 1;
  if (!fit_out) return;  // uniform over the cluster: no remote access follows
  gam = warp_sum(gam);
  if ((t & 31) == 0) red[4 + (t >> 5)] = gam;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < MC_NT / 32; ++w) s += red[4 + w];
    st_cluster(gam_slot + c, 0, s);
  }
  cluster_arrive();
  cluster_wait();
  if (c == 0 && t == 0) {
    double gamma = 0.0, beta = 0.0;
    for (int src = 0; src < MC_CS; ++src) {
      gamma += gam_slot[src];
      beta += beta_slot[src];
    }
    const double a = ldc<COH>(alpha);
    const double rad = a - 2.0 * beta + gamma;
    const double eps = a > 0.0 ? sqrt(fmax(0.0, rad) / a) : 0.0;
    fit_out[0] = eps;
    fit_out[1] = beta;
    fit_out[2] = gamma;
    if (rec.hist) {  // this iteration's history record (replaces a separate launch)
      const int it = *rec.counter;
      if (it < rec.cap) {
        rec.hist[3 * it + 0] = eps;
        rec.hist[3 * it + 1] = beta;
        rec.hist[3 * it + 2] = gamma;
        for (int q = 0; q < rec.N; ++q) rec.inner_hist[it * rec.N + q] = rec.inner_now[q];
      }
      *rec.counter = it + 1;
    }
  }
}

template <typename TA, int RP, int ALG>
__global__ void __launch_bounds__(MC_NT, 1)
mode_cluster_kernel(int rows, int R, int N, int n, double* __restrict__ G,
                    float* __restrict__ Gf, const TA* __restrict__ M, TA* __restrict__ H,
                    double* __restrict__ lam, int alg, double mu_eps, int pgd_steps, double tiny,
                    int32_t* __restrict__ inner, const double* __restrict__ alpha,
                    double* __restrict__ fit_out, int* __restrict__ err,
                    const double* __restrict__ nes_scr, int nes_kmax, double nes_tol,
                    const __grid_constant__ RecArgs rec, int* __restrict__ nflags) {
  mode_update_body<TA, RP, ALG>(rows, R, N, n, G, Gf, M, H, lam, alg, mu_eps, pgd_steps, tiny, inner,
                           alpha, fit_out, err, nes_scr, nes_kmax, nes_tol, rec, nflags);
}

// Batched form: cluster b (blocks MC_CS b .. MC_CS b + MC_CS - 1) updates mode n
// of instance b of a 3-way batch; after mode 3 it writes instance b's error
// identity for outer iteration `it` into its history.
__global__ void __launch_bounds__(MC_NT, 1)
mode_cluster_batch_kernel(const BatchInst* __restrict__ tab, int n, int it, int alg,
                          double mu_eps, int pgd_steps, int* __restrict__ err) {
  const BatchInst& b = tab[blockIdx.x / MC_CS];
  mode_update_body<float, 32>((int)b.I[n], b.R, 3, n, b.G, b.Gf, b.M, b.H[n], b.lam, alg, mu_eps,
                              pgd_steps, 1e-30, b.inner + 3 * it + n, b.alpha,
                              n == 2 ? b.hist + 3 * it : nullptr, err, nullptr, 0, 0.0);
}

template <typename TA, int RP>
cudaError_t run_mc(int rows, int R, int N, int n, double* G, float* Gf, const void* M, void* H,
                   double* lam, planc_nls_t alg, const planc_nls_opts& o, int32_t* inner,
                   const double* alpha, double* fit_out, int* err, const double* nes_scr,
                   const RecArgs& rec, int* flags, cudaStream_t st) {
  const size_t smem = McLayout<TA, RP>::bytes;
  auto kern = alg == PLANC_MU     ? mode_cluster_kernel<TA, RP, PLANC_MU>
              : alg == PLANC_HALS ? mode_cluster_kernel<TA, RP, PLANC_HALS>
              : alg == PLANC_PGD  ? mode_cluster_kernel<TA, RP, PLANC_PGD>
              : alg == PLANC_UCP  ? mode_cluster_kernel<TA, RP, PLANC_UCP>
              : alg == PLANC_ADMM ? mode_cluster_kernel<TA, RP, PLANC_ADMM>
              : alg == PLANC_BPP  ? mode_cluster_kernel<TA, RP, PLANC_BPP>
                                  : mode_cluster_kernel<TA, RP, PLANC_NES>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(MC_CS, 1, 1);
  cfg.blockDim = dim3(MC_NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = MC_CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 2 : 1;
  e = cudaLaunchKernelEx(&cfg, kern, rows, R, N, n, G, Gf, (const TA*)M, (TA*)H, lam, (int)alg,
                         o.mu_eps, std::max(1, o.pgd_steps), sizeof(TA) == 8 ? 1e-300 : 1e-30,
                         inner, alpha, fit_out, err, nes_scr,
                         alg == PLANC_ADMM
                             ? std::min(PLANC_MAX_ADMM_STEPS, std::max(1, o.admm_max_inner))
                             : std::min(PLANC_MAX_NES_STEPS, std::max(1, o.nes_max_inner)),
                         alg == PLANC_ADMM ? o.admm_tol : o.nes_tol, rec, flags);
  note_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}


// ---- the whole batched solve in one persistent launch ---------------------------------
// Cluster q of the grid (MC_CS CTAs) solves the instances clist[coff[q]] ..
// clist[coff[q + 1] - 1] one after another, each through all of its outer
// iterations: alpha = ||X||^2 and the Grams of the initial factors, then per
// iteration (Alg. 1 with the dimension tree of Alg. 3, N = 3, S = 2)
//   T^{1:2} = X_(1:2) H^(3)  over the CTAs' row blocks  -> M^(1) = T x_2 H^(2)
//   -> update of mode 1 -> M^(2) = T x_1 H^(1) -> update of mode 2
//   -> M^(3) = X_(1:2)^T (H^(2) . H^(1)) over the CTAs' slabs -> update of
//   mode 3 and the error identity of Alg. 4 (Sec. A.2) into the history,
// with the same device code as the per-phase kernels.  Consecutive phases are
// separated by cluster barriers (release / acquire at cluster scope, so one
// phase's global writes are visible to the next); no CTA ever waits on
// another cluster, so the launch needs no flag, no spin and no device-wide
// barrier.  mode 1 / 2 run only the left / right partial MTTKRP of every
// assigned instance at the current factors (timed by the schedule tuner;
// they leave the factors as they are).  sqpart: MC_CS doubles per instance.
constexpr int PB_MINB = 2;  // CTAs per SM the persistent kernel is compiled for (the update needs ~200 registers)
static_assert(kBatchClusterCtas == MC_CS, "the host sizes the alpha partials for this cluster size");

__device__ __forceinline__ void cluster_sync_all() {
  cluster_arrive();
  cluster_wait();
}

size_t batch_persistent_smem(int hmax, int h1max) {
  return std::max(McLayout<float, 32, false>::bytes, bdev::pm_smem_bytes(hmax, h1max));
}

template <int ALG>
__global__ void __launch_bounds__(MC_NT, PB_MINB)
batch_solve_kernel(const BatchInst* __restrict__ tab, const int* __restrict__ clist,
                   const int* __restrict__ coff, int iters, double mu_eps, int pgd_steps,
                   int sched_l, int sched_r, int mode, int hcap, int h1cap,
                   double* __restrict__ sqpart, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char mc_smem[];
  __shared__ double sred[MC_NT / 32];
  // the contractions' staged column and partial sums use the start of the
  // dynamic area, which no other phase holds while they run
  float* hcol = reinterpret_cast<float*>(mc_smem);                  // <= 1024 floats
  float* cpart = reinterpret_cast<float*>(mc_smem + 1024 * sizeof(float));  // MC_NT floats
  const int q = (int)(blockIdx.x / MC_CS);
  const int c = (int)cluster_rank();
  const int t = threadIdx.x;
  for (int j = coff[q]; j < coff[q + 1]; ++j) {
    const int bi = clist[j];
    const BatchInst& b = tab[bi];
    const int R = b.R;
    const int64_t L = b.I[0] * b.I[1];
    const int I3 = (int)b.I[2];
    // this CTA's left items (row blocks of 2 MC_NT rows) and right items (slabs)
    const int nyl = (int)((L + 2 * MC_NT - 1) / (2 * MC_NT));
    const int yl0 = nyl * c / MC_CS, yl1 = nyl * (c + 1) / MC_CS;
    const int yr0 = I3 * c / MC_CS, yr1 = I3 * (c + 1) / MC_CS;
    auto item = [bi](int y) { return make_int2(bi, y); };
    if (mode != 0) {
      if (mode == 1) bdev::pm_left_run<MC_NT>(tab, item, yl0, yl1, sched_l, mc_smem);
      else bdev::pm_right_run<MC_NT>(tab, item, yr0, yr1, sched_r, mc_smem, hcap, h1cap);
      cluster_sync_all();
      continue;
    }
    {  // alpha: FP64 partial of this CTA's share of the elements, summed in CTA order
      const int64_t n = L * I3;
      const int64_t e0 = n * c / MC_CS, e1 = n * (c + 1) / MC_CS;
      double acc = 0.0;
#pragma unroll 4
      for (int64_t e = e0 + t; e < e1; e += MC_NT) {
        const float x = bdev::ldx(b, e);
        acc += (double)(x * x);
      }
      acc = warp_sum(acc);
      if ((t & 31) == 0) sred[t >> 5] = acc;
      __syncthreads();
      if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < MC_NT / 32; ++w) s += sred[w];
        sqpart[(size_t)bi * MC_CS + c] = s;
      }
    }
    for (int e = c * MC_NT + t; e < 3 * R * R; e += MC_CS * MC_NT)
      bdev::initial_gram_entry(b, e / (R * R), e % (R * R));
    if (c == 0 && t < 32) b.lam[t] = 1.0;  // lambda starts at 1
    cluster_sync_all();
    if (c == 0 && t == 0) {  // read next by this thread, in the mode-3 update
      double s = 0.0;
      for (int k = 0; k < MC_CS; ++k) s += __ldcg(sqpart + (size_t)bi * MC_CS + k);
      *b.alpha = s;
    }
    for (int it = 0; it < iters; ++it) {
      for (int n = 0; n < 3; ++n) {
        if (n == 0) {
          bdev::pm_left_run<MC_NT>(tab, item, yl0, yl1, sched_l, mc_smem);
          cluster_sync_all();
          for (int r = c; r < R; r += MC_CS) bdev::contract_rest_item<MC_NT>(b, r, hcol, cpart);
        } else if (n == 1) {
          for (int r = c; r < R; r += MC_CS) bdev::contract_first_item<MC_NT>(b, r, hcol);
        } else {
          bdev::pm_right_run<MC_NT>(tab, item, yr0, yr1, sched_r, mc_smem, hcap, h1cap);
        }
        cluster_sync_all();  // M^(n) complete
        mode_update_body<float, 32, ALG, true>((int)b.I[n], R, 3, n, b.G, b.Gf, b.M, b.H[n], b.lam,
                                               ALG, mu_eps, pgd_steps, 1e-30, b.inner + 3 * it + n,
                                               b.alpha, n == 2 ? b.hist + 3 * it : nullptr, err,
                                               nullptr, 0, 0.0);
        cluster_sync_all();  // H^(n), G^(n), lambda written
      }
    }
  }
}

template <int ALG>
cudaError_t run_batch_persistent(const BatchInst* tab, const int* clist, const int* coff,
                                 int nclusters, int iters, const planc_nls_opts& o, int sched_l,
                                 int sched_r, int mode, int hmax, int h1max, double* sqpart,
                                 int* err, cudaStream_t st) {
  const size_t smem = batch_persistent_smem(hmax, h1max);
  cudaError_t e = cudaFuncSetAttribute(batch_solve_kernel<ALG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(MC_CS * nclusters), 1, 1);
  cfg.blockDim = dim3(MC_NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = MC_CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, batch_solve_kernel<ALG>, tab, clist, coff, iters, o.mu_eps,
                         std::max(1, o.pgd_steps), sched_l, sched_r, mode, hmax, h1max, sqpart,
                         err);
  note_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int ALG>
int max_clusters_persistent(int hmax, int h1max) {
  const size_t smem = batch_persistent_smem(hmax, h1max);
  if (cudaFuncSetAttribute(batch_solve_kernel<ALG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(batch_solve_kernel<ALG>,
                           cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(MC_CS, 1, 1);
  cfg.blockDim = dim3(MC_NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = MC_CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, batch_solve_kernel<ALG>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}
}  // namespace

cudaError_t launch_mode_batch(const BatchInst* tab, int count, int n, int it, planc_nls_t alg,
                              const planc_nls_opts& o, int* err, cudaStream_t st) {
  const size_t smem = McLayout<float, 32>::bytes;
  cudaError_t e = cudaFuncSetAttribute(mode_cluster_batch_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(MC_CS * count), 1, 1);
  cfg.blockDim = dim3(MC_NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = MC_CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, mode_cluster_batch_kernel, tab, n, it, (int)alg, o.mu_eps,
                         std::max(1, o.pgd_steps), err);
  note_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

int mode_batch_max_rows() { return MC_CS * MC_RPC; }

int batch_persistent_max_clusters(planc_nls_t alg, int hmax, int h1max) {
  return alg == PLANC_MU    ? max_clusters_persistent<PLANC_MU>(hmax, h1max)
         : alg == PLANC_PGD ? max_clusters_persistent<PLANC_PGD>(hmax, h1max)
                            : max_clusters_persistent<PLANC_HALS>(hmax, h1max);
}

cudaError_t launch_batch_persistent(const BatchInst* tab, const int* clist, const int* coff,
                                    int nclusters, int iters, planc_nls_t alg,
                                    const planc_nls_opts& o, int sched_l, int sched_r, int mode,
                                    int hmax, int h1max, double* sqpart, int* err,
                                    cudaStream_t st) {
  if (alg == PLANC_MU)
    return run_batch_persistent<PLANC_MU>(tab, clist, coff, nclusters, iters, o, sched_l, sched_r,
                                          mode, hmax, h1max, sqpart, err, st);
  if (alg == PLANC_PGD)
    return run_batch_persistent<PLANC_PGD>(tab, clist, coff, nclusters, iters, o, sched_l, sched_r,
                                           mode, hmax, h1max, sqpart, err, st);
  if (alg == PLANC_HALS)
    return run_batch_persistent<PLANC_HALS>(tab, clist, coff, nclusters, iters, o, sched_l,
                                            sched_r, mode, hmax, h1max, sqpart, err, st);
  return cudaErrorInvalidValue;
}

bool mode_fused_eligible(planc_nls_t alg, int64_t rows, int R, bool f64) {
  // the Nesterov and ADMM steps hold four row vectors in registers: FP64 up
  // to R = 16
  const bool steps_ok = (alg == PLANC_NES || alg == PLANC_ADMM) && (!f64 || R <= 16);
  return (alg == PLANC_MU || alg == PLANC_HALS || alg == PLANC_PGD || alg == PLANC_UCP ||
          alg == PLANC_BPP || steps_ok) && rows >= 1 &&
         rows <= (int64_t)MC_CS * MC_RPC && R <= 32;
}

cudaError_t launch_mode_fused(bool f64, int64_t rows, int R, int N, int n, const double* G,
                              float* Gf, const void* M, void* H, double* lam, planc_nls_t alg,
                              const planc_nls_opts& o, int32_t* inner, const double* alpha,
                              double* fit_out, int* err, const double* nes_scr,
                              const RecArgs& rec, int* flags, cudaStream_t st) {
  const int r = (int)rows;
  double* Gw = const_cast<double*>(G);
  if (f64) {
    if (R <= 16)
      return run_mc<double, 16>(r, R, N, n, Gw, Gf, M, H, lam, alg, o, inner, alpha, fit_out, err,
                                nes_scr, rec, flags, st);
    return run_mc<double, 32>(r, R, N, n, Gw, Gf, M, H, lam, alg, o, inner, alpha, fit_out, err,
                              nes_scr, rec, flags, st);
  }
  if (R <= 16)
    return run_mc<float, 16>(r, R, N, n, Gw, Gf, M, H, lam, alg, o, inner, alpha, fit_out, err,
                             nes_scr, rec, flags, st);
  return run_mc<float, 32>(r, R, N, n, Gw, Gf, M, H, lam, alg, o, inner, alpha, fit_out, err,
                           nes_scr, rec, flags, st);
}

}  // namespace planc
