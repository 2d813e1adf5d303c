// Fused per-mode update for small factor matrices: everything of Alg. 1 /
// Alg. 4 that follows the MTTKRP for mode n,
//   S^(n) = Hadamard of the other Grams,
//   Hhat  = NNLS-Update(S^(n), M^(n)) with warm start H^(n) diag(lambda)
//           (MU, Eq. muupd; HALS, Eq. halsupd; projected gradient),
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

#include "internal.h"

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
// reciprocal-square-root seed refined by two Newton-Raphson steps
// y <- y (3 - s y^2) / 2, each of which squares the relative error; FP64
// sqrt and division are avoided because this GPU's FP64 pipe is narrow.
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
  y = y * (1.5 - 0.5 * s * y * y);
  l = s * y;
  il = y;
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

template <typename TA, int RP>
struct McLayout {
  static constexpr int NB = RP / 4;                     // 4-column blocks
  static constexpr int NBLK = NB * (NB + 1) / 2;        // upper-triangle 4x4 tiles
  static constexpr int RCN = MC_NT / NBLK;              // row chunks of the Gram
  static constexpr int NP = RP * (RP + 1) / 2;          // packed pairs r <= s
  static constexpr int NPO = (NP + MC_CS - 1) / MC_CS;  // pairs owned per CTA
  // scratch `red`: [0, MC_NT) column partials, then 4 beta and 4 gamma warp sums
  static constexpr int RED = MC_NT + 8;
  // byte offsets
  static constexpr size_t oSs = 0;
  static constexpr size_t oHs = oSs + sizeof(TA) * RP * RP;
  static constexpr size_t oMs = oHs + sizeof(TA) * MC_RPC * RP;
  static constexpr size_t oTp = oMs + sizeof(TA) * MC_RPC * RP;
  static constexpr size_t oCs = oTp + sizeof(TA) * RCN * NBLK * 16;
  static constexpr size_t oGs = oCs + sizeof(double) * MC_CS * RP;
  static constexpr size_t oBeta = oGs + sizeof(double) * MC_CS * NPO;
  static constexpr size_t oGam = oBeta + sizeof(double) * MC_CS;
  static constexpr size_t oRed = oGam + sizeof(double) * MC_CS;
  static constexpr size_t bytes = oRed + sizeof(double) * RED;
  static_assert(MC_NT % RP == 0 && MC_NT == MC_RPC, "one row per thread");
};

// G: the N Grams (FP64, R x R each), Gf: the same in FP32.  Mode n's entries
// of both are overwritten with G^(n) of the updated factor.
template <typename TA, int RP>
__global__ void __launch_bounds__(MC_NT, 1)
mode_cluster_kernel(int rows, int R, int N, int n, double* __restrict__ G,
                    float* __restrict__ Gf, const TA* __restrict__ M, TA* __restrict__ H,
                    double* __restrict__ lam, int alg, double mu_eps, int pgd_steps, double tiny,
                    int32_t* __restrict__ inner, const double* __restrict__ alpha,
                    double* __restrict__ fit_out) {
  using L = McLayout<TA, RP>;
  using S = Swz<TA, RP>;
  extern __shared__ __align__(16) unsigned char mc_smem[];
  TA* Ss = reinterpret_cast<TA*>(mc_smem + L::oSs);                 // S^(n), RP x RP
  TA* Hs = reinterpret_cast<TA*>(mc_smem + L::oHs);                 // this CTA's rows
  TA* Ms = reinterpret_cast<TA*>(mc_smem + L::oMs);                 // its rows of M
  TA* tp = reinterpret_cast<TA*>(mc_smem + L::oTp);                 // Gram tile partials
  double* cs_slot = reinterpret_cast<double*>(mc_smem + L::oCs);    // [src CTA][r]
  double* g_slot = reinterpret_cast<double*>(mc_smem + L::oGs);     // [src CTA][owned pair]
  double* beta_slot = reinterpret_cast<double*>(mc_smem + L::oBeta);  // [src CTA] (CTA 0)
  double* gam_slot = reinterpret_cast<double*>(mc_smem + L::oGam);    // [src CTA] (CTA 0)
  double* red = reinterpret_cast<double*>(mc_smem + L::oRed);
  __shared__ double s_lam[RP];
  __shared__ TA s_lamt[RP], s_inv[RP];
  __shared__ TA s_rinv[RP];  // 1 / S(r, r), or 0 where S(r, r) <= tiny (column kept)
  __shared__ TA s_eta;
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

  // every CTA of the cluster must be running before any remote store
  cluster_arrive_relaxed();

  // ---- every global load of the prologue is issued up front: this CTA's
  // rows of M and H (coalesced), lambda, and the other Grams
  constexpr int LPT = MC_RPC * RP / MC_NT;  // staged elements per thread
  constexpr int EPT = RP * RP / MC_NT;      // entries of S per thread
  TA mv[LPT], hv[LPT];
#pragma unroll
  for (int j = 0; j < LPT; ++j) {
    const int e = t + j * MC_NT;
    mv[j] = e < nel ? M[(size_t)row0 * R + e] : TA(0);
    hv[j] = e < nel ? H[(size_t)row0 * R + e] : TA(0);
  }
  const double lam_t = t < R ? lam[t] : 0.0;
  // S^(n) = Hadamard of the other Grams, in TA (from the FP32 copies when TA
  // is FP32); entry (i, k) of S for e = t + j * MC_NT
  TA v[EPT];
  int off[EPT];
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int e = t + j * MC_NT, i = e / RP, k = e % RP;
    const bool in = i < R && k < R;
    v[j] = in ? TA(1) : TA(0);
    off[j] = in ? i * R + k : 0;
  }
#pragma unroll 4
  for (int qi = 0; qi + 1 < N; ++qi) {
    const size_t q = (size_t)(qi < n ? qi : qi + 1);
    TA g[EPT];
    if constexpr (sizeof(TA) == 4) {
#pragma unroll
      for (int j = 0; j < EPT; ++j) g[j] = Gf[q * RR + off[j]];
    } else {
#pragma unroll
      for (int j = 0; j < EPT; ++j) g[j] = G[q * RR + off[j]];
    }
#pragma unroll
    for (int j = 0; j < EPT; ++j) v[j] *= g[j];
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
  // staged rows; padding rows are zero (mv = hv = 0 past nel)
  {
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
      h[g * S::VPG + u] = hs[u] * s_lamt[g * S::VPG + u];  // warm start H diag(lambda)
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
  if ((t & 31) == 0) red[MC_NT + (t >> 5)] = bw;
  __syncthreads();

  // ---- column sums of squares of this CTA's rows: thread (r, chunk)
  constexpr int CH = MC_NT / RP;
  {
    constexpr int RPCH = MC_RPC / CH;
    const int r = t % RP, ch = t / RP;
    TA a = TA(0);
    for (int i = ch * RPCH; i < (ch + 1) * RPCH; ++i) {
      const TA x = Hs[S::idx(i, r)];
      a = fma(x, x, a);
    }
    red[ch * RP + r] = (double)a;
  }
  __syncthreads();
  cluster_wait();  // pairs with the arrive at kernel start: every CTA is running
  if (t < RP) {
    double s = 0.0;
    for (int ch = 0; ch < CH; ++ch) s += red[ch * RP + t];
    for (uint32_t dst = 0; dst < MC_CS; ++dst) st_cluster(cs_slot + c * RP + t, dst, s);
  }
  if (t == 0) {
    double b = 0.0;
    for (int w = 0; w < MC_NT / 32; ++w) b += red[MC_NT + w];
    st_cluster(beta_slot + c, 0, b);
  }
  cluster_arrive();
  cluster_wait();

  // ---- lambda (identical in every CTA: same slots, same order)
  if (t < RP) {
    double s = 0.0;
    for (int src = 0; src < MC_CS; ++src) s += cs_slot[src * RP + t];
    double l = 0.0, il = 0.0;  // a zero column keeps lambda = 0 and stays zero
    if (t < R) sqrt_and_inv(s, l, il);
    s_lam[t] = l;
    s_inv[t] = (TA)il;
    if (c == 0 && t < R) lam[t] = l;
  }
  __syncthreads();
  // ---- normalise this CTA's rows: H = Hhat diag(lambda)^-1
#pragma unroll
  for (int g = 0; g < S::GR; ++g) {
    TA* p = Hs + S::gidx(t, g);
#pragma unroll
    for (int u = 0; u < S::VPG; ++u) p[u] *= s_inv[g * S::VPG + u];
  }
  __syncthreads();
  {
    int a = a_0, k = k_0;
#pragma unroll 4
    for (int e = t; e < nel; e += MC_NT) {  // coalesced write of the R live columns
      H[(size_t)row0 * R + e] = Hs[S::idx(a, k)];
      a += q_step;
      k += k_step;
      if (k >= R) {
        k -= R;
        ++a;
      }
    }
  }

  // ---- Gram partial of this CTA: 4x4 tiles (rb <= sb) x row chunks, in TA
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
  // combine the chunks (in TA) and push each pair to its owner CTA (p % MC_CS)
  for (int p = t; p < L::NP; p += MC_NT) {
    int r, s;
    tri_unpack(p, RP, r, s);
    const int blk = tri_index(r / 4, s / 4, L::NB), e = (r % 4) * 4 + (s % 4);
    TA ga = TA(0);
    for (int ch = 0; ch < L::RCN; ++ch) ga += tp[(ch * L::NBLK + blk) * 16 + e];
    st_cluster(g_slot + c * L::NPO + p / MC_CS, (uint32_t)(p % MC_CS), (double)ga);
  }
  cluster_arrive();
  cluster_wait();

  // ---- owned pairs: G^(n) entries (FP64 across the CTAs), and the gamma
  // partial of the error identity with the FP64 entry of S^(n)
  double gam = 0.0;
  double* Gn = G + (size_t)n * RR;
  float* Gnf = Gf + (size_t)n * RR;
  for (int j = t; j < L::NPO; j += MC_NT) {
    const int p = j * MC_CS + (int)c;
    if (p >= L::NP) break;
    int r, s;
    tri_unpack(p, RP, r, s);
    if (s >= R) continue;
    double g = 0.0;
    for (int src = 0; src < MC_CS; ++src) g += g_slot[src * L::NPO + j];
    Gn[r * R + s] = g;
    Gn[s * R + r] = g;
    Gnf[r * R + s] = (float)g;
    Gnf[s * R + r] = (float)g;
    if (fit_out) {
      double sv = 1.0;
      for (int q = 0; q < N; ++q)
        if (q != n) sv *= G[(size_t)q * RR + r * R + s];
      gam += (r == s ? 1.0 : 2.0) * s_lam[r] * s_lam[s] * sv * g;
    }
  }
  if (c == 0 && t == 0 && inner) *inner = alg == PLANC_PGD ? pgd_steps : 1;
  if (!fit_out) return;  // uniform over the cluster: no remote access follows
  gam = warp_sum(gam);
  if ((t & 31) == 0) red[MC_NT + 4 + (t >> 5)] = gam;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < MC_NT / 32; ++w) s += red[MC_NT + 4 + w];
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
    const double a = *alpha;
    const double rad = a - 2.0 * beta + gamma;
    const double eps = a > 0.0 ? sqrt(fmax(0.0, rad) / a) : 0.0;
    fit_out[0] = eps;
    fit_out[1] = beta;
    fit_out[2] = gamma;
  }
}

template <typename TA, int RP>
cudaError_t run_mc(int rows, int R, int N, int n, double* G, float* Gf, const void* M, void* H,
                   double* lam, planc_nls_t alg, const planc_nls_opts& o, int32_t* inner,
                   const double* alpha, double* fit_out, cudaStream_t st) {
  const size_t smem = McLayout<TA, RP>::bytes;
  auto kern = mode_cluster_kernel<TA, RP>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(MC_CS, 1, 1);
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
  e = cudaLaunchKernelEx(&cfg, kern, rows, R, N, n, G, Gf, (const TA*)M, (TA*)H, lam, (int)alg,
                         o.mu_eps, std::max(1, o.pgd_steps), sizeof(TA) == 8 ? 1e-300 : 1e-30,
                         inner, alpha, fit_out);
  note_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

bool mode_fused_eligible(planc_nls_t alg, int64_t rows, int R) {
  return (alg == PLANC_MU || alg == PLANC_HALS || alg == PLANC_PGD) && rows >= 1 &&
         rows <= (int64_t)MC_CS * MC_RPC && R <= 32;
}

cudaError_t launch_mode_fused(bool f64, int64_t rows, int R, int N, int n, const double* G,
                              float* Gf, const void* M, void* H, double* lam, planc_nls_t alg,
                              const planc_nls_opts& o, int32_t* inner, const double* alpha,
                              double* fit_out, cudaStream_t st) {
  const int r = (int)rows;
  double* Gw = const_cast<double*>(G);
  if (f64) {
    if (R <= 16)
      return run_mc<double, 16>(r, R, N, n, Gw, Gf, M, H, lam, alg, o, inner, alpha, fit_out, st);
    return run_mc<double, 32>(r, R, N, n, Gw, Gf, M, H, lam, alg, o, inner, alpha, fit_out, st);
  }
  if (R <= 16)
    return run_mc<float, 16>(r, R, N, n, Gw, Gf, M, H, lam, alg, o, inner, alpha, fit_out, st);
  return run_mc<float, 32>(r, R, N, n, Gw, Gf, M, H, lam, alg, o, inner, alpha, fit_out, st);
}

}  // namespace planc
