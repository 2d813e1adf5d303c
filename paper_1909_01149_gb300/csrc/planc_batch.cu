// planc_batch_solve: many independent 3-way NNCP instances advanced together.
//
// Default (opts.batch_persistent): the whole solve is ONE persistent launch of
// thread-block clusters, each cluster solving whole instances in turn; the
// instances are dealt to the clusters longest-first onto the least-loaded
// cluster (LPT), by an estimate of each instance's work.  Otherwise every
// phase of an outer iteration is one launch over all instances (work tables
// of (instance, tile) items built here).  With opts.use_graph the launch
// sequence (one node, or all phases of all outer iterations) is captured once
// and launched as a CUDA graph.  The schedule (rank blocking of both partial
// MTTKRPs; for the per-phase launches also their tile shapes) is picked by
// timing the candidates on the batch itself the first time a batch of that
// signature is seen (the choice is cached for the process).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace planc {

cudaError_t launch_batch_sqnorm(const BatchInst* tab, int count, const int2* items, int nitems,
                                const int* first, double* part, int sm_count, cudaStream_t st);
cudaError_t launch_batch_gram(const BatchInst* tab, int count, cudaStream_t st);
cudaError_t launch_batch_pm_left(const BatchInst* tab, const int2* items, const int64_t* cumw,
                                 int nitems, int tl, int hmax, int sched, int sm_count,
                                 cudaStream_t st);
cudaError_t launch_batch_pm_right(const BatchInst* tab, const int2* items, const int64_t* cumw,
                                  int nitems, int nt, int hmax, int h1max, int sched, int sm_count,
                                  cudaStream_t st);
size_t batch_pm_smem(int hmax, int h1max);
cudaError_t launch_batch_contract(const BatchInst* tab, const int2* items, int nitems, bool rest,
                                  int sm_count, cudaStream_t st);

namespace {

constexpr int kTL[3] = {64, 128, 256};
constexpr int kNT[3] = {64, 128, 256};

struct TuneKey {
  int count;
  long long elems, rank_sum;
  int bf16_count;  // storage dtype mix (BF16 instances): tuned separately
  bool operator<(const TuneKey& o) const {
    return std::tie(count, elems, rank_sum, bf16_count) <
           std::tie(o.count, o.elems, o.rank_sum, o.bf16_count);
  }
};
// the schedule of the two partial MTTKRPs: tile candidate indices and rank
// blocking (0: every rank padded to 32; 1: classes 16, 32; 2: 8, 16, 32)
struct TuneChoice {
  int tl = 1, nt = 1, sched_left = 2, sched_right = 2;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune;    // per-phase launches
std::map<TuneKey, TuneChoice> g_tune_p;  // persistent launch (rank blocking only)
thread_local TuneChoice t_last_choice;
constexpr int kSchedules = 3;

struct Alloc {
  void* p = nullptr;
  ~Alloc() {
    if (p) cudaFree(p);
  }
};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// The persistent launch's deal of the instances to its clusters.  An
// instance's estimated cost per outer iteration is its partial-MTTKRP FMAs
// (elements x the two padded ranks, rank classes 8 / 16 / 32) plus a fixed
// share for the latency of its phases (about the FMAs of 8e6 at the rate of
// one cluster); instances are taken longest-first (ties in index order), each
// onto the least-loaded cluster (the lowest index on ties).  clist: count
// entries, cluster q's instances clist[coff[q]] .. clist[coff[q + 1] - 1];
// coff: nclusters + 1 entries; load (optional): the clusters' summed costs.
void batch_deal(const planc_batch_instance* inst, int count, int nclusters, int* clist, int* coff,
                double* load_out) {
  std::vector<double> cost(count);
  for (int b = 0; b < count; ++b) {
    const int R = inst[b].R;
    const double rc = R <= 8 ? 8.0 : R <= 16 ? 16.0 : 32.0;
    cost[b] = (double)(inst[b].dims[0] * inst[b].dims[1] * inst[b].dims[2]) * 2.0 * rc + 8e6;
  }
  std::vector<int> order(count);
  for (int b = 0; b < count; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<std::vector<int>> lists(nclusters);
  std::vector<double> load(nclusters, 0.0);
  for (int b : order) {
    int q = 0;
    for (int k = 1; k < nclusters; ++k)
      if (load[k] < load[q]) q = k;
    lists[q].push_back(b);
    load[q] += cost[b];
  }
  int n = 0;
  coff[0] = 0;
  for (int q = 0; q < nclusters; ++q) {
    for (int b : lists[q]) clist[n++] = b;
    coff[q + 1] = n;
    if (load_out) load_out[q] = load[q];
  }
}

planc_status_t bfail(planc_status_t st, const char* msg) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "planc_batch_solve: %s", msg);
  set_thread_error(buf);
  return st;
}

}  // namespace

}  // namespace planc

using namespace planc;

extern "C" planc_status_t planc_batch_solve(planc_batch_instance* inst, int count,
                                            const planc_solve_opts* opts, void* cuda_stream,
                                            planc_report* report) {
  if (!inst || count < 1 || !opts) return bfail(PLANC_E_INVALID, "bad arguments");
  const planc_solve_opts o = *opts;
  if (o.iters < 1 || o.iters > 100000) return bfail(PLANC_E_INVALID, "iters out of range");
  if (o.alg != PLANC_MU && o.alg != PLANC_HALS && o.alg != PLANC_PGD)
    return bfail(PLANC_E_UNSUPPORTED, "batched solve supports MU, HALS and PGD");
  const int maxrows = mode_batch_max_rows();
  int64_t maxC = 1, maxI2 = 1, maxI1 = 1;
  for (int b = 0; b < count; ++b) {
    const planc_batch_instance& in = inst[b];
    if (!in.X || !in.H[0] || !in.H[1] || !in.H[2]) return bfail(PLANC_E_INVALID, "NULL pointer");
    if (in.R < 1 || in.R > 32) return bfail(PLANC_E_SHAPE, "R must be 1..32");
    for (int n = 0; n < 3; ++n)
      if (in.dims[n] < 1 || in.dims[n] > maxrows) return bfail(PLANC_E_SHAPE, "dims must be 1..1024");
    if (in.x_dtype != PLANC_F32 && in.x_dtype != PLANC_BF16)
      return bfail(PLANC_E_DTYPE, "X must be F32 or BF16");
    if (reinterpret_cast<uintptr_t>(in.X) & 15u)
      return bfail(PLANC_E_INVALID, "X must start on a 16-byte boundary");
    maxC = std::max(maxC, in.dims[2]);
    maxI2 = std::max(maxI2, in.dims[1]);
    maxI1 = std::max(maxI1, in.dims[0]);
  }
  // graph capture needs a stream other than the legacy default stream
  struct OwnStream {
    cudaStream_t s = nullptr;
    ~OwnStream() {
      if (s) cudaStreamDestroy(s);
    }
  } own;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (st == nullptr) {
    if (cudaStreamCreateWithFlags(&own.s, cudaStreamNonBlocking) != cudaSuccess)
      return bfail(PLANC_E_CUDA, "stream creation failed");
    st = own.s;
  }
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return bfail(PLANC_E_CUDA, "no device");
  const int iters = o.iters;

  // ---- workspace: per-instance arrays, work tables, instance table
  std::vector<size_t> offT(count), offM(count), offG(count), offGf(count), offAlpha(count);
  size_t bytes = 0;
  for (int b = 0; b < count; ++b) {
    const planc_batch_instance& in = inst[b];
    const size_t L = (size_t)in.dims[0] * in.dims[1];
    const size_t R = in.R;
    const size_t maxI = std::max({in.dims[0], in.dims[1], in.dims[2]});
    offT[b] = bytes; bytes += align256(L * R * 4);
    offM[b] = bytes; bytes += align256(maxI * R * 4);
    offG[b] = bytes; bytes += align256(3 * R * R * 8);
    offGf[b] = bytes; bytes += align256(3 * R * R * 4);
    offAlpha[b] = bytes; bytes += 256;
  }
  // every instance's error history, inner counts and lambda, contiguous (one
  // clear and one copy back each)
  const size_t hist_per = (size_t)iters * 3;
  const size_t off_hist = bytes; bytes += align256(sizeof(double) * hist_per * count);
  const size_t off_inner = bytes; bytes += align256(sizeof(int32_t) * hist_per * count);
  const size_t off_lam = bytes; bytes += align256(sizeof(double) * 32 * count);
  // work tables; the partial-MTTKRP tables list the instances in rank order,
  // so that a CTA's contiguous run of items stays within one rank class
  std::vector<int> by_rank(count);
  for (int b = 0; b < count; ++b) by_rank[b] = b;
  std::stable_sort(by_rank.begin(), by_rank.end(),
                   [&](int a, int b) { return inst[a].R < inst[b].R; });
  std::vector<int2> sq_items, right_items, rc_items;
  std::vector<int> sq_first(count + 1, 0);
  for (int b = 0; b < count; ++b) {
    const int64_t n = inst[b].dims[0] * inst[b].dims[1] * inst[b].dims[2];
    sq_first[b] = (int)sq_items.size();
    for (int64_t c = 0; c * 65536 < n; ++c) sq_items.push_back(make_int2(b, (int)c));
    for (int r = 0; r < inst[b].R; ++r) rc_items.push_back(make_int2(b, r));
  }
  for (int b : by_rank)
    for (int64_t c = 0; c < inst[b].dims[2]; ++c) right_items.push_back(make_int2(b, (int)c));
  sq_first[count] = (int)sq_items.size();
  // prefix sums of the items' element counts: each CTA of the partial
  // MTTKRPs takes a contiguous run with an equal share of the elements
  std::vector<int64_t> right_cum(1, 0);
  for (int b : by_rank)
    for (int64_t c = 0; c < inst[b].dims[2]; ++c)
      right_cum.push_back(right_cum.back() + inst[b].dims[0] * inst[b].dims[1]);
  std::vector<int2> left_items[3];
  std::vector<int64_t> left_cum[3];
  for (int t = 0; t < 3; ++t) {
    left_cum[t].push_back(0);
    for (int b : by_rank) {
      const int64_t L = inst[b].dims[0] * inst[b].dims[1];
      for (int64_t y = 0; y * 2 * kTL[t] < L; ++y) {
        left_items[t].push_back(make_int2(b, (int)y));
        const int64_t rows = std::min<int64_t>(2 * kTL[t], L - y * 2 * kTL[t]);
        left_cum[t].push_back(left_cum[t].back() + rows * inst[b].dims[2]);
      }
    }
  }
  const size_t off_tab = bytes; bytes += align256(sizeof(BatchInst) * count);
  const size_t off_sq = bytes; bytes += align256(sizeof(int2) * sq_items.size());
  const size_t off_sqf = bytes; bytes += align256(sizeof(int) * (count + 1));
  const size_t off_sqp = bytes; bytes += align256(sizeof(double) * sq_items.size());
  const size_t off_right = bytes; bytes += align256(sizeof(int2) * right_items.size());
  const size_t off_rc = bytes; bytes += align256(sizeof(int2) * rc_items.size());
  const size_t off_rcum = bytes; bytes += align256(sizeof(int64_t) * right_cum.size());
  size_t off_left[3], off_lcum[3];
  for (int t = 0; t < 3; ++t) {
    off_left[t] = bytes;
    bytes += align256(sizeof(int2) * left_items[t].size());
    off_lcum[t] = bytes;
    bytes += align256(sizeof(int64_t) * left_cum[t].size());
  }
  const size_t off_err = bytes; bytes += 256;
  // persistent launch: alpha partials, and the instances dealt to the clusters
  const size_t off_sqpart = bytes; bytes += align256(sizeof(double) * kBatchClusterCtas * count);
  const size_t off_clist = bytes; bytes += align256(sizeof(int) * count);
  const size_t off_coff = bytes; bytes += align256(sizeof(int) * (count + 1));

  Alloc ws;
  if (cudaMalloc(&ws.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return bfail(PLANC_E_NOMEM, "workspace allocation failed");
  }
  char* base = static_cast<char*>(ws.p);
  std::vector<BatchInst> tab(count);
  for (int b = 0; b < count; ++b) {
    const planc_batch_instance& in = inst[b];
    BatchInst& t = tab[b];
    t.X = in.X;
    for (int n = 0; n < 3; ++n) {
      t.I[n] = in.dims[n];
      t.H[n] = static_cast<float*>(in.H[n]);
    }
    t.R = in.R;
    t.xbf16 = in.x_dtype == PLANC_BF16 ? 1 : 0;
    t.T = reinterpret_cast<float*>(base + offT[b]);
    t.M = reinterpret_cast<float*>(base + offM[b]);
    t.G = reinterpret_cast<double*>(base + offG[b]);
    t.Gf = reinterpret_cast<float*>(base + offGf[b]);
    t.lam = reinterpret_cast<double*>(base + off_lam) + (size_t)32 * b;
    t.alpha = reinterpret_cast<double*>(base + offAlpha[b]);
    t.hist = reinterpret_cast<double*>(base + off_hist) + hist_per * b;
    t.inner = reinterpret_cast<int32_t*>(base + off_inner) + hist_per * b;
  }
  const BatchInst* d_tab = reinterpret_cast<const BatchInst*>(base + off_tab);
  const int2* d_sq = reinterpret_cast<const int2*>(base + off_sq);
  const int* d_sqf = reinterpret_cast<const int*>(base + off_sqf);
  double* d_sqp = reinterpret_cast<double*>(base + off_sqp);
  const int2* d_right = reinterpret_cast<const int2*>(base + off_right);
  const int2* d_rc = reinterpret_cast<const int2*>(base + off_rc);
  int* d_err = reinterpret_cast<int*>(base + off_err);
  auto h2d = [&](size_t off, const void* src, size_t n) {
    return cudaMemcpyAsync(base + off, src, n, cudaMemcpyHostToDevice, st);
  };
  if (h2d(off_tab, tab.data(), sizeof(BatchInst) * count) != cudaSuccess ||
      h2d(off_sq, sq_items.data(), sizeof(int2) * sq_items.size()) != cudaSuccess ||
      h2d(off_sqf, sq_first.data(), sizeof(int) * (count + 1)) != cudaSuccess ||
      h2d(off_right, right_items.data(), sizeof(int2) * right_items.size()) != cudaSuccess ||
      h2d(off_rc, rc_items.data(), sizeof(int2) * rc_items.size()) != cudaSuccess ||
      h2d(off_rcum, right_cum.data(), sizeof(int64_t) * right_cum.size()) != cudaSuccess ||
      cudaMemsetAsync(base + off_err, 0, 256, st) != cudaSuccess)
    return bfail(PLANC_E_CUDA, "table upload failed");
  for (int t = 0; t < 3; ++t)
    if (h2d(off_left[t], left_items[t].data(), sizeof(int2) * left_items[t].size()) != cudaSuccess ||
        h2d(off_lcum[t], left_cum[t].data(), sizeof(int64_t) * left_cum[t].size()) != cudaSuccess)
      return bfail(PLANC_E_CUDA, "table upload failed");
  if (cudaMemsetAsync(base + off_hist, 0, sizeof(double) * hist_per * count, st) != cudaSuccess)
    return bfail(PLANC_E_CUDA, "memset failed");

  const int hmax_left = (int)maxC, hmax_right = (int)maxI2;
  if (batch_pm_smem(std::max(hmax_left, hmax_right), 0) > 227 * 1024)
    return bfail(PLANC_E_SHAPE, "a mode is too long for the staged factor");
  // the right branch also stages H1 when it fits next to H2 (otherwise its
  // epilogue reads H1 from global memory)
  constexpr size_t kStageBudget = 160 * 1024;
  const int h1max_right = batch_pm_smem(hmax_right, (int)maxI1) <= kStageBudget ? (int)maxI1 : 0;
  const int64_t* d_rcum = reinterpret_cast<const int64_t*>(base + off_rcum);
  const int nleft[3] = {(int)left_items[0].size(), (int)left_items[1].size(),
                        (int)left_items[2].size()};
  const int nright = (int)right_items.size(), nrc = (int)rc_items.size();

  // ---- the persistent launch: clusters that fit at once, instances dealt
  // longest-first onto the least-loaded cluster (batch_deal)
  const bool persistent = o.batch_persistent != 0;
  const int hmax_p = (int)std::max(maxC, maxI2);
  const int h1max_p = batch_pm_smem(hmax_p, (int)maxI1) <= kStageBudget ? (int)maxI1 : 0;
  int nclusters = 0;
  if (persistent) {
    nclusters = std::min(count, batch_persistent_max_clusters(o.alg, hmax_p, h1max_p));
    if (nclusters < 1) return bfail(PLANC_E_CUDA, "the persistent launch does not fit on this GPU");
    std::vector<int> clist(count), coff(nclusters + 1);
    batch_deal(inst, count, nclusters, clist.data(), coff.data(), nullptr);
    if (h2d(off_clist, clist.data(), sizeof(int) * count) != cudaSuccess ||
        h2d(off_coff, coff.data(), sizeof(int) * (nclusters + 1)) != cudaSuccess)
      return bfail(PLANC_E_CUDA, "table upload failed");
  }
  const int* d_clist = reinterpret_cast<const int*>(base + off_clist);
  const int* d_coff = reinterpret_cast<const int*>(base + off_coff);
  double* d_sqpart = reinterpret_cast<double*>(base + off_sqpart);

  // ---- schedule: every candidate of each partial MTTKRP timed on this batch
  // (second of two runs), cached per batch signature.  Per-phase launches:
  // (tile, rank blocking) of each kernel; persistent launch: the rank
  // blocking of each branch (the launch run with only that branch).
  TuneKey key{count, 0, 0, 0};
  for (int b = 0; b < count; ++b) {
    key.elems += inst[b].dims[0] * inst[b].dims[1] * inst[b].dims[2];
    key.rank_sum += inst[b].R;
    key.bf16_count += inst[b].x_dtype == PLANC_BF16 ? 1 : 0;
  }
  std::map<TuneKey, TuneChoice>& cache = persistent ? g_tune_p : g_tune;
  TuneChoice ch;
  bool tuned = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      ch = it->second;
      tuned = true;
    }
  }
  if (!tuned) {
    struct Events {  // released on every return path
      cudaEvent_t e[2] = {nullptr, nullptr};
      ~Events() {
        for (cudaEvent_t x : e)
          if (x) cudaEventDestroy(x);
      }
    } ev;
    if (cudaEventCreate(&ev.e[0]) != cudaSuccess || cudaEventCreate(&ev.e[1]) != cudaSuccess)
      return bfail(PLANC_E_CUDA, "event creation failed");
    const cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
    float best_l = 1e30f, best_r = 1e30f;
    auto time_it = [&](auto&& launch, float& ms) -> bool {
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, st);
        const cudaError_t ce = launch();
        cudaEventRecord(e1, st);
        if (ce != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return false;
        cudaEventElapsedTime(&ms, e0, e1);
      }
      return true;
    };
    if (persistent) {
      ch.tl = 1;  // 128 threads per CTA, two rows each (fixed by the launch)
      ch.nt = 1;
      for (int sc = 0; sc < kSchedules; ++sc) {
        float ms = 0.f;
        if (!time_it([&] { return launch_batch_persistent(d_tab, d_clist, d_coff, nclusters, 1,
                                                          o.alg, o.nls, sc, sc, 1, hmax_p,
                                                          h1max_p, d_sqpart, d_err, st); }, ms))
          return bfail(PLANC_E_CUDA, "tuning launch failed");
        if (ms < best_l) { best_l = ms; ch.sched_left = sc; }
        if (!time_it([&] { return launch_batch_persistent(d_tab, d_clist, d_coff, nclusters, 1,
                                                          o.alg, o.nls, sc, sc, 2, hmax_p,
                                                          h1max_p, d_sqpart, d_err, st); }, ms))
          return bfail(PLANC_E_CUDA, "tuning launch failed");
        if (ms < best_r) { best_r = ms; ch.sched_right = sc; }
      }
    } else {
      for (int t = 0; t < 3; ++t)
        for (int sc = 0; sc < kSchedules; ++sc) {
          const int2* items = reinterpret_cast<const int2*>(base + off_left[t]);
          const int64_t* lcum = reinterpret_cast<const int64_t*>(base + off_lcum[t]);
          float ms = 0.f;
          if (!time_it([&] { return launch_batch_pm_left(d_tab, items, lcum, nleft[t], kTL[t],
                                                         hmax_left, sc, sms, st); }, ms))
            return bfail(PLANC_E_CUDA, "tuning launch failed");
          if (ms < best_l) { best_l = ms; ch.tl = t; ch.sched_left = sc; }
          if (!time_it([&] { return launch_batch_pm_right(d_tab, d_right, d_rcum, nright, kNT[t],
                                                          hmax_right, h1max_right, sc, sms,
                                                          st); }, ms))
            return bfail(PLANC_E_CUDA, "tuning launch failed");
          if (ms < best_r) { best_r = ms; ch.nt = t; ch.sched_right = sc; }
        }
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    cache[key] = ch;
  }
  // PLANC_BATCH_RANK_BLOCKING="l,r" forces the rank blocking of the two
  // kernels (tests compare every schedule; the tile choice stays tuned)
  if (const char* env = std::getenv("PLANC_BATCH_RANK_BLOCKING")) {
    int l = -1, r = -1;
    if (std::sscanf(env, "%d,%d", &l, &r) == 2 && l >= 0 && l < kSchedules && r >= 0 &&
        r < kSchedules) {
      ch.sched_left = l;
      ch.sched_right = r;
    }
  }
  t_last_choice = ch;
  const int tl_idx = ch.tl;
  const int2* d_left = reinterpret_cast<const int2*>(base + off_left[tl_idx]);
  const int64_t* d_lcum = reinterpret_cast<const int64_t*>(base + off_lcum[tl_idx]);
  const int tl = kTL[tl_idx], nt = kNT[ch.nt];

  const long long c_start = launch_count();
  // ---- the solve as a launch sequence
  auto enqueue = [&]() -> cudaError_t {
    if (persistent)
      return launch_batch_persistent(d_tab, d_clist, d_coff, nclusters, iters, o.alg, o.nls,
                                     ch.sched_left, ch.sched_right, 0, hmax_p, h1max_p, d_sqpart,
                                     d_err, st);
    cudaError_t e;
    if ((e = launch_batch_sqnorm(d_tab, count, d_sq, (int)sq_items.size(), d_sqf, d_sqp, sms, st)) != cudaSuccess) return e;
    if ((e = launch_batch_gram(d_tab, count, st)) != cudaSuccess) return e;
    for (int it = 0; it < iters; ++it) {
      if ((e = launch_batch_pm_left(d_tab, d_left, d_lcum, nleft[tl_idx], tl, hmax_left, ch.sched_left, sms, st)) != cudaSuccess) return e;
      if ((e = launch_batch_contract(d_tab, d_rc, nrc, true, sms, st)) != cudaSuccess) return e;
      if ((e = launch_mode_batch(d_tab, count, 0, it, o.alg, o.nls, d_err, st)) != cudaSuccess) return e;
      if ((e = launch_batch_contract(d_tab, d_rc, nrc, false, sms, st)) != cudaSuccess) return e;
      if ((e = launch_mode_batch(d_tab, count, 1, it, o.alg, o.nls, d_err, st)) != cudaSuccess) return e;
      if ((e = launch_batch_pm_right(d_tab, d_right, d_rcum, nright, nt, hmax_right, h1max_right, ch.sched_right, sms, st)) != cudaSuccess) return e;
      if ((e = launch_mode_batch(d_tab, count, 2, it, o.alg, o.nls, d_err, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  cudaError_t ce;
  if (o.use_graph) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      const cudaError_t ee = enqueue();
      ce = cudaStreamEndCapture(st, &g);
      if (ee != cudaSuccess) ce = ee;
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&ge, g, 0);
    if (ce == cudaSuccess) ce = cudaGraphLaunch(ge, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
  } else {
    ce = enqueue();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  }
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return bfail(PLANC_E_CUDA, cudaGetErrorString(ce));
  }
  const long long launches = launch_count() - c_start;

  // ---- results (one copy of every history, one of every lambda)
  int err = 0;
  std::vector<double> hist(hist_per * count), lam((size_t)32 * count);
  if (cudaMemcpy(&err, d_err, sizeof err, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hist.data(), base + off_hist, hist.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(lam.data(), base + off_lam, lam.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return bfail(PLANC_E_CUDA, "D2H failed");
  double worst = 0.0;
  for (int b = 0; b < count; ++b) {
    const double* hb = hist.data() + hist_per * b;
    inst[b].rel_err = hb[3 * (iters - 1)];
    worst = std::max(worst, inst[b].rel_err);
    if (inst[b].rel_err_hist)
      for (int i = 0; i < iters; ++i) inst[b].rel_err_hist[i] = hb[3 * i];
    if (inst[b].lambda)
      for (int r = 0; r < inst[b].R; ++r) inst[b].lambda[r] = lam[(size_t)32 * b + r];
  }
  if (report) {
    std::memset(report, 0, sizeof *report);
    report->iters_done = iters;
    report->rel_err = worst;
    report->fit = 1.0 - worst;
    report->launches = launches;
  }
  if (err != 0) return bfail(PLANC_E_TIMEOUT, "a bounded wait in the mode update gave up");
  return PLANC_OK;
}

extern "C" planc_status_t planc_batch_plan(const planc_batch_instance* inst, int count,
                                           int nclusters, int* clist, int* coff, double* load) {
  if (!inst || !clist || !coff || count < 1) return bfail(PLANC_E_INVALID, "bad arguments");
  if (nclusters < 1 || nclusters > count) return bfail(PLANC_E_INVALID, "nclusters must be 1..count");
  for (int b = 0; b < count; ++b) {
    if (inst[b].R < 1) return bfail(PLANC_E_SHAPE, "R must be >= 1");
    for (int n = 0; n < 3; ++n)
      if (inst[b].dims[n] < 1) return bfail(PLANC_E_SHAPE, "dims must be >= 1");
  }
  planc::batch_deal(inst, count, nclusters, clist, coff, load);
  return PLANC_OK;
}

extern "C" planc_status_t planc_batch_schedule(int* out) {
  if (!out) return PLANC_E_INVALID;
  const planc::TuneChoice& c = planc::t_last_choice;
  out[0] = 2 * planc::kTL[c.tl];  // two rows per thread
  out[1] = planc::kNT[c.nt];      // (the persistent launch: 128 threads per CTA)
  out[2] = c.sched_left;
  out[3] = c.sched_right;
  return PLANC_OK;
}
