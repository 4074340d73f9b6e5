// Batches of many patterns of uneven size: host planning, the schedule of
// grouped launches, CUDA-graph replay and the schedule autotuner.
//
// Every pattern gets an ordinary transform plan (exact SNF and tables, the
// same device code as pfft_forward) restricted to the generic shared-memory
// kernels, whose tables are sub-allocated from one arena.  A schedule turns
// the plans into grouped launches: for each pass, the patterns are grouped by
// the shared-memory footprint of their tile into at most kMaxBuckets
// launches (so that small tiles are not held to the occupancy of the largest
// one), those launches run concurrently on forked streams, and inside a
// launch the CTAs of the costliest tiles come first.  The split level of every
// pattern is one more grouped launch.  The autotuner times candidate tile
// budgets and orders on the real batch and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pfft.h"
#include "batch.hpp"
#include "plan_internal.hpp"

using namespace pfft;

namespace {
constexpr int kMaxBuckets = 5;
// upper ends of the shared-memory classes of a grouped pass launch (bytes)
constexpr int kSmemClass[kMaxBuckets] = {24 * 1024, 48 * 1024, 72 * 1024, 112 * 1024, kGroupedMaxDynSmem};

struct Bucket {
  int cols = 0, n = 0, nctas = 0, threads = 0, smem = 0;
  size_t items_off = 0, cta0_off = 0;  // byte offsets into the schedule buffer
};
}  // namespace

struct pfft_batch_s {
  int n = 0, dtype = 0;
  unsigned flags = 0;
  Arena arena;  // declared first: destroyed after the plans are released
  std::vector<pfft_plan_s*> plans;
  std::vector<int64_t> m, off;
  int64_t total = 0;
  bool has_split = false;
  std::vector<SplitItem> sitems;   // patterns whose dilation has |det J| = 2
  std::vector<PrimeItem> pitems;   // |det J| = p > 2
  std::vector<int> split_pat, prime_pat;  // pattern of each split item
  std::vector<int> p;              // |det J_i| (0 without dilations)
  std::vector<int64_t> sc_off, wv_off;
  int64_t sc_total = 0, wv_total = 0;
  void* ws = nullptr;
  void* sched = nullptr;  // device: items and first-CTA tables of all launches
  std::vector<Bucket> rows, cols, splits, primes;
  int row_budget = 8192, col_budget = 8192, order = 1, max2 = 16;
  std::vector<int> ident;  // patterns with m = 1 (the transform is a copy)
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  cudaGraphExec_t exec = nullptr;
  const void* key[4] = {nullptr, nullptr, nullptr, nullptr};
  // single launch (PFFT_BATCH_ONE_LAUNCH): the queue's tables in the schedule
  // buffer (pointers filled per call), its counters and status word
  QueueArgs q{};
  int q_units = 0, q_smem = 0;
  size_t q_off[14] = {};
  int* qmem = nullptr;  // [0] status, then the counters of QueueArgs
  unsigned spin_limit = kSpinLimit;

  ~pfft_batch_s() {
    for (auto* P : plans) plan_release(P);
    if (exec) cudaGraphExecDestroy(exec);
    for (auto e : events) cudaEventDestroy(e);
    for (auto s : streams) cudaStreamDestroy(s);
    if (cap) cudaStreamDestroy(cap);
    if (qmem) cudaFree(qmem);
    if (sched) cudaFree(sched);
    if (ws) cudaFree(ws);
  }
};

namespace {

size_t ebytes(int dtype) { return dtype == PFFT_C64 ? 8 : 16; }

// Relative cost of one CTA of a pass: its elements times the per-element work
// of its stages (direct prime stages cost about R / 4 radix-2 butterflies).
double tile_cost(const PassArgs& a) {
  double w = 0;
  for (int i = 0; i < a.nstages; ++i) {
    const int R = a.st[i].R;
    w += R >= kMinDirectRadix ? R / 4.0 : std::log2(double(R));
  }
  return double(a.T) * a.L * (w + 2.0);
}

struct Item {
  PassArgs a;
  int pattern;
  double cost;
};

// Group items into launches by shared-memory class; order each launch.
void make_buckets(std::vector<Item>& items, int cols, int order, std::vector<Bucket>& out,
                  std::vector<std::vector<Item>>& groups) {
  std::vector<std::vector<Item>> g(kMaxBuckets);
  for (auto& it : items) {
    int c = 0;
    while (c + 1 < kMaxBuckets && it.a.smem_bytes > kSmemClass[c]) ++c;
    g[c].push_back(it);
  }
  for (auto& v : g) {
    if (v.empty()) continue;
    if (order == 1)
      std::stable_sort(v.begin(), v.end(), [](const Item& x, const Item& y) { return x.cost > y.cost; });
    Bucket b;
    b.cols = cols;
    b.n = int(v.size());
    int tmax = 1;
    for (auto& it : v) {
      b.nctas += it.a.groups;
      b.threads = std::max(b.threads, it.a.nthreads);
      b.smem = std::max(b.smem, it.a.smem_bytes);
      tmax = std::max(tmax, it.a.T);
    }
    // a column pass keeps one column per thread: the block size must be a
    // multiple of every item's T (powers of two up to 512)
    if (cols && b.threads % tmax) b.threads = (b.threads + tmax - 1) / tmax * tmax;
    out.push_back(b);
    groups.push_back(std::move(v));
  }
}

pfft_status build_schedule(pfft_batch_s& B) {
  const size_t eb = ebytes(B.dtype);
  std::vector<Item> rows, cols;
  for (int i = 0; i < B.n; ++i) {
    pfft_plan_s* P = B.plans[i];
    if (P->D == 0) continue;
    pfft_status st = plan_retile(*P, B.row_budget, B.col_budget, B.max2);
    if (st != PFFT_OK) return st;
    const double scale = 1.0 / std::sqrt(double(P->m));
    const uintptr_t boff = uintptr_t(B.off[i]) * eb;
    PassArgs r = P->rowp;
    r.batch = 1;
    r.load_mode = MAP_BOX_H;
    r.conj_in = r.conj_out = 0;
    r.in_sel = 0;
    r.in = reinterpret_cast<const void*>(boff);
    r.out = reinterpret_cast<void*>(boff);
    if (P->pen.empty()) {
      r.store_mode = MAP_BOX_G;
      r.scale = scale;
      r.out_sel = 2;
    } else {
      r.store_mode = MAP_WS;
      r.scale = 1.0;
      r.out_sel = 1;
    }
    rows.push_back({r, i, tile_cost(r)});
    if (!P->pen.empty()) {
      PassArgs c = P->colp;
      c.batch = 1;
      c.load_mode = MAP_WS;
      c.store_mode = MAP_BOX_G;
      c.conj_in = c.conj_out = 0;
      c.scale = scale;
      c.in_sel = 1;
      c.out_sel = 2;
      c.in = reinterpret_cast<const void*>(boff);
      c.out = reinterpret_cast<void*>(boff);
      cols.push_back({c, i, tile_cost(c)});
    }
  }
  std::vector<Bucket> rb, cb, sb;
  std::vector<std::vector<Item>> rg, cg;
  make_buckets(rows, 0, B.order, rb, rg);
  make_buckets(cols, 1, B.order, cb, cg);
  // split launch: one item per pattern, costliest first
  std::vector<int> sorder;
  for (int i = 0; i < int(B.sitems.size()); ++i) sorder.push_back(i);
  if (B.order == 1)
    std::stable_sort(sorder.begin(), sorder.end(),
                     [&](int x, int y) { return B.sitems[x].L.mN > B.sitems[y].L.mN; });
  // lay out the schedule buffer
  std::vector<char> host;
  auto put = [&](const void* p, size_t bytes) {
    const size_t o = (host.size() + 255) & ~size_t(255);
    host.resize(o + bytes);
    std::memcpy(host.data() + o, p, bytes);
    return o;
  };
  // prefix table of first CTAs (n + 1 ints, padded to an even count), then
  // the (item, tile) pair of every CTA (cta_item in batch_kernels.cu)
  auto with_map = [](std::vector<int> c0) {
    const int n = int(c0.size()) - 1;
    if (c0.size() & 1) c0.push_back(0);
    for (int k = 0; k < n; ++k)
      for (int t = 0; t < c0[k + 1] - c0[k]; ++t) {
        c0.push_back(k);
        c0.push_back(t);
      }
    return c0;
  };
  auto put_group = [&](Bucket& b, const std::vector<Item>& v) {
    std::vector<PassArgs> a(v.size());
    std::vector<int> c0(v.size() + 1, 0);
    for (size_t k = 0; k < v.size(); ++k) {
      a[k] = v[k].a;
      c0[k + 1] = c0[k] + v[k].a.groups;
    }
    b.items_off = put(a.data(), a.size() * sizeof(PassArgs));
    const std::vector<int> t = with_map(c0);
    b.cta0_off = put(t.data(), t.size() * sizeof(int));
  };
  for (size_t k = 0; k < rb.size(); ++k) put_group(rb[k], rg[k]);
  for (size_t k = 0; k < cb.size(); ++k) put_group(cb[k], cg[k]);
  if (!sorder.empty()) {
    std::vector<SplitItem> si;
    std::vector<int> c0(1, 0);
    for (int i : sorder) {
      si.push_back(B.sitems[i]);
      const int per_cta = kSplitThreads * kSplitPerThread;
      c0.push_back(c0.back() + int((B.sitems[i].L.mN + per_cta - 1) / per_cta));
    }
    Bucket b;
    b.n = int(si.size());
    b.nctas = c0.back();
    b.threads = kSplitThreads;
    b.items_off = put(si.data(), si.size() * sizeof(SplitItem));
    const std::vector<int> t = with_map(c0);
    b.cta0_off = put(t.data(), t.size() * sizeof(int));
    sb.push_back(b);
  }
  // prime split launch: one item per pattern with |det J| > 2, costliest first
  std::vector<Bucket> pb;
  if (!B.pitems.empty()) {
    std::vector<int> porder;
    for (int i = 0; i < int(B.pitems.size()); ++i) porder.push_back(i);
    auto work = [&](int i) { return (long long)B.pitems[i].P.mN * B.pitems[i].P.nch; };
    if (B.order == 1) std::stable_sort(porder.begin(), porder.end(), [&](int x, int y) { return work(x) > work(y); });
    std::vector<PrimeItem> pi;
    std::vector<int> c0(1, 0);
    for (int i : porder) {
      pi.push_back(B.pitems[i]);
      c0.push_back(c0.back() + int((work(i) + kSplitThreads - 1) / kSplitThreads));
    }
    Bucket b;
    b.n = int(pi.size());
    b.nctas = c0.back();
    b.threads = kSplitThreads;
    b.items_off = put(pi.data(), pi.size() * sizeof(PrimeItem));
    const std::vector<int> t = with_map(c0);
    b.cta0_off = put(t.data(), t.size() * sizeof(int));
    pb.push_back(b);
  }
  // the single-launch queue: rows, columns, p = 2 splits, prime splits, each
  // list in the buckets' order, with first units, patterns and the patterns'
  // tile counts
  if (B.flags & PFFT_BATCH_ONE_LAUNCH) {
    std::vector<PassArgs> qa;
    std::vector<int> u0(1, 0), pat, need_r(B.n, 0), need_c(B.n, 0);
    int smem = 0;
    auto pass_list = [&](const std::vector<std::vector<Item>>& groups, std::vector<int>& need, size_t* o) {
      qa.clear();
      u0.assign(1, 0);
      pat.clear();
      for (auto& v : groups)
        for (auto& it : v) {
          qa.push_back(it.a);
          u0.push_back(u0.back() + it.a.groups);
          pat.push_back(it.pattern);
          need[it.pattern] += it.a.groups;
          smem = std::max(smem, it.a.smem_bytes);
        }
      o[0] = qa.empty() ? 0 : put(qa.data(), qa.size() * sizeof(PassArgs));
      o[1] = put(u0.data(), u0.size() * sizeof(int));
      o[2] = pat.empty() ? 0 : put(pat.data(), pat.size() * sizeof(int));
      return std::make_pair(int(qa.size()), u0.back());
    };
    const auto r = pass_list(rg, need_r, B.q_off + 0);
    const auto c = pass_list(cg, need_c, B.q_off + 3);
    B.q.nrow = r.first;
    B.q.u_rows = r.second;
    B.q.ncol = c.first;
    B.q.u_cols = c.second;
    // split units
    {
      std::vector<SplitItem> si;
      std::vector<int> su0(1, 0), spat;
      for (int i : sorder) {
        si.push_back(B.sitems[i]);
        su0.push_back(su0.back() + int((B.sitems[i].L.mN + kQueueSplitFibres - 1) / kQueueSplitFibres));
        spat.push_back(B.split_pat[i]);
      }
      B.q_off[6] = si.empty() ? 0 : put(si.data(), si.size() * sizeof(SplitItem));
      B.q_off[7] = put(su0.data(), su0.size() * sizeof(int));
      B.q_off[8] = spat.empty() ? 0 : put(spat.data(), spat.size() * sizeof(int));
      B.q.nsplit = int(si.size());
      B.q.u_splits = su0.back();
    }
    {
      std::vector<int> porder;
      for (int i = 0; i < int(B.pitems.size()); ++i) porder.push_back(i);
      auto work = [&](int i) { return (long long)B.pitems[i].P.mN * B.pitems[i].P.nch; };
      if (B.order == 1) std::stable_sort(porder.begin(), porder.end(), [&](int x, int y) { return work(x) > work(y); });
      std::vector<PrimeItem> pi;
      std::vector<int> pu0(1, 0), ppat;
      for (int i : porder) {
        pi.push_back(B.pitems[i]);
        pu0.push_back(pu0.back() + int((work(i) + kMaxThreads - 1) / kMaxThreads));
        ppat.push_back(B.prime_pat[i]);
      }
      B.q_off[9] = pi.empty() ? 0 : put(pi.data(), pi.size() * sizeof(PrimeItem));
      B.q_off[10] = put(pu0.data(), pu0.size() * sizeof(int));
      B.q_off[11] = ppat.empty() ? 0 : put(ppat.data(), ppat.size() * sizeof(int));
      B.q.nprime = int(pi.size());
      B.q.u_primes = pu0.back();
    }
    B.q_off[12] = put(need_r.data(), need_r.size() * sizeof(int));
    B.q_off[13] = put(need_c.data(), need_c.size() * sizeof(int));
    B.q.npat = B.n;
    B.q_smem = smem;
    B.q_units = B.q.u_rows + B.q.u_cols + B.q.u_splits + B.q.u_primes;
  }
  void* dev = nullptr;
  if (!host.empty()) {
    if (int e = device_alloc(&dev, host.size())) return pfft_status(e);
    if (cudaMemcpy(dev, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(dev);
      return PFFT_ERR_CUDA;
    }
  }
  if (B.sched) cudaFree(B.sched);
  B.sched = dev;
  B.rows = rb;
  B.cols = cb;
  B.splits = sb;
  B.primes = pb;
  if (B.exec) {  // the graph refers to the old schedule
    cudaGraphExecDestroy(B.exec);
    B.exec = nullptr;
  }
  return PFFT_OK;
}

// Queue the whole batch on stream s (directly, or into a capture of s).
pfft_status enqueue(pfft_batch_s& B, const void* in, void* chat, void* sc, void* wv, cudaStream_t s) {
  const size_t eb = ebytes(B.dtype);
  for (int i : B.ident)
    if (cudaMemcpyAsync(static_cast<char*>(chat) + B.off[i] * eb, static_cast<const char*>(in) + B.off[i] * eb, eb,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return PFFT_ERR_CUDA;
  const char* sched = static_cast<const char*>(B.sched);
  if (B.flags & PFFT_BATCH_ONE_LAUNCH) {
    QueueArgs q = B.q;
    auto at = [&](int i) { return static_cast<const void*>(sched + B.q_off[i]); };
    q.rows = static_cast<const PassArgs*>(at(0));
    q.row_u0 = static_cast<const int*>(at(1));
    q.row_pat = static_cast<const int*>(at(2));
    q.cols = static_cast<const PassArgs*>(at(3));
    q.col_u0 = static_cast<const int*>(at(4));
    q.col_pat = static_cast<const int*>(at(5));
    q.splits = static_cast<const SplitItem*>(at(6));
    q.split_u0 = static_cast<const int*>(at(7));
    q.split_pat = static_cast<const int*>(at(8));
    q.primes = static_cast<const PrimeItem*>(at(9));
    q.prime_u0 = static_cast<const int*>(at(10));
    q.prime_pat = static_cast<const int*>(at(11));
    q.need_rows = static_cast<const int*>(at(12));
    q.need_cols = static_cast<const int*>(at(13));
    q.status = B.qmem;
    q.counters = B.qmem + 1;
    q.spin_limit = B.spin_limit;
    q.base[0] = in;
    q.base[1] = B.ws;
    q.base[2] = chat;
    q.sc = sc;
    q.wv = wv;
    if (!(sc && wv)) q.u_splits = q.u_primes = 0;
    const int units = q.u_rows + q.u_cols + q.u_splits + q.u_primes;
    if (cudaMemsetAsync(q.counters, 0, sizeof(int) * size_t(2 + 2 * B.n), s) != cudaSuccess) return PFFT_ERR_CUDA;
    return launch_batch_queue(q, B.dtype, units, B.q_smem, s) == 0 ? PFFT_OK : PFFT_ERR_CUDA;
  }
  auto phase = [&](const std::vector<Bucket>& bs) -> pfft_status {
    auto launch = [&](const Bucket& b, cudaStream_t st) {
      GroupArgs g;
      g.items = reinterpret_cast<const PassArgs*>(sched + b.items_off);
      g.cta0 = reinterpret_cast<const int*>(sched + b.cta0_off);
      g.n = b.n;
      g.base[0] = in;
      g.base[1] = B.ws;
      g.base[2] = chat;
      return launch_grouped_pass(g, b.cols, B.dtype, b.nctas, b.threads, b.smem, st);
    };
    if (bs.empty()) return PFFT_OK;
    if (bs.size() == 1) return launch(bs[0], s) == 0 ? PFFT_OK : PFFT_ERR_CUDA;
    if (cudaEventRecord(B.events[0], s) != cudaSuccess) return PFFT_ERR_CUDA;
    for (size_t k = 0; k < bs.size(); ++k) {
      if (cudaStreamWaitEvent(B.streams[k], B.events[0], 0) != cudaSuccess) return PFFT_ERR_CUDA;
      if (launch(bs[k], B.streams[k]) != 0) return PFFT_ERR_CUDA;
      if (cudaEventRecord(B.events[1 + k], B.streams[k]) != cudaSuccess) return PFFT_ERR_CUDA;
    }
    for (size_t k = 0; k < bs.size(); ++k)
      if (cudaStreamWaitEvent(s, B.events[1 + k], 0) != cudaSuccess) return PFFT_ERR_CUDA;
    return PFFT_OK;
  };
  pfft_status st = phase(B.rows);
  if (st != PFFT_OK) return st;
  st = phase(B.cols);
  if (st != PFFT_OK) return st;
  if (sc && wv && !B.splits.empty()) {
    const Bucket& b = B.splits[0];
    if (launch_grouped_split(reinterpret_cast<const SplitItem*>(sched + b.items_off),
                             reinterpret_cast<const int*>(sched + b.cta0_off), b.n, b.nctas, chat, sc, wv, B.dtype,
                             s) != 0)
      return PFFT_ERR_CUDA;
  }
  if (sc && wv && !B.primes.empty()) {
    const Bucket& b = B.primes[0];
    if (launch_grouped_prime_split(reinterpret_cast<const PrimeItem*>(sched + b.items_off),
                                   reinterpret_cast<const int*>(sched + b.cta0_off), b.n, b.nctas, chat, sc, wv,
                                   B.dtype, s) != 0)
      return PFFT_ERR_CUDA;
  }
  return PFFT_OK;
}

pfft_status run_graph(pfft_batch_s& B, const void* in, void* chat, void* sc, void* wv, cudaStream_t s) {
  const void* key[4] = {in, chat, sc, wv};
  if (!B.exec || std::memcmp(key, B.key, sizeof(key)) != 0) {
    if (cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PFFT_ERR_CUDA;
    pfft_status st = enqueue(B, in, chat, sc, wv, B.cap);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(B.cap, &g);
    if (st != PFFT_OK || ce != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return st != PFFT_OK ? st : PFFT_ERR_CUDA;
    }
    if (B.exec) cudaGraphExecDestroy(B.exec);
    B.exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&B.exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      B.exec = nullptr;
      return PFFT_ERR_CUDA;
    }
    std::memcpy(B.key, key, sizeof(key));
  }
  return cudaGraphLaunch(B.exec, s) == cudaSuccess ? PFFT_OK : PFFT_ERR_CUDA;
}

// Mean time (ms) of `reps` direct runs of the current schedule.
pfft_status time_schedule(pfft_batch_s& B, const void* in, void* chat, void* sc, void* wv, int reps, float* ms) {
  cudaStream_t s = B.cap;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PFFT_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PFFT_ERR_CUDA;
  }
  pfft_status st = enqueue(B, in, chat, sc, wv, s);  // warm-up
  if (st == PFFT_OK) cudaEventRecord(e0, s);
  for (int r = 0; r < reps && st == PFFT_OK; ++r) st = enqueue(B, in, chat, sc, wv, s);
  if (st == PFFT_OK) {
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      st = PFFT_ERR_CUDA;
    *ms /= float(reps);
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

// Coordinate search over the row budget, the column budget, the launch order
// and the largest power-of-two radix (16 or 8).
pfft_status autotune(pfft_batch_s& B) {
  const size_t eb = ebytes(B.dtype);
  void *in = nullptr, *chat = nullptr, *sc = nullptr, *wv = nullptr;
  pfft_status st = PFFT_OK;
  auto fail = [&](pfft_status e) {
    for (void* p : {in, chat, sc, wv})
      if (p) cudaFree(p);
    return e;
  };
  if (int e = device_alloc(&in, size_t(B.total) * eb)) return fail(pfft_status(e));
  if (int e = device_alloc(&chat, size_t(B.total) * eb)) return fail(pfft_status(e));
  if (B.has_split) {
    if (int e = device_alloc(&sc, size_t(std::max<int64_t>(B.sc_total, 1)) * eb)) return fail(pfft_status(e));
    if (int e = device_alloc(&wv, size_t(std::max<int64_t>(B.wv_total, 1)) * eb)) return fail(pfft_status(e));
  }
  if (cudaMemset(in, 0, size_t(B.total) * eb) != cudaSuccess) return fail(PFFT_ERR_CUDA);
  const int budgets[] = {2048, 4096, 8192, 16384};
  float best = 1e30f;
  int br = B.row_budget, bc = B.col_budget, bo = B.order, bx = B.max2;
  auto trial = [&](int r, int c, int o, int x) -> pfft_status {
    B.row_budget = r;
    B.col_budget = c;
    B.order = o;
    B.max2 = x;
    pfft_status e = build_schedule(B);
    if (e != PFFT_OK) return e;
    float ms = 0;
    e = time_schedule(B, in, chat, sc, wv, 3, &ms);
    if (e != PFFT_OK) return e;
    if (ms < best) {
      best = ms;
      br = r;
      bc = c;
      bo = o;
      bx = x;
    }
    return PFFT_OK;
  };
  for (int r : budgets)
    if ((st = trial(r, bc, bo, bx)) != PFFT_OK) return fail(st);
  for (int c : budgets)
    if ((st = trial(br, c, bo, bx)) != PFFT_OK) return fail(st);
  if ((st = trial(br, bc, 1 - bo, bx)) != PFFT_OK) return fail(st);
  if ((st = trial(br, bc, bo, bx == 16 ? 8 : 16)) != PFFT_OK) return fail(st);
  B.row_budget = br;
  B.col_budget = bc;
  B.order = bo;
  B.max2 = bx;
  st = build_schedule(B);
  return fail(st);
}

}  // namespace

extern "C" pfft_status pfft_batch_create(pfft_batch* out, int n, const int* d, const int64_t* M, const int64_t* J,
                                         int symbol, double eta, int dtype, unsigned flags) {
  if (!out || n < 1 || !d || !M || (dtype != PFFT_C64 && dtype != PFFT_C128) ||
      (flags & ~unsigned(PFFT_BATCH_NO_GRAPH | PFFT_BATCH_AUTOTUNE | PFFT_BATCH_RADIX8 | PFFT_BATCH_ONE_LAUNCH)))
    return PFFT_ERR_ARG;
  if (J && (symbol != PWT_DIRICHLET && symbol != PWT_DLVP)) return PFFT_ERR_ARG;
  if (J && symbol == PWT_DLVP && !(eta > 0.0 && eta < 1.0)) return PFFT_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (d[i] < 1 || d[i] > 4) return PFFT_ERR_ARG;
  pfft_batch_s* B = new (std::nothrow) pfft_batch_s;
  if (!B) return PFFT_ERR_OOM;
  B->n = n;
  B->dtype = dtype;
  B->flags = flags;
  if (flags & PFFT_BATCH_RADIX8) B->max2 = 8;
  B->has_split = J != nullptr;
  auto fail = [&](pfft_status st) {
    delete B;
    return st;
  };
  if (prepare_grouped(dtype) != 0) return fail(PFFT_ERR_CUDA);
  if ((flags & PFFT_BATCH_ONE_LAUNCH) && prepare_queue(dtype) != 0) return fail(PFFT_ERR_CUDA);
  size_t mo = 0;
  bool need_ws = false;
  for (int i = 0; i < n; ++i) {
    pfft_plan_s* P = new (std::nothrow) pfft_plan_s;
    if (!P) return fail(PFFT_ERR_OOM);
    B->plans.push_back(P);
    P->batch = 1;
    P->dtype = dtype;
    P->arena = &B->arena;
    P->generic_only = true;
    P->own_workspace = false;
    // grouped kernels: 16 complex64 points per thread (64 registers, two
    // 512-thread CTAs per SM) to hide the latency of the table-driven passes
    P->ept_c64 = kGroupedEptC64;
    pfft_status st;
    try {
      st = plan_host(*P, d[i], M + mo);
      if (st == PFFT_OK) st = plan_device(*P);
    } catch (const LatticeError& e) {
      st = pfft_status(e.code);
    }
    if (st != PFFT_OK) return fail(st);
    B->m.push_back(P->m);
    B->off.push_back(B->total);
    B->total += P->m;
    if (P->D == 0) B->ident.push_back(i);
    if (!P->pen.empty()) need_ws = true;
    if (J) {
      i64 pdet = 0;
      try {
        IMat Jm(d[i]);
        for (int k = 0; k < d[i] * d[i]; ++k) Jm.a[k] = J[mo + k];
        pdet = determinant(Jm);
      } catch (const LatticeError& e) {
        return fail(pfft_status(e.code));
      }
      if (pdet < 0) pdet = -pdet;
      if (pdet < 2 || pdet > (i64(1) << 20) || P->m % pdet != 0) return fail(pdet == 0 ? PFFT_ERR_SINGULAR
                                                                                     : PFFT_ERR_NOT_INTEGRAL);
      const int64_t n_i = P->m / pdet;
      if (pdet == 2) {
        SplitItem it;
        std::memset(&it, 0, sizeof(it));
        st = describe_split_level(d[i], M + mo, J + mo, symbol, eta, &it.L);
        if (st != PFFT_OK) return fail(st);
        void* tab = nullptr;  // phase tables in the arena, as single plans have them
        if (int e = B->arena.alloc(&tab, split_table_elems(it.L) * ebytes(dtype))) return fail(pfft_status(e));
        if (launch_split_tables(it.L, tab, dtype) != 0) return fail(PFFT_ERR_CUDA);
        it.in_off = B->off[i];
        it.sc_off = B->sc_total;
        it.wv_off = B->wv_total;
        B->sitems.push_back(it);
        B->split_pat.push_back(i);
      } else {
        if (symbol != PWT_DIRICHLET) return fail(PFFT_ERR_UNSUPPORTED);  // built-in bands: Dirichlet only
        PrimeItem it;
        std::memset(&it, 0, sizeof(it));
        try {
          st = describe_prime_level(d[i], M + mo, J + mo, &it.P);
        } catch (const LatticeError& e) {
          st = pfft_status(e.code);
        }
        if (st != PFFT_OK) return fail(st);
        it.in_off = B->off[i];
        it.sc_off = B->sc_total;
        it.wv_off = B->wv_total;
        B->pitems.push_back(it);
        B->prime_pat.push_back(i);
      }
      B->p.push_back(int(pdet));
      B->sc_off.push_back(B->sc_total);
      B->wv_off.push_back(B->wv_total);
      B->sc_total += n_i;
      B->wv_total += (pdet - 1) * n_i;
    }
    mo += size_t(d[i]) * d[i];
  }
  if (B->total >= (int64_t(1) << 40)) return fail(PFFT_ERR_OVERFLOW);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(PFFT_ERR_CUDA);  // tables built
  if (need_ws)
    if (int e = device_alloc(&B->ws, size_t(B->total) * ebytes(dtype))) return fail(pfft_status(e));
  if (flags & PFFT_BATCH_ONE_LAUNCH) {  // status word and queue counters
    if (int e = device_alloc(reinterpret_cast<void**>(&B->qmem), sizeof(int) * size_t(3 + 2 * n)))
      return fail(pfft_status(e));
    if (cudaMemset(B->qmem, 0, sizeof(int) * size_t(3 + 2 * n)) != cudaSuccess) return fail(PFFT_ERR_CUDA);
  }
  if (cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(PFFT_ERR_CUDA);
  for (int k = 0; k < kMaxBuckets; ++k) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(PFFT_ERR_CUDA);
    B->streams.push_back(s);
  }
  for (int k = 0; k < kMaxBuckets + 1; ++k) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(PFFT_ERR_CUDA);
    B->events.push_back(e);
  }
  pfft_status st = (flags & PFFT_BATCH_AUTOTUNE) ? autotune(*B) : build_schedule(*B);
  if (st != PFFT_OK) return fail(st);
  *out = B;
  return PFFT_OK;
}

extern "C" pfft_status pfft_batch_info(pfft_batch b, int64_t* m, int64_t* total) {
  if (!b) return PFFT_ERR_ARG;
  if (m)
    for (int i = 0; i < b->n; ++i) m[i] = b->m[i];
  if (total) *total = b->total;
  return PFFT_OK;
}

extern "C" pfft_status pfft_batch_split_layout(pfft_batch b, int* p, int64_t* scaling_off, int64_t* wavelet_off,
                                               int64_t* scaling_total, int64_t* wavelet_total) {
  if (!b) return PFFT_ERR_ARG;
  for (int i = 0; i < b->n; ++i) {
    const bool has = b->has_split;
    if (p) p[i] = has ? b->p[i] : 0;
    if (scaling_off) scaling_off[i] = has ? b->sc_off[i] : 0;
    if (wavelet_off) wavelet_off[i] = has ? b->wv_off[i] : 0;
  }
  if (scaling_total) *scaling_total = b->sc_total;
  if (wavelet_total) *wavelet_total = b->wv_total;
  return PFFT_OK;
}

extern "C" pfft_status pfft_batch_schedule(pfft_batch b, int* row_budget, int* col_budget, int* order,
                                           int* max_radix) {
  if (!b) return PFFT_ERR_ARG;
  if (row_budget) *row_budget = b->row_budget;
  if (col_budget) *col_budget = b->col_budget;
  if (order) *order = b->order;
  if (max_radix) *max_radix = b->max2;
  return PFFT_OK;
}

extern "C" pfft_status pfft_batch_forward(pfft_batch b, const void* in, void* c_hat, void* scaling, void* wavelet,
                                          void* stream) {
  if (!b || !in || !c_hat || in == c_hat) return PFFT_ERR_ARG;
  if ((scaling == nullptr) != (wavelet == nullptr)) return PFFT_ERR_ARG;
  if (scaling && !b->has_split) return PFFT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (b->flags & PFFT_BATCH_NO_GRAPH) return enqueue(*b, in, c_hat, scaling, wavelet, s);
  return run_graph(*b, in, c_hat, scaling, wavelet, s);
}

extern "C" pfft_status pfft_batch_destroy(pfft_batch b) {
  if (!b) return PFFT_ERR_ARG;
  delete b;
  return PFFT_OK;
}

extern "C" pfft_status pfft_batch_set_wait_limit(pfft_batch b, int64_t spins) {
  if (!b) return PFFT_ERR_ARG;
  if (!(b->flags & PFFT_BATCH_ONE_LAUNCH)) return PFFT_ERR_UNSUPPORTED;
  b->spin_limit = spins < 0 ? kSpinLimit : unsigned(std::min<int64_t>(spins, int64_t(UINT32_MAX)));
  if (b->exec) {  // the graph holds the old limit
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return PFFT_OK;
}

extern "C" pfft_status pfft_batch_device_status(pfft_batch b, void* stream) {
  if (!b) return PFFT_ERR_ARG;
  if (!b->qmem) return PFFT_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int v = 0;
  if (cudaMemcpyAsync(&v, b->qmem, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemsetAsync(b->qmem, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return PFFT_ERR_CUDA;
  return pfft_status(v);
}
