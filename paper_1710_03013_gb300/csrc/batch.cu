// kkm_fit_batch: many independent fits (separate data sets, or restarts of
// one data set with different seeds) on one GPU at once.
//
// Each problem is an ordinary kkm_fit call, so its results are those of the
// same call made alone: every kernel of a fit runs on that fit's own stream,
// and the reductions inside a fit are in a fixed order that does not depend
// on what else occupies the GPU.
//
// Scheduling.  W worker threads each own one non-blocking CUDA stream and
// take problems from a shared list, longest first (LPT: the estimated
// algorithmic work of a fit is sum_i N_i |L_i| (iters + 2) kernel-block
// entries read plus the N d input), which keeps the large fits from being the
// last to start.  Small fits are bound by launch latency and host round
// trips, not by the GPU, so several of them in flight on separate streams
// fill the SMs that one alone leaves idle; the large ones stream the HBM.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace kkm {

// ------------------------------------------- rows per assign CTA, by timing
// A work-list assign CTA takes 1, 2, 4 or 8 blocks of 32 rows of its loop.
// Every 32-row block does the same work and writes the same partial sums
// whichever CTA takes it, so the choice changes no result, only time: few
// rows per CTA spread a small round over the SMs, more rows amortise a CTA's
// fixed work (cluster tables, barriers, its ticket) in a round of many loops.
// Per key (the CTA width and the launch's row-block count rounded down to a
// power of two; a fit's own assign launches and the work lists' are keyed
// apart) each candidate is timed on kTuneSamples live launches with events,
// and the one with the least time per row block is kept for the process.  KKM_TUNE_CACHE names a file the choices are read from when the
// first executor starts and written back to when an executor stops (lines
// "assign_rows <key> <rows>"); KKM_ASSIGN_ROWS forces one candidate.
struct RowTuner {
  static constexpr int kCand[4] = {1, 2, 4, 8};
  static constexpr int kTuneSamples = 3;
  struct Entry {
    int best = 0;  // 0: still timing
    double us_per_block[4] = {0.0, 0.0, 0.0, 0.0};
    int n[4] = {0, 0, 0, 0};
  };
  std::mutex mu;
  std::map<long long, Entry> table;
  bool loaded = false;

  static long long key(int nw, int blocks) {
    int lg = 0;
    while ((2LL << lg) <= blocks) ++lg;
    return (long long)nw * 64 + lg;
  }
  static int forced() {
    const char* f = getenv("KKM_ASSIGN_ROWS");
    if (!f) return 0;
    const int v = atoi(f);
    for (int c : kCand)
      if (c == v) return v;
    return 0;
  }
  void load() {
    std::lock_guard<std::mutex> lk(mu);
    if (loaded) return;
    loaded = true;
    const char* path = getenv("KKM_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char name[32];
    long long k;
    int v;
    while (fscanf(f, "%31s %lld %d", name, &k, &v) == 3)
      if (!strcmp(name, "assign_rows"))
        for (int c : kCand)
          if (c == v) table[k].best = v;
    fclose(f);
  }
  void save() {
    const char* path = getenv("KKM_TUNE_CACHE");
    if (!path) return;
    std::lock_guard<std::mutex> lk(mu);
    FILE* f = fopen(path, "w");
    if (!f) return;
    for (auto& kv : table)
      if (kv.second.best) fprintf(f, "assign_rows %lld %d\n", kv.first, kv.second.best);
    fclose(f);
  }
  // The candidate for a launch; *timed: this launch is a timing sample.
  int choose(long long k, bool* timed) {
    *timed = false;
    if (const int f = forced()) return f;
    std::lock_guard<std::mutex> lk(mu);
    Entry& e = table[k];
    if (e.best) return e.best;
    int c = 0;
    for (int q = 1; q < 4; ++q)
      if (e.n[q] < e.n[c]) c = q;
    *timed = true;
    return kCand[c];
  }
  void sample(long long k, int rows, int blocks, float ms) {
    std::lock_guard<std::mutex> lk(mu);
    Entry& e = table[k];
    if (e.best) return;
    int c = 0;
    while (kCand[c] != rows) ++c;
    e.us_per_block[c] += 1e3 * ms / std::max(blocks, 1);
    ++e.n[c];
    for (int q = 0; q < 4; ++q)
      if (e.n[q] < kTuneSamples) return;
    int b = 0;
    for (int q = 1; q < 4; ++q)
      if (e.us_per_block[q] < e.us_per_block[b]) b = q;
    e.best = kCand[b];
  }
};
static RowTuner g_row_tuner;
int assign_rows_choose(long long key, bool* timed) {
  g_row_tuner.load();
  return g_row_tuner.choose(key, timed);
}
void assign_rows_sample(long long key, int rows, int blocks, float ms) { g_row_tuner.sample(key, rows, blocks, ms); }
long long assign_rows_key(int nw, int blocks, bool solo) { return RowTuner::key(nw, blocks) + (solo ? (1LL << 20) : 0); }
void assign_rows_load() { g_row_tuner.load(); }
void assign_rows_save() { g_row_tuner.save(); }

// ------------------------------------------------ inner loops as work lists
// The fits of a batch hand their split-form inner loops to one executor
// thread, which runs them in rounds on its own stream: per round one f_hat
// stream launch over every loop in flight (one per block type present), then
// one assign launch for all of them (as wide as the widest, each CTA working
// with its own loop's warp count, so its CTAs do what that loop's own launch
// would: same results as a fit alone).  A loop joins at the next
// round once the work before it on its fit's stream has finished (its event
// is polled, so a fit still computing its block holds up no other loop) and
// leaves after its iteration count; its fit's stream then waits for the
// round that ran its last iteration.  At most two rounds are queued ahead of
// the GPU, so a loop that becomes ready joins within about two rounds, and
// the many small loops of a batch share launches instead of each paying two
// launches per iteration.  The support sort after a landmark label change
// runs in a third launch per round, one full CTA per loop, instead of in the
// last CTA of the loop's assign.
struct LoopExecutor {
  struct Req {
    LoopItem item;
    int iters = 0;
    cudaEvent_t ready = nullptr, done = nullptr;
    bool finished = false;
    kkm_status status = KKM_OK;
    std::string error;
  };
  static constexpr int kMirror = 1024;  // pinned copies of admitted items, reused round-robin
  std::mutex mu;
  std::condition_variable cv_submit, cv_done;
  std::vector<Req*> incoming;
  bool stopping = false;
  int device = 0;
  cudaStream_t st = nullptr;
  LoopItem* slots = nullptr;   // device [kRoundMaxItems]
  LoopItem* mirror = nullptr;  // pinned [kMirror]
  int mirror_next = 0;
  cudaEvent_t round_ev[4] = {};
  std::thread th;
  // timing samples of the row tuner still in flight
  struct Sample {
    long long key;
    int rows, blocks;
    cudaEvent_t a, b;
  };
  std::vector<Sample> samples;
  std::vector<cudaEvent_t> ev_pool;

  kkm_status start(int dev) {
    device = dev;
    KKM_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    KKM_CK(cudaMalloc(&slots, sizeof(LoopItem) * kRoundMaxItems));
    KKM_CK(cudaHostAlloc(reinterpret_cast<void**>(&mirror), sizeof(LoopItem) * kMirror, cudaHostAllocDefault));
    for (auto& e : round_ev) KKM_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    g_row_tuner.load();
    th = std::thread([this] { loop(); });
    return KKM_OK;
  }
  // after every submitter has returned
  void stop() {
    if (th.joinable()) {
      {
        std::lock_guard<std::mutex> lk(mu);
        stopping = true;
      }
      cv_submit.notify_all();
      th.join();
    }
    if (st) cudaStreamSynchronize(st);
    collect_samples();
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    ev_pool.clear();
    g_row_tuner.save();
    for (auto& e : round_ev)
      if (e) cudaEventDestroy(e);
    if (slots) cudaFree(slots);
    if (mirror) cudaFreeHost(mirror);
    if (st) cudaStreamDestroy(st);
    cudaGetLastError();
    st = nullptr;
    slots = nullptr;
    mirror = nullptr;
    for (auto& e : round_ev) e = nullptr;
  }

  kkm_status run(const LoopItem& item, int iters, cudaStream_t fit_st) {
    if (iters <= 0) return KKM_OK;
    Req r;
    r.item = item;
    r.iters = iters;
    KKM_CK(cudaEventCreateWithFlags(&r.ready, cudaEventDisableTiming));
    cudaError_t e = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r.ready, fit_st);
    if (e != cudaSuccess) {
      cudaEventDestroy(r.ready);
      if (r.done) cudaEventDestroy(r.done);
      return cuda_fail(e, "loop executor: event", __FILE__, __LINE__);
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      incoming.push_back(&r);
    }
    cv_submit.notify_one();
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_done.wait(lk, [&] { return r.finished; });
    }
    kkm_status s = r.status;
    if (s == KKM_OK) {
      e = cudaStreamWaitEvent(fit_st, r.done, 0);
      if (e != cudaSuccess) s = cuda_fail(e, "cudaStreamWaitEvent", __FILE__, __LINE__);
    } else {
      set_error(r.error);
    }
    cudaEventDestroy(r.ready);
    cudaEventDestroy(r.done);
    return s;
  }

 private:
  struct Active {
    Req* r;
    int slot;
    int left;
  };
  void finish(Req* r, kkm_status s, const char* what, cudaError_t e) {
    std::lock_guard<std::mutex> lk(mu);
    r->status = s;
    if (s != KKM_OK) r->error = std::string("loop executor: ") + what + ": " + cudaGetErrorString(e);
    r->finished = true;
    cv_done.notify_all();
  }
  // one iteration of every active loop
  cudaError_t round(const std::vector<Active>& act) {
    for (int half = 1; half >= 0; --half) {
      RoundList L;
      L.cta_off[0] = 0;
      for (const Active& a : act)
        if (a.r->item.half == half) {
          L.slot[L.n] = a.slot;
          L.cta_off[L.n + 1] = L.cta_off[L.n] + a.r->item.units * a.r->item.n_strips;
          ++L.n;
        }
      if (L.n == 0) continue;
      ProfScope ps("fhat_multi", st);
      const cudaError_t e = launch_fhat_multi(slots, L, half != 0, st);
      if (e != cudaSuccess) return e;
    }
    // one assign launch for every loop of the round, as wide as its widest
    // loop: each CTA works with its own loop's warp count (the results of
    // a launch of that width), so loops of small C no longer wait for
    // launches of their own
    {
      int blocks = 0, nw = 1, smem = 0;
      for (const Active& a : act) {
        blocks += a.r->item.assign_ctas;
        nw = std::max(nw, a.r->item.nw);
        smem = std::max(smem, a.r->item.assign_smem);
      }
      const long long key = RowTuner::key(nw, blocks);
      bool timed = false;
      const int RG = g_row_tuner.choose(key, &timed);
      RoundList L;
      L.cta_off[0] = 0;
      for (const Active& a : act) {
        L.slot[L.n] = a.slot;
        L.cta_off[L.n + 1] = L.cta_off[L.n] + (a.r->item.assign_ctas + RG - 1) / RG;
        ++L.n;
      }
      Sample smp{key, RG, blocks, nullptr, nullptr};
      if (timed) {
        smp.a = take_event();
        smp.b = take_event();
        if (smp.a && smp.b) cudaEventRecord(smp.a, st);
      }
      ProfScope ps("assign_multi", st);
      const cudaError_t e = launch_assign_multi(slots, L, nw, smem, RG, st);
      if (e != cudaSuccess) return e;
      if (timed && smp.a && smp.b) {
        cudaEventRecord(smp.b, st);
        samples.push_back(smp);
      }
    }
    RoundList L;
    for (const Active& a : act) {
      L.slot[L.n] = a.slot;
      L.cta_off[L.n] = L.n;
      ++L.n;
    }
    L.cta_off[L.n] = L.n;
    ProfScope ps("sort_multi", st);
    return launch_sort_multi(slots, L, st);
  }
  cudaEvent_t take_event() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
  // timing samples whose launches have finished go to the tuner
  void collect_samples() {
    for (size_t q = 0; q < samples.size();) {
      Sample& m = samples[q];
      const cudaError_t e = cudaEventQuery(m.b);
      if (e == cudaErrorNotReady) {
        ++q;
        continue;
      }
      float ms = 0.0f;
      if (e == cudaSuccess && cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess)
        g_row_tuner.sample(m.key, m.rows, m.blocks, ms);
      cudaGetLastError();
      ev_pool.push_back(m.a);
      ev_pool.push_back(m.b);
      samples.erase(samples.begin() + (std::ptrdiff_t)q);
    }
  }
  void loop() {
    cudaSetDevice(device);
    std::vector<Req*> pending;
    std::vector<Active> act;
    std::vector<int> free_slots;
    for (int q = kRoundMaxItems - 1; q >= 0; --q) free_slots.push_back(q);
    long long rounds = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        if (act.empty() && pending.empty() && incoming.empty()) {
          if (stopping) break;
          cv_submit.wait(lk, [&] { return stopping || !incoming.empty(); });
          continue;
        }
        pending.insert(pending.end(), incoming.begin(), incoming.end());
        incoming.clear();
      }
      // admit the loops whose preceding work has finished
      for (size_t q = 0; q < pending.size() && !free_slots.empty();) {
        Req* r = pending[q];
        const cudaError_t e = cudaEventQuery(r->ready);
        if (e == cudaErrorNotReady) {
          ++q;
          continue;
        }
        pending.erase(pending.begin() + (std::ptrdiff_t)q);
        if (e != cudaSuccess) {
          cudaGetLastError();
          finish(r, KKM_ECUDA, "the work before a loop", e);
          continue;
        }
        const int slot = free_slots.back();
        LoopItem* m = mirror + (mirror_next++ % kMirror);
        *m = r->item;
        const cudaError_t c = cudaMemcpyAsync(slots + slot, m, sizeof(LoopItem), cudaMemcpyHostToDevice, st);
        if (c != cudaSuccess) {
          cudaGetLastError();
          finish(r, KKM_ECUDA, "item upload", c);
          continue;
        }
        free_slots.pop_back();
        act.push_back(Active{r, slot, r->iters});
      }
      if (act.empty()) {
        std::this_thread::yield();
        continue;
      }
      if (rounds >= 2) cudaEventSynchronize(round_ev[(rounds - 2) & 3]);
      if (!samples.empty()) collect_samples();
      cudaError_t e = round(act);
      if (e == cudaSuccess) e = cudaEventRecord(round_ev[rounds & 3], st);
      ++rounds;
      for (size_t q = 0; q < act.size();) {
        Active& a = act[q];
        if (e != cudaSuccess || --a.left == 0) {
          cudaError_t d = e;
          if (d == cudaSuccess) d = cudaEventRecord(a.r->done, st);
          free_slots.push_back(a.slot);
          finish(a.r, d == cudaSuccess ? KKM_OK : KKM_ECUDA, "round launch", d);
          act.erase(act.begin() + (std::ptrdiff_t)q);
        } else {
          ++q;
        }
      }
      if (e != cudaSuccess) cudaGetLastError();
    }
  }
};

static thread_local LoopExecutor* t_loop_exec = nullptr;
LoopExecutor* current_loop_executor() { return t_loop_exec; }
kkm_status loop_executor_run(LoopExecutor* ex, const LoopItem& item, int iters, cudaStream_t st) {
  return ex->run(item, iters, st);
}

// Default number of concurrent streams for a batch.
// (32: a fit waits while the work lists run its inner loop, so more fits are
// in flight than loops; measured on 256 uneven problems: 8 -> 200 ms,
// 16 -> 177 ms, 32 -> 171 ms, 64 -> 174 ms)
constexpr int kBatchStreams = 32;
constexpr int kBatchMaxStreams = 64;

// Number of work-list chains (executors, each with its own thread and
// stream); worker w hands its loops to chain w mod E.  The rounds of one
// chain run in order, so while one chain's assign launch (bound by its CTAs'
// fixed work, not by bytes) occupies part of the GPU, another chain's f_hat
// stream can use the rest.  KKM_LOOP_CHAINS overrides the default.
constexpr int kLoopChains = 1;
constexpr int kLoopChainsMax = 8;
static int loop_chains(int W) {
  int e = kLoopChains;
  if (const char* v = getenv("KKM_LOOP_CHAINS")) {
    const int x = atoi(v);
    if (x >= 1 && x <= kLoopChainsMax) e = x;
  }
  return std::max(1, std::min(e, W));
}

static double fit_work(const kkm_problem& p) {
  if (p.N < 1 || p.B < 1 || p.B > p.N) return 0.0;
  double w = (double)p.N * (double)p.d;
  for (int32_t i = 0; i < p.B; ++i) {
    const double Ni = (double)((p.N - i + p.B - 1) / p.B);
    const double nl = std::min(std::max(std::ceil(p.s * Ni - 1e-9), 1.0), Ni);
    w += Ni * nl * (double)(std::max(p.iters, 0) + 2);
  }
  return w;
}

static kkm_status batch_impl(const kkm_problem* P, int32_t n, int32_t n_streams, kkm_model** models_out,
                             kkm_status* status_out, cudaStream_t caller, bool no_work_lists = false) {
  if (n < 0) {
    set_error("n must be >= 0");
    return KKM_EINVAL;
  }
  if (n > 0 && (!P || !status_out)) {
    set_error("problems and status_out must not be NULL");
    return KKM_EINVAL;
  }
  if (n_streams < 0 || n_streams > kBatchMaxStreams) {
    set_error("n_streams must be in [0, 64]");
    return KKM_EINVAL;
  }
  if (n == 0) return KKM_OK;
  for (int32_t p = 0; p < n; ++p) {
    status_out[p] = KKM_EINTERNAL;
    if (models_out) models_out[p] = nullptr;
  }
  int dev = 0;
  KKM_CK(cudaGetDevice(&dev));

  std::vector<double> work(n);
  for (int32_t p = 0; p < n; ++p) work[p] = fit_work(P[p]);
  std::vector<int32_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return work[a] > work[b]; });

  const int W = std::min<int>(n, n_streams > 0 ? n_streams : kBatchStreams);
  // the inputs may still be in flight on the caller's stream
  cudaEvent_t ready = nullptr;
  KKM_CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  KKM_CK(cudaEventRecord(ready, caller));
  std::atomic<int32_t> next{0};
  std::vector<std::string> errors(n);
  std::vector<std::string> worker_err(W);
  const bool use_exec = !no_work_lists;
  std::vector<std::unique_ptr<LoopExecutor>> execs;
  if (use_exec) {
    const int E = loop_chains(W);
    for (int c = 0; c < E; ++c) {
      execs.emplace_back(new LoopExecutor());
      const kkm_status es = execs.back()->start(dev);
      if (es != KKM_OK) {
        for (auto& x : execs) x->stop();
        cudaEventDestroy(ready);
        return es;
      }
    }
  }

  auto worker = [&](int w) {
    t_loop_exec = use_exec ? execs[w % execs.size()].get() : nullptr;
    cudaStream_t st = nullptr;
    if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamWaitEvent(st, ready, 0) != cudaSuccess) {
      cudaGetLastError();
      worker_err[w] = "worker could not create its stream";
      return;
    }
    for (;;) {
      const int32_t q = next.fetch_add(1);
      if (q >= n) break;
      const int32_t p = order[q];
      const kkm_problem& pr = P[p];
      kkm_options opt = pr.opt;
      opt.stream = st;
      opt.pipeline = side_by_side_pipeline(opt.pipeline);
      opt.iteration = side_by_side_iteration(opt.iteration);
      kkm_model* m = nullptr;
      const kkm_status s = kkm_fit(pr.X, pr.N, pr.d, pr.C, pr.B, pr.s, &pr.kernel, pr.iters, pr.seed, &opt,
                                   pr.labels_out, models_out ? &m : nullptr);
      status_out[p] = s;
      if (s != KKM_OK) errors[p] = kkm_last_error();
      if (models_out) models_out[p] = m;
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    t_loop_exec = nullptr;
  };
  std::vector<std::thread> threads;
  threads.reserve(W);
  for (int w = 0; w < W; ++w) threads.emplace_back(worker, w);
  for (auto& t : threads) t.join();
  for (auto& x : execs) x->stop();
  cudaEventDestroy(ready);

  for (int w = 0; w < W; ++w)
    if (!worker_err[w].empty()) {
      set_error(worker_err[w]);
      return KKM_ECUDA;
    }
  for (int32_t p = 0; p < n; ++p)
    if (status_out[p] != KKM_OK) {
      set_error("problem " + std::to_string(p) + ": " + errors[p]);
      return status_out[p];
    }
  return KKM_OK;
}

}  // namespace kkm

extern "C" kkm_status kkm_fit_batch(const kkm_problem* problems, int32_t n, int32_t n_streams,
                                    kkm_model** models_out, kkm_status* status_out, void* stream) {
  kkm::set_error("");
  try {
    return kkm::batch_impl(problems, n, n_streams, models_out, status_out, (cudaStream_t)stream);
  } catch (...) {
    kkm::set_error("internal exception");
    return KKM_EINTERNAL;
  }
}
