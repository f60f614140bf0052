// kkm_server: a request loop for fit and assign jobs on one GPU.
//
// Jobs arrive on any host thread (kkm_server_submit_*) and are queued.  W
// worker threads, each owning one non-blocking CUDA stream, take jobs as
// soon as a worker is free AND the job's device-memory estimate fits in what
// the HBM budget has left after the resident models and the jobs already
// running (admission by budget).  Jobs that arrive while others run are
// admitted as workers and memory free up, so their work overlaps on the
// device (continuous batching, not a queue drained one job at a time).
//
// Assign jobs against the same resident model and mode that are waiting
// together are fused: their rows are copied into one device buffer and
// labelled by one kkm_assign call.  Every row's result depends only on that
// row and the model (the kernel block, the segmented sums and the argmin are
// per row, in a fixed order), so a request gets bit-for-bit what it would
// get alone.
//
// Admission is first-come first-served, except that a job that does not fit
// yet may be passed by later jobs that do -- at most kMaxPass times, after
// which nothing passes it until it has started.  A job that could never fit
// (its estimate plus the resident models exceeds the budget) is refused at
// submission with KKM_EBUDGET.
//
// The paper has no serving layer; this is a library service around its
// Algorithm 1 (fits) and Eq. 15 (assignment of new samples).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace kkm {

constexpr int kServerWorkers = 4;
constexpr int kServerMaxWorkers = 64;
constexpr int64_t kServerMaxBatchRows = 65536;
constexpr int kMaxPass = 16;
constexpr uint64_t kSlackBytes = 8ull << 20;  // per job: small buffers, allocator rounding

using Clock = std::chrono::steady_clock;

static int64_t lm_count(int64_t Ni, double s) {
  return std::min<int64_t>(std::max<int64_t>((int64_t)std::ceil(s * (double)Ni - 1e-9), 1), Ni);
}

// Device bytes one kkm_fit call holds at its peak (its workspace plus the
// input copy and the model it returns).
static uint64_t fit_bytes(const kkm_problem& p) {
  const int64_t N = p.N, d = p.d, B = std::max<int32_t>(p.B, 1), C = p.C;
  const int64_t dp = p.kernel.kind == KKM_RMSD ? round_up(d, 24) : round_up(d, 8);
  const int64_t Nmax = (N + B - 1) / B, nL = lm_count(Nmax, p.s);
  const int64_t ldk = round_up(Nmax, 32);
  const int64_t units = ceil_div(nL, kUnitRows) + C;
  const int64_t strips = ceil_div(ldk, kStripCols);
  // one set of kernel-block buffers (two when the fit overlaps the next
  // block with the current inner loop)
  uint64_t blk = 4ull * Nmax * dp + 12ull * Nmax;  // X^i, norms, ids
  blk += 4ull * nL * dp + 12ull * nL;               // landmark rows
  blk += 4ull * nL * ldk;                           // the kernel block
  if (p.opt.precision != KKM_FP32 && p.kernel.kind == KKM_RBF && d < kBf16TensorMinDim)
    blk += 2ull * nL * ldk;  // short rows: the FP16 block beside its FP32 values
  if (p.opt.precision == KKM_BF16) blk += 2ull * (Nmax + nL) * dp + 4ull * (Nmax + nL);
  if (p.opt.precision == KKM_FP8) blk += (uint64_t)(Nmax + nL) * round_up(dp, 16) + 8ull * (Nmax + nL);
  if (p.kernel.kind == KKM_RMSD)  // tensor-core MD path: split-BF16 planes, rotations, refine plan
    blk += 24ull * round_up(p.kernel.n_atoms, 64) * (Nmax + nL) + 16ull * nL * ldk + 8ull * nL +
           4ull * ceil_div(nL, 32) * ceil_div(Nmax, 64);
  const bool two = fit_overlaps(side_by_side_pipeline(p.opt.pipeline), (int)B, p.kernel.kind, p.opt.precision);
  uint64_t b = blk * (two ? 2 : 1);
  b += 4ull * N * d + 4ull * N + 4ull * Nmax;   // input copy, labels out, labels
  b += 4ull * 2 * C * ldk + 8ull * C * dp;       // Eq. 8 / Eq. 12 blocks, medoid rows
  b += 4ull * units * ldk + 8ull * units * strips + 4ull * 6 * ldk;  // inner-loop buffers
  b += 24ull * Nmax;                             // k-means++ scratch
  b += 4ull * nL * dp + 64ull * nL + 8ull * C * dp;  // the model
  if (!(p.kernel.sigma > 0.0f)) {  // the median rule's sample, distances and split-K products
    const int64_t M = std::min<int64_t>(N, 2048);
    const bool split = p.kernel.kind != KKM_RMSD && dp >= kDistSplitMinDp;
    b += 4ull * M * dp + 4ull * M * round_up(M, 4) * (split ? 1 + kDistSplit : 1);
  }
  return b + kSlackBytes;
}

// Device bytes of one kkm_assign call on M rows (device input and outputs
// included), following its chunking of the kernel block.
static uint64_t assign_bytes(const kkm_model* m, int64_t M, int32_t mode) {
  const int64_t rows_ref = mode == KKM_ASSIGN_SUPPORTS ? m->nL : m->C;
  const int64_t chunk = std::max<int64_t>(1024, std::min<int64_t>(M, ((int64_t)1 << 27) / std::max<int64_t>(rows_ref, 1)));
  const int64_t ldm = round_up(std::min(chunk, M), 32);
  const int64_t units = ceil_div(m->nL, kUnitRows) + m->C;
  uint64_t b = 4ull * M * m->d + 8ull * M;     // rows and outputs on the device
  b += 4ull * ldm * (m->dp + 1) + 4ull * rows_ref * ldm;
  if (mode == KKM_ASSIGN_SUPPORTS) b += 4ull * units * ldm + 8ull * units * ceil_div(ldm, kStripCols);
  if (m->kind == KKM_RMSD)  // tensor-core MD path
    b += 24ull * round_up(m->n_atoms, 64) * (rows_ref + ldm) + 16ull * rows_ref * ldm + 8ull * rows_ref +
         4ull * ceil_div(rows_ref, 32) * ceil_div(ldm, 64);
  return b + kSlackBytes;
}

static uint64_t model_bytes(const kkm_model* m) {
  return 4ull * m->nL * m->dp + 64ull * m->nL + 8ull * m->C * m->dp + 256ull * m->C + (64ull << 10);
}

struct Job {
  enum Kind { FIT, ASSIGN } kind;
  uint64_t ticket = 0;
  // fit
  kkm_problem fit{};
  int32_t keep_model = 0;
  int32_t model_out = -1;
  // assign
  int32_t model_id = -1;
  const float* X = nullptr;
  int64_t M = 0;
  int32_t mode = 0;
  int32_t* labels_out = nullptr;
  float* dist_out = nullptr;
  // bookkeeping
  uint64_t bytes = 0;
  int passed = 0;
  double evals = 0.0;
  Clock::time_point t_submit, t_start, t_end;
  bool done = false;
  kkm_status status = KKM_OK;
  std::string error;
};

struct ModelEntry {
  kkm_model* m = nullptr;
  uint64_t bytes = 0;
  int busy = 0;
  bool retired = false;
};

}  // namespace kkm

struct kkm_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<kkm::Job>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<kkm::Job>> jobs;  // submitted, not yet collected
  std::unordered_map<int32_t, kkm::ModelEntry> models;
  int32_t next_model = 0;
  uint64_t next_ticket = 1;
  uint64_t budget = 0, in_use = 0, peak = 0;
  int64_t max_batch_rows = kkm::kServerMaxBatchRows;
  bool stop = false;
  int device = 0;
  std::vector<std::thread> workers;
  // statistics
  std::vector<double> lat_fit, lat_assign;  // ms, submit to completion
  int64_t done_fit = 0, done_assign = 0, failed = 0, refused = 0, fused_launches = 0;
  double evals = 0.0;
  kkm::Clock::time_point t0;
};

namespace kkm {

static double fit_evals(const kkm_problem& p) {
  double e = 0.0;
  const int64_t B = p.B;
  for (int64_t i = 0; i < B; ++i) {
    const int64_t Ni = (p.N - i + B - 1) / B;
    e += (double)Ni * (double)lm_count(Ni, p.s) + 2.0 * (double)Ni * p.C;
  }
  return e + (double)(p.C - 1) * (double)((p.N + B - 1) / B);
}

// Takes the next admissible job (and, for an assign, the waiting assigns it
// can be fused with).  Called with the lock held.
static std::vector<std::shared_ptr<Job>> take_jobs(kkm_server* s) {
  std::vector<std::shared_ptr<Job>> out;
  // Fits that keep their model make the resident set grow after admission
  // checks were made: a queued job that can no longer fit at all fails now.
  uint64_t resident = 0;
  for (auto& kv : s->models) resident += kv.second.bytes;
  bool refused = false;
  for (size_t qi = 0; qi < s->queue.size();) {
    auto& J = s->queue[qi];
    if (resident + J->bytes > s->budget) {
      J->status = KKM_EBUDGET;
      J->error = "the resident models grew: the job no longer fits in the budget";
      J->done = true;
      J->t_start = J->t_end = Clock::now();
      s->refused += 1;
      s->queue.erase(s->queue.begin() + qi);
      refused = true;
    } else {
      ++qi;
    }
  }
  if (refused) s->cv_done.notify_all();
  for (size_t qi = 0; qi < s->queue.size(); ++qi) {
    auto& J = s->queue[qi];
    if (s->in_use + J->bytes > s->budget) {
      if (J->passed >= kMaxPass) return out;  // nothing may pass it any more
      continue;
    }
    for (size_t k = 0; k < qi; ++k) s->queue[k]->passed += 1;
    out.push_back(J);
    s->in_use += J->bytes;
    s->queue.erase(s->queue.begin() + qi);
    if (J->kind == Job::ASSIGN) {
      // fuse the later waiting assigns on the same model and mode
      int64_t rows = J->M;
      for (size_t k = 0; k < s->queue.size();) {
        auto& K = s->queue[k];
        if (K->kind == Job::ASSIGN && K->model_id == J->model_id && K->mode == J->mode &&
            rows + K->M <= s->max_batch_rows && s->in_use + K->bytes <= s->budget) {
          rows += K->M;
          s->in_use += K->bytes;
          out.push_back(K);
          s->queue.erase(s->queue.begin() + k);
        } else {
          ++k;
        }
      }
      s->models[J->model_id].busy += 1;
    }
    break;
  }
  s->peak = std::max(s->peak, s->in_use);
  return out;
}

static kkm_status run_fit(kkm_server* s, Job& J, cudaStream_t st) {
  kkm_problem p = J.fit;
  kkm_options opt = p.opt;
  opt.stream = st;
  opt.pipeline = side_by_side_pipeline(opt.pipeline);
  opt.iteration = side_by_side_iteration(opt.iteration);
  kkm_model* m = nullptr;
  const kkm_status r = kkm_fit(p.X, p.N, p.d, p.C, p.B, p.s, &p.kernel, p.iters, p.seed, &opt, p.labels_out,
                               J.keep_model ? &m : nullptr);
  if (r != KKM_OK) {
    J.error = kkm_last_error();
    return r;
  }
  J.evals = fit_evals(p);
  if (m) {
    std::lock_guard<std::mutex> lk(s->mu);
    const int32_t id = s->next_model++;
    ModelEntry& e = s->models[id];
    e.m = m;
    e.bytes = model_bytes(m);
    s->in_use += e.bytes;
    s->peak = std::max(s->peak, s->in_use);
    J.model_out = id;
  }
  return KKM_OK;
}

// One kkm_assign over the concatenated rows of the fused jobs.
static kkm_status run_assigns(kkm_server* s, std::vector<std::shared_ptr<Job>>& js, cudaStream_t st,
                              std::string* err) {
  kkm_model* m = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    m = s->models[js[0]->model_id].m;
  }
  const int64_t d = m->d;
  int64_t R = 0;
  for (auto& J : js) R += J->M;
  if (R == 0) return KKM_OK;
  float* X = nullptr;
  int32_t* lab = nullptr;
  float* dist = nullptr;
  auto fail = [&](cudaError_t e, const char* what) {
    cudaGetLastError();
    *err = std::string(what) + ": " + cudaGetErrorString(e);
    return KKM_ECUDA;
  };
  cudaError_t e = cudaMallocAsync(&X, (size_t)R * d * 4, st);
  if (e != cudaSuccess) return fail(e, "cudaMallocAsync");
  e = cudaMallocAsync(&lab, (size_t)R * 4, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&dist, (size_t)R * 4, st);
  kkm_status r = KKM_OK;
  if (e != cudaSuccess) {
    r = fail(e, "cudaMallocAsync");
  } else {
    int64_t off = 0;
    for (auto& J : js) {
      e = cudaMemcpyAsync(X + off * d, J->X, (size_t)J->M * d * 4, cudaMemcpyDefault, st);
      if (e != cudaSuccess) break;
      off += J->M;
    }
    if (e != cudaSuccess) {
      r = fail(e, "cudaMemcpyAsync");
    } else {
      r = kkm_assign(m, X, R, js[0]->mode, lab, dist, st);
      if (r != KKM_OK) {
        *err = kkm_last_error();
      } else {
        off = 0;
        for (auto& J : js) {
          if (J->labels_out)
            e = cudaMemcpyAsync(J->labels_out, lab + off, (size_t)J->M * 4, cudaMemcpyDefault, st);
          if (e == cudaSuccess && J->dist_out)
            e = cudaMemcpyAsync(J->dist_out, dist + off, (size_t)J->M * 4, cudaMemcpyDefault, st);
          if (e != cudaSuccess) break;
          off += J->M;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = fail(e, "copy-out");
      }
    }
  }
  if (X) cudaFreeAsync(X, st);
  if (lab) cudaFreeAsync(lab, st);
  if (dist) cudaFreeAsync(dist, st);
  cudaStreamSynchronize(st);
  const int64_t nref = js[0]->mode == KKM_ASSIGN_SUPPORTS ? m->nL : m->C;
  for (auto& J : js) J->evals = (double)J->M * (double)nref;
  return r;
}

static void worker_loop(kkm_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    st = nullptr;
  }
  for (;;) {
    std::vector<std::shared_ptr<Job>> js;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        if (s->stop && s->queue.empty()) return true;
        js = take_jobs(s);
        return !js.empty();
      });
      if (js.empty()) break;  // stopping, queue drained
    }
    const auto t_start = Clock::now();
    for (auto& J : js) J->t_start = t_start;
    kkm_status r = KKM_OK;
    std::string err;
    if (!st) {
      r = KKM_ECUDA;
      err = "worker stream unavailable";
    } else if (js[0]->kind == Job::FIT) {
      NvtxRange nv("server fit job");
      r = run_fit(s, *js[0], st);
      err = js[0]->error;
    } else {
      NvtxRange nv("server assign batch");
      r = run_assigns(s, js, st, &err);
    }
    const auto t_end = Clock::now();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto& J : js) {
        s->in_use -= J->bytes;
        J->t_end = t_end;
        J->status = r;
        J->error = err;
        J->done = true;
        const double ms = std::chrono::duration<double, std::milli>(t_end - J->t_submit).count();
        if (r == KKM_OK) {
          (J->kind == Job::FIT ? s->lat_fit : s->lat_assign).push_back(ms);
          (J->kind == Job::FIT ? s->done_fit : s->done_assign) += 1;
          s->evals += J->evals;
        } else {
          s->failed += 1;
        }
      }
      if (js[0]->kind == Job::ASSIGN) {
        s->fused_launches += 1;
        auto it = s->models.find(js[0]->model_id);
        if (it != s->models.end()) {
          it->second.busy -= 1;
          if (it->second.retired && it->second.busy == 0) {
            s->in_use -= it->second.bytes;
            kkm_model_free(it->second.m);
            s->models.erase(it);
          }
        }
      }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();  // memory was released: others may now fit
  }
  if (st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
}

static kkm_status enqueue(kkm_server* s, std::shared_ptr<Job> J, uint64_t* ticket) {
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    set_error("server is shutting down");
    return KKM_EINVAL;
  }
  uint64_t resident = 0;
  for (auto& kv : s->models) resident += kv.second.bytes;
  if (resident + J->bytes > s->budget) {
    s->refused += 1;
    set_error("job needs about " + std::to_string(J->bytes >> 20) + " MiB of device memory; the budget leaves " +
              std::to_string((s->budget - std::min(s->budget, resident)) >> 20) + " MiB beside the resident models");
    return KKM_EBUDGET;
  }
  J->ticket = s->next_ticket++;
  J->t_submit = Clock::now();
  s->jobs[J->ticket] = J;
  s->queue.push_back(J);
  *ticket = J->ticket;
  s->cv_work.notify_one();
  return KKM_OK;
}

static double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t lo = (size_t)std::floor(pos), hi = (size_t)std::ceil(pos);
  return v[lo] + (v[hi] - v[lo]) * (pos - (double)lo);
}

}  // namespace kkm

using namespace kkm;

extern "C" {

kkm_status kkm_server_create(const kkm_server_config* cfg, kkm_server** out) {
  set_error("");
  if (!cfg || !out) {
    set_error("cfg and out must not be NULL");
    return KKM_EINVAL;
  }
  *out = nullptr;
  const int W = cfg->n_workers > 0 ? cfg->n_workers : kServerWorkers;
  if (cfg->n_workers < 0 || W > kServerMaxWorkers || cfg->budget_bytes == 0 || cfg->max_batch_rows < 0 ||
      cfg->reserved != 0) {
    set_error("n_workers must be in [0, 64], budget_bytes > 0, max_batch_rows >= 0, reserved == 0");
    return KKM_EINVAL;
  }
  try {
    auto* s = new kkm_server();
    s->budget = cfg->budget_bytes;
    s->max_batch_rows = cfg->max_batch_rows > 0 ? cfg->max_batch_rows : kServerMaxBatchRows;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      set_error("no CUDA device");
      return KKM_ECUDA;
    }
    s->t0 = Clock::now();
    for (int w = 0; w < W; ++w) s->workers.emplace_back(worker_loop, s);
    *out = s;
    return KKM_OK;
  } catch (...) {
    set_error("could not start the worker threads");
    return KKM_EINTERNAL;
  }
}

void kkm_server_destroy(kkm_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->models) kkm_model_free(kv.second.m);
  delete s;
}

kkm_status kkm_server_add_model(kkm_server* s, kkm_model* m, int32_t* model_id) {
  set_error("");
  if (!s || !m || !model_id) {
    set_error("server, model and model_id must not be NULL");
    return KKM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  const uint64_t b = model_bytes(m);
  uint64_t resident = 0;
  for (auto& kv : s->models) resident += kv.second.bytes;
  if (resident + b > s->budget) {
    set_error("the resident models would exceed the budget");
    return KKM_EBUDGET;
  }
  const int32_t id = s->next_model++;
  s->models[id] = ModelEntry{m, b, 0, false};
  s->in_use += b;
  s->peak = std::max(s->peak, s->in_use);
  *model_id = id;
  return KKM_OK;
}

kkm_status kkm_server_remove_model(kkm_server* s, int32_t model_id) {
  set_error("");
  if (!s) return KKM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->models.find(model_id);
  if (it == s->models.end() || it->second.retired) {
    set_error("unknown model id");
    return KKM_EINVAL;
  }
  bool queued = false;
  for (auto& J : s->queue) queued |= (J->kind == Job::ASSIGN && J->model_id == model_id);
  if (queued) {
    set_error("jobs for this model are still queued");
    return KKM_EINVAL;
  }
  if (it->second.busy > 0) {
    it->second.retired = true;  // freed when its running jobs finish
  } else {
    s->in_use -= it->second.bytes;
    kkm_model_free(it->second.m);
    s->models.erase(it);
  }
  return KKM_OK;
}

kkm_status kkm_server_submit_fit(kkm_server* s, const kkm_problem* p, int32_t keep_model, uint64_t* ticket) {
  set_error("");
  if (!s || !p || !ticket) {
    set_error("server, problem and ticket must not be NULL");
    return KKM_EINVAL;
  }
  if (p->N < 1 || p->d < 1 || p->C < 1 || p->B < 1 || p->B > p->N || !(p->s > 0.0 && p->s <= 1.0)) {
    set_error("bad problem sizes");
    return KKM_EINVAL;
  }
  auto J = std::make_shared<Job>();
  J->kind = Job::FIT;
  J->fit = *p;
  J->keep_model = keep_model;
  J->bytes = fit_bytes(*p);
  return enqueue(s, J, ticket);
}

kkm_status kkm_server_submit_assign(kkm_server* s, int32_t model_id, const float* X, int64_t M, int32_t mode,
                                    int32_t* labels_out, float* dist_out, uint64_t* ticket) {
  set_error("");
  if (!s || !ticket || (M > 0 && (!X || !labels_out)) || M < 0) {
    set_error("bad arguments");
    return KKM_EINVAL;
  }
  if (mode != KKM_ASSIGN_SUPPORTS && mode != KKM_ASSIGN_MEDOIDS) {
    set_error("unknown assign mode");
    return KKM_EINVAL;
  }
  auto J = std::make_shared<Job>();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->models.find(model_id);
    if (it == s->models.end() || it->second.retired) {
      set_error("unknown model id");
      return KKM_EINVAL;
    }
    J->bytes = assign_bytes(it->second.m, M, mode);
  }
  J->kind = Job::ASSIGN;
  J->model_id = model_id;
  J->X = X;
  J->M = M;
  J->mode = mode;
  J->labels_out = labels_out;
  J->dist_out = dist_out;
  return enqueue(s, J, ticket);
}

kkm_status kkm_server_wait(kkm_server* s, uint64_t ticket, int32_t timeout_ms, kkm_status* job_status,
                           int32_t* model_id_out) {
  set_error("");
  if (!s || !job_status) return KKM_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) {
    set_error("unknown ticket (never issued, or already collected)");
    return KKM_EINVAL;
  }
  std::shared_ptr<Job> J = it->second;
  auto ready = [&] { return J->done; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    set_error("job not finished yet");
    return KKM_ETIMEOUT;
  }
  *job_status = J->status;
  if (model_id_out) *model_id_out = J->model_out;
  if (J->status != KKM_OK) set_error(J->error);
  s->jobs.erase(ticket);
  return KKM_OK;
}

kkm_status kkm_server_stats(kkm_server* s, kkm_serving_stats* out) {
  set_error("");
  if (!s || !out) return KKM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out->completed_fit = s->done_fit;
  out->completed_assign = s->done_assign;
  out->failed = s->failed;
  out->refused = s->refused;
  out->fused_assign_launches = s->fused_launches;
  out->queued = (int64_t)s->queue.size();
  out->p50_fit_ms = percentile(s->lat_fit, 0.50);
  out->p99_fit_ms = percentile(s->lat_fit, 0.99);
  out->p50_assign_ms = percentile(s->lat_assign, 0.50);
  out->p99_assign_ms = percentile(s->lat_assign, 0.99);
  out->kernel_evals = s->evals;
  out->seconds = std::chrono::duration<double>(Clock::now() - s->t0).count();
  out->bytes_in_use = s->in_use;
  out->peak_bytes = s->peak;
  return KKM_OK;
}

kkm_status kkm_server_reset_stats(kkm_server* s) {
  if (!s) return KKM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_fit.clear();
  s->lat_assign.clear();
  s->done_fit = s->done_assign = s->failed = s->refused = s->fused_launches = 0;
  s->evals = 0.0;
  s->peak = s->in_use;
  s->t0 = Clock::now();
  return KKM_OK;
}

}  // extern "C"
