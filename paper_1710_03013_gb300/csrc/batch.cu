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
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace kkm {

// Default number of concurrent streams for a batch.
constexpr int kBatchStreams = 8;
constexpr int kBatchMaxStreams = 64;

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
                             kkm_status* status_out, cudaStream_t caller) {
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

  auto worker = [&](int w) {
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
  };
  std::vector<std::thread> threads;
  threads.reserve(W);
  for (int w = 0; w < W; ++w) threads.emplace_back(worker, w);
  for (auto& t : threads) t.join();
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
