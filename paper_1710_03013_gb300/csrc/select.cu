// Model selection around Algorithm 1: restarts that keep the solution of
// minimum cost (Section 4.5) and the number of clusters by the elbow
// criterion over a range of C (Sections 4.4, 4.5).  Every fit is an ordinary
// kkm_fit run through kkm_fit_batch (the restarts and the (C, restart) pairs
// are independent problems on one GPU at once); the costs are kkm_cost
// (Eq. 1 against the final global medoids).  Only the choice among a few
// costs is made on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <string>
#include <vector>

#include "internal.h"

namespace kkm {

static kkm_status sel_invalid(const std::string& msg) {
  set_error(msg);
  return KKM_EINVAL;
}

// Device view of X: the pointer itself, or one copy for every fit of the
// selection (so the restarts do not each copy a host input).
struct DeviceX {
  const float* p = nullptr;
  float* own = nullptr;
  ~DeviceX() {
    if (own) cudaFree(own);
  }
  kkm_status init(const float* X, int64_t n, cudaStream_t st) {
    cudaPointerAttributes a;
    const bool dev = cudaPointerGetAttributes(&a, X) == cudaSuccess &&
                     (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev) {
      p = X;
      return KKM_OK;
    }
    KKM_CK(cudaMalloc(&own, (size_t)n * sizeof(float)));
    KKM_CK(cudaMemcpyAsync(own, X, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, st));
    KKM_CK(cudaStreamSynchronize(st));
    p = own;
    return KKM_OK;
  }
};

// Restart seeds: the first n outputs of SplitMix64(seed).
static std::vector<uint64_t> restart_seeds(uint64_t seed, int n) {
  SplitMix64 g(seed);
  std::vector<uint64_t> s((size_t)n);
  for (auto& v : s) v = g.next();
  return s;
}

// The kernel every fit of a selection uses: the median rule resolved once
// (seed's bandwidth stream) when sigma <= 0, so the costs compare fits of one
// kernel.
static kkm_status shared_kernel(const float* Xd, int64_t N, int64_t d, const kkm_kernel* k, uint64_t seed,
                                kkm_kernel* out) {
  *out = *k;
  if (k->kind != KKM_LINEAR && !(k->sigma > 0.0f)) {
    float sig = 0.0f;
    KKM_TRY(kkm_median_bandwidth(Xd, N, d, k, seed, &sig));
    out->sigma = sig;
  }
  return KKM_OK;
}

// Fits the given problems as one batch and returns each one's Eq. 1 cost
// against its final medoids; models_keep[r] (nullable entries) receive the
// models the caller keeps, the others are freed.
static kkm_status fit_and_cost(std::vector<kkm_problem>& P, const float* Xd, int64_t N, cudaStream_t st,
                               std::vector<double>* costs, std::vector<kkm_model*>* models) {
  const int n = (int)P.size();
  models->assign(n, nullptr);
  std::vector<kkm_status> status(n, KKM_OK);
  const kkm_status bs = kkm_fit_batch(P.data(), n, std::min(n, 8), models->data(), status.data(), st);
  if (bs != KKM_OK) {
    for (auto* m : *models) kkm_model_free(m);
    models->assign(n, nullptr);
    return bs;
  }
  costs->assign(n, 0.0);
  for (int r = 0; r < n; ++r) {
    const kkm_status cs = kkm_cost((*models)[r], Xd, N, KKM_ASSIGN_MEDOIDS, &(*costs)[r], st);
    if (cs != KKM_OK) {
      for (auto* m : *models) kkm_model_free(m);
      models->assign(n, nullptr);
      return cs;
    }
  }
  return KKM_OK;
}

static kkm_status check_common(const float* X, int64_t N, int64_t d, int32_t n_restarts, const kkm_options* opt) {
  if (!X) return sel_invalid("X is NULL");
  if (N < 1 || d < 1) return sel_invalid("N and d must be >= 1");
  if (n_restarts < 1 || n_restarts > 1024) return sel_invalid("n_restarts must be in [1, 1024]");
  if (opt && opt->init_medoids) return sel_invalid("restarts differ by their k-means++ seeding: init_medoids must be NULL");
  return KKM_OK;
}

static kkm_status restarts_impl(const float* X, int64_t N, int64_t d, int32_t C, int32_t B, double s,
                                const kkm_kernel* k, int32_t iters, uint64_t seed, int32_t R,
                                const kkm_options* opt_in, int32_t* labels_out, kkm_model** model_out,
                                double* costs_out, int32_t* best_out) {
  KKM_TRY(check_common(X, N, d, R, opt_in));
  if (!k) return sel_invalid("kernel is NULL");
  kkm_options opt;
  kkm_options_default(&opt);
  if (opt_in) opt = *opt_in;
  cudaStream_t st = (cudaStream_t)opt.stream;
  DeviceX xd;
  KKM_TRY(xd.init(X, N * d, st));
  kkm_kernel kk;
  KKM_TRY(shared_kernel(xd.p, N, d, k, seed, &kk));
  // per-restart labels on the device when the caller wants the winner's
  int32_t* lab = nullptr;
  std::unique_ptr<void, void (*)(void*)> lab_guard(nullptr, [](void* q) { cudaFree(q); });
  if (labels_out) {
    KKM_CK(cudaMalloc(&lab, (size_t)R * N * sizeof(int32_t)));
    lab_guard.reset(lab);
  }
  const std::vector<uint64_t> seeds = restart_seeds(seed, R);
  std::vector<kkm_problem> P((size_t)R);
  for (int r = 0; r < R; ++r) {
    kkm_problem& p = P[r];
    p.X = xd.p;
    p.N = N;
    p.d = d;
    p.C = C;
    p.B = B;
    p.s = s;
    p.kernel = kk;
    p.iters = iters;
    p.seed = seeds[r];
    p.opt = opt;
    p.labels_out = lab ? lab + (size_t)r * N : nullptr;
  }
  std::vector<double> costs;
  std::vector<kkm_model*> models;
  KKM_TRY(fit_and_cost(P, xd.p, N, st, &costs, &models));
  int best = 0;
  for (int r = 1; r < R; ++r)
    if (costs[r] < costs[best]) best = r;  // lowest restart on ties
  if (costs_out)
    for (int r = 0; r < R; ++r) costs_out[r] = costs[r];
  if (best_out) *best_out = best;
  for (int r = 0; r < R; ++r)
    if (r != best || !model_out) kkm_model_free(models[r]);
  if (model_out) *model_out = models[best];
  if (labels_out) {
    KKM_CK(cudaMemcpyAsync(labels_out, lab + (size_t)best * N, (size_t)N * sizeof(int32_t), cudaMemcpyDefault, st));
    KKM_CK(cudaStreamSynchronize(st));
  }
  return KKM_OK;
}

// The elbow of a cost curve over consecutive C: the point farthest below the
// chord joining its end points, both axes scaled to [0, 1] (lowest C on ties).
static int elbow_index(const std::vector<double>& y) {
  const int n = (int)y.size();
  if (n <= 2) return 0;
  const double lo = *std::min_element(y.begin(), y.end()), hi = *std::max_element(y.begin(), y.end());
  if (!(hi > lo)) return 0;
  const double y0 = (y[0] - lo) / (hi - lo), y1 = (y[n - 1] - lo) / (hi - lo);
  int best = 0;
  double gap = -INFINITY;
  for (int q = 0; q < n; ++q) {
    const double x = (double)q / (double)(n - 1);
    const double g = (y0 + (y1 - y0) * x) - (y[q] - lo) / (hi - lo);
    if (g > gap) {
      gap = g;
      best = q;
    }
  }
  return best;
}

static kkm_status elbow_impl(const float* X, int64_t N, int64_t d, int32_t C_lo, int32_t C_hi, int32_t B, double s,
                             const kkm_kernel* k, int32_t iters, uint64_t seed, int32_t R, const kkm_options* opt_in,
                             double* costs_out, int32_t* C_out) {
  KKM_TRY(check_common(X, N, d, R, opt_in));
  if (!k) return sel_invalid("kernel is NULL");
  if (C_lo < 1 || C_hi <= C_lo || C_hi > kMaxC) return sel_invalid("need 1 <= C_lo < C_hi <= 256");
  kkm_options opt;
  kkm_options_default(&opt);
  if (opt_in) opt = *opt_in;
  cudaStream_t st = (cudaStream_t)opt.stream;
  DeviceX xd;
  KKM_TRY(xd.init(X, N * d, st));
  kkm_kernel kk;
  KKM_TRY(shared_kernel(xd.p, N, d, k, seed, &kk));
  const std::vector<uint64_t> seeds = restart_seeds(seed, R);
  const int nC = C_hi - C_lo + 1;
  std::vector<kkm_problem> P((size_t)nC * R);
  for (int c = 0; c < nC; ++c)
    for (int r = 0; r < R; ++r) {
      kkm_problem& p = P[(size_t)c * R + r];
      p.X = xd.p;
      p.N = N;
      p.d = d;
      p.C = C_lo + c;
      p.B = B;
      p.s = s;
      p.kernel = kk;
      p.iters = iters;
      p.seed = seeds[r];
      p.opt = opt;
      p.labels_out = nullptr;
    }
  std::vector<double> costs;
  std::vector<kkm_model*> models;
  KKM_TRY(fit_and_cost(P, xd.p, N, st, &costs, &models));
  for (auto* m : models) kkm_model_free(m);
  std::vector<double> best((size_t)nC);
  for (int c = 0; c < nC; ++c) {
    best[c] = costs[(size_t)c * R];
    for (int r = 1; r < R; ++r) best[c] = std::min(best[c], costs[(size_t)c * R + r]);
  }
  if (costs_out)
    for (int c = 0; c < nC; ++c) costs_out[c] = best[c];
  if (C_out) *C_out = C_lo + elbow_index(best);
  return KKM_OK;
}

}  // namespace kkm

extern "C" kkm_status kkm_fit_restarts(const float* X, int64_t N, int64_t d, int32_t C, int32_t B, double s,
                                       const kkm_kernel* k, int32_t iters, uint64_t seed, int32_t n_restarts,
                                       const kkm_options* opt, int32_t* labels_out, kkm_model** model_out,
                                       double* costs_out, int32_t* best_out) {
  kkm::set_error("");
  try {
    return kkm::restarts_impl(X, N, d, C, B, s, k, iters, seed, n_restarts, opt, labels_out, model_out, costs_out,
                              best_out);
  } catch (...) {
    kkm::set_error("internal exception");
    return KKM_EINTERNAL;
  }
}

extern "C" kkm_status kkm_elbow(const float* X, int64_t N, int64_t d, int32_t C_lo, int32_t C_hi, int32_t B,
                                double s, const kkm_kernel* k, int32_t iters, uint64_t seed, int32_t n_restarts,
                                const kkm_options* opt, double* costs_out, int32_t* C_out) {
  kkm::set_error("");
  try {
    return kkm::elbow_impl(X, N, d, C_lo, C_hi, B, s, k, iters, seed, n_restarts, opt, costs_out, C_out);
  } catch (...) {
    kkm::set_error("internal exception");
    return KKM_EINTERNAL;
  }
}
