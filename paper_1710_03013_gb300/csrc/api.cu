// C-ABI entry points and host orchestration of Algorithm 1.
//
// The host side only validates arguments, draws the random numbers of the
// method (SplitMix64, Steele, Lea & Flood 2014: landmark sets, k-means++
// draws, the bandwidth sample), allocates stream-ordered device memory and
// enqueues kernels.  Every step of the clustering itself runs on the device;
// one mini-batch needs no host synchronisation between its kernels (early stop
// is a device flag that makes the remaining launches return at once).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <mutex>
#include <type_traits>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"

// The opaque model (struct kkm_model) is defined in internal.h.

namespace kkm {

// ======================================================================
// Errors
// ======================================================================
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
kkm_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  cudaGetLastError();
  set_error(std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
            ") in " + what + " at " + file + ":" + std::to_string(line));
  return e == cudaErrorMemoryAllocation ? KKM_ENOMEM : KKM_ECUDA;
}
static kkm_status invalid(const std::string& msg) {
  set_error(msg);
  return KKM_EINVAL;
}

// ======================================================================
// Profiling (per-kernel CUDA-event timing)
// ======================================================================
struct ProfEntry {
  int64_t launches = 0;
  double ms = 0.0;
  double work = 0.0;  // data-dependent work units reported by the kernel's host code
};
struct Pending {
  const char* name;
  cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static int g_prof_on = 0;  // 0 off, 1 time every launch, 2 count all, time the heavy kernels

static bool heavy_kernel(const char* name) {
  return !strcmp(name, "gram_block") || !strcmp(name, "rmsd_block") || !strcmp(name, "rmsd_exact") ||
         !strcmp(name, "fhat_partial") || !strcmp(name, "iterate") || !strcmp(name, "fhat_multi");
}
static std::unordered_map<std::string, ProfEntry> g_prof;
static std::vector<Pending> g_pending;
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// the name of the innermost profiled launch of this thread
static thread_local const char* t_prof_scope = nullptr;

void prof_more_launches(int k) {
  if (!g_prof_on || !t_prof_scope || k <= 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof[t_prof_scope].launches += k;
}

ProfScope::ProfScope(const char* n, cudaStream_t s) : name(n), stream(s) {
  prev_scope = t_prof_scope;
  t_prof_scope = n;
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_prof_on == 2 && !heavy_kernel(name)) {
    g_prof[name].launches += 1;
    return;
  }
  a = take_event();
  b = take_event();
  cudaEventRecord(a, s);
}
// The pair is queued only once both events are recorded, so a concurrent
// prof_collect (another thread's call) never sees a half-recorded pair.
ProfScope::~ProfScope() {
  t_prof_scope = prev_scope;
  if (!a) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEventRecord(b, stream);
  g_pending.push_back(Pending{name, a, b});
}
void prof_collect() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& p : g_pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      auto& e = g_prof[p.name];
      e.launches += 1;
      e.ms += ms;
    }
    cudaGetLastError();
    g_event_pool.push_back(p.a);
    g_event_pool.push_back(p.b);
  }
  g_pending.clear();
}

bool prof_on() { return g_prof_on != 0; }
void prof_add_work(const char* name, double units) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof[name].work += units;
}

#define KKM_RUN(name, st, call)                 \
  do {                                          \
    ::kkm::ProfScope _ps(name, st);             \
    KKM_CK(call);                               \
  } while (0)

// First k entries of a partial Fisher-Yates shuffle of [0, n): step a swaps
// positions a and a + floor(u (n - a)).  When k is small against n only the
// positions the swaps touched are held (open addressing, identity elsewhere),
// so drawing a few thousand of N samples costs O(k), not O(N).
static std::vector<int64_t> partial_shuffle(int64_t n, int64_t k, SplitMix64& rng) {
  if (k * 8 >= n) {
    std::vector<int64_t> idx((size_t)n);
    for (int64_t a = 0; a < n; ++a) idx[(size_t)a] = a;
    for (int64_t a = 0; a < k; ++a) {
      const int64_t r = a + (int64_t)floor(rng.u01() * (double)(n - a));
      std::swap(idx[(size_t)a], idx[(size_t)r]);
    }
    idx.resize((size_t)k);
    return idx;
  }
  size_t cap = 16;
  int bits = 4;
  while (cap < (size_t)(4 * k)) cap <<= 1, ++bits;
  std::vector<int64_t> key(cap, -1), val(cap, 0);
  auto at = [&](int64_t pos) -> int64_t& {
    size_t h = (size_t)(((uint64_t)pos * 0x9E3779B97F4A7C15ull) >> (64 - bits));
    while (key[h] != pos) {
      if (key[h] < 0) {
        key[h] = pos;
        val[h] = pos;
        break;
      }
      h = (h + 1) & (cap - 1);
    }
    return val[h];
  };
  for (int64_t a = 0; a < k; ++a) {
    const int64_t r = a + (int64_t)floor(rng.u01() * (double)(n - a));
    int64_t& va = at(a);
    int64_t& vr = at(r);
    std::swap(va, vr);
  }
  std::vector<int64_t> out((size_t)k);
  for (int64_t a = 0; a < k; ++a) out[(size_t)a] = at(a);
  return out;
}

// The same k picks in increasing order, by a bitmap over [0, n) (a sort of
// thousands of random indices costs far more on the host).
static void sorted_picks(int64_t n, int64_t k, SplitMix64& rng, int32_t* out) {
  const std::vector<int64_t> p = partial_shuffle(n, k, rng);
  std::vector<uint64_t> bm((size_t)((n + 63) / 64), 0);
  for (int64_t v : p) bm[(size_t)(v >> 6)] |= 1ull << (v & 63);
  int64_t c = 0;
  for (size_t w = 0; w < bm.size(); ++w)
    for (uint64_t b = bm[w]; b; b &= b - 1) out[c++] = (int32_t)((int64_t)w * 64 + __builtin_ctzll(b));
}

// Eq. 18 solved for |L|.
static int64_t n_landmarks(int64_t Ni, double s) {
  int64_t nl = (int64_t)ceil(s * (double)Ni - 1e-9);
  return std::min<int64_t>(std::max<int64_t>(nl, 1), Ni);
}

// ======================================================================
// Device memory helpers
// ======================================================================
static void setup_pool_once(int dev) {
  static std::mutex mu;
  static std::vector<int> done;
  std::lock_guard<std::mutex> lk(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done.push_back(dev);
}

// Stream-ordered scratch of one call, freed in stream order when the call
// returns.  Buffers of up to 64 KB are carved (256-byte aligned) from 1 MB
// slabs: a fit asks for some forty small arrays, and one pool allocation
// each costs more host time than the kernels that use them.
struct Workspace {
  static constexpr size_t kSlab = 1u << 20, kSmall = 64u << 10, kAlign = 256;
  cudaStream_t st;
  std::vector<void*> ptrs;
  char* slab = nullptr;
  size_t slab_used = kSlab;
  explicit Workspace(cudaStream_t s) : st(s) {}
  ~Workspace() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
  template <typename T>
  kkm_status alloc(T** p, int64_t n) {
    void* q = nullptr;
    const size_t bytes = (size_t)std::max<int64_t>(n, 1) * sizeof(T);
    if (bytes <= kSmall) {
      const size_t rounded = (bytes + kAlign - 1) / kAlign * kAlign;
      if (slab_used + rounded > kSlab) {
        void* fresh = nullptr;
        KKM_CK(cudaMallocAsync(&fresh, kSlab, st));
        ptrs.push_back(fresh);
        slab = static_cast<char*>(fresh);
        slab_used = 0;
      }
      q = slab + slab_used;
      slab_used += rounded;
    } else {
      KKM_CK(cudaMallocAsync(&q, bytes, st));
      ptrs.push_back(q);
    }
    *p = reinterpret_cast<T*>(q);
    return KKM_OK;
  }
};

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller input: the pointer itself if it is device memory,
// otherwise a workspace copy.
template <typename T>
static kkm_status device_input(Workspace& ws, const T* p, int64_t n, const T** out) {
  if (n <= 0 || is_device_ptr(p)) {
    *out = p;
    return KKM_OK;
  }
  T* d = nullptr;
  KKM_TRY(ws.alloc(&d, n));
  KKM_CK(cudaMemcpyAsync(d, p, (size_t)n * sizeof(T), cudaMemcpyHostToDevice, ws.st));
  *out = d;
  return KKM_OK;
}

// Caller input X (n floats) on the device, with *bad set when it holds NaN
// or Inf (checked before any other work).  Device memory is checked in
// place; pinned host memory is copied and checked by one kernel that reads
// it directly; other host memory is copied, then checked.
// Pinned host words for the finite-input flag of a call whose host work goes
// on while the check runs (a pool shared by all threads; never freed).
static std::mutex g_flag_mu;
static std::vector<int*> g_flag_free;
static int* pinned_flag_acquire() {
  std::lock_guard<std::mutex> lk(g_flag_mu);
  if (g_flag_free.empty()) {
    int* blk = nullptr;
    if (cudaHostAlloc(&blk, 64 * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (int q = 0; q < 64; ++q) g_flag_free.push_back(blk + q);
  }
  int* f = g_flag_free.back();
  g_flag_free.pop_back();
  return f;
}
static void pinned_flag_release(int* f) {
  if (!f) return;
  std::lock_guard<std::mutex> lk(g_flag_mu);
  g_flag_free.push_back(f);
}
// Pinned host buffers for the read-backs at the end of a call: the copies
// into them are asynchronous, so one synchronisation covers them all (a copy
// into pageable memory returns only once it is done).  A pool shared by all
// threads, never freed; a buffer grows when a call needs more.
struct PinnedStage {
  char* p = nullptr;
  size_t cap = 0;
};
static std::vector<PinnedStage> g_stage_free;
static PinnedStage pinned_stage_acquire(size_t bytes) {
  PinnedStage b;
  {
    std::lock_guard<std::mutex> lk(g_flag_mu);
    if (!g_stage_free.empty()) {
      b = g_stage_free.back();
      g_stage_free.pop_back();
    }
  }
  if (b.cap < bytes) {
    if (b.p) cudaFreeHost(b.p);
    b.cap = std::max<size_t>(bytes, 64u << 10);
    if (cudaHostAlloc(reinterpret_cast<void**>(&b.p), b.cap, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      b = PinnedStage();
    }
  }
  return b;
}
static void pinned_stage_release(const PinnedStage& b) {
  if (!b.p) return;
  std::lock_guard<std::mutex> lk(g_flag_mu);
  g_stage_free.push_back(b);
}
// Device -> host copies of one call gathered in a pinned stage: add() lays
// out the pieces (16-byte aligned), run() issues the copies and waits once,
// then copies every piece to its destination.
struct Readback {
  struct Piece {
    void* dst;
    const void* src;
    size_t bytes, off;
  };
  std::vector<Piece> pieces;
  size_t total = 0;
  void add(void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return;
    pieces.push_back({dst, src, bytes, total});
    total += (bytes + 15) & ~size_t(15);
  }
  kkm_status run(cudaStream_t st) {
    PinnedStage b = pinned_stage_acquire(total);
    if (!b.p) {  // no pinned memory: pageable copies
      for (auto& q : pieces) KKM_CK(cudaMemcpyAsync(q.dst, q.src, q.bytes, cudaMemcpyDeviceToHost, st));
      KKM_CK(cudaStreamSynchronize(st));
      return KKM_OK;
    }
    for (auto& q : pieces) {
      const cudaError_t e = cudaMemcpyAsync(b.p + q.off, q.src, q.bytes, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        pinned_stage_release(b);
        return cuda_fail(e, "cudaMemcpyAsync (read-back)", __FILE__, __LINE__);
      }
    }
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
      for (auto& q : pieces) memcpy(q.dst, b.p + q.off, q.bytes);
    pinned_stage_release(b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize (read-back)", __FILE__, __LINE__);
    return KKM_OK;
  }
};

// The answer of a finite-input check enqueued without waiting for it.
struct PendingCheck {
  int* flag = nullptr;  // pinned
  cudaStream_t st = nullptr;
  ~PendingCheck() { pinned_flag_release(flag); }
  kkm_status wait(bool* bad) {
    *bad = false;
    if (!flag) return KKM_OK;
    KKM_CK(cudaStreamSynchronize(st));
    *bad = *flag != 0;
    return KKM_OK;
  }
};

// With `pending`, the check is only enqueued (its flag lands in pinned host
// memory) and pending->wait gives the answer; else this call waits for it.
// With pull_flag (a caller that fetches every row of X through
// prep_rows), pinned host X 16-byte aligned is used in place: *out is its
// device address, nothing is copied or checked here, and *pull_flag is a
// zeroed device word for the rows' check.
static kkm_status device_input_checked(Workspace& ws, const float* p, int64_t n, const float** out, bool* bad,
                                       PendingCheck* pending = nullptr, int** pull_flag = nullptr) {
  cudaStream_t st = ws.st;
  *bad = false;
  *out = p;
  if (pull_flag) *pull_flag = nullptr;
  if (n <= 0) return KKM_OK;
  int* flag;
  KKM_TRY(ws.alloc(&flag, 1));
  KKM_CK(cudaMemsetAsync(flag, 0, 4, st));
  cudaPointerAttributes a;
  const bool known = cudaPointerGetAttributes(&a, p) == cudaSuccess;
  if (!known) cudaGetLastError();
  if (pull_flag && known && a.type == cudaMemoryTypeHost && a.devicePointer &&
      (reinterpret_cast<uintptr_t>(a.devicePointer) & 15) == 0) {
    *out = static_cast<const float*>(a.devicePointer);
    *pull_flag = flag;
    return KKM_OK;
  }
  if (known && (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
    KKM_RUN("check_finite", st, launch_check_finite(p, n, flag, st));
  } else {
    float* d = nullptr;
    KKM_TRY(ws.alloc(&d, n));
    *out = d;
    const float* mapped = (known && a.type == cudaMemoryTypeHost) ? static_cast<const float*>(a.devicePointer) : nullptr;
    if (mapped && (reinterpret_cast<uintptr_t>(mapped) & 15) == 0) {
      KKM_RUN("copy_check", st, launch_copy_check(mapped, d, n, flag, st));
    } else {
      KKM_CK(cudaMemcpyAsync(d, p, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, st));
      KKM_RUN("check_finite", st, launch_check_finite(d, n, flag, st));
    }
  }
  if (pending) {
    int* hf = pinned_flag_acquire();
    if (hf) {
      pending->flag = hf;
      pending->st = st;
      KKM_CK(cudaMemcpyAsync(hf, flag, 4, cudaMemcpyDeviceToHost, st));
      return KKM_OK;
    }
  }
  int h = 0;
  KKM_CK(cudaMemcpyAsync(&h, flag, 4, cudaMemcpyDeviceToHost, st));
  KKM_CK(cudaStreamSynchronize(st));
  *bad = h != 0;
  return KKM_OK;
}

// ======================================================================
// Small kernels of the host orchestration
// ======================================================================
__global__ void iota32_kernel(int32_t* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = i;
}
__global__ void iota64_kernel(int64_t* out, int64_t start, int64_t step, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = start + i * step;
}
__global__ void gather_i64_kernel(const int64_t* in, const int32_t* idx, int64_t n, int64_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = idx[i] >= 0 ? in[idx[i]] : -1;
}
__global__ void gather_i32_kernel(const int32_t* in, const int32_t* idx, int64_t n, int32_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[idx[i]];
}
// Rows ids[0..C) of the row-major n x d matrix X, packed into out [C][d].
__global__ void gather_raw_rows_kernel(const float* __restrict__ X, int64_t d, const int64_t* __restrict__ ids,
                                       int C, float* __restrict__ out) {
  const int64_t n = (int64_t)C * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / d;
    out[t] = X[ids[r] * d + (t - r * d)];
  }
}
// Resets a mini-batch's loop state in one launch: the landmark column maps
// (col_label, col_ord = -1 over ldk columns), the early-stop flag, the
// fixed-point g_hat numerators, the Eq. 10 keys and member counts (each
// nullable).
__global__ void loop_reset_kernel(int32_t* col_label, int32_t* col_ord, int64_t ldk, int32_t* done,
                                  unsigned long long* gfix, unsigned long long* keys, int32_t* cnt, int C) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ldk) {
    col_label[t] = -1;
    col_ord[t] = -1;
  }
  if (t < C) {
    if (gfix) gfix[t] = 0ull;
    if (keys) keys[t] = ~0ull;
    if (cnt) cnt[t] = 0;
  }
  if (t == 0 && done) *done = 0;
}
// Up to kCopyMax device-to-device copies in one launch (blockIdx.y = copy;
// 4-byte words; every size a multiple of 4 bytes, every address 4-byte
// aligned).
constexpr int kCopyMax = 16;
struct CopyList {
  int n = 0;
  const void* src[kCopyMax];
  void* dst[kCopyMax];
  int64_t words[kCopyMax];
};
__global__ void copy_many_kernel(CopyList L) {
  const int q = blockIdx.y;
  const uint32_t* __restrict__ s = static_cast<const uint32_t*>(L.src[q]);
  uint32_t* __restrict__ d = static_cast<uint32_t*>(L.dst[q]);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < L.words[q]; t += (int64_t)gridDim.x * blockDim.x)
    d[t] = s[t];
}
__global__ void clamp_idx_kernel(const int32_t* in, int n, int32_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i] >= 0 ? in[i] : 0;
}

static unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

// ======================================================================
// Kernel-function dispatch (RBF / linear via the Gram product, MD via RMSD)
// ======================================================================
struct KernelSpec {
  int precision = KKM_FP32;
  int kind;       // kkm_kernel_kind
  float sigma;
  int n_atoms;
  int64_t d;
  int dp;         // prepared row length
  int ap;         // padded atoms (RMSD)
  float neg_scale() const { return (float)(-1.4426950408889634 / (2.0 * (double)sigma * (double)sigma)); }
  bool gaussian() const { return kind != KKM_LINEAR; }
};

static kkm_status make_spec(const kkm_kernel* k, int64_t d, KernelSpec* sp) {
  if (!k) return invalid("kernel is NULL");
  sp->kind = k->kind;
  sp->sigma = k->sigma;
  sp->n_atoms = k->n_atoms;
  sp->d = d;
  if (d < 1) return invalid("d must be >= 1");
  if (k->kind == KKM_RBF || k->kind == KKM_LINEAR) {
    sp->dp = (int)round_up(d, 8);
    sp->ap = 0;
  } else if (k->kind == KKM_RMSD) {
    if (k->n_atoms < 1 || (int64_t)3 * k->n_atoms != d)
      return invalid("KKM_RMSD needs n_atoms >= 1 and d == 3 * n_atoms");
    sp->ap = (int)round_up(k->n_atoms, 8);
    sp->dp = 3 * sp->ap;
  } else {
    return invalid("unknown kernel kind");
  }
  if (sp->dp > (1 << 20)) return invalid("d too large");
  return KKM_OK;
}

// Prepared rows start + l*step of X (device) -> out [n][dp], aux [n].
// pull_bad: X is pinned host memory fetched by the copy engine, *pull_bad set
// for a NaN or Inf among the rows; MD frames go through `stage` ([n][d]
// floats) and are prepared from there.
static kkm_status prep_rows(const KernelSpec& sp, const float* X, int64_t start, int64_t step,
                            int64_t n, float* out, float* aux, cudaStream_t st, int* pull_bad = nullptr,
                            float* stage = nullptr) {
  if (pull_bad && sp.kind == KKM_RMSD) {
    if (n <= 0) return KKM_OK;
    KKM_CK(cudaMemcpy2DAsync(stage, (size_t)sp.d * 4, X + start * sp.d, (size_t)(step * sp.d) * 4, (size_t)sp.d * 4,
                             (size_t)n, cudaMemcpyDefault, st));
    KKM_RUN("check_finite", st, launch_check_finite(stage, n * sp.d, pull_bad, st));
    KKM_RUN("rmsd_prep", st, launch_rmsd_prep_rows(stage, sp.n_atoms, 0, 1, n, out, sp.ap, aux, st));
  } else if (pull_bad)
    KKM_RUN("gather_rows", st, launch_gather_rows_pull(X, sp.d, start, step, n, out, sp.dp, aux, pull_bad, st));
  else if (sp.kind == KKM_RMSD)
    KKM_RUN("rmsd_prep", st, launch_rmsd_prep_rows(X, sp.n_atoms, start, step, n, out, sp.ap, aux, st));
  else
    KKM_RUN("gather_rows", st, launch_gather_rows(X, sp.d, start, step, n, out, sp.dp, aux, st));
  return KKM_OK;
}
static kkm_status prep_ids(const KernelSpec& sp, const float* X, const int64_t* ids, int64_t n,
                           float* out, float* aux, cudaStream_t st) {
  if (sp.kind == KKM_RMSD)
    KKM_RUN("rmsd_prep", st, launch_rmsd_prep_idx64(X, sp.n_atoms, ids, n, out, sp.ap, aux, st));
  else
    KKM_RUN("gather_rows", st, launch_gather_idx64(X, sp.d, ids, n, out, sp.dp, aux, st));
  return KKM_OK;
}
// Copies of already prepared rows (the row's sum of squares is its aux value
// for both layouts: squared norm, or G of a centred frame).
static kkm_status copy_prepared(const KernelSpec& sp, const float* Xp, const int32_t* idx, int64_t n,
                                float* out, float* aux, cudaStream_t st) {
  KKM_RUN("gather_rows", st, launch_gather_idx32(Xp, sp.dp, idx, n, out, sp.dp, aux, st));
  return KKM_OK;
}
// out[a*ldo + b] = K(A_a, B_b).  dist != 0 gives distances instead.
// Scratch of the MD kernel's tensor-core path (sized for the largest call):
// BF16 planes of both sides, their squared radii, the refine flags and the
// tensor-core error word.
struct RmsdTcScratch {
  __nv_bfloat16* P = nullptr;  // [nP_cap][4][3 kp] split-BF16 references
  __nv_bfloat16* Q = nullptr;  // [nQ_cap][4][3 kp] split-BF16 samples
  float4* quat = nullptr;      // [nP_cap][ld_cap] rotations of the pairs to refine
  int* flags = nullptr;
  int* key = nullptr;    // [nP_cap] reference sort keys
  int* order = nullptr;  // [nP_cap] reference order of the exact pass
  int* err = nullptr;
  int64_t nP_cap = 0, nQ_cap = 0, ld_cap = 0;
  int kp = 0;
};

// Reference sets at least this large take the tensor-core MD path, for
// bandwidths at least this wide (the screen's rounding margin).
constexpr int64_t kRmsdTcMinRefs = 32;
constexpr float kRmsdTcMinSigma = 0.5f;

static kkm_status alloc_rmsd_tc(Workspace& ws, const KernelSpec& sp, int64_t nP_cap, int64_t nQ_cap,
                                int64_t ld_cap, RmsdTcScratch* t) {
  t->kp = (int)round_up(sp.n_atoms, 64);
  t->nP_cap = nP_cap;
  t->nQ_cap = nQ_cap;
  t->ld_cap = ld_cap;
  KKM_TRY(ws.alloc(&t->P, nP_cap * 4 * 3 * t->kp));
  KKM_TRY(ws.alloc(&t->Q, nQ_cap * 4 * 3 * t->kp));
  KKM_TRY(ws.alloc(&t->quat, nP_cap * ld_cap));
  KKM_TRY(ws.alloc(&t->flags, ceil_div(nP_cap, 32) * ceil_div(nQ_cap, 64)));
  KKM_TRY(ws.alloc(&t->key, nP_cap));
  KKM_TRY(ws.alloc(&t->order, nP_cap));
  KKM_TRY(ws.alloc(&t->err, 1));
  KKM_CK(cudaMemsetAsync(t->err, 0, 4, ws.st));
  return KKM_OK;
}

// MD kernel block on the tensor cores: a BF16 screen of every pair, then the
// exact FP32 two-pass kernel only on the 32 x 64 tiles holding a pair the
// screen could not certify as far (the others keep 0; their true values are
// below 1e-5), with the references reordered so that near pairs gather in
// few tiles.
static kkm_status rmsd_block_tc(const KernelSpec& sp, const float* A, const float* auxA, const int64_t* idA,
                                int64_t nA, const float* Bm, const float* auxB, const int64_t* idB, int64_t nB,
                                float* out, int64_t ldo, const RmsdTcScratch& t, bool block, cudaStream_t st);

static kkm_status kernel_block(const KernelSpec& sp, const float* A, const float* auxA,
                               const int64_t* idA, int64_t nA, const float* Bm, const float* auxB,
                               const int64_t* idB, int64_t nB, float* out, int64_t ldo,
                               cudaStream_t st, bool dist = false, bool block = false,
                               const RmsdTcScratch* tc = nullptr) {
  if (sp.kind == KKM_RMSD) {
    if (tc && !dist && nA >= kRmsdTcMinRefs && nA <= tc->nP_cap && nB <= tc->nQ_cap && sp.sigma >= kRmsdTcMinSigma)
      return rmsd_block_tc(sp, A, auxA, idA, nA, Bm, auxB, idB, nB, out, ldo, *tc, block, st);
    KKM_RUN(block ? "rmsd_block" : "rmsd_gram", st,
            launch_rmsd_gram(dist ? DK_DIST : DK_RBF, A, nA, Bm, nB, sp.ap, sp.n_atoms, auxA, auxB, idA,
                             idB, sp.neg_scale(), out, ldo, st));
  } else {
    const int dk = dist ? DK_DIST : (sp.kind == KKM_LINEAR ? DK_LINEAR : DK_RBF);
    KKM_RUN(block ? "gram_block" : "gram", st,
            launch_gram(dk, A, nA, Bm, nB, sp.dp, auxA, auxB, idA, idB, sp.neg_scale(), out, ldo, st));
  }
  return KKM_OK;
}

static int sm_count() {
  static const int n = []() {
    int dev = 0, v = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) v = 1;
    cudaGetLastError();
    return v;
  }();
  return n;
}

static kkm_status rmsd_block_tc(const KernelSpec& sp, const float* A, const float* auxA, const int64_t* idA,
                                int64_t nA, const float* Bm, const float* auxB, const int64_t* idB, int64_t nB,
                                float* out, int64_t ldo, const RmsdTcScratch& t, bool block, cudaStream_t st) {
  if (ldo > t.ld_cap) return invalid("internal: MD scratch too small");
  KKM_RUN("rmsd_to_bf16", st, launch_rmsd_to_bf16(A, nA, sp.ap, sp.n_atoms, t.P, t.kp, 0, st));
  KKM_RUN("rmsd_to_bf16", st, launch_rmsd_to_bf16(Bm, nB, sp.ap, sp.n_atoms, t.Q, t.kp, 1, st));
  KKM_RUN(block ? "rmsd_block" : "rmsd_gram", st,
          launch_rmsd_tc_estimate(t.P, nA, t.Q, nB, 3 * t.kp, auxA, auxB, sp.n_atoms, sp.neg_scale(), out, t.quat,
                                  ldo, t.err, sm_count(), st));
  KKM_RUN("rmsd_plan", st, launch_rmsd_refine_plan(out, ldo, (int)nA, (int)nB, t.key, t.order, t.flags, st));
  KKM_RUN("rmsd_exact", st,
          launch_rmsd_gram(DK_RBF, A, nA, Bm, nB, sp.ap, sp.n_atoms, auxA, auxB, idA, idB, sp.neg_scale(), out, ldo,
                           st, t.flags, t.order, t.quat));
  if (prof_on()) {  // pairs the exact pass recomputed (profiling only: a read-back)
    const int64_t nf = ceil_div(nA, 32) * ceil_div(nB, 64);
    std::vector<int> f((size_t)nf);
    KKM_CK(cudaMemcpyAsync(f.data(), t.flags, (size_t)nf * 4, cudaMemcpyDeviceToHost, st));
    KKM_CK(cudaStreamSynchronize(st));
    int64_t tiles = 0;
    for (int v : f) tiles += v != 0;
    prof_add_work("rmsd_exact", (double)tiles * 32.0 * 64.0);
  }
  return KKM_OK;
}

// The kernel block on the tensor cores: P (reference rows) and Q (sample
// rows) are prepared FP32 rows; their BF16 copies and rounded norms go to the
// given scratch.  out[n*ldo + m] = K(P_n, Q_m).
// L (nullable): local sample positions of the reference rows; their diagonal
// entries are then set to exactly 1 (Gaussian kernels).
// converted: Pb/Qb and their norms already hold the rounded rows.
static kkm_status kernel_block_bf16(const KernelSpec& sp, const float* P, const int32_t* L, int64_t nP,
                                    const float* Q, int64_t nQ, void* out, bool out_half, int64_t ldo,
                                    __nv_bfloat16* Pb, float* nPb, __nv_bfloat16* Qb, float* nQb, int* err,
                                    cudaStream_t st, int n_sms = 0, bool converted = false) {
  if (!converted) {
    KKM_RUN("to_bf16", st, launch_to_bf16(P, nP, sp.dp, Pb, nPb, st));
    KKM_RUN("to_bf16", st, launch_to_bf16(Q, nQ, sp.dp, Qb, nQb, st));
  }
  const int dk = (int)sp.d;
  KKM_RUN("gram_block", st,
          launch_gram_tc(sp.kind == KKM_LINEAR ? DK_LINEAR : DK_RBF, Pb, nP, Qb, nQ, dk, sp.dp, nPb, nQb,
                         sp.neg_scale(), out, out_half, ldo, err, n_sms > 0 ? n_sms : sm_count(), st));
  if (L && sp.kind != KKM_LINEAR) KKM_RUN("set_diag", st, launch_set_diag(out, out_half, ldo, L, (int)nP, st));
  return KKM_OK;
}

// The same from e4m3 rows with a scale per row (KKM_FP8): P8 / Q8 [n][ld8]
// codes, their scales and the squared norms of the decoded rows go to the
// given scratch.
static kkm_status kernel_block_fp8(const KernelSpec& sp, const float* P, const int32_t* L, int64_t nP, const float* Q,
                                   int64_t nQ, void* out, bool out_half, int64_t ldo, uint8_t* P8, float* sP,
                                   float* nP8, uint8_t* Q8, float* sQ, float* nQ8, int* err, cudaStream_t st,
                                   bool converted = false) {
  const int ld8 = (int)round_up(sp.dp, 16);
  if (!converted) {
    KKM_RUN("to_fp8", st, launch_to_fp8(P, nP, sp.dp, ld8, P8, sP, nP8, st));
    KKM_RUN("to_fp8", st, launch_to_fp8(Q, nQ, sp.dp, ld8, Q8, sQ, nQ8, st));
  }
  KKM_RUN("gram_block", st,
          launch_gram_tc_fp8(sp.kind == KKM_LINEAR ? DK_LINEAR : DK_RBF, P8, nP, Q8, nQ, (int)sp.d, ld8, nP8, nQ8, sP,
                             sQ, sp.neg_scale(), out, out_half, ldo, err, sm_count(), st));
  if (L && sp.kind != KKM_LINEAR) KKM_RUN("set_diag", st, launch_set_diag(out, out_half, ldo, L, (int)nP, st));
  return KKM_OK;
}

int l2_keep_rows(int64_t ldk, int rows, double share, int elem_bytes) {
  static const int l2 = []() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev) != cudaSuccess) v = 0;
    cudaGetLastError();
    return v;
  }();
  const double row_bytes = (double)ldk * (double)elem_bytes;
  return (int)std::min<double>(rows, std::floor(share * (double)l2 / row_bytes));
}

// Rows whose low-precision margin d2 - d1 is below this fraction of
// max(|d2|, K_ii + g_hat) are re-scored with exact FP32 kernel values.
constexpr float kRescoreMargin = 1e-3f;
// The same for a block of FP32-exact values stored in FP16 (the storage
// rounding alone, <= 2^-12 relative per value, averaged by the segment sums).
constexpr float kRescoreMarginHalf = 3e-4f;
// The same for the FP8 block: e4m3 keeps 3 significand bits (rounding error
// up to 2^-4 relative per coordinate), and its kernel values were measured
// up to 1e-2 from those of the unrounded rows; d = K_ii - 2 f_hat + g_hat
// then moves by at most three times that, which this window covers.
constexpr float kRescoreMarginFp8 = 3e-2f;
// Share of L2 given to kernel-block rows that stay resident through the inner
// loop (loaded evict_last; the other rows evict_first).  Measured on the
// MNIST-shaped fit: the 180 MB FP32 block streams fastest at 0.5 (11.0 ms per
// fit against 11.8 ms at 0.7); the 90 MB FP16 block is the same from 0.4 to
// 0.7.
constexpr double kL2KeepShare = 0.50;
constexpr double kL2KeepShareHalf = 0.70;

// ======================================================================
// Bandwidth rule
// ======================================================================
// Median rule enqueued on ws.st: the distances of min(N, 2048) samples drawn
// from the bandwidth stream and their median.  The answer lands in
// *sigma_host (pinned host memory) when the stream reaches it; it is read
// with median_sigma_of after a wait.  NaN or Inf rows give a meaningless
// answer but no fault (the select bins bit patterns).
static kkm_status median_bandwidth_enqueue(const KernelSpec& sp, const float* X, int64_t N, uint64_t bw_seed,
                                           Workspace& ws, float* sigma_host) {
  const int64_t M = std::min<int64_t>(N, 2048);
  if (M < 2) {
    *sigma_host = 1.0f;
    return KKM_OK;
  }
  SplitMix64 bw(bw_seed);
  std::vector<int64_t> pick = partial_shuffle(N, M, bw);
  cudaStream_t st = ws.st;
  int64_t* ids;
  float *P, *aux, *D, *out;
  uint32_t* scratch;
  const int64_t ld = round_up(M, 4);
  KKM_TRY(ws.alloc(&ids, M));
  KKM_TRY(ws.alloc(&P, M * sp.dp));
  KKM_TRY(ws.alloc(&aux, M));
  KKM_TRY(ws.alloc(&D, M * ld));
  KKM_TRY(ws.alloc(&out, 1));
  KKM_TRY(ws.alloc(&scratch, 1024));
  KKM_CK(cudaMemcpyAsync(ids, pick.data(), (size_t)M * 8, cudaMemcpyHostToDevice, st));
  KKM_TRY(prep_ids(sp, X, ids, M, P, aux, st));
  if (sp.kind == KKM_RMSD)
    KKM_TRY(kernel_block(sp, P, aux, ids, M, P, aux, ids, M, D, ld, st, /*dist=*/true));
  else {  // the select reads the strict upper triangle only
    float* part = nullptr;
    if (sp.dp >= kDistSplitMinDp) KKM_TRY(ws.alloc(&part, (int64_t)kDistSplit * M * ld));
    KKM_RUN("gram", st, launch_gram_dist_upper(P, M, sp.dp, aux, ids, D, ld, part, st));
  }
  const int64_t pairs = M * (M - 1) / 2;
  KKM_RUN("median_select", st, launch_select_upper(D, (int)M, ld, (pairs - 1) / 2, scratch, out, st));
  KKM_CK(cudaMemcpyAsync(sigma_host, out, 4, cudaMemcpyDeviceToHost, st));
  return KKM_OK;
}
// The bandwidth from the median (1 when it is not a positive finite number).
static float median_sigma_of(float m) { return (m > 0.0f && isfinite(m)) ? m : 1.0f; }

static kkm_status median_bandwidth_dev(const KernelSpec& sp, const float* X, int64_t N, uint64_t bw_seed,
                                       Workspace& ws, float* sigma_out) {
  int* slot = pinned_flag_acquire();
  float pageable = 0.0f;
  float* h = slot ? reinterpret_cast<float*>(slot) : &pageable;
  kkm_status r = median_bandwidth_enqueue(sp, X, N, bw_seed, ws, h);
  if (r == KKM_OK) {
    const cudaError_t e = cudaStreamSynchronize(ws.st);
    if (e != cudaSuccess) r = cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
  }
  if (r == KKM_OK) *sigma_out = median_sigma_of(*h);
  pinned_flag_release(slot);
  return r;
}

// ======================================================================
// Per-problem device state of the inner loop
// ======================================================================
struct LoopBuffers {
  Supports S{};
  IterState I{};
  int32_t* n_copy = nullptr;  // [C]
  int max_units = 0;
};

// gaussian: the kernel's values lie in [0, 1], so the g_hat numerators are
// accumulated in fixed point (IterState::gfix); else per-cluster tickets.
static kkm_status alloc_loop(Workspace& ws, int nLmax, int C, int64_t ldk, int trace_cap, LoopBuffers* lb,
                             bool gaussian = false) {
  Supports& S = lb->S;
  IterState& I = lb->I;
  const int mu = max_units_for(nLmax, C);
  lb->max_units = mu;
  S.C = C;
  S.max_units = mu;
  KKM_TRY(ws.alloc(&S.perm, nLmax));
  KKM_TRY(ws.alloc(&S.seg_off, C + 1));
  KKM_TRY(ws.alloc(&S.n_j, C));
  KKM_TRY(ws.alloc(&S.unit_j, mu));
  KKM_TRY(ws.alloc(&S.unit_kb, mu));
  KKM_TRY(ws.alloc(&S.unit_ke, mu));
  KKM_TRY(ws.alloc(&S.seg_unit, C + 1));
  KKM_TRY(ws.alloc(&S.n_units, 1));
  KKM_TRY(ws.alloc(&S.col_label, ldk));
  KKM_TRY(ws.alloc(&S.col_ord, ldk));
  KKM_TRY(ws.alloc(&S.lab, nLmax));
  KKM_TRY(ws.alloc(&lb->n_copy, C));
  I.n_strips = (int)ceil_div(ldk, kStripCols);
  I.assign_grid = (int)ceil_div(ldk, 32);
  // per-CTA slots serve the assign (one CTA per 32 rows) and the fused
  // iteration (at most one CTA per SM)
  I.fused_cap = sm_count();
  const int parts = std::max(I.assign_grid, I.fused_cap);
  KKM_TRY(ws.alloc(&I.partial, (int64_t)mu * ldk));
  KKM_TRY(ws.alloc(&I.gpart, (int64_t)mu * I.n_strips));
  KKM_TRY(ws.alloc(&I.omega_part, parts));
  KKM_TRY(ws.alloc(&I.changed_part, parts));
  KKM_TRY(ws.alloc(&I.lm_part, parts));
  KKM_TRY(ws.alloc(&I.gcta, (int64_t)I.fused_cap * C));
  KKM_TRY(ws.alloc(&I.facc, 2 * (C + 3)));
  if (gaussian) KKM_TRY(ws.alloc(&I.lm_list, 2 * (int64_t)nLmax));
  KKM_TRY(ws.alloc(&I.bar, 1));
  KKM_TRY(ws.alloc(&I.err, 1));
  KKM_CK(cudaMemsetAsync(I.bar, 0, 4, ws.st));
  KKM_CK(cudaMemsetAsync(I.err, 0, 4, ws.st));
  KKM_TRY(ws.alloc(&I.ghat_cur, C));
  KKM_TRY(ws.alloc(&I.gtick, C));
  KKM_CK(cudaMemsetAsync(I.gtick, 0, (size_t)C * 4, ws.st));
  if (gaussian) {
    KKM_TRY(ws.alloc(&I.gfix, C));
    KKM_CK(cudaMemsetAsync(I.gfix, 0, (size_t)C * 8, ws.st));
    I.gfix_shift = gfix_shift_for(nLmax);
  }
  KKM_TRY(ws.alloc(&I.ticket, 1));
  KKM_TRY(ws.alloc(&I.done, 1));
  KKM_TRY(ws.alloc(&I.trace_omega, std::max(trace_cap, 1)));
  KKM_TRY(ws.alloc(&I.trace_changed, std::max(trace_cap, 1)));
  KKM_TRY(ws.alloc(&I.trace_count, 1));
  KKM_CK(cudaMemsetAsync(I.ticket, 0, 4, ws.st));
  KKM_CK(cudaMemsetAsync(I.done, 0, 4, ws.st));
  KKM_CK(cudaMemsetAsync(I.trace_count, 0, 4, ws.st));
  return KKM_OK;
}

// Kernel k-means++ on prepared rows Xi (picks[0] already on the device).
// D2 needs 2*Ni + ceil(Ni/256) doubles (D^2, block prefixes, block totals).
// D2 holds 2 Ni + ceil(Ni / 32) doubles; *ticket is zero.  The RBF and linear
// kernels take one launch per round; the RMSD kernel evaluates the column of
// the last pick with its own block kernel first.
static kkm_status kmeanspp_dev(const KernelSpec& sp, const float* Xi, const float* aux_i, int Ni, int C,
                               const float* kself, float* rowbuf, float* rowaux, float* kcol,
                               int64_t ldk, double* D2, int32_t* picks, const double* draws_d,
                               uint32_t* ticket, cudaStream_t st) {
  double* P = D2 + Ni;
  double* bsum = P + Ni;
  if (sp.kind != KKM_RMSD) {
    for (int r = 1; r < C; ++r)
      KKM_RUN("kpp_round", st,
              launch_kpp_fused_round(Xi, sp.dp, Ni, sp.kind == KKM_LINEAR, sp.neg_scale(), kself, D2, P, bsum, picks,
                                     draws_d, r, ticket, st));
    return KKM_OK;
  }
  for (int r = 1; r < C; ++r) {
    KKM_TRY(copy_prepared(sp, Xi, picks + (r - 1), 1, rowbuf, rowaux, st));
    KKM_TRY(kernel_block(sp, rowbuf, rowaux, nullptr, 1, Xi, aux_i, nullptr, Ni, kcol, ldk, st));
    KKM_RUN("kpp_round", st, launch_kpp_round(kcol, Ni, kself, D2, P, bsum, picks, draws_d, r, st));
  }
  return KKM_OK;
}

struct BatchGeom {
  int64_t start, step, Ni;
};

static std::vector<BatchGeom> batch_geometry(int64_t N, int B, int sampling) {
  std::vector<BatchGeom> g;
  if (sampling == KKM_STRIDE) {
    for (int i = 0; i < B; ++i) g.push_back({i, B, (N - i + B - 1) / B});
  } else {
    const int64_t base = N / B, extra = N % B;
    int64_t start = 0;
    for (int i = 0; i < B; ++i) {
      const int64_t n = base + (i < extra ? 1 : 0);
      g.push_back({start, 1, n});
      start += n;
    }
  }
  return g;
}

// ======================================================================
// kkm_fit
// ======================================================================
// Buffers of one mini-batch's kernel block: its prepared rows and ids, the
// landmark rows and ids, the block itself (FP16 on the reduced-precision RBF
// path) and the block kernels' scratch.
struct BlockBufs {
  float *Xi = nullptr, *aux_i = nullptr, *XL = nullptr, *auxL = nullptr, *KT = nullptr;
  __half* KTh = nullptr;
  int64_t *gid = nullptr, *gidL = nullptr;
  __nv_bfloat16 *Xib = nullptr, *XLb = nullptr;
  float *nXib = nullptr, *nXLb = nullptr;     // norms of the reduced-precision rows (BF16 or FP8)
  uint8_t *Xi8 = nullptr, *XL8 = nullptr;    // FP8: e4m3 codes [n][round_up(dp, 16)]
  float *sXi = nullptr, *sXL = nullptr;      // FP8: row scales
  RmsdTcScratch rtc;
};

// keep32: a block computed in FP32 and stored in FP16 keeps its FP32 values
// too (b->KT), for the near-tie re-score.
static kkm_status alloc_block_bufs(Workspace& ws, const KernelSpec& sp, int64_t Nmax, int64_t nLmax, int64_t ldk,
                                   bool kt_half, bool use_rtc, BlockBufs* b, bool keep32 = false) {
  KKM_TRY(ws.alloc(&b->Xi, Nmax * sp.dp));
  KKM_TRY(ws.alloc(&b->aux_i, Nmax));
  KKM_TRY(ws.alloc(&b->gid, Nmax));
  KKM_TRY(ws.alloc(&b->XL, nLmax * sp.dp));
  KKM_TRY(ws.alloc(&b->auxL, nLmax));
  KKM_TRY(ws.alloc(&b->gidL, nLmax));
  if (kt_half)
    KKM_TRY(ws.alloc(&b->KTh, nLmax * ldk));
  if (!kt_half || keep32)
    KKM_TRY(ws.alloc(&b->KT, nLmax * ldk));
  if (sp.precision == KKM_BF16) {
    KKM_TRY(ws.alloc(&b->Xib, Nmax * sp.dp));
    KKM_TRY(ws.alloc(&b->XLb, nLmax * sp.dp));
  }
  if (sp.precision == KKM_FP8) {
    const int64_t ld8 = round_up(sp.dp, 16);
    KKM_TRY(ws.alloc(&b->Xi8, Nmax * ld8));
    KKM_TRY(ws.alloc(&b->XL8, nLmax * ld8));
    KKM_TRY(ws.alloc(&b->sXi, Nmax));
    KKM_TRY(ws.alloc(&b->sXL, nLmax));
  }
  if (sp.precision != KKM_FP32) {
    KKM_TRY(ws.alloc(&b->nXib, Nmax));
    KKM_TRY(ws.alloc(&b->nXLb, nLmax));
  }
  if (use_rtc) KKM_TRY(alloc_rmsd_tc(ws, sp, nLmax, Nmax, ldk, &b->rtc));
  return KKM_OK;
}

// How a fit stores and evaluates its kernel block: the reduced-precision RBF
// path keeps the block in FP16 (values in [0, 1], an 11-bit significand,
// finer than the BF16 inputs' rounding), so the inner loop streams half the
// bytes; short rows keep the FP32 Gram on the FFMA pipes and only round the
// stored values.
struct BlockMode {
  bool kt_half = false, fp32_half_block = false, use_rtc = false;
  BlockMode(const KernelSpec& sp, int64_t nLmax) {
    kt_half = sp.precision != KKM_FP32 && sp.kind == KKM_RBF;
    fp32_half_block = kt_half && sp.d < kBf16TensorMinDim;
    use_rtc = sp.kind == KKM_RMSD && nLmax >= kRmsdTcMinRefs;
  }
  // near-tie window of the re-score (0: no re-score, FP32 blocks)
  float flag_tau(const KernelSpec& sp) const {
    if (sp.precision == KKM_FP32) return 0.0f;
    if (fp32_half_block) return kRescoreMarginHalf;
    return sp.precision == KKM_FP8 ? kRescoreMarginFp8 : kRescoreMargin;
  }
};

// Alg. 1 line 3 on already prepared rows: the kernel block K(L, X^i) of the
// buffer set b (its Xi, XL, ids filled) into b.KT or b.KTh.
// n_sms > 0 limits the tensor-core block to that many CTAs (SMs), e.g. those
// a concurrent one-launch inner loop leaves free.
// The reduced-precision copies of a mini-batch's rows and landmark rows
// that the tensor-core block reads (none for the FP32 Gram kernels); they do
// not depend on the bandwidth.
static kkm_status block_convert(const KernelSpec& sp, const BlockMode& bm, const BlockBufs& b, int nL, int Ni,
                                cudaStream_t bs) {
  if (bm.fp32_half_block) return KKM_OK;
  if (sp.precision == KKM_BF16) {
    KKM_RUN("to_bf16", bs, launch_to_bf16(b.XL, nL, sp.dp, b.XLb, b.nXLb, bs));
    KKM_RUN("to_bf16", bs, launch_to_bf16(b.Xi, Ni, sp.dp, b.Xib, b.nXib, bs));
  } else if (sp.precision == KKM_FP8) {
    const int ld8 = (int)round_up(sp.dp, 16);
    KKM_RUN("to_fp8", bs, launch_to_fp8(b.XL, nL, sp.dp, ld8, b.XL8, b.sXL, b.nXLb, bs));
    KKM_RUN("to_fp8", bs, launch_to_fp8(b.Xi, Ni, sp.dp, ld8, b.Xi8, b.sXi, b.nXib, bs));
  }
  return KKM_OK;
}

// converted: block_convert has run for these buffers.
static kkm_status block_kernel(const KernelSpec& sp, const BlockMode& bm, const BlockBufs& b, const int32_t* Ld,
                               int nL, int Ni, int64_t ldk, int* tc_err, cudaStream_t bs, int n_sms = 0,
                               bool converted = false) {
  if (bm.fp32_half_block)
    KKM_RUN("gram_block", bs,
            launch_gram_rbf_half(b.XL, nL, b.Xi, Ni, sp.dp, b.auxL, b.aux_i, b.gidL, b.gid, sp.neg_scale(), b.KTh,
                                 ldk, bs, b.KT));
  else if (sp.precision == KKM_BF16)
    KKM_TRY(kernel_block_bf16(sp, b.XL, Ld, nL, b.Xi, Ni, bm.kt_half ? (void*)b.KTh : (void*)b.KT, bm.kt_half, ldk,
                              b.XLb, b.nXLb, b.Xib, b.nXib, tc_err, bs, n_sms, converted));
  else if (sp.precision == KKM_FP8)
    KKM_TRY(kernel_block_fp8(sp, b.XL, Ld, nL, b.Xi, Ni, bm.kt_half ? (void*)b.KTh : (void*)b.KT, bm.kt_half, ldk,
                             b.XL8, b.sXL, b.nXLb, b.Xi8, b.sXi, b.nXib, tc_err, bs, converted));
  else
    KKM_TRY(kernel_block(sp, b.XL, b.auxL, b.gidL, nL, b.Xi, b.aux_i, b.gid, Ni, b.KT, ldk, bs, false, true,
                         bm.use_rtc ? &b.rtc : nullptr));
  return KKM_OK;
}

// Re-score inputs of the reduced-precision path: the FP32 rows of the
// mini-batch and of its landmarks, and the FP32 values of a block computed in
// FP32 and stored in FP16.
static RescoreArgs rescore_args(const KernelSpec& sp, const BlockBufs& b, int64_t ldk) {
  RescoreArgs R;
  if (sp.precision == KKM_FP32) return R;
  if (b.KTh && b.KT) {
    R.K32 = b.KT;
    R.ldk32 = ldk;
  }
  R.kind = sp.kind == KKM_LINEAR ? DK_LINEAR : DK_RBF;
  R.dp = sp.dp;
  R.Xi = b.Xi;
  R.nXi = b.aux_i;
  R.XL = b.XL;
  R.nXL = b.auxL;
  R.neg_scale = sp.neg_scale();
  return R;
}

// Whether the inner iterations of a mini-batch run fused (one cooperative
// launch each) for this option and block shape.
// Inner-loop forms (kkm_iteration): the split pair of launches per
// iteration, the one-launch loop on the CUDA cores, the one-launch loop with
// the tensor-core f_hat sums.
enum LoopForm { kLoopSplit = 0, kLoopFused = 1, kLoopTc = 2 };

static bool fused_applies(int Ni, int nL, int C, int esize) {
  FusedShape F;
  size_t smem = 0;
  return fused_shape(Ni, nL, C, esize, sm_count(), &F, &smem);
}
// The tensor-core loop needs the FP16 Gaussian block and its fixed-point sums.
static bool tc_applies(const KernelSpec& sp, const BlockMode& bm, int Ni, int nL, int C) {
  int ns = 0;
  size_t smem = 0;
  return bm.kt_half && sp.kind == KKM_RBF && tc_iter_shape(Ni, nL, C, sm_count(), &ns, &smem);
}
// The loop form for an iteration option; -1 when a form asked for does not
// apply to the shape.
static int loop_form(int iteration, const KernelSpec& sp, const BlockMode& bm, int Ni, int nL, int C) {
  const bool tc = tc_applies(sp, bm, Ni, nL, C);
  switch (iteration) {
    case KKM_ITER_TC:
      return tc ? kLoopTc : -1;
    case KKM_ITER_FUSED:
      return fused_applies(Ni, nL, C, bm.kt_half ? 2 : 4) ? kLoopFused : -1;
    case KKM_ITER_SPLIT:
      return kLoopSplit;
    default:  // AUTO: the tensor-core loop where it applies (measured 2x faster per iteration)
      return tc ? kLoopTc : kLoopSplit;
  }
}

// The inner loop of a mini-batch (Alg. 1 lines 9-16; Eq. 15-17) over the
// block of the buffer set b: `iters` iterations fused in one launch, or per
// iteration the streaming partial sums and the assign.  Either way every
// iteration closes on the device (trace, early stop, support re-sort).
// With the tensor-core form and `med` (keys preset to ~0, counts to 0), the
// loop also leaves the Eq. 10 keys, member counts, g_hat and n_j of the final
// supports, and the rest of the support structure is rebuilt only when
// `need_supports`.
struct MedoidOut {
  unsigned long long* keys = nullptr;
  int32_t* cnt = nullptr;
  double* ghat = nullptr;
  bool need_supports = true;
};

static kkm_status inner_loop(const BlockMode& bm, const BlockBufs& b, int64_t ldk, int Ni, const Supports& S,
                             const IterState& I, int form, int iters, const float* kself, int32_t* u,
                             float* margin, float* fhat_out, double* ghat_out, int early_stop, const RescoreArgs& R,
                             cudaStream_t st, const MedoidOut& med = MedoidOut()) {
  if (form == kLoopTc) {
    KKM_RUN("iterate", st,
            launch_iterate_tc(b.KTh, ldk, Ni, S, I, iters, u, margin, fhat_out, ghat_out, early_stop, sm_count(), st,
                              R, med.keys, med.cnt, med.ghat));
    // the landmark labels are final: the rest of the support structure
    if (med.need_supports || !med.keys) KKM_RUN("build_supports", st, launch_build_supports(S, st));
    return KKM_OK;
  }
  if (form == kLoopFused) {
    KKM_RUN("iterate", st,
            bm.kt_half ? launch_iterate(b.KTh, ldk, Ni, S, I, iters, kself, u, margin, fhat_out, ghat_out, early_stop,
                                        sm_count(), st, R)
                       : launch_iterate(b.KT, ldk, Ni, S, I, iters, kself, u, margin, fhat_out, ghat_out, early_stop,
                                        sm_count(), st, R));
    return KKM_OK;
  }
  LoopExecutor* ex = current_loop_executor();
  if (ex && !margin && !fhat_out && !ghat_out) {  // a fit of a batch: the batch's work lists run the loop
    LoopItem item;
    KKM_CK(make_loop_item(bm.kt_half ? static_cast<const void*>(b.KTh) : static_cast<const void*>(b.KT), bm.kt_half,
                          ldk, Ni, S, I, kself, u, early_stop, R, &item));
    return loop_executor_run(ex, item, iters, st);
  }
  for (int t = 0; t < iters; ++t) {
    KKM_RUN("fhat_partial", st,
            bm.kt_half ? launch_fhat_partial(b.KTh, ldk, Ni, S, I, st) : launch_fhat_partial(b.KT, ldk, Ni, S, I, st));
    // the assign's last CTA closes the iteration and re-sorts the supports
    // when a landmark label changed
    KKM_RUN("assign", st,
            launch_assign(ldk, Ni, S, I, kself, u, margin, nullptr, fhat_out, ghat_out, early_stop, /*trace=*/1, st,
                          R));
  }
  return KKM_OK;
}

// Streams of one fit.  With the block pipeline (Section 4, Fig. 3: the next
// mini-batch's kernel block is produced while the current one iterates) the
// inner loops run on a high-priority stream and the blocks on a low-priority
// one, so that a loop kernel's CTAs are scheduled ahead of a block kernel's
// as SMs free up.  Both start after the work queued so far on the caller's
// stream; join() (or the destructor, on an error return) orders the caller's
// stream after both, so the workspace is released only when they are done.
// Without the pipeline all three are the caller's stream.
// High- and low-priority stream pairs of the block pipeline, reused across
// fits (creating two streams costs tens of microseconds, a small fit's whole
// run).  A pair is taken for one fit and given back once the caller's stream
// is ordered after it; work still in flight on a returned pair only orders
// the next fit that takes it after that work.
struct StreamPair {
  cudaStream_t main = nullptr, side = nullptr;
  int device = -1;
};
static std::mutex g_pair_mu;
static std::vector<StreamPair> g_pairs;

static kkm_status take_pair(StreamPair* out) {
  int dev = 0;
  KKM_CK(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(g_pair_mu);
    for (size_t q = 0; q < g_pairs.size(); ++q)
      if (g_pairs[q].device == dev) {
        *out = g_pairs[q];
        g_pairs.erase(g_pairs.begin() + (std::ptrdiff_t)q);
        return KKM_OK;
      }
  }
  int least = 0, greatest = 0;
  KKM_CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  StreamPair p;
  p.device = dev;
  KKM_CK(cudaStreamCreateWithPriority(&p.main, cudaStreamNonBlocking, greatest));
  const cudaError_t e = cudaStreamCreateWithPriority(&p.side, cudaStreamNonBlocking, least);
  if (e != cudaSuccess) {
    cudaStreamDestroy(p.main);
    KKM_CK(e);
  }
  *out = p;
  return KKM_OK;
}

static void give_pair(const StreamPair& p) {
  std::lock_guard<std::mutex> lk(g_pair_mu);
  g_pairs.push_back(p);
}

// Streams of one fit.  With the block pipeline (Section 4, Fig. 3: the next
// mini-batch's kernel block is produced while the current one iterates) the
// inner loops run on a high-priority stream and the blocks on a low-priority
// one, so that a loop kernel's CTAs are scheduled ahead of a block kernel's
// as SMs free up.  Both start after the work queued so far on the caller's
// stream; join() (or the destructor, on an error return) orders the caller's
// stream after both, so the workspace is released only when they are done.
// Without the pipeline all three are the caller's stream.
struct FitStreams {
  cudaStream_t user = nullptr, main = nullptr, side = nullptr;
  StreamPair pair;
  bool own = false;

  // `later` waits for the work queued so far on `first`.
  static kkm_status after(cudaStream_t first, cudaStream_t later) {
    if (first == later) return KKM_OK;
    cudaEvent_t e;
    KKM_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaError_t r = cudaEventRecord(e, first);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(later, e, 0);
    cudaEventDestroy(e);  // released once recorded work completes; the wait stands
    KKM_CK(r);
    return KKM_OK;
  }
  kkm_status start(cudaStream_t u, bool pipelined) {
    user = main = side = u;
    if (!pipelined) return KKM_OK;
    KKM_TRY(take_pair(&pair));
    main = pair.main;
    side = pair.side;
    own = true;
    KKM_TRY(after(user, main));
    KKM_TRY(after(user, side));
    return KKM_OK;
  }
  kkm_status join() {
    if (!own) return KKM_OK;
    own = false;
    const kkm_status a = after(main, user), b = after(side, user);
    if (a != KKM_OK || b != KKM_OK) {
      // the caller's stream cannot be ordered after them: wait on the host
      cudaStreamSynchronize(main);
      cudaStreamSynchronize(side);
    }
    give_pair(pair);
    main = side = user;
    return a != KKM_OK ? a : b;
  }
  ~FitStreams() { join(); }
};

kkm_status model_alloc_device(kkm_model* m, cudaStream_t st) {
  const int64_t nL = m->nL, C = m->C, dp = m->dp, mu = m->max_units;
  // one allocation for the resident arrays (256-byte aligned pieces)
  std::vector<std::pair<void**, size_t>> parts;
  auto A = [&](auto** p, int64_t n) {
    using T = std::remove_reference_t<decltype(**p)>;
    parts.emplace_back(reinterpret_cast<void**>(p), (size_t)std::max<int64_t>(n, 1) * sizeof(T));
  };
  A(&m->sup, nL * dp);
  A(&m->sup_aux, nL);
  A(&m->sup_ids, nL);
  A(&m->sup_labels, nL);
  A(&m->L_ident, nL);
  A(&m->perm, nL);
  A(&m->seg_off, C + 1);
  A(&m->n_j, C);
  A(&m->unit_j, mu);
  A(&m->unit_kb, mu);
  A(&m->unit_ke, mu);
  A(&m->seg_unit, C + 1);
  A(&m->n_units, 1);
  A(&m->ghat, C);
  A(&m->med, C * dp);
  A(&m->med_aux, C);
  size_t total = 0;
  for (auto& pr : parts) total += (pr.second + 255) & ~size_t(255);
  // from the device's stream-ordered pool (its release threshold keeps the
  // memory mapped), so that freeing a model does not unmap it
  setup_pool_once(m->device);
  KKM_CK(cudaMallocAsync(&m->arena, total, st));
  size_t off = 0;
  for (auto& pr : parts) {
    *pr.first = static_cast<unsigned char*>(m->arena) + off;
    off += (pr.second + 255) & ~size_t(255);
  }
  return KKM_OK;
}

static kkm_status fit_impl(const float* X_in, int64_t N, int64_t d, int32_t C, int32_t B, double s,
                           const kkm_kernel* k, int32_t iters, uint64_t seed, const kkm_options* opt_in,
                           int32_t* labels_out, kkm_model** model_out, const kkm_checkpoint* from = nullptr,
                           int32_t stop = -1, kkm_checkpoint** ckpt_out = nullptr) {
  kkm_options opt;
  kkm_options_default(&opt);
  if (opt_in) opt = *opt_in;
  if (!X_in) return invalid("X is NULL");
  if (N < 1 || N > INT32_MAX) return invalid("N must be in [1, 2^31)");
  if (C < 1 || C > kMaxC) return invalid("C must be in [1, 256]");
  if (B < 1 || B > N) return invalid("B must be in [1, N]");
  if (!(s > 0.0 && s <= 1.0)) return invalid("s must be in (0, 1]");
  if (iters < 0) return invalid("iters must be >= 0");
  if (opt.pipeline != KKM_PIPE_AUTO && opt.pipeline != KKM_PIPE_SERIAL && opt.pipeline != KKM_PIPE_OVERLAP)
    return invalid("unknown pipeline");
  if (opt.sampling != KKM_STRIDE && opt.sampling != KKM_BLOCK) return invalid("unknown sampling");
  if (opt.iteration != KKM_ITER_AUTO && opt.iteration != KKM_ITER_FUSED && opt.iteration != KKM_ITER_SPLIT &&
      opt.iteration != KKM_ITER_TC)
    return invalid("unknown iteration form");
  KernelSpec sp;
  KKM_TRY(make_spec(k, d, &sp));
  if (opt.precision != KKM_FP32 && opt.precision != KKM_BF16 && opt.precision != KKM_FP8)
    return invalid("precision must be KKM_FP32, KKM_BF16 or KKM_FP8");
  if (opt.precision != KKM_FP32 && sp.kind == KKM_RMSD)
    return invalid("KKM_BF16 and KKM_FP8 apply to the RBF and linear kernels");
  sp.precision = opt.precision;
  if (sp.kind != KKM_LINEAR && !isfinite(sp.sigma)) return invalid("sigma must be finite");
  const std::vector<BatchGeom> geo = batch_geometry(N, B, opt.sampling);
  int64_t Nmax = 0, Nmin = INT64_MAX, nLmax = 0;
  for (auto& g : geo) {
    Nmax = std::max(Nmax, g.Ni);
    Nmin = std::min(Nmin, g.Ni);
    nLmax = std::max(nLmax, n_landmarks(g.Ni, s));
  }
  if (C > Nmin) return invalid("C exceeds the size of a mini-batch");
  std::vector<int64_t> init;
  if (opt.init_medoids) {
    init.assign(opt.init_medoids, opt.init_medoids + C);
    for (int64_t v : init)
      if (v < 0 || v >= N) return invalid("init_medoids out of range");
  }
  // the mini-batches of this call: [start, stop) (a checkpoint resumes at its
  // next mini-batch; the call must repeat the arguments it was made with)
  if (stop < 0) stop = B;
  const int start = from ? from->next_batch : 0;
  if (from) {
    const bool same = from->N == N && from->d == d && from->C == C && from->B == B && from->s == s &&
                      from->kind == k->kind && from->n_atoms == k->n_atoms &&
                      (k->kind == KKM_LINEAR || from->sigma_arg == k->sigma) && from->iters == iters &&
                      from->seed == seed && from->precision == opt.precision && from->sampling == opt.sampling &&
                      from->early_stop == opt.early_stop && from->had_init == (opt.init_medoids ? 1 : 0);
    if (!same) return invalid("the checkpoint was made by a fit with other arguments");
    if ((int64_t)from->M.size() != C || (int64_t)from->W.size() != C ||
        (int64_t)from->displacement.size() != start || from->omega.size() != from->changed.size() ||
        (int64_t)from->omega.size() > (int64_t)start * iters || start < 1 || start >= B)
      return invalid("inconsistent checkpoint");
  }
  if (stop <= start || stop > B) return invalid("the mini-batch range is empty or beyond B");
  if (model_out && stop != B) return invalid("a model needs the last mini-batch (stop == B)");

  cudaStream_t st = (cudaStream_t)opt.stream;
  int dev = 0;
  KKM_CK(cudaGetDevice(&dev));
  setup_pool_once(dev);
  Workspace ws(st);

  // ---- inputs on the device; the finite check (then the median rule) runs
  // while the host draws the random numbers and sets up the workspace, and
  // a fit whose X holds NaN or Inf returns before any step of Alg. 1
  // Pinned host X (feature rows of a multiple of 4 floats, or MD frames)
  // stays on the host in a whole fit: each mini-batch's rows cross the link
  // when they are gathered (the next mini-batch's during the current loop)
  // and are checked there; the fit reports NaN or Inf at its end, writing no
  // output.
  const float* X = nullptr;
  PendingCheck chk;
  int* pull_bad = nullptr;
  {
    bool bad = false;
    // (a call over part of the mini-batches reads rows it does not gather:
    // it checks all of X up front)
    const bool may_pull = (sp.kind == KKM_RMSD || d % 4 == 0) && start == 0 && stop == B;
    KKM_TRY(device_input_checked(ws, X_in, N * d, &X, &bad, &chk, may_pull ? &pull_bad : nullptr));
    if (bad) return invalid("X holds NaN or Inf");
  }

  // ---- block buffers and streams (Alg. 1 line 3 is the first device work
  // of a fit whose X stays on the host: its first rows cross the link while
  // the median rule runs and the host draws the landmarks)
  const int64_t ldk = round_up(Nmax, 32);
  // AUTO overlaps the next block with the inner loop when the loop is the
  // tensor-core one, which holds one SM per 128 samples and leaves the rest
  // to the block (measured 4 % faster on the MNIST-shaped fit)
  const int first_nl = (int)n_landmarks(geo[0].Ni, s);
  const bool tc_loop = opt.iteration == KKM_ITER_AUTO || opt.iteration == KKM_ITER_TC
                           ? tc_applies(sp, BlockMode(sp, nLmax), (int)geo[0].Ni, first_nl, C)
                           : false;
  const bool overlap = fit_overlaps(opt.pipeline, B, sp.kind, sp.precision) ||
                       (opt.pipeline == KKM_PIPE_AUTO && B >= 2 && tc_loop);
  // the block of the next mini-batch takes the SMs the tensor-core loop leaves
  const int side_sms = overlap && tc_loop ? std::max(16, sm_count() - (int)ceil_div(Nmax, 128)) : 0;
  // The BF16 path keeps a Gaussian block in FP16 (values in [0, 1], 11-bit
  // significand, finer than the BF16 inputs' rounding): the inner loop
  // streams half the bytes.
  const BlockMode bm(sp, nLmax);
  const bool kt_half = bm.kt_half;
  const bool use_rtc = bm.use_rtc;
  // one set of block buffers, or two when the next mini-batch's block is
  // computed while the current one iterates
  BlockBufs bb[2];
  const int nbuf = overlap ? 2 : 1;
  for (int q = 0; q < nbuf; ++q)
    KKM_TRY(alloc_block_bufs(ws, sp, Nmax, nLmax, ldk, kt_half, use_rtc, &bb[q], bm.fp32_half_block));
  NvtxRange nv_fit("kkm_fit");
  FitStreams fs;
  KKM_TRY(fs.start(st, overlap));
  const cudaStream_t ms = fs.main;
  // MD frames fetched from the host are staged, then prepared (one stream
  // fetches at a time: the side stream, or the main one without the pipeline)
  float* pull_stage = nullptr;
  if (pull_bad && sp.kind == KKM_RMSD) KKM_TRY(ws.alloc(&pull_stage, Nmax * d));
  const bool first_fetched = pull_bad != nullptr;
  if (first_fetched) {
    const BatchGeom& g0 = geo[start];
    const BlockBufs& b0 = bb[start % nbuf];
    KKM_TRY(prep_rows(sp, X, g0.start, g0.step, g0.Ni, b0.Xi, b0.aux_i, overlap ? fs.side : ms, pull_bad,
                      pull_stage));
  }

  // ---- random numbers (Section 3.1, 3.2): k-means++, bandwidth, landmarks
  SplitMix64 master(seed);
  SplitMix64 kpp(master.next());
  const uint64_t bw_seed = master.next();
  // ---- bandwidth: the median rule runs behind the check while the host
  // draws the landmarks (a resumed fit keeps the bandwidth it started with)
  const float sigma_arg = sp.sigma;
  const bool need_median = !from && sp.kind != KKM_LINEAR && !(sp.sigma > 0.0f);
  struct PinnedWord {
    int* p = pinned_flag_acquire();
    ~PinnedWord() { pinned_flag_release(p); }
  } sig_slot;
  float sig_pageable = 1.0f;
  float* const sig_h = sig_slot.p ? reinterpret_cast<float*>(sig_slot.p) : &sig_pageable;
  if (need_median) KKM_TRY(median_bandwidth_enqueue(sp, X, N, bw_seed, ws, sig_h));
  std::vector<SplitMix64> lm;
  for (int i = 0; i < B; ++i) lm.emplace_back(master.next());
  std::vector<int64_t> L_off(B + 1, 0);
  std::vector<int32_t> L_all;
  for (int i = 0; i < B; ++i) {
    const int64_t Ni = geo[i].Ni, nl = n_landmarks(Ni, s);
    if (nl == Ni) {
      for (int64_t a = 0; a < Ni; ++a) L_all.push_back((int32_t)a);
    } else {
      const size_t at = L_all.size();
      L_all.resize(at + (size_t)nl);
      sorted_picks(Ni, nl, lm[i], L_all.data() + at);
    }
    L_off[i + 1] = (int64_t)L_all.size();
  }
  const bool do_kpp = init.empty() && start == 0;
  std::vector<double> draws(C, 0.0);
  std::vector<int32_t> pick0(1, 0);
  if (do_kpp) {
    for (int r = 0; r < C; ++r) draws[r] = kpp.u01();
    pick0[0] = (int32_t)floor(draws[0] * (double)geo[0].Ni);
  }


  // ---- workspace
  const int trace_cap = B * iters;
  float *Kt, *Kmi, *MX, *auxM, *MIX, *auxMI, *rowbuf, *rowaux, *kcol, *MXn, *auxMn, *Kmn;
  int64_t *Mg, *W, *idMI, *Mg_prev;
  double* disp;
  int32_t *u, *Ld_all, *mi, *mi_safe, *cnt, *picks, *labels_dev = nullptr;
  unsigned long long* keys;
  double *ghat, *D2 = nullptr, *draws_d = nullptr;
  uint32_t* kpp_ticket = nullptr;
  KKM_TRY(ws.alloc(&Kt, (int64_t)C * ldk));
  KKM_TRY(ws.alloc(&Kmi, (int64_t)C * ldk));
  KKM_TRY(ws.alloc(&MX, (int64_t)C * sp.dp));
  KKM_TRY(ws.alloc(&auxM, C));
  KKM_TRY(ws.alloc(&MIX, (int64_t)C * sp.dp));
  KKM_TRY(ws.alloc(&auxMI, C));
  KKM_TRY(ws.alloc(&idMI, C));
  KKM_TRY(ws.alloc(&Mg, C));
  KKM_TRY(ws.alloc(&W, C));
  // centre displacement per mini-batch (Section 4.1, Fig. 4b)
  const int64_t ldc = round_up(C, 32);
  KKM_TRY(ws.alloc(&Mg_prev, C));
  KKM_TRY(ws.alloc(&MXn, (int64_t)C * sp.dp));
  KKM_TRY(ws.alloc(&auxMn, C));
  KKM_TRY(ws.alloc(&Kmn, (int64_t)C * ldc));
  KKM_TRY(ws.alloc(&disp, B));
  KKM_TRY(ws.alloc(&u, Nmax));
  KKM_TRY(ws.alloc(&Ld_all, (int64_t)L_all.size()));
  KKM_TRY(ws.alloc(&mi, C));
  KKM_TRY(ws.alloc(&mi_safe, C));
  KKM_TRY(ws.alloc(&cnt, C));
  KKM_TRY(ws.alloc(&keys, C));
  KKM_TRY(ws.alloc(&ghat, C));
  KKM_TRY(ws.alloc(&picks, C));
  KKM_TRY(ws.alloc(&rowbuf, sp.dp));
  KKM_TRY(ws.alloc(&rowaux, 1));
  KKM_TRY(ws.alloc(&kcol, ldk));
  int* tc_err = nullptr;
  if (sp.precision != KKM_FP32) {
    KKM_TRY(ws.alloc(&tc_err, 1));
    KKM_CK(cudaMemsetAsync(tc_err, 0, 4, st));
  }
  LoopBuffers lb;
  KKM_TRY(alloc_loop(ws, (int)nLmax, C, ldk, trace_cap, &lb, sp.gaussian()));
  Supports& S = lb.S;
  IterState& I = lb.I;
  if (from) {
    // the outer loop's state after mini-batch start - 1: medoids, counts, the
    // trace and the displacements so far
    const int32_t tc0 = (int32_t)from->omega.size();
    KKM_CK(cudaMemcpyAsync(Mg, from->M.data(), (size_t)C * 8, cudaMemcpyHostToDevice, st));
    KKM_CK(cudaMemcpyAsync(W, from->W.data(), (size_t)C * 8, cudaMemcpyHostToDevice, st));
    if (tc0 > 0) {
      KKM_CK(cudaMemcpyAsync(I.trace_omega, from->omega.data(), (size_t)tc0 * 8, cudaMemcpyHostToDevice, st));
      KKM_CK(cudaMemcpyAsync(I.trace_changed, from->changed.data(), (size_t)tc0 * 4, cudaMemcpyHostToDevice, st));
    }
    KKM_CK(cudaMemcpyAsync(disp, from->displacement.data(), (size_t)start * 8, cudaMemcpyHostToDevice, st));
    KKM_CK(cudaMemcpyAsync(I.trace_count, &tc0, 4, cudaMemcpyHostToDevice, st));
    KKM_CK(cudaStreamSynchronize(st));  // tc0 lives on this stack frame
  } else if (do_kpp) {
    KKM_TRY(ws.alloc(&D2, 2 * geo[0].Ni + ceil_div(geo[0].Ni, 32)));
    KKM_TRY(ws.alloc(&draws_d, C));
    KKM_TRY(ws.alloc(&kpp_ticket, 1));
    KKM_CK(cudaMemsetAsync(kpp_ticket, 0, 4, st));
    KKM_CK(cudaMemcpyAsync(draws_d, draws.data(), (size_t)C * 8, cudaMemcpyHostToDevice, st));
    KKM_CK(cudaMemcpyAsync(picks, pick0.data(), 4, cudaMemcpyHostToDevice, st));
  } else {
    KKM_CK(cudaMemcpyAsync(Mg, init.data(), (size_t)C * 8, cudaMemcpyHostToDevice, st));
  }
  KKM_CK(cudaMemcpyAsync(Ld_all, L_all.data(), L_all.size() * 4, cudaMemcpyHostToDevice, st));
  if (!from) KKM_CK(cudaMemsetAsync(W, 0, (size_t)C * 8, st));
  const bool labels_on_host = labels_out && !is_device_ptr(labels_out);
  if (labels_out) {
    if (labels_on_host) {
      KKM_TRY(ws.alloc(&labels_dev, N));
      // a partial range writes only its own rows: the others keep the
      // caller's values
      if (start > 0 || stop < B)
        KKM_CK(cudaMemcpyAsync(labels_dev, labels_out, (size_t)N * 4, cudaMemcpyHostToDevice, st));
    } else {
      labels_dev = labels_out;
    }
  }
  // Feature kernels carry the medoid rows from one mini-batch to the next
  // (the rows after the merge are rows of the mini-batch just done); MD
  // frames are prepared again from X.
  const bool rows_carried = sp.kind != KKM_RMSD;
  bool mx_ready = false;  // MX/auxM hold the rows of Mg

  // Alg. 1 line 3 for mini-batch i on stream `bs`, in two parts: its rows,
  // landmark rows, ids and reduced-precision copies (no bandwidth needed),
  // then the kernel block into the buffer set b.
  auto block_rows = [&](int i, const BlockBufs& b, cudaStream_t bs) -> kkm_status {
    const BatchGeom& g = geo[i];
    const int Ni = (int)g.Ni;
    const int nL = (int)(L_off[i + 1] - L_off[i]);
    const int32_t* Ld = Ld_all + L_off[i];
    if (!(first_fetched && i == start))
      KKM_TRY(prep_rows(sp, X, g.start, g.step, Ni, b.Xi, b.aux_i, bs, pull_bad, pull_stage));  // fetch X^i
    KKM_RUN("iota", bs, (iota64_kernel<<<blocks_for(Ni), 256, 0, bs>>>(b.gid, g.start, g.step, Ni), cudaGetLastError()));
    KKM_TRY(copy_prepared(sp, b.Xi, Ld, nL, b.XL, b.auxL, bs));                 // landmarks
    KKM_RUN("gather_ids", bs, (gather_i64_kernel<<<blocks_for(nL), 256, 0, bs>>>(b.gid, Ld, nL, b.gidL), cudaGetLastError()));
    return block_convert(sp, bm, b, nL, Ni, bs);
  };
  auto block_gram = [&](int i, const BlockBufs& b, cudaStream_t bs, bool side) -> kkm_status {
    const int Ni = (int)geo[i].Ni;
    const int nL = (int)(L_off[i + 1] - L_off[i]);
    return block_kernel(sp, bm, b, Ld_all + L_off[i], nL, Ni, ldk, tc_err, bs, side ? side_sms : 0,
                        /*converted=*/true);
  };
  auto block_step = [&](int i, const BlockBufs& b, cudaStream_t bs, bool side) -> kkm_status {
    KKM_TRY(block_rows(i, b, bs));
    return block_gram(i, b, bs, side);
  };

  // ---- Algorithm 1
  // both streams after the uploads and fills of the workspace on st
  KKM_TRY(FitStreams::after(st, ms));
  KKM_TRY(FitStreams::after(st, fs.side));
  // the first mini-batch's rows need no bandwidth: they are gathered while
  // the host waits for the finite check and the median rule.  With the
  // pipeline, k-means++ and the Eq. 8 labels of that mini-batch (which read
  // its rows, not its block) then run beside its kernel block.
  struct OwnedEvent {
    cudaEvent_t e = nullptr;
    ~OwnedEvent() {
      if (e) cudaEventDestroy(e);
    }
  } rows_ready, block_ready;
  KKM_TRY(block_rows(start, bb[start % nbuf], overlap ? fs.side : ms));
  if (overlap) {
    KKM_CK(cudaEventCreateWithFlags(&rows_ready.e, cudaEventDisableTiming));
    KKM_CK(cudaEventCreateWithFlags(&block_ready.e, cudaEventDisableTiming));
    KKM_CK(cudaEventRecord(rows_ready.e, fs.side));
  }
  {
    bool bad = false;
    KKM_TRY(chk.wait(&bad));
    if (bad) return invalid("X holds NaN or Inf");
  }
  if (from) {
    sp.sigma = from->sigma;
  } else if (need_median) {
    KKM_CK(cudaStreamSynchronize(st));  // at once when the check's wait already covered it
    sp.sigma = median_sigma_of(*sig_h);
  }
  if (overlap) {
    KKM_TRY(block_gram(start, bb[start % nbuf], fs.side, false));  // no loop to overlap yet
    KKM_CK(cudaEventRecord(block_ready.e, fs.side));
  }
  for (int i = start; i < stop; ++i) {
    NvtxRange nv_batch("mini-batch");
    const BatchGeom& g = geo[i];
    const int Ni = (int)g.Ni;
    const int nL = (int)(L_off[i + 1] - L_off[i]);
    const int32_t* Ld = Ld_all + L_off[i];
    const BlockBufs& bk = bb[i % nbuf];
    if (overlap) {
      // the block of mini-batch i is ready (the first one: its rows; the
      // block is waited for before the loop)
      if (i == start) KKM_CK(cudaStreamWaitEvent(ms, rows_ready.e, 0));
      else KKM_TRY(FitStreams::after(fs.side, ms));
    } else if (i == start) {
      KKM_TRY(block_gram(i, bk, ms, false));  // its rows are gathered above
    } else {
      KKM_TRY(block_step(i, bk, ms, false));
    }
    float* const Xi = bk.Xi;
    float* const aux_i = bk.aux_i;
    int64_t* const gid = bk.gid;
    const float* kself = sp.kind == KKM_LINEAR ? aux_i : nullptr;
    if (i == 0 && do_kpp) {                                                   // Alg. 1 lines 4-6
      KKM_TRY(kmeanspp_dev(sp, Xi, aux_i, Ni, C, kself, rowbuf, rowaux, kcol, ldk, D2, picks, draws_d, kpp_ticket,
                           ms));
      KKM_RUN("local_to_global", ms, launch_local_to_global(picks, C, g.start, g.step, Mg, ms));
    }
    // the side stream produces the next block into the other buffer set,
    // whose last reader (mini-batch i - 1) is queued on the main stream
    // before this point; in the first mini-batch only after k-means++, whose
    // rounds re-read X^i from L2 (a fetch of the next rows beside them, from
    // host memory in particular, would push X^i out)
    if (overlap && i + 1 < stop) {
      KKM_TRY(FitStreams::after(ms, fs.side));
      KKM_TRY(block_step(i + 1, bb[(i + 1) % nbuf], fs.side, true));
    }
    // Eq. 8: auxiliary block K~ = K(M, X^i) and nearest-medoid labels
    const float* kmm = sp.kind == KKM_LINEAR ? auxM : nullptr;
    if (!mx_ready) KKM_TRY(prep_ids(sp, X, Mg, C, MX, auxM, ms));
    KKM_TRY(kernel_block(sp, MX, auxM, Mg, C, Xi, aux_i, gid, Ni, Kt, ldk, ms));
    KKM_RUN("nearest", ms, launch_nearest(Kt, ldk, Ni, C, kself, kmm, u, nullptr, ms));

    // supports of the initial labels
    S.L = Ld;
    S.nL = nL;
    // column maps, early stop, g_hat numerators (the last mini-batch's medoid
    // step read them), the Eq. 10 keys and counts
    KKM_RUN("loop_reset", ms,
            (loop_reset_kernel<<<blocks_for(std::max<int64_t>(ldk, C)), 256, 0, ms>>>(S.col_label, S.col_ord, ldk, I.done,
                                                                                   I.gfix, keys, cnt, C),
             cudaGetLastError()));
    KKM_RUN("landmark_maps", ms, launch_landmark_maps(S, u, ms));
    KKM_RUN("build_supports", ms, launch_build_supports(S, ms));
    I.keep_rows = kt_half ? l2_keep_rows(ldk, nL, kL2KeepShareHalf, 2) : l2_keep_rows(ldk, nL, kL2KeepShare, 4);
    I.flag_tau = bm.flag_tau(sp);
    const RescoreArgs R = rescore_args(sp, bk, ldk);
    const int form = loop_form(opt.iteration, sp, bm, Ni, nL, C);
    if (form < 0)
      return invalid(opt.iteration == KKM_ITER_TC
                         ? "KKM_ITER_TC does not apply to this shape (RBF with KKM_BF16 or KKM_FP8, C <= 16, at most "
                           "128 samples per SM in a mini-batch, about 3,000 landmarks)"
                         : "KKM_ITER_FUSED does not apply to this shape (C <= 64 and a mini-batch of at most one "
                           "column per thread of one CTA per SM)");
    NvtxRange nv_loop("inner loop");
    MedoidOut med;
    if (form == kLoopTc) {  // the loop leaves the Eq. 10 keys itself (reset above)
      med.keys = keys;
      med.cnt = cnt;
      med.ghat = ghat;
      med.need_supports = i == B - 1 && model_out;  // the model keeps the final support structure
    }
    if (overlap && i == start) KKM_CK(cudaStreamWaitEvent(ms, block_ready.e, 0));
    KKM_TRY(inner_loop(bm, bk, ldk, Ni, S, I, form, iters, kself, u, nullptr, nullptr, nullptr,  // Alg. 1 lines 9-16
                       opt.early_stop, R, ms, med));
    I.flag_tau = 0.0f;
    if (form != kLoopTc) {
      // Eq. 10: f_hat of the final labels and the mini-batch medoids
      IterState Ifin = I;
      Ifin.done = nullptr;
      KKM_RUN("fhat_partial", ms,
              kt_half ? launch_fhat_partial(bk.KTh, ldk, Ni, S, Ifin, ms)
                      : launch_fhat_partial(bk.KT, ldk, Ni, S, Ifin, ms));
      KKM_RUN("medoid_keys", ms, launch_medoid_keys(ldk, Ni, S, Ifin, kself, u, keys, cnt, ghat, ms));
    }
    if (rows_carried) {
      KKM_RUN("medoid_rows", ms,
              launch_medoid_rows(keys, cnt, S.n_j, C, mi, mi_safe, Xi, aux_i, sp.dp, gid, MIX, auxMI, idMI, ms));
    } else {
      KKM_RUN("medoid_pick", ms, launch_medoid_pick(keys, cnt, S.n_j, C, mi, ms, /*reset_keys=*/true));
      KKM_RUN("clamp_idx", ms, (clamp_idx_kernel<<<blocks_for(C), 256, 0, ms>>>(mi, C, mi_safe), cudaGetLastError()));
      KKM_TRY(copy_prepared(sp, Xi, mi_safe, C, MIX, auxMI, ms));
      KKM_RUN("gather_ids", ms, (gather_i64_kernel<<<blocks_for(C), 256, 0, ms>>>(gid, mi, C, idMI), cudaGetLastError()));
    }
    // Eq. 12: K(X^i, m^i) and the convex merge
    KKM_TRY(kernel_block(sp, MIX, auxMI, idMI, C, Xi, aux_i, gid, Ni, Kmi, ldk, ms));
    KKM_RUN("merge_keys", ms, launch_merge_keys(Kt, Kmi, ldk, Ni, C, kself, mi, cnt, W, keys, ms));
    KKM_RUN("merge_apply", ms, launch_merge_apply(keys, mi, cnt, C, g.start, g.step, Mg, W, ms, Mg_prev));
    // how far the global medoids moved in this outer iteration (Fig. 4b):
    // K(old medoid row, new medoid row) per cluster
    if (rows_carried) {
      KKM_RUN("displacement", ms,
              launch_displacement_rows(MX, auxM, Xi, aux_i, sp.dp, C, keys, mi, Mg_prev, Mg, sp.kind == KKM_LINEAR,
                                       sp.neg_scale(), disp + i, MXn, auxMn, ms));
      std::swap(MX, MXn);  // the rows of the medoids after the merge
      std::swap(auxM, auxMn);
      mx_ready = true;
    } else {
      KKM_TRY(prep_ids(sp, X, Mg, C, MXn, auxMn, ms));
      KKM_TRY(kernel_block(sp, MX, auxM, Mg_prev, C, MXn, auxMn, Mg, C, Kmn, ldc, ms));
      KKM_RUN("displacement", ms,
              launch_displacement(Kmn, ldc, C, kmm, sp.kind == KKM_LINEAR ? auxMn : nullptr, Mg_prev, Mg, disp + i,
                                  ms));
    }
    if (labels_dev)
      KKM_RUN("scatter_labels", ms, launch_scatter_labels(u, Ni, g.start, g.step, labels_dev, ms));
    if (i == B - 1 && model_out) {
      // keep the final supports of the last mini-batch
      kkm_model* m = new kkm_model();
      m->C = C;
      m->d = d;
      m->kind = sp.kind;
      m->sigma = sp.sigma;
      m->n_atoms = sp.n_atoms;
      m->dp = sp.dp;
      m->nL = nL;
      m->device = dev;
      std::unique_ptr<kkm_model> guard(m);
      m->max_units = lb.max_units;
      KKM_TRY(model_alloc_device(m, ms));
      const int mu = m->max_units;
      // the resident arrays, copied by one launch
      CopyList cl;
      auto cp = [&](void* dst, const void* src, size_t bytes) {
        cl.src[cl.n] = src;
        cl.dst[cl.n] = dst;
        cl.words[cl.n] = (int64_t)(bytes / 4);
        ++cl.n;
      };
      cp(m->sup, bk.XL, (size_t)nL * sp.dp * 4);
      cp(m->sup_aux, bk.auxL, (size_t)nL * 4);
      cp(m->sup_ids, bk.gidL, (size_t)nL * 8);
      cp(m->perm, S.perm, (size_t)nL * 4);
      cp(m->seg_off, S.seg_off, (size_t)(C + 1) * 4);
      cp(m->n_j, S.n_j, (size_t)C * 4);
      cp(m->unit_j, S.unit_j, (size_t)mu * 4);
      cp(m->unit_kb, S.unit_kb, (size_t)mu * 4);
      cp(m->unit_ke, S.unit_ke, (size_t)mu * 4);
      cp(m->seg_unit, S.seg_unit, (size_t)(C + 1) * 4);
      cp(m->n_units, S.n_units, 4);
      cp(m->ghat, ghat, (size_t)C * 8);
      KKM_RUN("copy_model", ms,
              (copy_many_kernel<<<dim3(2 * (unsigned)sm_count(), (unsigned)cl.n), 256, 0, ms>>>(cl),
               cudaGetLastError()));
      KKM_RUN("gather_labels", ms, (gather_i32_kernel<<<blocks_for(nL), 256, 0, ms>>>(u, Ld, nL, m->sup_labels), cudaGetLastError()));
      KKM_RUN("iota", ms, (iota32_kernel<<<blocks_for(nL), 256, 0, ms>>>(m->L_ident, nL), cudaGetLastError()));
      *model_out = guard.release();
    }
  }

  KKM_TRY(fs.join());

  // ---- results: every read-back through one pinned stage, one wait
  if (pull_bad) {  // the rows' finite check, before any output is written
    int h = 0;
    KKM_CK(cudaMemcpyAsync(sig_h, pull_bad, 4, cudaMemcpyDeviceToHost, st));
    KKM_CK(cudaStreamSynchronize(st));
    memcpy(&h, sig_h, 4);
    if (h) {
      if (model_out && *model_out) {
        delete *model_out;
        *model_out = nullptr;
      }
      return invalid("X holds NaN or Inf");
    }
  }
  kkm_model* const mres = model_out ? *model_out : nullptr;
  const int32_t tcap = std::max(trace_cap, 1);
  int32_t tc = 0;
  std::vector<double> om_h;
  std::vector<int32_t> ch_h;
  int tc_err_h = 0, rtc_err_h[2] = {0, 0}, it_err_h = 0;
  std::unique_ptr<kkm_checkpoint> ck;
  Readback rb;
  if (mres) {
    kkm_model* m = mres;
    if (mx_ready) {
      KKM_CK(cudaMemcpyAsync(m->med, MX, (size_t)C * sp.dp * 4, cudaMemcpyDeviceToDevice, st));
      KKM_CK(cudaMemcpyAsync(m->med_aux, auxM, (size_t)C * 4, cudaMemcpyDeviceToDevice, st));
    } else {
      KKM_TRY(prep_ids(sp, X, Mg, C, m->med, m->med_aux, st));
    }
    float* coords = nullptr;  // medoid rows in the caller's layout
    KKM_TRY(ws.alloc(&coords, (int64_t)C * d));
    KKM_RUN("gather_rows", st,
            (gather_raw_rows_kernel<<<blocks_for((int64_t)C * d), 256, 0, st>>>(X, d, Mg, C, coords),
             cudaGetLastError()));
    m->medoids.resize(C);
    m->W.resize(C);
    m->displacement.resize(B);
    m->sup_labels_h.resize(m->nL);
    m->ghat_h.resize(C);
    m->n_h.resize(C);
    m->med_coords_h.resize((size_t)C * d);
    rb.add(m->medoids.data(), Mg, (size_t)C * 8);
    rb.add(m->W.data(), W, (size_t)C * 8);
    rb.add(m->displacement.data(), disp, (size_t)B * 8);
    rb.add(m->sup_labels_h.data(), m->sup_labels, (size_t)m->nL * 4);
    rb.add(m->ghat_h.data(), m->ghat, (size_t)C * 8);
    rb.add(m->n_h.data(), m->n_j, (size_t)C * 4);
    rb.add(m->med_coords_h.data(), coords, (size_t)C * d * 4);
  }
  if (ckpt_out) {
    ck.reset(new kkm_checkpoint());
    kkm_checkpoint* c = ck.get();
    c->N = N;
    c->d = d;
    c->C = C;
    c->B = B;
    c->s = s;
    c->kind = k->kind;
    c->n_atoms = k->n_atoms;
    c->iters = iters;
    c->sigma_arg = sigma_arg;
    c->seed = seed;
    c->precision = opt.precision;
    c->sampling = opt.sampling;
    c->early_stop = opt.early_stop;
    c->had_init = opt.init_medoids ? 1 : 0;
    c->next_batch = stop;
    c->sigma = sp.sigma;
    c->M.resize(C);
    c->W.resize(C);
    c->displacement.resize(stop);
    rb.add(c->M.data(), Mg, (size_t)C * 8);
    rb.add(c->W.data(), W, (size_t)C * 8);
    rb.add(c->displacement.data(), disp, (size_t)stop * 8);
  }
  if (mres || ckpt_out) {  // the whole trace capacity; the count says how much of it is used
    om_h.resize(tcap);
    ch_h.resize(tcap);
    rb.add(&tc, I.trace_count, 4);
    rb.add(om_h.data(), I.trace_omega, (size_t)tcap * 8);
    rb.add(ch_h.data(), I.trace_changed, (size_t)tcap * 4);
  }
  if (labels_on_host)
    KKM_CK(cudaMemcpyAsync(labels_out, labels_dev, (size_t)N * 4, cudaMemcpyDeviceToHost, st));
  if (tc_err) rb.add(&tc_err_h, tc_err, 4);
  rb.add(&it_err_h, I.err, 4);
  for (int q = 0; q < nbuf; ++q)
    if (use_rtc) rb.add(&rtc_err_h[q], bb[q].rtc.err, 4);
  KKM_TRY(rb.run(st));
  tc_err_h |= rtc_err_h[0] | rtc_err_h[1];
  if (tc_err_h) {
    set_error("tensor-core kernel block: a bounded pipeline wait gave up (code " + std::to_string(tc_err_h) + ")");
    return KKM_ETIMEOUT;
  }
  if (it_err_h) {
    set_error("fused inner iteration: the bounded grid-barrier wait gave up");
    return KKM_ETIMEOUT;
  }
  tc = std::min(std::max(tc, 0), tcap);
  if (mres) {
    mres->omega.assign(om_h.begin(), om_h.begin() + tc);
    mres->changed.assign(ch_h.begin(), ch_h.begin() + tc);
  }
  if (ck) {
    ck->omega.assign(om_h.begin(), om_h.begin() + tc);
    ck->changed.assign(ch_h.begin(), ch_h.begin() + tc);
    *ckpt_out = ck.release();
  }
  prof_collect();
  return KKM_OK;
}

}  // namespace kkm

namespace kkm {

// ======================================================================
// kkm_assign / kkm_cost
// ======================================================================
static kkm_status assign_impl(const kkm_model* m, const float* Xnew_in, int64_t M, int32_t mode,
                              int32_t* labels_out, float* dist_out, double* omega_out,
                              cudaStream_t st) {
  NvtxRange nv("kkm_assign");
  if (!m) return invalid("model is NULL");
  if (M < 0 || M > INT32_MAX) return invalid("M must be in [0, 2^31)");
  if (mode != KKM_ASSIGN_SUPPORTS && mode != KKM_ASSIGN_MEDOIDS) return invalid("unknown assign mode");
  if (M == 0) {
    if (omega_out) *omega_out = 0.0;
    return KKM_OK;
  }
  if (!Xnew_in) return invalid("X is NULL");
  kkm_kernel kk{m->kind, m->sigma, m->n_atoms};
  KernelSpec sp;
  KKM_TRY(make_spec(&kk, m->d, &sp));
  const int64_t d = m->d;
  const int C = m->C;
  int dev = 0;
  KKM_CK(cudaGetDevice(&dev));
  setup_pool_once(dev);
  Workspace ws(st);
  const float* X = nullptr;
  {
    bool bad = false;
    KKM_TRY(device_input_checked(ws, Xnew_in, M * d, &X, &bad));
    if (bad) return invalid("X holds NaN or Inf");
  }
  int32_t* lab = nullptr;
  float* dist = nullptr;
  const bool lab_host = labels_out && !is_device_ptr(labels_out);
  const bool dist_host = dist_out && !is_device_ptr(dist_out);
  if (!labels_out || lab_host) KKM_TRY(ws.alloc(&lab, M)); else lab = labels_out;
  if (!dist_out || dist_host) KKM_TRY(ws.alloc(&dist, M)); else dist = dist_out;

  const int rows_ref = mode == KKM_ASSIGN_SUPPORTS ? m->nL : C;
  const int64_t budget_floats = (int64_t)1 << 27;  // 512 MB of kernel values per chunk
  const int64_t chunk = std::max<int64_t>(1024, std::min<int64_t>(M, budget_floats / std::max(rows_ref, 1)));
  const int64_t ldm = round_up(std::min(chunk, M), 32);
  float *Xc, *auxc, *Kb;
  KKM_TRY(ws.alloc(&Xc, ldm * sp.dp));
  KKM_TRY(ws.alloc(&auxc, ldm));
  KKM_TRY(ws.alloc(&Kb, (int64_t)rows_ref * ldm));
  const float* kself = sp.kind == KKM_LINEAR ? auxc : nullptr;
  RmsdTcScratch rtc;
  const bool use_rtc = sp.kind == KKM_RMSD && rows_ref >= kRmsdTcMinRefs;
  if (use_rtc) KKM_TRY(alloc_rmsd_tc(ws, sp, rows_ref, ldm, ldm, &rtc));
  LoopBuffers lb;
  if (mode == KKM_ASSIGN_SUPPORTS) {
    KKM_TRY(alloc_loop(ws, m->nL, C, ldm, 1, &lb));
    Supports& S = lb.S;
    S.L = m->L_ident;
    S.nL = m->nL;
    S.perm = m->perm;
    S.seg_off = m->seg_off;
    S.n_j = m->n_j;
    S.unit_j = m->unit_j;
    S.unit_kb = m->unit_kb;
    S.unit_ke = m->unit_ke;
    S.seg_unit = m->seg_unit;
    S.n_units = m->n_units;
    S.col_label = nullptr;
    S.col_ord = nullptr;
    S.lab = nullptr;
    lb.I.ghat_in = m->ghat;
    lb.I.done = nullptr;
  }
  for (int64_t c0 = 0; c0 < M; c0 += chunk) {
    const int n = (int)std::min<int64_t>(chunk, M - c0);
    KKM_TRY(prep_rows(sp, X, c0, 1, n, Xc, auxc, st));
    if (mode == KKM_ASSIGN_SUPPORTS) {
      KKM_TRY(kernel_block(sp, m->sup, m->sup_aux, nullptr, m->nL, Xc, auxc, nullptr, n, Kb, ldm, st, false, false,
                           use_rtc ? &rtc : nullptr));
      KKM_RUN("fhat_partial", st, launch_fhat_partial(Kb, ldm, n, lb.S, lb.I, st));
      KKM_RUN("assign", st,
              launch_assign(ldm, n, lb.S, lb.I, kself, lab + c0, nullptr, dist + c0, nullptr, nullptr, 0,
                            /*rebuild=*/0, st));
    } else {
      KKM_TRY(kernel_block(sp, m->med, m->med_aux, nullptr, C, Xc, auxc, nullptr, n, Kb, ldm, st, false, false,
                           use_rtc ? &rtc : nullptr));
      KKM_RUN("nearest", st,
              launch_nearest(Kb, ldm, n, C, kself, sp.kind == KKM_LINEAR ? m->med_aux : nullptr, lab + c0,
                             dist + c0, st));
    }
  }
  double* omega_d = nullptr;
  if (omega_out) {
    double* part;
    KKM_TRY(ws.alloc(&part, 256));
    KKM_TRY(ws.alloc(&omega_d, 1));
    KKM_RUN("sum", st, launch_sum_f32_to_f64(dist, M, part, 256, omega_d, st));
    KKM_CK(cudaMemcpyAsync(omega_out, omega_d, 8, cudaMemcpyDeviceToHost, st));
  }
  if (lab_host) KKM_CK(cudaMemcpyAsync(labels_out, lab, (size_t)M * 4, cudaMemcpyDeviceToHost, st));
  if (dist_host) KKM_CK(cudaMemcpyAsync(dist_out, dist, (size_t)M * 4, cudaMemcpyDeviceToHost, st));
  int rtc_err_h = 0;
  if (use_rtc) KKM_CK(cudaMemcpyAsync(&rtc_err_h, rtc.err, 4, cudaMemcpyDeviceToHost, st));
  KKM_CK(cudaStreamSynchronize(st));
  prof_collect();
  if (rtc_err_h) {
    set_error("tensor-core MD estimate: a bounded pipeline wait gave up");
    return KKM_ETIMEOUT;
  }
  return KKM_OK;
}

// ======================================================================
// kkm_kernel_matrix
// ======================================================================
static kkm_status kernel_matrix_impl(const float* A_in, int64_t nA, const float* B_in, int64_t nB, int64_t d,
                                     const kkm_kernel* k, int32_t precision, float* out, cudaStream_t st) {
  KernelSpec sp;
  KKM_TRY(make_spec(k, d, &sp));
  if (precision != KKM_FP32 && precision != KKM_BF16 && precision != KKM_FP8)
    return invalid("precision must be KKM_FP32, KKM_BF16 or KKM_FP8");
  if (precision != KKM_FP32 && sp.kind == KKM_RMSD)
    return invalid("KKM_BF16 and KKM_FP8 apply to the RBF and linear kernels");
  sp.precision = precision;
  if (nA < 0 || nB < 0 || nA > INT32_MAX || nB > INT32_MAX) return invalid("bad sizes");
  if (sp.kind != KKM_LINEAR && !(sp.sigma > 0.0f && isfinite(sp.sigma))) return invalid("sigma must be > 0");
  if (nA == 0 || nB == 0) return KKM_OK;
  if (!A_in || !B_in || !out) return invalid("NULL pointer");
  int dev = 0;
  KKM_CK(cudaGetDevice(&dev));
  setup_pool_once(dev);
  Workspace ws(st);
  const float *A, *Bm;
  KKM_TRY(device_input(ws, A_in, nA * d, &A));
  KKM_TRY(device_input(ws, B_in, nB * d, &Bm));
  float *Ap, *Bp, *aA, *aB, *o;
  KKM_TRY(ws.alloc(&Ap, nA * sp.dp));
  KKM_TRY(ws.alloc(&Bp, nB * sp.dp));
  KKM_TRY(ws.alloc(&aA, nA));
  KKM_TRY(ws.alloc(&aB, nB));
  const bool host_out = !is_device_ptr(out);
  if (host_out) KKM_TRY(ws.alloc(&o, nA * nB)); else o = out;
  KKM_TRY(prep_rows(sp, A, 0, 1, nA, Ap, aA, st));
  KKM_TRY(prep_rows(sp, Bm, 0, 1, nB, Bp, aB, st));
  int tc_err_h = 0;
  if (precision == KKM_BF16) {
    __nv_bfloat16 *Ab, *Bb;
    float *nAb, *nBb;
    int* err;
    KKM_TRY(ws.alloc(&Ab, nA * sp.dp));
    KKM_TRY(ws.alloc(&Bb, nB * sp.dp));
    KKM_TRY(ws.alloc(&nAb, nA));
    KKM_TRY(ws.alloc(&nBb, nB));
    KKM_TRY(ws.alloc(&err, 1));
    KKM_CK(cudaMemsetAsync(err, 0, 4, st));
    KKM_TRY(kernel_block_bf16(sp, Ap, nullptr, nA, Bp, nB, o, false, nB, Ab, nAb, Bb, nBb, err, st));
    KKM_CK(cudaMemcpyAsync(&tc_err_h, err, 4, cudaMemcpyDeviceToHost, st));
  } else if (precision == KKM_FP8) {
    const int64_t ld8 = round_up(sp.dp, 16);
    uint8_t *A8, *B8;
    float *sA, *sB, *nA8, *nB8;
    int* err;
    KKM_TRY(ws.alloc(&A8, nA * ld8));
    KKM_TRY(ws.alloc(&B8, nB * ld8));
    KKM_TRY(ws.alloc(&sA, nA));
    KKM_TRY(ws.alloc(&sB, nB));
    KKM_TRY(ws.alloc(&nA8, nA));
    KKM_TRY(ws.alloc(&nB8, nB));
    KKM_TRY(ws.alloc(&err, 1));
    KKM_CK(cudaMemsetAsync(err, 0, 4, st));
    KKM_TRY(kernel_block_fp8(sp, Ap, nullptr, nA, Bp, nB, o, false, nB, A8, sA, nA8, B8, sB, nB8, err, st));
    KKM_CK(cudaMemcpyAsync(&tc_err_h, err, 4, cudaMemcpyDeviceToHost, st));
  } else if (sp.kind == KKM_RMSD && nA >= kRmsdTcMinRefs) {
    // the MD kernel takes the same tensor-core estimate + exact-refine path as a fit
    RmsdTcScratch rtc;
    KKM_TRY(alloc_rmsd_tc(ws, sp, nA, nB, nB, &rtc));
    KKM_TRY(kernel_block(sp, Ap, aA, nullptr, nA, Bp, aB, nullptr, nB, o, nB, st, false, false, &rtc));
    KKM_CK(cudaMemcpyAsync(&tc_err_h, rtc.err, 4, cudaMemcpyDeviceToHost, st));
  } else {
    KKM_TRY(kernel_block(sp, Ap, aA, nullptr, nA, Bp, aB, nullptr, nB, o, nB, st));
  }
  if (host_out) KKM_CK(cudaMemcpyAsync(out, o, (size_t)nA * nB * 4, cudaMemcpyDeviceToHost, st));
  KKM_CK(cudaStreamSynchronize(st));
  prof_collect();
  if (tc_err_h) {
    set_error("tensor-core kernel block: a bounded pipeline wait gave up");
    return KKM_ETIMEOUT;
  }
  return KKM_OK;
}

// ======================================================================
// kkm_debug_step (teacher-forced inner iteration)
// ======================================================================
static kkm_status debug_step_impl(const float* Xb_in, int64_t Ni, int64_t d, const int32_t* L, int32_t nL,
                                  const kkm_kernel* k, int32_t C, int32_t precision, int32_t iteration,
                                  const int32_t* u_in,
                                  int32_t* u_out, float* fhat_out, float* margin_out, double* ghat_out,
                                  int32_t* n_out, double* omega_out, int32_t* changed_out, cudaStream_t st) {
  KernelSpec sp;
  KKM_TRY(make_spec(k, d, &sp));
  if (Ni < 1 || Ni > INT32_MAX) return invalid("Ni must be >= 1");
  if (C < 1 || C > kMaxC) return invalid("C must be in [1, 256]");
  if (nL < 1 || nL > Ni || !L || !u_in || !Xb_in) return invalid("bad landmarks or NULL pointer");
  if (precision != KKM_FP32 && precision != KKM_BF16 && precision != KKM_FP8)
    return invalid("precision must be KKM_FP32, KKM_BF16 or KKM_FP8");
  if (precision != KKM_FP32 && sp.kind == KKM_RMSD)
    return invalid("KKM_BF16 and KKM_FP8 apply to the RBF and linear kernels");
  if (iteration != KKM_ITER_AUTO && iteration != KKM_ITER_FUSED && iteration != KKM_ITER_SPLIT &&
      iteration != KKM_ITER_TC)
    return invalid("unknown iteration form");
  sp.precision = precision;
  if (sp.kind != KKM_LINEAR && !(sp.sigma > 0.0f && isfinite(sp.sigma))) return invalid("sigma must be > 0");
  for (int q = 0; q < nL; ++q)
    if (L[q] < 0 || L[q] >= Ni || (q > 0 && L[q] <= L[q - 1])) return invalid("L must be sorted, in [0, Ni)");
  for (int64_t q = 0; q < Ni; ++q)
    if (u_in[q] < 0 || u_in[q] >= C) return invalid("labels must be in [0, C)");
  int dev = 0;
  KKM_CK(cudaGetDevice(&dev));
  setup_pool_once(dev);
  Workspace ws(st);
  const float* X;
  KKM_TRY(device_input(ws, Xb_in, Ni * d, &X));
  const int64_t ldk = round_up(Ni, 32);
  // the fit's block buffers and block evaluation for this precision
  const BlockMode bm(sp, nL);
  BlockBufs b;
  KKM_TRY(alloc_block_bufs(ws, sp, Ni, nL, ldk, bm.kt_half, bm.use_rtc, &b, bm.fp32_half_block));
  float *fh, *mg;
  int32_t *Ld, *u;
  double* gh;
  int* tc_err = nullptr;
  KKM_TRY(ws.alloc(&Ld, nL));
  KKM_TRY(ws.alloc(&u, Ni));
  KKM_TRY(ws.alloc(&fh, Ni * C));
  KKM_TRY(ws.alloc(&mg, Ni));
  KKM_TRY(ws.alloc(&gh, C));
  if (sp.precision != KKM_FP32) {
    KKM_TRY(ws.alloc(&tc_err, 1));
    KKM_CK(cudaMemsetAsync(tc_err, 0, 4, st));
  }
  KKM_CK(cudaMemcpyAsync(Ld, L, (size_t)nL * 4, cudaMemcpyHostToDevice, st));
  KKM_CK(cudaMemcpyAsync(u, u_in, (size_t)Ni * 4, cudaMemcpyHostToDevice, st));
  KKM_TRY(prep_rows(sp, X, 0, 1, Ni, b.Xi, b.aux_i, st));
  KKM_RUN("iota", st, (iota64_kernel<<<blocks_for(Ni), 256, 0, st>>>(b.gid, 0, 1, Ni), cudaGetLastError()));
  KKM_TRY(copy_prepared(sp, b.Xi, Ld, nL, b.XL, b.auxL, st));
  KKM_RUN("gather_ids", st, (gather_i64_kernel<<<blocks_for(nL), 256, 0, st>>>(b.gid, Ld, nL, b.gidL), cudaGetLastError()));
  KKM_TRY(block_kernel(sp, bm, b, Ld, nL, (int)Ni, ldk, tc_err, st));
  LoopBuffers lb;
  KKM_TRY(alloc_loop(ws, nL, C, ldk, 1, &lb, sp.gaussian()));
  lb.S.L = Ld;
  lb.S.nL = nL;
  KKM_RUN("fill", st, launch_fill_i32(lb.S.col_label, -1, ldk, st));
  KKM_RUN("fill", st, launch_fill_i32(lb.S.col_ord, -1, ldk, st));
  KKM_RUN("landmark_maps", st, launch_landmark_maps(lb.S, u, st));
  KKM_RUN("build_supports", st, launch_build_supports(lb.S, st));
  KKM_CK(cudaMemcpyAsync(lb.n_copy, lb.S.n_j, (size_t)C * 4, cudaMemcpyDeviceToDevice, st));
  const float* kself = sp.kind == KKM_LINEAR ? b.aux_i : nullptr;
  lb.I.keep_rows = 0;
  lb.I.flag_tau = bm.flag_tau(sp);
  const RescoreArgs R = rescore_args(sp, b, ldk);
  const int form = loop_form(iteration, sp, bm, (int)Ni, nL, C);
  if (form < 0) return invalid("the iteration form asked for does not apply to this shape");
  KKM_TRY(inner_loop(bm, b, ldk, (int)Ni, lb.S, lb.I, form, 1, kself, u, mg, fh, gh, 0, R, st));
  if (u_out) KKM_CK(cudaMemcpyAsync(u_out, u, (size_t)Ni * 4, cudaMemcpyDeviceToHost, st));
  if (fhat_out) KKM_CK(cudaMemcpyAsync(fhat_out, fh, (size_t)Ni * C * 4, cudaMemcpyDeviceToHost, st));
  if (margin_out) KKM_CK(cudaMemcpyAsync(margin_out, mg, (size_t)Ni * 4, cudaMemcpyDeviceToHost, st));
  if (ghat_out) KKM_CK(cudaMemcpyAsync(ghat_out, gh, (size_t)C * 8, cudaMemcpyDeviceToHost, st));
  if (n_out) KKM_CK(cudaMemcpyAsync(n_out, lb.n_copy, (size_t)C * 4, cudaMemcpyDeviceToHost, st));
  if (omega_out) KKM_CK(cudaMemcpyAsync(omega_out, lb.I.trace_omega, 8, cudaMemcpyDeviceToHost, st));
  if (changed_out) KKM_CK(cudaMemcpyAsync(changed_out, lb.I.trace_changed, 4, cudaMemcpyDeviceToHost, st));
  int tc_err_h = 0, it_err_h = 0;
  if (tc_err) KKM_CK(cudaMemcpyAsync(&tc_err_h, tc_err, 4, cudaMemcpyDeviceToHost, st));
  KKM_CK(cudaMemcpyAsync(&it_err_h, lb.I.err, 4, cudaMemcpyDeviceToHost, st));
  KKM_CK(cudaStreamSynchronize(st));
  if (tc_err_h) {
    set_error("tensor-core kernel block: a bounded pipeline wait gave up (code " + std::to_string(tc_err_h) + ")");
    return KKM_ETIMEOUT;
  }
  if (it_err_h) {
    set_error("fused inner iteration: the bounded grid-barrier wait gave up");
    return KKM_ETIMEOUT;
  }
  prof_collect();
  return KKM_OK;
}

static kkm_status debug_kmeanspp_impl(const float* X0_in, int64_t N0, int64_t d, const kkm_kernel* k, int32_t C,
                                      uint64_t seed, int64_t* picks_out, cudaStream_t st) {
  KernelSpec sp;
  KKM_TRY(make_spec(k, d, &sp));
  if (N0 < 1 || N0 > INT32_MAX || C < 1 || C > N0 || C > kMaxC || !X0_in || !picks_out)
    return invalid("bad sizes or NULL pointer");
  if (sp.kind != KKM_LINEAR && !(sp.sigma > 0.0f && isfinite(sp.sigma))) return invalid("sigma must be > 0");
  SplitMix64 master(seed);
  SplitMix64 kpp(master.next());
  std::vector<double> draws(C);
  for (int r = 0; r < C; ++r) draws[r] = kpp.u01();
  const int32_t p0 = (int32_t)floor(draws[0] * (double)N0);
  int dev = 0;
  KKM_CK(cudaGetDevice(&dev));
  setup_pool_once(dev);
  Workspace ws(st);
  const float* X;
  KKM_TRY(device_input(ws, X0_in, N0 * d, &X));
  const int64_t ldk = round_up(N0, 32);
  float *Xi, *aux, *rowbuf, *rowaux, *kcol;
  double *D2, *draws_d;
  int32_t* picks;
  KKM_TRY(ws.alloc(&Xi, N0 * sp.dp));
  KKM_TRY(ws.alloc(&aux, N0));
  KKM_TRY(ws.alloc(&rowbuf, sp.dp));
  KKM_TRY(ws.alloc(&rowaux, 1));
  KKM_TRY(ws.alloc(&kcol, ldk));
  uint32_t* ticket;
  KKM_TRY(ws.alloc(&D2, 2 * N0 + ceil_div(N0, 32)));
  KKM_TRY(ws.alloc(&draws_d, C));
  KKM_TRY(ws.alloc(&picks, C));
  KKM_TRY(ws.alloc(&ticket, 1));
  KKM_CK(cudaMemsetAsync(ticket, 0, 4, st));
  KKM_CK(cudaMemcpyAsync(draws_d, draws.data(), (size_t)C * 8, cudaMemcpyHostToDevice, st));
  KKM_CK(cudaMemcpyAsync(picks, &p0, 4, cudaMemcpyHostToDevice, st));
  KKM_TRY(prep_rows(sp, X, 0, 1, N0, Xi, aux, st));
  KKM_TRY(kmeanspp_dev(sp, Xi, aux, (int)N0, C, sp.kind == KKM_LINEAR ? aux : nullptr, rowbuf, rowaux, kcol,
                       ldk, D2, picks, draws_d, ticket, st));
  std::vector<int32_t> ph(C);
  KKM_CK(cudaMemcpyAsync(ph.data(), picks, (size_t)C * 4, cudaMemcpyDeviceToHost, st));
  KKM_CK(cudaStreamSynchronize(st));
  for (int r = 0; r < C; ++r) picks_out[r] = ph[r];
  prof_collect();
  return KKM_OK;
}

template <typename F>
static kkm_status guarded(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return KKM_ENOMEM;
  } catch (...) {
    set_error("internal exception");
    return KKM_EINTERNAL;
  }
}

}  // namespace kkm

// ======================================================================
// extern "C"
// ======================================================================
using namespace kkm;

extern "C" {

void kkm_options_default(kkm_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = KKM_FP32;
  opt->sampling = KKM_STRIDE;
  opt->early_stop = 1;
}

kkm_status kkm_fit(const float* X, int64_t N, int64_t d, int32_t C, int32_t B, double s, const kkm_kernel* k,
                   int32_t iters, uint64_t seed, const kkm_options* opt, int32_t* labels_out,
                   kkm_model** model_out) {
  set_error("");
  if (model_out) *model_out = nullptr;
  kkm_status r = guarded([&] { return fit_impl(X, N, d, C, B, s, k, iters, seed, opt, labels_out, model_out); });
  if (r != KKM_OK && model_out && *model_out) {
    delete *model_out;
    *model_out = nullptr;
  }
  return r;
}

kkm_status kkm_fit_range(const float* X, int64_t N, int64_t d, int32_t C, int32_t B, double s, const kkm_kernel* k,
                         int32_t iters, uint64_t seed, const kkm_options* opt, const kkm_checkpoint* from,
                         int32_t stop, int32_t* labels_out, kkm_model** model_out, kkm_checkpoint** ckpt_out) {
  set_error("");
  if (model_out) *model_out = nullptr;
  if (ckpt_out) *ckpt_out = nullptr;
  if (stop < 1) return invalid("stop must be >= 1");
  if (from && from->next_batch >= from->B) return invalid("the checkpoint's fit is complete (next_batch == B)");
  kkm_status r = guarded(
      [&] { return fit_impl(X, N, d, C, B, s, k, iters, seed, opt, labels_out, model_out, from, stop, ckpt_out); });
  if (r != KKM_OK) {
    if (model_out && *model_out) {
      delete *model_out;
      *model_out = nullptr;
    }
    if (ckpt_out && *ckpt_out) {
      delete *ckpt_out;
      *ckpt_out = nullptr;
    }
  }
  return r;
}

kkm_status kkm_checkpoint_info(const kkm_checkpoint* c, int32_t* next_batch, int32_t* B, int32_t* C, float* sigma,
                               int64_t* medoids_out) {
  set_error("");
  if (!c) return invalid("checkpoint is NULL");
  if (next_batch) *next_batch = c->next_batch;
  if (B) *B = c->B;
  if (C) *C = c->C;
  if (sigma) *sigma = c->sigma;
  if (medoids_out) memcpy(medoids_out, c->M.data(), c->M.size() * 8);
  return KKM_OK;
}

void kkm_checkpoint_free(kkm_checkpoint* c) { delete c; }

kkm_status kkm_assign(const kkm_model* m, const float* Xnew, int64_t M, int32_t mode, int32_t* labels_out,
                      float* dist_out, void* stream) {
  set_error("");
  if (!labels_out) return invalid("labels_out is NULL");
  return guarded([&] { return assign_impl(m, Xnew, M, mode, labels_out, dist_out, nullptr, (cudaStream_t)stream); });
}

kkm_status kkm_cost(const kkm_model* m, const float* X, int64_t N, int32_t mode, double* omega_out, void* stream) {
  set_error("");
  if (!omega_out) return invalid("omega_out is NULL");
  return guarded([&] { return assign_impl(m, X, N, mode, nullptr, nullptr, omega_out, (cudaStream_t)stream); });
}

kkm_status kkm_model_info(const kkm_model* m, int32_t* C, int64_t* d, int32_t* n_support, float* sigma) {
  if (!m) return invalid("model is NULL");
  if (C) *C = m->C;
  if (d) *d = m->d;
  if (n_support) *n_support = m->nL;
  if (sigma) *sigma = m->sigma;
  return KKM_OK;
}

kkm_status kkm_model_medoids(const kkm_model* m, int64_t* idx_out, int64_t* counts_out, float* coords_out) {
  if (!m) return invalid("model is NULL");
  if (idx_out) memcpy(idx_out, m->medoids.data(), m->medoids.size() * 8);
  if (counts_out) memcpy(counts_out, m->W.data(), m->W.size() * 8);
  if (coords_out) {
    cudaError_t e = cudaMemcpy(coords_out, m->med_coords_h.data(), m->med_coords_h.size() * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy", __FILE__, __LINE__);
  }
  return KKM_OK;
}

kkm_status kkm_model_supports(const kkm_model* m, int32_t* labels_out, double* ghat_out, int32_t* n_out) {
  if (!m) return invalid("model is NULL");
  if (labels_out) memcpy(labels_out, m->sup_labels_h.data(), m->sup_labels_h.size() * 4);
  if (ghat_out) memcpy(ghat_out, m->ghat_h.data(), m->ghat_h.size() * 8);
  if (n_out) memcpy(n_out, m->n_h.data(), m->n_h.size() * 4);
  return KKM_OK;
}

kkm_status kkm_model_displacement(const kkm_model* m, double* out, int32_t cap, int32_t* n_out) {
  set_error("");
  if (!m || !n_out) return invalid("model and n_out must not be NULL");
  const int n = (int)m->displacement.size();
  *n_out = n;
  if (out)
    for (int q = 0; q < std::min(n, std::max(cap, 0)); ++q) out[q] = m->displacement[q];
  return KKM_OK;
}

kkm_status kkm_model_trace(const kkm_model* m, double* omega, int32_t* changed, int32_t cap, int32_t* n_out) {
  if (!m) return invalid("model is NULL");
  const int32_t n = (int32_t)m->omega.size();
  if (n_out) *n_out = n;
  const int32_t c = std::min(n, std::max(cap, 0));
  if (omega) memcpy(omega, m->omega.data(), (size_t)c * 8);
  if (changed) memcpy(changed, m->changed.data(), (size_t)c * 4);
  return KKM_OK;
}

void kkm_model_free(kkm_model* m) { delete m; }

kkm_status kkm_kernel_matrix(const float* A, int64_t nA, const float* Bm, int64_t nB, int64_t d, const kkm_kernel* k,
                             int32_t precision, float* out, void* stream) {
  set_error("");
  return guarded([&] { return kernel_matrix_impl(A, nA, Bm, nB, d, k, precision, out, (cudaStream_t)stream); });
}

kkm_status kkm_median_bandwidth(const float* X, int64_t N, int64_t d, const kkm_kernel* k, uint64_t seed,
                                float* sigma_out) {
  set_error("");
  return guarded([&]() -> kkm_status {
    KernelSpec sp;
    KKM_TRY(make_spec(k, d, &sp));
    if (N < 1 || N > INT32_MAX || !X || !sigma_out) return invalid("bad sizes or NULL pointer");
    SplitMix64 master(seed);
    master.next();
    const uint64_t bw_seed = master.next();
    int dev = 0;
    KKM_CK(cudaGetDevice(&dev));
    setup_pool_once(dev);
    Workspace ws(nullptr);
    const float* Xd;
    KKM_TRY(device_input(ws, X, N * d, &Xd));
    KKM_TRY(median_bandwidth_dev(sp, Xd, N, bw_seed, ws, sigma_out));
    prof_collect();
    return KKM_OK;
  });
}

kkm_status kkm_debug_step(const float* Xb, int64_t Ni, int64_t d, const int32_t* L, int32_t nL, const kkm_kernel* k,
                          int32_t C, int32_t precision, int32_t iteration, const int32_t* u_in, int32_t* u_out,
                          float* fhat_out, float* margin_out, double* ghat_out, int32_t* n_out, double* omega_out,
                          int32_t* changed_out, void* stream) {
  set_error("");
  return guarded([&] {
    return debug_step_impl(Xb, Ni, d, L, nL, k, C, precision, iteration, u_in, u_out, fhat_out, margin_out, ghat_out,
                           n_out, omega_out, changed_out, (cudaStream_t)stream);
  });
}

kkm_status kkm_debug_kmeanspp(const float* X0, int64_t N0, int64_t d, const kkm_kernel* k, int32_t C, uint64_t seed,
                              int64_t* picks_out, void* stream) {
  set_error("");
  return guarded([&] { return debug_kmeanspp_impl(X0, N0, d, k, C, seed, picks_out, (cudaStream_t)stream); });
}

kkm_status kkm_minibatch_plan(int64_t N, int32_t B, int32_t sampling, double s, uint64_t seed, int32_t batch,
                              int64_t* start_out, int64_t* step_out, int64_t* n_out, int32_t* L_out,
                              int64_t* nl_out) {
  set_error("");
  return guarded([&]() -> kkm_status {
    if (N < 1 || B < 1 || B > N || batch < 0 || batch >= B) return invalid("bad N, B or batch");
    if (sampling != KKM_STRIDE && sampling != KKM_BLOCK) return invalid("unknown sampling");
    if (!(s > 0.0 && s <= 1.0)) return invalid("s must be in (0, 1]");
    const std::vector<BatchGeom> geo = batch_geometry(N, B, sampling);
    const BatchGeom& g = geo[batch];
    if (start_out) *start_out = g.start;
    if (step_out) *step_out = g.step;
    if (n_out) *n_out = g.Ni;
    SplitMix64 master(seed);
    master.next();
    master.next();
    uint64_t lm_seed = 0;
    for (int i = 0; i <= batch; ++i) lm_seed = master.next();
    SplitMix64 lm(lm_seed);
    const int64_t nl = n_landmarks(g.Ni, s);
    if (nl_out) *nl_out = nl;
    if (L_out) {
      if (nl == g.Ni) {
        for (int64_t a = 0; a < nl; ++a) L_out[a] = (int32_t)a;
      } else {
        sorted_picks(g.Ni, nl, lm, L_out);
      }
    }
    return KKM_OK;
  });
}

const char* kkm_status_string(kkm_status s) {
  switch (s) {
    case KKM_OK: return "KKM_OK";
    case KKM_EINVAL: return "KKM_EINVAL";
    case KKM_ENOMEM: return "KKM_ENOMEM";
    case KKM_EBUDGET: return "KKM_EBUDGET";
    case KKM_ECUDA: return "KKM_ECUDA";
    case KKM_ETIMEOUT: return "KKM_ETIMEOUT";
    case KKM_EINTERNAL: return "KKM_EINTERNAL";
  }
  return "KKM_UNKNOWN";
}

const char* kkm_last_error(void) { return g_last_error.c_str(); }

void kkm_prof_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = (on == 1 || on == 2) ? on : 0;
}
void kkm_prof_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.clear();
}
int32_t kkm_prof_read(const char* name, int64_t* launches, double* ms) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  auto it = g_prof.find(name ? name : "");
  if (it == g_prof.end()) {
    if (launches) *launches = 0;
    if (ms) *ms = 0.0;
    return 0;
  }
  if (launches) *launches = it->second.launches;
  if (ms) *ms = it->second.ms;
  return 1;
}
double kkm_prof_work(const char* name) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  auto it = g_prof.find(name ? name : "");
  return it == g_prof.end() ? 0.0 : it->second.work;
}
int32_t kkm_prof_names(char* buf, int32_t cap) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::string all;
  for (auto& kv : g_prof) {
    if (!all.empty()) all += ",";
    all += kv.first;
  }
  if (buf && cap > 0) {
    const size_t n = std::min<size_t>(all.size(), (size_t)cap - 1);
    memcpy(buf, all.data(), n);
    buf[n] = 0;
  }
  return (int32_t)all.size();
}

}  // extern "C"
