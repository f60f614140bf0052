// kkm_assign_noalloc: labelling new samples against a fitted model without
// any device allocation.
//
// Who needs it: a caller on a request path that must not call cudaMalloc --
// cudaMalloc can synchronise the whole device and stall every other stream --
// or a caller whose device memory is owned by another framework's pool, where
// a private allocation may fail even though memory is free in that pool.
// kkm_assign allocates its working buffers per call; this entry point uses one
// fixed scratch area instead.
//
// The scratch is the file-scope array below.  Every GPU that loads this
// library holds it (about 21 MB) until the process exits.  All calls share it
// and it keeps the contents of the last call, so two calls whose work overlaps
// on the GPU (different streams, or threads calling concurrently) race on it;
// calls on one stream, one after the other, are safe.  What must start at zero
// (the non-finite-input flag) is cleared by every call.
//
// In host code the array's name is only a host-side stand-in, not a device
// address, so the first call on each device, with that device current, asks
// the runtime for the array's device address (cudaGetSymbolAddress) and keeps
// it.  That first call may load this module onto the device; make it before
// any stream capture.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "internal.h"

namespace kkm {

constexpr int64_t kNaRows = KKM_NOALLOC_MAX_ROWS;      // query rows per call
constexpr int64_t kNaRef = KKM_NOALLOC_MAX_REF;        // reference rows (supports or medoids)
constexpr int64_t kNaRowLen = KKM_NOALLOC_MAX_ROWLEN;  // prepared row length
constexpr int64_t kNaUnits = (kNaRef + kUnitRows - 1) / kUnitRows + kMaxC;
constexpr int64_t kNaGrid = kNaRows / 32;              // assign CTAs (32 rows each)

constexpr size_t na_align(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffRows = 0;                                               // float [rows][rowlen]
constexpr size_t kOffAux = na_align(kOffRows + sizeof(float) * kNaRows * kNaRowLen);  // float [rows]
constexpr size_t kOffK = na_align(kOffAux + sizeof(float) * kNaRows);         // float [ref][rows]
constexpr size_t kOffPart = na_align(kOffK + sizeof(float) * kNaRef * kNaRows);  // float [units][rows]
constexpr size_t kOffOmega = na_align(kOffPart + sizeof(float) * kNaUnits * kNaRows);  // float2 [grid]
constexpr size_t kOffChanged = na_align(kOffOmega + sizeof(float2) * kNaGrid);   // int [grid]
constexpr size_t kOffFlag = na_align(kOffChanged + sizeof(int32_t) * kNaGrid);   // int [1]
constexpr size_t kNaBytes = na_align(kOffFlag + sizeof(int32_t));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

static std::mutex g_na_mu;
static unsigned char* g_na_dev[256] = {nullptr};

// Device address of the scratch array on the current device (resolved on the
// first call per device).
static kkm_status scratch_address(unsigned char** out) {
  int dev = 0;
  KKM_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) {
    set_error("device ordinal out of range");
    return KKM_EINTERNAL;
  }
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_dev[dev]) {
    void* p = nullptr;
    KKM_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_na_dev[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_na_dev[dev];
  return KKM_OK;
}

// True when p is device (or managed) memory of device `dev`.
static bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

static kkm_status na_invalid(const char* msg) {
  set_error(msg);
  return KKM_EINVAL;
}

static kkm_status assign_noalloc_impl(const kkm_model* m, const float* X, int64_t M, int32_t mode,
                                      int32_t* labels_out, float* dist_out, cudaStream_t st) {
  if (!m) return na_invalid("model is NULL");
  if (mode != KKM_ASSIGN_SUPPORTS && mode != KKM_ASSIGN_MEDOIDS) return na_invalid("unknown assign mode");
  if (M < 0 || M > kNaRows) return na_invalid("M exceeds KKM_NOALLOC_MAX_ROWS (split the query into chunks)");
  if (M == 0) return KKM_OK;
  if (!X || !labels_out) return na_invalid("X or labels_out is NULL");
  // the model's arrays live on m->device: the scratch address is taken on
  // the current device, so both must be that device, and so must the buffers
  int cur = -1;
  KKM_CK(cudaGetDevice(&cur));
  if (cur != m->device) return na_invalid("the current device is not the model's device");
  if (!on_device(X, cur) || !on_device(labels_out, cur) || (dist_out && !on_device(dist_out, cur)))
    return na_invalid("kkm_assign_noalloc needs X, labels_out and dist_out in the model device's memory");
  const int rows_ref = mode == KKM_ASSIGN_SUPPORTS ? m->nL : m->C;
  if (rows_ref > kNaRef) return na_invalid("model has more reference rows than KKM_NOALLOC_MAX_REF");
  if (m->dp > kNaRowLen) return na_invalid("model rows are longer than KKM_NOALLOC_MAX_ROWLEN");
  if (m->C > kMaxC) return na_invalid("too many clusters");

  unsigned char* base = nullptr;
  KKM_TRY(scratch_address(&base));
  float* Xc = reinterpret_cast<float*>(base + kOffRows);
  float* auxc = reinterpret_cast<float*>(base + kOffAux);
  float* Kb = reinterpret_cast<float*>(base + kOffK);
  float* partial = reinterpret_cast<float*>(base + kOffPart);
  float2* omega_part = reinterpret_cast<float2*>(base + kOffOmega);
  int32_t* changed_part = reinterpret_cast<int32_t*>(base + kOffChanged);
  int* flag = reinterpret_cast<int*>(base + kOffFlag);

  // non-finite inputs are rejected (the flag must start at zero every call)
  KKM_CK(cudaMemsetAsync(flag, 0, sizeof(int), st));
  KKM_CK(launch_check_finite(X, M * m->d, flag, st));
  int bad = 0;
  KKM_CK(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  KKM_CK(cudaStreamSynchronize(st));
  if (bad) return na_invalid("X holds NaN or Inf");

  const int64_t ldm = round_up(M, 32);
  const bool rmsd = m->kind == KKM_RMSD;
  const int ap = rmsd ? m->dp / 3 : 0;
  const float neg_scale = (float)(-1.4426950408889634 / (2.0 * (double)m->sigma * (double)m->sigma));
  const int dk = rmsd ? DK_RBF : (m->kind == KKM_LINEAR ? DK_LINEAR : DK_RBF);
  if (rmsd)
    KKM_CK(launch_rmsd_prep_rows(X, m->n_atoms, 0, 1, M, Xc, ap, auxc, st));
  else
    KKM_CK(launch_gather_rows(X, m->d, 0, 1, M, Xc, m->dp, auxc, st));
  const float* kself = m->kind == KKM_LINEAR ? auxc : nullptr;
  const float* P = mode == KKM_ASSIGN_SUPPORTS ? m->sup : m->med;
  const float* Paux = mode == KKM_ASSIGN_SUPPORTS ? m->sup_aux : m->med_aux;
  if (rmsd)
    KKM_CK(launch_rmsd_gram(dk, P, rows_ref, Xc, M, ap, m->n_atoms, Paux, auxc, nullptr, nullptr, neg_scale, Kb,
                            ldm, st));
  else
    KKM_CK(launch_gram(dk, P, rows_ref, Xc, M, m->dp, Paux, auxc, nullptr, nullptr, neg_scale, Kb, ldm, st));

  if (mode == KKM_ASSIGN_SUPPORTS) {
    Supports S{};
    S.L = m->L_ident;
    S.nL = m->nL;
    S.C = m->C;
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
    S.max_units = max_units_for(m->nL, m->C);
    IterState I{};
    I.partial = partial;
    I.gpart = nullptr;
    I.omega_part = omega_part;
    I.changed_part = changed_part;
    I.ghat_in = m->ghat;
    I.n_strips = (int)ceil_div(ldm, kStripCols);
    I.assign_grid = (int)ceil_div(ldm, 32);
    KKM_CK(launch_fhat_partial(Kb, ldm, (int)M, S, I, st));
    KKM_CK(launch_assign(ldm, (int)M, S, I, kself, labels_out, nullptr, dist_out, nullptr, nullptr, 0,
                         /*trace=*/0, st));
  } else {
    KKM_CK(launch_nearest(Kb, ldm, (int)M, m->C, kself, m->kind == KKM_LINEAR ? m->med_aux : nullptr, labels_out,
                          dist_out, st));
  }
  KKM_CK(cudaStreamSynchronize(st));
  return KKM_OK;
}

}  // namespace kkm

extern "C" kkm_status kkm_assign_noalloc(const kkm_model* m, const float* Xnew, int64_t M, int32_t mode,
                                         int32_t* labels_out, float* dist_out, void* stream) {
  kkm::set_error("");
  try {
    return kkm::assign_noalloc_impl(m, Xnew, M, mode, labels_out, dist_out, (cudaStream_t)stream);
  } catch (...) {
    kkm::set_error("internal exception");
    return KKM_EINTERNAL;
  }
}
