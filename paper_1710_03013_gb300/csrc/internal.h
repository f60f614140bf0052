// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/kkm.h"

// The state of Algorithm 1's outer loop between two mini-batches (kkm_fit_range):
// the arguments it was started with (a resume must repeat them), the next
// mini-batch, the bandwidth in use, the global medoids and their counts, and
// the trace so far.
struct kkm_checkpoint {
  int64_t N = 0, d = 0;
  int32_t C = 0, B = 0;
  double s = 0.0;
  int32_t kind = 0, n_atoms = 0, iters = 0;
  float sigma_arg = 0.0f;       // the sigma the fit was called with (<= 0: median rule)
  uint64_t seed = 0;
  int32_t precision = 0, sampling = 0, early_stop = 0, had_init = 0;
  int32_t next_batch = 0;
  float sigma = 0.0f;           // the bandwidth in use
  std::vector<int64_t> M, W;    // [C] global medoids, cumulative counts
  std::vector<double> omega;
  std::vector<int32_t> changed;
  std::vector<double> displacement;  // [next_batch]
};

// The model behind the opaque kkm_model handle: device copies of what
// kkm_assign / kkm_cost need, plus host copies of the reported results.
struct kkm_model {
  int C = 0;
  int64_t d = 0;
  int kind = 0;
  float sigma = 1.0f;
  int n_atoms = 0;
  int dp = 0;  // prepared row length (padded)
  int nL = 0;
  int max_units = 0;  // capacity of the unit tables
  int device = 0;
  float* sup = nullptr;        // [nL][dp] prepared landmark rows
  float* sup_aux = nullptr;    // [nL] squared norms (RBF/linear) or G (RMSD)
  int64_t* sup_ids = nullptr;  // [nL] global sample ids of the landmarks
  int32_t* sup_labels = nullptr;
  int32_t* L_ident = nullptr;  // [nL] 0..nL-1
  int32_t* perm = nullptr;
  int32_t* seg_off = nullptr;
  int32_t* n_j = nullptr;
  int32_t* unit_j = nullptr;
  int32_t* unit_kb = nullptr;
  int32_t* unit_ke = nullptr;
  int32_t* seg_unit = nullptr;
  int32_t* n_units = nullptr;
  double* ghat = nullptr;      // [C]
  float* med = nullptr;        // [C][dp]
  float* med_aux = nullptr;    // [C]
  std::vector<int64_t> medoids, W;
  std::vector<double> omega;
  std::vector<int32_t> changed;
  std::vector<double> displacement;  // [B] average centre displacement per mini-batch (Fig. 4b)
  std::vector<int32_t> sup_labels_h;
  std::vector<double> ghat_h;
  std::vector<int32_t> n_h;
  std::vector<float> med_coords_h;  // [C][d]
  void* arena = nullptr;            // one device allocation holding every array above
  ~kkm_model() {
    // like cudaFree: every launch that may still read the model finishes
    // first; the memory then goes back to the stream-ordered pool
    if (arena) {
      cudaDeviceSynchronize();
      cudaFreeAsync(arena, nullptr);
      cudaGetLastError();
    }
  }
};

namespace kkm {

// One device allocation (m->arena) for the model's resident arrays, sized from
// C, dp, nL and max_units, ordered on stream st (m->device must be set); the
// array pointers point into it.
kkm_status model_alloc_device(kkm_model* m, cudaStream_t st = nullptr);

// ------------------------------------------------------- random numbers ---
// SplitMix64 (Steele, Lea & Flood 2014) from its published definition; u01
// takes the top 53 bits.  The host draws every random number of the method.
struct SplitMix64 {
  uint64_t state;
  explicit SplitMix64(uint64_t s) : state(s) {}
  uint64_t next() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double u01() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

// ---------------------------------------------------------------- errors ---
void set_error(const std::string& msg);
kkm_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define KKM_CK(expr)                                                        \
  do {                                                                      \
    cudaError_t _e = (expr);                                                \
    if (_e != cudaSuccess) return ::kkm::cuda_fail(_e, #expr, __FILE__, __LINE__); \
  } while (0)

#define KKM_TRY(expr)                      \
  do {                                     \
    kkm_status _s = (expr);                \
    if (_s != KKM_OK) return _s;           \
  } while (0)

// ------------------------------------------------------------- profiling ---
// Brackets one kernel launch with events when profiling is on.
struct ProfScope {
  ProfScope(const char* name, cudaStream_t s);
  ~ProfScope();
  const char* name;
  cudaEvent_t a = nullptr, b = nullptr;  // null: not timed
  cudaStream_t stream;
  const char* prev_scope = nullptr;
};
void prof_collect();  // after a stream sync: fold finished events into totals

// NVTX range for the phases of a call (visible to a profiler attached to the
// process; header-only, no cost when none is).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
bool prof_on();
void prof_add_work(const char* name, double units);  // data-dependent work of a kernel
// A launcher that starts k kernels beyond its first reports them here; they
// are counted under the enclosing profiled launch (launch counts are kernels).
void prof_more_launches(int k);

// Launch check after every kernel launch.
#define KKM_LAUNCH_CK() KKM_CK(cudaGetLastError())

// --------------------------------------------------------------- layouts ---
constexpr int kUnitRows = 64;     // landmark rows per f_hat streaming unit
constexpr int kStripCols = 512;   // narrowest f_hat strip (FP32: 128 threads x 4 columns); sizes gpart
constexpr int kMaxC = 256;     // clusters per problem (one scan slot per thread of a 256-thread CTA)

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Whether kkm_fit computes the next mini-batch's kernel block while the
// current one iterates (two block buffers; the server sizes fits by it).
// KKM_PIPE_AUTO overlaps for B >= 2 unless the block is the reduced-precision
// RBF/linear block on the tensor cores: that block is a few percent of a fit,
// and its writes would push the inner loop's cached block out of L2.
inline bool fit_overlaps(int pipeline, int B, int kind, int precision) {
  if (B < 2 || pipeline == KKM_PIPE_SERIAL) return false;
  if (pipeline == KKM_PIPE_OVERLAP) return true;
  return kind == KKM_RMSD || precision == KKM_FP32;
}
// Fits that run side by side (kkm_fit_batch, the server's workers) overlap
// one another; inside each, AUTO means serial blocks (a low-priority block
// stream would wait behind the other fits' high-priority inner loops).
inline int side_by_side_pipeline(int pipeline) { return pipeline == KKM_PIPE_AUTO ? KKM_PIPE_SERIAL : pipeline; }
// The one-launch loop forms hold their CTAs at grid barriers, which needs the
// whole grid resident at once; beside other fits' one-launch loops that is
// not assured (each could hold part of the SMs while waiting for the rest), so
// fits that run side by side take the split form.
inline int side_by_side_iteration(int iteration) { (void)iteration; return KKM_ITER_SPLIT; }

// The reduced-precision path computes the block of short rows (d below this)
// in FP32 on the FFMA pipes and stores it in FP16, keeping the FP32 values for
// the near-tie re-score: at these lengths the block is a small share of a fit,
// while the BF16 rounding of the rows would widen the near-tie window (and the
// re-scores) of every inner iteration.
constexpr int64_t kBf16TensorMinDim = 129;

// Kernel-function codes used on the device.
enum DevKind { DK_RBF = 0, DK_LINEAR = 1, DK_DIST = 2, DK_RMSD_EST = 3, DK_RAW = 4 /* plain products */ };

// --------------------------------------------------------- kernel launchers
// (all asynchronous on `st`; they return a CUDA error code of the launch)

// Rows of X chosen as start + l*step (l < n) copied to out [n][dp], zero-padded,
// with FP64-accumulated squared norms (normsq nullable).
cudaError_t launch_gather_rows(const float* X, int64_t d, int64_t start, int64_t step,
                               int64_t n, float* out, int dp, float* normsq, cudaStream_t st);
// The same rows from pinned host memory (X its device address; d and dp
// multiples of 4, both 16-byte aligned), fetched by the copy engine, *bad set
// when a value is NaN or Inf.
cudaError_t launch_gather_rows_pull(const float* X, int64_t d, int64_t start, int64_t step, int64_t n, float* out,
                                    int dp, float* normsq, int* bad, cudaStream_t st);
// Rows X[idx[l]] (device indices, int64 or int32) copied like above.
cudaError_t launch_gather_idx64(const float* X, int64_t d, const int64_t* idx, int64_t n,
                                float* out, int dp, float* normsq, cudaStream_t st);
cudaError_t launch_gather_idx32(const float* Xp, int dp_in, const int32_t* idx, int64_t n,
                                float* out, int dp, float* normsq, cudaStream_t st);
// Sets *flag = 1 if any of the n floats is NaN or Inf.
cudaError_t launch_check_finite(const float* X, int64_t n, int* flag, cudaStream_t st);
// Copies n floats from host memory the GPU can read (pinned; src and dst
// 16-byte aligned, else cudaErrorInvalidValue) and sets *flag = 1 if any is
// NaN or Inf, in one pass.
cudaError_t launch_copy_check(const float* src, float* dst, int64_t n, int* flag, cudaStream_t st);

// out[a*ldo + b] = kappa(A_a, B_b) for a < nA, b < nB (A [nA][dp], B [nB][dp]).
// kind: DK_RBF (neg_scale = -log2(e)/(2 sigma^2)), DK_LINEAR, DK_DIST (sqrt of
// squared distance).  idA/idB (nullable) are sample ids: equal ids give K = 1
// exactly for RBF and 0 for DIST.
// Euclidean distances of the rows of A among themselves, only the entries
// above the diagonal (out[a*ldo + b], b > a, written; the tiles wholly at or
// below it are skipped).  Rows of at least kDistSplitMinDp floats split K
// kDistSplit ways (scratch: kDistSplit * n * ldo floats of partial products;
// NULL for shorter rows).
constexpr int kDistSplit = 4;
constexpr int kDistSplitMinDp = 256;
cudaError_t launch_gram_dist_upper(const float* A, int64_t n, int dp, const float* normA, const int64_t* idA,
                                   float* out, int64_t ldo, float* scratch, cudaStream_t st);
cudaError_t launch_gram(int kind, const float* A, int64_t nA, const float* Bm, int64_t nB,
                        int dp, const float* normA, const float* normB, const int64_t* idA,
                        const int64_t* idB, float neg_scale, float* out, int64_t ldo,
                        cudaStream_t st);

// The FP32 RBF block (tiled FFMA kernel, ids force the exact diagonal) stored
// in FP16: the reduced-precision path's block for short rows; out32
// (nullable, same leading dimension) gets the FP32 values too.
cudaError_t launch_gram_rbf_half(const float* A, int64_t nA, const float* Bm, int64_t nB, int dp, const float* normA,
                                 const float* normB, const int64_t* idA, const int64_t* idB, float neg_scale,
                                 __half* out, int64_t ldo, cudaStream_t st, float* out32 = nullptr);

// ---- tensor-core (tcgen05) BF16 kernel block ----------------------------
// out[n*ldo + m] = kappa(P_n, Q_m) for BF16 rows P [nP][ldb], Q [nQ][ldb]
// (dk valid columns), with the squared norms of the BF16 rows; out is float,
// or __half when out_half (Gaussian kernel only: values in [0, 1]).  *err gets
// a nonzero code if a bounded wait gave up.
cudaError_t launch_gram_tc(int kind, const __nv_bfloat16* P, int64_t nP, const __nv_bfloat16* Q, int64_t nQ,
                           int dk, int ldb, const float* normP, const float* normQ, float neg_scale, void* out,
                           bool out_half, int64_t ldo, int* err, int n_sms, cudaStream_t st);
// MD kernel screen on the tensor cores: P [4 nP][kp] and Q [4 nQ][kp] hold
// split-BF16 centred frames (planes x, y, z and a zero plane; kp = 3 segments
// of the padded atom count, see launch_rmsd_to_bf16), gP / gQ their squared
// radii.  out[l*ldo + s] = 0 where the correlation certifies exp(-rmsd^2 /
// (2 sigma^2)) < kRmsdRefine, else 1 with the optimal rotation as a unit
// quaternion in quat[l*ldo + s]; the pairs marked 1 are recomputed exactly
// (launch_rmsd_refine_plan, then launch_rmsd_gram with tile flags and quat).
// The split operands give the correlation to ~1e-5 relative, so the
// rotation's error enters the exact residual at ~1e-10; the certificate's
// margin holds for sigma >= 0.5 A and coordinates within ~100 A of the centroid.
constexpr float kRmsdRefine = 1e-6f;
cudaError_t launch_rmsd_tc_estimate(const __nv_bfloat16* P, int64_t nP, const __nv_bfloat16* Q, int64_t nQ, int kp,
                                    const float* gP, const float* gQ, int n_atoms, float neg_scale, float* out,
                                    float4* quat, int64_t ldo, int* err, int n_sms, cudaStream_t st);
// out[k*ldo + L[k]] = 1 (the exact diagonal of a Gaussian kernel block).
cudaError_t launch_set_diag(void* out, bool out_half, int64_t ldo, const int32_t* L, int nL, cudaStream_t st);
// FP8 e4m3 operands with a scale per row (rows [ld8] bytes, ld8 a multiple of
// 16): out[n*ldo + m] = kappa(P_n, Q_m) of the decoded rows s * e4m3, from
// their squared norms and scales.  RBF (FP32 or FP16 out) and linear.
cudaError_t launch_gram_tc_fp8(int kind, const uint8_t* P, int64_t nP, const uint8_t* Q, int64_t nQ, int dk, int ld8,
                               const float* normP, const float* normQ, const float* scaleP, const float* scaleQ,
                               float neg_scale, void* out, bool out_half, int64_t ldo, int* err, int n_sms,
                               cudaStream_t st);
// e4m3 rows [n][ld8] of FP32 rows [n][dp] with a scale per row (max |x| /
// 448) and the squared norms of the decoded rows.
cudaError_t launch_to_fp8(const float* src, int64_t n, int dp, int ld8, uint8_t* dst, float* scale, float* normsq,
                          cudaStream_t st);
// BF16 copy of FP32 rows [n][dp] with the squared norms of the rounded rows.
cudaError_t launch_to_bf16(const float* src, int64_t n, int dp, __nv_bfloat16* dst, float* normsq,
                           cudaStream_t st);

// ---- MD kernel (RMSD) -----------------------------------------------------
// Frames [n][n_atoms][3] (rows start + l*step of X) -> centred SoA [n][3][ap]
// (ap = padded atom count) with G = sum |x_a|^2 in gsq.
cudaError_t launch_rmsd_prep_rows(const float* X, int n_atoms, int64_t start, int64_t step,
                                  int64_t n, float* out, int ap, float* gsq, cudaStream_t st);
cudaError_t launch_rmsd_prep_idx64(const float* X, int n_atoms, const int64_t* idx, int64_t n,
                                   float* out, int ap, float* gsq, cudaStream_t st);
// kind DK_RBF: out = exp(-rmsd^2/(2 sigma^2)) via neg_scale; DK_DIST: rmsd.
// tile_flag (nullable): only the tiles of 32 A-frames x 64 B-frames whose
// flag is set are computed ([ceil(nA/32)][ceil(nB/64)], A-tile major); arow
// (nullable): A tile rows are the frames arow[0..nA) in that order; quat
// (nullable, with tile_flag): rotations of the screen for the pairs it
// marked 1 in out, so only the residual pass runs (pairs marked 0 keep 0).
cudaError_t launch_rmsd_gram(int kind, const float* A, int64_t nA, const float* Bm, int64_t nB,
                             int ap, int n_atoms, const float* gA, const float* gB,
                             const int64_t* idA, const int64_t* idB, float neg_scale,
                             float* out, int64_t ldo, cudaStream_t st, const int* tile_flag = nullptr,
                             const int* arow = nullptr, const float4* quat = nullptr);
// From the estimate block est [nA][ldo]: the reference order that groups
// references near the same samples (key [nA], order [nA]) and the refine flag
// of every (reference tile of that order, sample tile) ([ceil(nA/32)][ceil(nB/64)]).
cudaError_t launch_rmsd_refine_plan(const float* est, int64_t ldo, int nA, int nB, int* key, int* order, int* flag,
                                    cudaStream_t st);
// Centred SoA frames [n][3][ap] (FP32) -> split BF16 rows [n][4][3 kp]
// (fourth plane and atoms past n_atoms zero): segments (hi, lo, hi) for
// side 0 (references), (hi, hi, lo) for side 1 (samples).
cudaError_t launch_rmsd_to_bf16(const float* src, int64_t n, int ap, int n_atoms, __nv_bfloat16* dst, int kp,
                                int side, cudaStream_t st);

// ---- inner iteration ---------------------------------------------------------
struct Supports {
  // landmark structure of one mini-batch, all device memory
  const int32_t* L;      // [nL] local positions of landmarks (sorted)
  int nL;
  int C;
  int32_t* perm;         // [nL] landmark ordinals k sorted by label (stable)
  int32_t* seg_off;      // [C+1]
  int32_t* n_j;          // [C]
  int32_t* unit_j;       // [max_units]
  int32_t* unit_kb;      // [max_units]
  int32_t* unit_ke;      // [max_units]
  int32_t* seg_unit;     // [C+1] first unit of each segment
  int32_t* n_units;      // [1]
  int32_t* col_label;    // [ldk] label of the landmark in column i, else -1;
                         // NULL: no g_hat numerators are needed
  int32_t* col_ord;      // [ldk] landmark ordinal of column i, else -1 (NULL: none)
  int32_t* lab;          // [nL] landmark labels, written by assign
  int max_units;
};
inline int max_units_for(int nL, int C) { return (int)(ceil_div(nL, kUnitRows) + C); }
// Fixed-point scale of the Gaussian g_hat numerators for up to nL landmarks:
// a numerator is at most n_j^2 <= nL^2, kept below 2^61 after scaling.
inline int gfix_shift_for(int64_t nL) {
  int b = 0;
  while (b < 40 && ((int64_t)1 << b) <= nL) ++b;  // nL < 2^b
  return std::max(8, std::min(40, 61 - 2 * b));
}

struct IterState {
  float* partial;        // [max_units][ldk]
  float2* gpart;         // [max_units][n_strips] g_hat numerators, double-float (hi, lo)
  float2* omega_part;    // [assign grid] cost per CTA, double-float (hi, lo)
  int32_t* changed_part; // [assign grid]
  uint32_t* ticket;      // [1], zero between launches
  int32_t* done;         // [1] early-stop flag (device)
  double* trace_omega;   // [trace cap]
  int32_t* trace_changed;// [trace cap]
  int32_t* trace_count;  // [1]
  const double* ghat_in = nullptr;  // g_hat given (assign against a model), else from gpart
  int32_t* lm_part = nullptr;       // [assign grid] landmark label changes per CTA
  // near-tie re-score (low-precision kernel blocks): rows whose margin is
  // below flag_tau * max(|d2|, K_ii + g_hat) are re-scored in FP32 by assign
  float flag_tau = 0.0f;
  double* ghat_cur = nullptr;       // [C] g_hat of the current supports (written by fhat_partial)
  uint32_t* gtick = nullptr;        // [C] per-cluster tile tickets of fhat_partial, zero between launches
  // Gaussian kernels (values in [0, 1]): the g_hat numerators as fixed-point
  // integers (value * 2^gfix_shift), one integer atomic per stream CTA, so
  // the sum is exact and order-free; the assign divides by n_j^2 and its
  // last CTA zeroes them for the next stream.  NULL: tickets and ghat_cur.
  unsigned long long* gfix = nullptr;  // [C]
  int gfix_shift = 0;
  int keep_rows = 0;                // block rows kept in L2 across iterations (evict_last)
  int assign_grid;
  int n_strips;
  // fused iteration (launch_iterate): per-CTA g_hat shares, the grid barrier
  // counter (zero between launches) and the error word of its bounded wait
  float2* gcta = nullptr;           // [fused_cap][C] double-float (linear kernel)
  unsigned long long* facc = nullptr;  // [2][C + 3] fixed-point shares (Gaussian kernels)
  int fom_shift = 0;                // fixed-point scale of the cost shares (set per launch)
  uint32_t* bar = nullptr;          // [1]
  int32_t* err = nullptr;           // [1]
  int fused_cap = 0;                // CTAs the fused buffers hold (omega_part etc. hold at least as many)
  // tensor-core iteration (launch_iterate_tc): landmark label changes of the
  // two alternating iterations, (ordinal << 8) | (old << 4) | new
  int32_t* lm_list = nullptr;       // [2][nL]
};
// Rows of a [rows][ldk] float block that fit in the given share of L2.
int l2_keep_rows(int64_t ldk, int rows, double share, int elem_bytes = 4);

// Builds perm/seg/units/col_label from the landmark labels S.lab (one CTA).
cudaError_t launch_build_supports(const Supports& S, cudaStream_t st);
// col_ord[L[k]] = k (col_ord pre-filled with -1) and lab[k] = u[L[k]].
cudaError_t launch_landmark_maps(const Supports& S, const int32_t* u, cudaStream_t st);
// Streams K^T [nL][ldk] once: per unit partial sums of the f_hat numerators.
cudaError_t launch_fhat_partial(const float* KT, int64_t ldk, int Ni, const Supports& S,
                                const IterState& I, cudaStream_t st);
// The same over a kernel block stored in FP16 (the BF16 path's Gaussian block).
cudaError_t launch_fhat_partial(const __half* KT, int64_t ldk, int Ni, const Supports& S,
                                const IterState& I, cudaStream_t st);
// FP32 rows for the near-tie re-score of a low-precision kernel block
// (Xi == NULL: no re-score).
struct RescoreArgs {
  int kind = DK_RBF;           // DK_RBF or DK_LINEAR
  int dp = 0;
  const float* Xi = nullptr;   // [Ni][dp] sample rows
  const float* nXi = nullptr;  // squared norms
  const float* XL = nullptr;   // [nL][dp] landmark rows (by ordinal)
  const float* nXL = nullptr;
  float neg_scale = 0.0f;
  // the FP32 values of the block when it was computed in FP32 and stored in
  // FP16 ([nL][ldk32], K32[k][i] = K(landmark k, sample i)): the re-score
  // reads them instead of recomputing them from the rows
  const float* K32 = nullptr;
  int64_t ldk32 = 0;
};

// f_hat, distances, argmin, margin, Omega; updates u in place.  With
// trace == 1 the last CTA also writes the trace entry, the early-stop flag and
// the count of changed landmark labels, and re-sorts the supports (as
// build_supports) when a landmark label changed.  Uses ceil(Ni/32) CTAs
// (omega_part/changed_part/lm_part need that many slots).
cudaError_t launch_assign(int64_t ldk, int Ni, const Supports& S, const IterState& I,
                          const float* kself, int32_t* u, float* margin, float* dmin,
                          float* fhat_out, double* ghat_out, int early_stop, int trace,
                          cudaStream_t st, const RescoreArgs& R = RescoreArgs());

// ---------------------------------------------- inner loops as work lists
// One mini-batch's inner loop (split form) as an item of a work-list launch:
// what fhat_partial and assign take for it.  A launch over a RoundList runs
// one iteration's f_hat stream (or assign) of every listed item, each item's
// CTAs doing exactly what its own launch would, so results are unchanged.
struct alignas(16) LoopItem {
  const void* KT = nullptr;  // [nL][ldk] kernel block (__half when half, else float)
  int64_t ldk = 0;
  int Ni = 0;
  int half = 0;
  int n_strips = 0;  // column strips of the f_hat stream
  int units = 0;     // unit rows of the f_hat stream (S.max_units)
  int nw = 0;        // warps of an assign CTA
  int early_stop = 0;
  int assign_ctas = 0;
  int assign_smem = 0;  // dynamic shared memory of an assign CTA
  double gfix_scale = 0.0;
  const float* kself = nullptr;
  int32_t* u = nullptr;
  Supports S{};
  IterState I{};
  RescoreArgs R{};
};
constexpr int kRoundMaxItems = 64;
// The items of one launch: device slots and their first CTAs (cta_off[n] is
// the grid size).
struct RoundList {
  int n = 0;
  int slot[kRoundMaxItems];
  int cta_off[kRoundMaxItems + 1];
};
// Fills the item of one mini-batch's loop (arguments as launch_fhat_partial
// and launch_assign take them in a fit).
cudaError_t make_loop_item(const void* KT, bool half, int64_t ldk, int Ni, const Supports& S, const IterState& I,
                           const float* kself, int32_t* u, int early_stop, const RescoreArgs& R, LoopItem* out);
// One f_hat stream of every item in L (items: device array of slots; all
// items of one launch have the same block type).
cudaError_t launch_fhat_multi(const LoopItem* items, const RoundList& L, bool half, cudaStream_t st);
// One assign (trace on) of every item in L; the items share nw and the
// dynamic shared memory is the largest they need.  Each CTA takes RG blocks
// of 32 rows of its item (cta_off counts ceil(row blocks / RG) per item); RG
// changes no result.
cudaError_t launch_assign_multi(const LoopItem* items, const RoundList& L, int nw, int smem, int RG,
                                cudaStream_t st);
// The support sort of every listed item whose landmark labels changed in the
// assign launches before it (their last CTAs leave it to this launch).
cudaError_t launch_sort_multi(const LoopItem* items, const RoundList& L, cudaStream_t st);
// The work-list runner of a batch's inner loops (batch.cu).  A fit whose
// thread has one (set by kkm_fit_batch's workers) hands every split-form
// inner loop to it: run() returns once the loop's last iteration is queued,
// with the fit's stream ordered after it.
struct LoopExecutor;
LoopExecutor* current_loop_executor();
// Rows per assign CTA (1, 2, 4 or 8 blocks of 32; no effect on results),
// chosen by timing per key (batch.cu): the choice for a launch (*timed: time
// it and report with assign_rows_sample), keys, the cache file.
long long assign_rows_key(int nw, int blocks, bool solo);
int assign_rows_choose(long long key, bool* timed);
void assign_rows_sample(long long key, int rows, int blocks, float ms);
void assign_rows_load();
void assign_rows_save();
kkm_status loop_executor_run(LoopExecutor* ex, const LoopItem& item, int iters, cudaStream_t st);

// The whole inner loop of a mini-batch (up to `iters` iterations: f_hat,
// g_hat, d, argmin, margin, re-score, Omega, trace, early stop, support
// re-sort) in one cooperative launch of at most one CTA per SM, each owning a
// strip of columns over every landmark row.  Applies when fused_shape() says
// so (C <= kFusedMaxC, a strip of at most one column per thread); *I.err
// becomes 1 if one of its bounded grid-barrier waits gave up.
constexpr int kFusedMaxC = 64;
constexpr int kFusedMaxDynSmem = 200 * 1024;
struct FusedShape {
  int n_cta;   // CTAs (<= n_sms)
  int groups;  // 16-byte column groups holding the Ni samples
  int gmax;    // most groups of one CTA
  int R;       // row streams of a CTA
};
bool fused_shape(int Ni, int nL, int C, int esize, int n_sms, FusedShape* F, size_t* smem);
cudaError_t launch_iterate(const float* KT, int64_t ldk, int Ni, const Supports& S, const IterState& I, int iters,
                           const float* kself, int32_t* u, float* margin, float* fhat_out, double* ghat_out,
                           int early_stop, int n_sms, cudaStream_t st, const RescoreArgs& R = RescoreArgs());
cudaError_t launch_iterate(const __half* KT, int64_t ldk, int Ni, const Supports& S, const IterState& I, int iters,
                           const float* kself, int32_t* u, float* margin, float* fhat_out, double* ghat_out,
                           int early_stop, int n_sms, cudaStream_t st, const RescoreArgs& R = RescoreArgs());
// The inner loop in one cooperative launch with the f_hat numerators formed on
// the tensor cores as the product of the FP16 Gaussian block and the one-hot
// label matrix (one CTA per 128-sample tile).  Applies when tc_iter_shape()
// says so (C <= 16, at most one tile per SM, the one-hot tiles fit in shared
// memory) and needs the fixed-point accumulators (I.facc, I.gfix_shift) and
// I.lm_list.  S.lab holds the final landmark labels afterwards; the caller
// rebuilds the rest of the support structure from it.  With keys != NULL the
// loop also leaves the Eq. 10 inputs of the final supports: keys[j] = the
// smallest pack_key(K_ii - 2 f_hat_ij, i) over the samples (keys preset to
// ~0), kcount[j] += the members of cluster j (preset to 0), ghat_final[j] and
// S.n_j.  *I.err becomes non-zero if a bounded wait gave up.
bool tc_iter_shape(int Ni, int nL, int C, int n_sms, int* nstages, size_t* smem);
cudaError_t launch_iterate_tc(const __half* KT, int64_t ldk, int Ni, const Supports& S, const IterState& I, int iters,
                              int32_t* u, float* margin, float* fhat_out, double* ghat_out, int early_stop,
                              int n_sms, cudaStream_t st, const RescoreArgs& R, unsigned long long* keys = nullptr,
                              int32_t* kcount = nullptr, double* ghat_final = nullptr);

// ---- mini-batch boundary -----------------------------------------------------
// Eq. 8: u[l] = argmin_j kself[l] - 2 Kt[j][l] + kmm[j]; dmin (nullable).
cudaError_t launch_nearest(const float* Kt, int64_t ldk, int Ni, int C, const float* kself,
                           const float* kmm, int32_t* u, float* dmin, cudaStream_t st);
// Eq. 10 keys and member counts c_j (keys/c must be reset by the caller).
cudaError_t launch_medoid_keys(int64_t ldk, int Ni, const Supports& S, const IterState& I,
                               const float* kself, const int32_t* u, unsigned long long* keys,
                               int32_t* c, double* ghat_out, cudaStream_t st);
// mi[j] = local index of the Eq. 10 medoid, or -1 when empty; with
// reset_keys the keys are left at ~0 (ready for the merge keys).
cudaError_t launch_medoid_pick(unsigned long long* keys, const int32_t* c, const int32_t* n_j, int C, int32_t* mi,
                               cudaStream_t st, bool reset_keys = false);
// Eq. 12 keys.
cudaError_t launch_merge_keys(const float* Kt, const float* Kmi, int64_t ldk, int Ni, int C,
                              const float* kself, const int32_t* mi, const int32_t* c,
                              const int64_t* W, unsigned long long* keys, cudaStream_t st);
// Applies the merge: M[j] = start + l*step for non-empty j, W += c; prev
// (nullable) gets M before the update.
cudaError_t launch_merge_apply(const unsigned long long* keys, const int32_t* mi, const int32_t* c,
                               int C, int64_t start, int64_t step, int64_t* M, int64_t* W,
                               cudaStream_t st, int64_t* prev = nullptr);
// Average centre displacement across one mini-batch (Section 4.1, Fig. 4b)
// from K[a][b] = K(old_a, cur_b) (C x C, row pitch ldk) into *out (device).
// Eq. 10 medoids of the mini-batch with their rows (feature kernels): mi,
// mi_safe, the keys reset, the medoid rows and norms copied from Xi/aux_i,
// their global ids idMI (dp a multiple of 4).
cudaError_t launch_medoid_rows(unsigned long long* keys, const int32_t* c, const int32_t* n_j, int C, int32_t* mi,
                               int32_t* mi_safe, const float* Xi, const float* aux_i, int dp, const int64_t* gid,
                               float* MIX, float* auxMI, int64_t* idMI, cudaStream_t st);
// The displacement of a mini-batch from the medoid rows before (MX) and the
// mini-batch rows (Gaussian or linear kernel); NX/nauxM get the medoid rows
// after the merge (the next mini-batch's MX).
cudaError_t launch_displacement_rows(const float* MX, const float* auxM, const float* Xi, const float* aux_i, int dp,
                                     int C, const unsigned long long* keys, const int32_t* mi, const int64_t* old,
                                     const int64_t* cur, bool linear, float neg_scale, double* out, float* NX,
                                     float* nauxM, cudaStream_t st);
cudaError_t launch_displacement(const float* K, int64_t ldk, int C, const float* selfA, const float* selfB,
                                const int64_t* old, const int64_t* cur, double* out, cudaStream_t st);
// labels_out[start + l*step] = u[l]
cudaError_t launch_scatter_labels(const int32_t* u, int Ni, int64_t start, int64_t step,
                                  int32_t* labels_out, cudaStream_t st);
cudaError_t launch_fill_u64(unsigned long long* p, unsigned long long v, int n, cudaStream_t st);
cudaError_t launch_fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t st);
cudaError_t launch_fill_f32(float* p, float v, int64_t n, cudaStream_t st);
// kernel k-means++ round r (1..C-1): D2 update with column Kc and the next pick.
// P [N0] and bsum [ceil(N0/256)] are scratch.
cudaError_t launch_kpp_round(const float* Kc, int N0, const float* kself, double* D2, double* P,
                             double* bsum, int32_t* picks, const double* draws, int r, cudaStream_t st);
// One whole k-means++ round on prepared rows (RBF or linear kernel), the next
// pick drawn by the last CTA; *ticket is zero between launches.  D2 holds
// N0 + N0 + ceil(N0 / 32) doubles (D^2, running sums, CTA totals).
cudaError_t launch_kpp_fused_round(const float* X, int dp, int N0, bool linear, float neg_scale, const float* kself,
                                   double* D2, double* P, double* bsum, int32_t* picks, const double* draws, int r,
                                   uint32_t* ticket, cudaStream_t st);
// picks (local) -> global ids start + p*step
cudaError_t launch_local_to_global(const int32_t* picks, int C, int64_t start, int64_t step,
                                   int64_t* M, cudaStream_t st);
// sum of n doubles in a fixed order into *out (device)
cudaError_t launch_sum_f32_to_f64(const float* v, int64_t n, double* part, int parts,
                                  double* out, cudaStream_t st);

// ---- bandwidth ----------------------------------------------------------------
// k-th smallest (0-based) of the upper-triangle entries of D [M][ld] (j > i),
// written to *out (device); scratch >= 4 KB.
cudaError_t launch_select_upper(const float* D, int M, int64_t ld, int64_t k, uint32_t* scratch,
                                float* out, cudaStream_t st);

}  // namespace kkm
