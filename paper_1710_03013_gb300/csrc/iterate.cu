// Inner iteration of the approximate mini-batch kernel k-means (Eq. 15-17)
// and the mini-batch boundary steps (Eq. 8, 10, 12, kernel k-means++).
//
// Layout.  The kernel block of mini-batch i is stored transposed,
// KT[k][l] = K(x_{L_k}, x_l) for landmark ordinal k < |L| and sample l < N_i,
// with a row pitch ldk that is a multiple of 32 floats.  Landmarks are kept
// sorted by label in `perm` (a stable counting sort), so the support S_j of
// cluster j is the contiguous segment perm[seg_off[j] .. seg_off[j+1]).  The
// segment is cut into units of at most kUnitRows landmark rows.
//
// One iteration is two launches:
//   fhat_partial  streams KT once (the HBM-bound step): every CTA sums the
//                 rows of one unit over a strip of columns (16-byte loads,
//                 FP32 or FP16 storage) and writes the partial numerators of
//                 f_hat (Eq. 17) and the part of the g_hat numerator (Eq. 16)
//                 on landmark columns of the same cluster (an exact
//                 fixed-point sum for Gaussian kernels; for the linear kernel
//                 the last CTA of a cluster forms g_hat_j);
//   assign        adds the partials of each segment in a fixed order, forms
//                 d_ij = K_ii - 2 f_hat_ij + g_hat_j, takes the argmin (lowest
//                 j on ties), the margin and the FP64 cost partials, and
//                 updates the labels in place.  Its last CTA to finish (atomic
//                 ticket, no waiting) sums the cost in a fixed order, records
//                 the trace, raises the early-stop flag and, when a landmark
//                 label changed, re-sorts the landmarks by their new labels
//                 for the next iteration (build_supports does the same sort
//                 for the initial labels of a mini-batch).
// Every sum has a fixed order, so results are bit-reproducible.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace kkm {

template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

constexpr int kSortThreads = 1024;  // build_supports: one CTA of 32 warps
constexpr int kLabRegs = 8;         // landmark labels held in registers per thread
constexpr int kAssignThreads = 256;
constexpr int kStreamThreads = 128;  // fhat_partial CTA

// Exclusive scan of one int per thread over the whole CTA (blockDim a
// multiple of 32, at most 1024).  `sh` needs 32 slots.  Returns the
// exclusive prefix; *total gets the CTA total.
__device__ __forceinline__ int block_excl_scan(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  const int off = w > 0 ? sh[w - 1] : 0;
  *total = sh[nw - 1];
  __syncthreads();
  return off + x - v;
}

// Stable counting sort of the landmark ordinals by label, done by one CTA
// (any multiple of 32 threads with blockDim.x >= C): n_j, the segment and
// unit tables, perm, and the label of every landmark column.  Shared
// scratch: cnt[C], base[C], wtab[(blockDim.x / 32) * C], scan_sh[32].
__device__ void sort_supports_cta(const Supports& S, int* cnt, int* base, int* wtab, int* scan_sh) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int nt = blockDim.x, nw = nt >> 5;
  const int C = S.C, nL = S.nL;
  for (int j = tid; j < C; j += nt) cnt[j] = 0;
  __syncthreads();
  // the first kLabRegs * nt landmark labels of this thread stay in registers;
  // larger landmark sets reload the rest from global memory in pass 2
  int labr[kLabRegs];
#pragma unroll
  for (int q = 0; q < kLabRegs; ++q) {
    const int k = q * nt + tid;
    labr[q] = k < nL ? __ldcg(S.lab + k) : -1;
  }
  // pass 1: counts (one shared atomic per distinct label and warp)
  for (int start = 0, q = 0; start < nL; start += nt, ++q) {
    const int k = start + tid;
    int lab = -1;
#pragma unroll
    for (int qq = 0; qq < kLabRegs; ++qq)
      if (qq == q) lab = labr[qq];
    if (q >= kLabRegs) lab = k < nL ? __ldcg(S.lab + k) : -1;
    if (k < nL) S.col_label[S.L[k]] = lab;
    const unsigned peers = __match_any_sync(kFull, lab);
    if (lab >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[lab], __popc(peers));
  }
  __syncthreads();
  // segment offsets and units (one cluster per thread)
  const int cj = tid < C ? cnt[tid] : 0;
  int total;
  const int off = block_excl_scan(cj, scan_sh, &total);
  const int nu = (cj + kUnitRows - 1) / kUnitRows;
  int nunits;
  const int uoff = block_excl_scan(nu, scan_sh, &nunits);
  if (tid < C) {
    base[tid] = off;
    S.seg_off[tid] = off;
    S.n_j[tid] = cj;
    S.seg_unit[tid] = uoff;
    for (int r = 0; r < nu; ++r) {
      const int un = uoff + r;
      S.unit_j[un] = tid;
      S.unit_kb[un] = off + r * kUnitRows;
      S.unit_ke[un] = min(off + (r + 1) * kUnitRows, off + cj);
    }
  }
  if (tid == 0) {
    S.seg_off[C] = nL;
    S.seg_unit[C] = nunits;
    *S.n_units = nunits;
  }
  __syncthreads();
  // pass 2: stable scatter, nt landmarks at a time in landmark order
  for (int start = 0, q = 0; start < nL; start += nt, ++q) {
    const int k = start + tid;
    int lab = -1;
#pragma unroll
    for (int qq = 0; qq < kLabRegs; ++qq)
      if (qq == q) lab = labr[qq];
    if (q >= kLabRegs) lab = k < nL ? __ldcg(S.lab + k) : -1;
    const unsigned peers = __match_any_sync(kFull, lab);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    for (int e = tid; e < nw * C; e += nt) wtab[e] = 0;
    __syncthreads();
    if (lab >= 0 && rank == 0) wtab[w * C + lab] = __popc(peers);
    __syncthreads();
    // per label, an exclusive scan over the warps (one warp per label, lane =
    // warp index)
    for (int j = w; j < C; j += nw) {
      const int v = lane < nw ? wtab[lane * C + j] : 0;
      int x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
      }
      const int b = base[j];
      if (lane < nw) wtab[lane * C + j] = b + x - v;
      const int tot = __shfl_sync(kFull, x, 31);
      __syncwarp();
      if (lane == 0) base[j] = b + tot;
    }
    __syncthreads();
    if (lab >= 0) S.perm[wtab[w * C + lab] + rank] = k;
    __syncthreads();
  }
}

// Rebuilds the support structure of the landmarks from their labels (the
// sort above) in one CTA of kSortThreads threads.
__global__ void __launch_bounds__(kSortThreads) build_supports_kernel(Supports S) {
  __shared__ int cnt[kMaxC];
  __shared__ int base[kMaxC];
  __shared__ int wtab[32 * kMaxC];
  __shared__ int scan_sh[32];
  griddep_wait();
  griddep_launch();
  sort_supports_cta(S, cnt, base, wtab, scan_sh);
}

cudaError_t launch_build_supports(const Supports& S, cudaStream_t st) {
  return launch_pdl(build_supports_kernel, dim3(1), dim3(kSortThreads), 0, st, S);
}

__global__ void landmark_maps_kernel(Supports S, const int32_t* __restrict__ u) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S.nL) return;
  const int l = S.L[k];
  S.col_ord[l] = k;
  S.lab[k] = u[l];
}

cudaError_t launch_landmark_maps(const Supports& S, const int32_t* u, cudaStream_t st) {
  if (S.nL <= 0) return cudaSuccess;
  landmark_maps_kernel<<<(unsigned)ceil_div(S.nL, 256), 256, 0, st>>>(S, u);
  return cudaGetLastError();
}

// --------------------------------------------------------- f_hat streaming
// 16-byte load with an L2 eviction-priority policy (createpolicy).
// Streaming shape per stored type: a thread adds `kCols` consecutive columns
// (one 16-byte load per block row), loading `kDepth` rows before adding
// them; a CTA of kStreamThreads threads covers kStrip columns.
template <typename T>
struct StreamCfg {
  static constexpr int kCols = 16 / (int)sizeof(T);   // FP32: 4, FP16: 8
  static constexpr int kDepth = 8;  // rows loaded before their additions
  static constexpr int kStrip = kStreamThreads * kCols;
};

__device__ __forceinline__ void ld16_policy(const float* p, uint64_t pol, float (&v)[4]) {
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
               : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld16_policy(const __half* p, uint64_t pol, uint4& u) {
  asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(u.x), "=r"(u.y), "=r"(u.z), "=r"(u.w)
               : "l"(p), "l"(pol));
}

// acc[c] += KT[rows[q]][col + c] for q < n (n == D when FULL), loading all
// rows of the chunk before adding any; rows below keep_rows with the
// evict_last policy, the rest evict_first.  FP16 storage converts to FP32
// before the additions.
template <typename T, int D, bool FULL>
__device__ __forceinline__ void stream_rows(const T* base, int64_t ldk, const int* rows, int n, int keep_rows,
                                            uint64_t keep, uint64_t stream, float (&acc)[16 / sizeof(T)]) {
  if constexpr (sizeof(T) == 4) {
    float v[D][4];
#pragma unroll
    for (int q = 0; q < D; ++q) {
      if (FULL || q < n) {
        const int r = rows[q];
        ld16_policy(base + (int64_t)r * ldk, r < keep_rows ? keep : stream, v[q]);
      } else {
        v[q][0] = v[q][1] = v[q][2] = v[q][3] = 0.0f;
      }
    }
#pragma unroll
    for (int q = 0; q < D; ++q)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] += v[q][c];
  } else {
    uint4 v[D];
#pragma unroll
    for (int q = 0; q < D; ++q) {
      if (FULL || q < n) {
        const int r = rows[q];
        ld16_policy(base + (int64_t)r * ldk, r < keep_rows ? keep : stream, v[q]);
      } else {
        v[q] = make_uint4(0u, 0u, 0u, 0u);  // +0.0 in FP16
      }
    }
#pragma unroll
    for (int q = 0; q < D; ++q) {
      const uint32_t w[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[c]));
        acc[2 * c] += f.x;
        acc[2 * c + 1] += f.y;
      }
    }
  }
}

// f_hat numerators: partial[u][l] = sum over the landmark rows k of unit u of
// KT[k][l] (in the unit's row order, FP32), for one strip of kStrip columns
// per CTA; plus the tile's g_hat numerator (its landmark columns of the same
// cluster), reduced in double-float in a fixed order.  Rows below keep_rows
// are loaded with an L2 evict_last policy (they stay resident across
// iterations), the rest evict_first.  With gfix (Gaussian kernels) each
// tile's numerator is added to gfix[j] as a fixed-point integer (exact and
// order-free; the assign forms g_hat_j = numerator / n_j^2, Eq. 16);
// otherwise the last CTA of cluster j to finish (atomic ticket, no waiting)
// forms g_hat_j in FP64 from the per-tile numerators, in a fixed order.
// Up to eight CTAs per SM (the whole grid of the MNIST-shaped block resident
// at once); the occupancy bound also lets the compiler keep a chunk's loads
// in flight together instead of interleaving them with the additions.
// Chunks of 8 rows measured faster than 4, 12 or 16, and than two chunks in
// flight with a register double buffer.
// The body takes its (strip, unit) tile explicitly, so that one launch can
// also cover the tiles of many mini-batches (fhat_partial_multi_kernel).
template <typename T>
__device__ __forceinline__ void fhat_partial_body(const T* __restrict__ KT, int64_t ldk, int Ni, const Supports& S,
                                                  float* __restrict__ partial, float2* __restrict__ gpart,
                                                  int n_strips, const int32_t* __restrict__ skip, int keep_rows,
                                                  uint32_t* __restrict__ gtick, double* __restrict__ ghat,
                                                  unsigned long long* __restrict__ gfix, double gfix_scale, int strip,
                                                  int unit) {
  using Cfg = StreamCfg<T>;
  constexpr int NC = Cfg::kCols, DEPTH = Cfg::kDepth;
  __shared__ int rows[kUnitRows];
  __shared__ float2 red[kStreamThreads / 32];
  __shared__ double redd[kStreamThreads / 32];
  __shared__ int last;
  griddep_wait();
  if (skip && *skip) return;
  // unit tables are allocated for max_units entries, so these loads stay in
  // bounds even for the units this launch does not use
  const int nu = *S.n_units;
  const int j = S.unit_j[unit], kb = S.unit_kb[unit], ke = S.unit_ke[unit];
  if (unit >= nu) return;
  const int nrow = ke - kb;
  for (int t = threadIdx.x; t < nrow; t += kStreamThreads) rows[t] = S.perm[kb + t];
  __syncthreads();
  uint64_t keep, stream;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream));
  const int col = (strip * kStreamThreads + threadIdx.x) * NC;
  float acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0f;
  // landmark labels of this thread's columns, loaded ahead of the stream (the
  // g_hat numerator needs them after it); col is a multiple of NC and the
  // label array has ldk (a multiple of 32) entries
  int clab[NC];
#pragma unroll
  for (int c = 0; c < NC; c += 4) {
    int4 v = make_int4(-1, -1, -1, -1);
    if (S.col_label && col < Ni) v = __ldg(reinterpret_cast<const int4*>(S.col_label + col + c));
    clab[c] = v.x;
    clab[c + 1] = v.y;
    clab[c + 2] = v.z;
    clab[c + 3] = v.w;
  }
  if (col < Ni) {
    const T* base = KT + col;
    // whole chunks of DEPTH rows: all loads issued before any is used, no
    // predicates between them; then the last partial chunk.  Rows are added
    // in the unit's order either way.
    int k = 0;
    for (; k + DEPTH <= nrow; k += DEPTH)
      stream_rows<T, DEPTH, true>(base, ldk, rows + k, DEPTH, keep_rows, keep, stream, acc);
    if (k < nrow) stream_rows<T, DEPTH, false>(base, ldk, rows + k, nrow - k, keep_rows, keep, stream, acc);
    float* out = partial + (int64_t)unit * ldk + col;
#pragma unroll
    for (int c = 0; c < NC; c += 4)
      *reinterpret_cast<float4*>(out + c) = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
  }
  // The assign may launch once every CTA has streamed its rows: its CTAs
  // then land on SMs this launch has left, evenly, while the g_hat tail runs.
  griddep_launch();
  // g_hat numerator: landmark columns of the same cluster
  if (!S.col_label) return;
  float2 g = make_float2(0.0f, 0.0f);
  if (col < Ni) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (col + c < Ni && clab[c] == j) g = df_add(g, make_float2(acc[c], 0.0f));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    g = df_add(g, make_float2(__shfl_xor_sync(kFull, g.x, o), __shfl_xor_sync(kFull, g.y, o)));
  if (lane == 0) red[w] = g;
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 t = red[0];
    for (int q = 1; q < kStreamThreads / 32; ++q) t = df_add(t, red[q]);
    last = 0;
    if (gfix) {
      // non-negative (Gaussian kernel values); the scale is a power of two
      atomicAdd(gfix + j, (unsigned long long)llrint(((double)t.x + (double)t.y) * gfix_scale));
    } else {
      gpart[(int64_t)unit * n_strips + strip] = t;
    }
    if (gtick && !gfix) {
      __threadfence();
      const uint32_t expect = (uint32_t)(S.seg_unit[j + 1] - S.seg_unit[j]) * (uint32_t)n_strips;
      last = atomicAdd(gtick + j, 1u) + 1u == expect;
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int64_t e0 = (int64_t)S.seg_unit[j] * n_strips, e1 = (int64_t)S.seg_unit[j + 1] * n_strips;
  double a2 = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += kStreamThreads) {
    const float2 v = __ldcg(gpart + e);
    a2 += (double)v.x + (double)v.y;
  }
  a2 = block_sum(a2, redd);
  if (threadIdx.x == 0) {
    const int n = S.n_j[j];
    ghat[j] = n > 0 ? a2 / ((double)n * (double)n) : __longlong_as_double(0x7ff8000000000000LL);
    gtick[j] = 0u;  // ready for the next launch
  }
}

template <typename T>
__global__ void __launch_bounds__(kStreamThreads, 8)
fhat_partial_kernel(const T* __restrict__ KT, int64_t ldk, int Ni, Supports S,
                    float* __restrict__ partial, float2* __restrict__ gpart, int n_strips,
                    const int32_t* __restrict__ skip, int keep_rows, uint32_t* __restrict__ gtick,
                    double* __restrict__ ghat, unsigned long long* __restrict__ gfix, double gfix_scale) {
  fhat_partial_body<T>(KT, ldk, Ni, S, partial, gpart, n_strips, skip, keep_rows, gtick, ghat, gfix, gfix_scale,
                       (int)blockIdx.x, (int)blockIdx.y);
}

template <typename T>
static cudaError_t launch_fhat_t(const T* KT, int64_t ldk, int Ni, const Supports& S, const IterState& I,
                                 cudaStream_t st) {
  const int n_strips = (int)ceil_div(ldk, StreamCfg<T>::kStrip);
  if (n_strips > I.n_strips) return cudaErrorInvalidValue;  // gpart capacity
  dim3 grid((unsigned)n_strips, (unsigned)S.max_units);
  return launch_pdl(fhat_partial_kernel<T>, grid, dim3(kStreamThreads), 0, st, KT, ldk, Ni, S, I.partial,
                    I.gpart, n_strips, (const int32_t*)I.done, I.keep_rows,
                    S.col_label ? I.gtick : (uint32_t*)nullptr, I.ghat_cur,
                    S.col_label ? I.gfix : (unsigned long long*)nullptr, ldexp(1.0, I.gfix_shift));
}
cudaError_t launch_fhat_partial(const float* KT, int64_t ldk, int Ni, const Supports& S,
                                const IterState& I, cudaStream_t st) {
  return launch_fhat_t(KT, ldk, Ni, S, I, st);
}
cudaError_t launch_fhat_partial(const __half* KT, int64_t ldk, int Ni, const Supports& S,
                                const IterState& I, cudaStream_t st) {
  return launch_fhat_t(KT, ldk, Ni, S, I, st);
}

// ------------------------------------------------------------------ assign
// Loads n_j, the unit ranges and g_hat (Eq. 16) into shared memory.
struct AssignShared {
  double gh[kMaxC];
  float ghf[kMaxC];
  int nj[kMaxC];
  int su[kMaxC + 1];
};

// g_hat_j (Eq. 16) of a non-empty cluster: given (an assign against a model),
// from the fixed-point numerator, or as formed by the f_hat stream.
__device__ __forceinline__ double cluster_ghat(const IterState& I, int j, int n) {
  if (I.ghat_in) return I.ghat_in[j];
  if (I.gfix) return (double)I.gfix[j] * ldexp(1.0, -I.gfix_shift) / ((double)n * (double)n);
  return I.ghat_cur[j];
}

// n_j, unit ranges and g_hat into shared memory (g_hat given for an assign
// against a model, else formed by fhat_partial for this iteration; NaN for an
// empty cluster).
__device__ __forceinline__ void load_cluster_stats(AssignShared& sh, const Supports& S,
                                                   const IterState& I) {
  const int C = S.C;
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    const int n = S.n_j[j];
    sh.nj[j] = n;
    sh.su[j] = S.seg_unit[j];
    sh.gh[j] = n > 0 ? cluster_ghat(I, j, n) : __longlong_as_double(0x7ff8000000000000LL);
    sh.ghf[j] = (float)sh.gh[j];
  }
  if (threadIdx.x == 0) sh.su[C] = S.seg_unit[C];
  __syncthreads();
}

__device__ __forceinline__ float partial_at(const float* __restrict__ partial, int64_t ldk, int un, int i) {
  return partial[(int64_t)un * ldk + i];
}

__device__ __forceinline__ float fhat_of(const AssignShared& sh, const float* __restrict__ partial,
                                         int64_t ldk, int i, int j) {
  float f = 0.0f;
  int un = sh.su[j];
  const int e = sh.su[j + 1];
  for (; un + 4 <= e; un += 4) {
    const float v0 = partial[(int64_t)un * ldk + i], v1 = partial[(int64_t)(un + 1) * ldk + i];
    const float v2 = partial[(int64_t)(un + 2) * ldk + i], v3 = partial[(int64_t)(un + 3) * ldk + i];
    f += v0;
    f += v1;
    f += v2;
    f += v3;
  }
  for (; un < e; ++un) f += partial[(int64_t)un * ldk + i];
  return f / (float)sh.nj[j];
}

// One CTA per 32 rows (up to 8 warps, so every CTA of a launch is resident at
// once): warp w forms d_ij for a contiguous range of clusters of its 32 rows
// (lane = row; each unit's partials are one coalesced 128-byte line); warp 0
// then takes the argmin over the clusters from shared memory.
//
// Near-tie re-score (low-precision kernel blocks, R.Xi != NULL): a row's
// candidates are the clusters j with d_j - d_best below
// flag_tau * max(|d_j|, K_ii + g_hat_best) (the best one included); a row
// with two or more is flagged, and the whole CTA recomputes its candidates'
// distances from exact FP32 kernel values over their supports (dot products
// of the FP32 rows, the same norm expansion and exponential as the FP32
// block; warp w takes landmarks w, w + nw, ... of the segment, warp sums
// added in warp order).  The other clusters are farther than the window, so
// the low-precision error (well inside it) cannot make one of them the best.
constexpr int kAssignRows = 32;

constexpr int kAssignWarps = 8;
constexpr int kCandCap = 512;  // near-tie re-score pairs listed per CTA

// 4-byte words of the assign kernel's distance tile, or of the support sort's
// scratch that reuses it (cnt[C], base[C], wtab[nw * C], scan[32]), rounded
// to 16 bytes; the re-score row follows.
__host__ __device__ inline int assign_dist_words(int C, int nw) {
  const int w = C * kAssignRows > (2 + nw) * C + 32 ? C * kAssignRows : (2 + nw) * C + 32;
  return (w + 3) & ~3;
}
// largest dynamic shared memory an assign launch may ask for
constexpr int kAssignMaxDynSmem = 160 * 1024;

// The body takes its row block bx and the number of row blocks G of its
// mini-batch explicitly, so that one launch can also cover the row blocks of
// many mini-batches (assign_multi_kernel).  nw_item > 0 sets the warps that
// work (the others only pass the barriers): a launch as wide as its widest
// item then runs every item exactly as its own launch of nw_item warps would,
// every split over warps and every thread-strided sum taken with nw_item.
__device__ __forceinline__ void assign_body(int64_t ldk, int Ni, const Supports& S, const IterState& I,
                                            const float* __restrict__ kself, int32_t* __restrict__ u,
                                            float* __restrict__ margin, float* __restrict__ dmin,
                                            float* __restrict__ fhat_out, double* __restrict__ ghat_out,
                                            int early_stop, int trace, const RescoreArgs& R, int bx, int G,
                                            bool defer_sort = false, int RG = 1, int nw_item = 0) {
  const int nw = nw_item > 0 ? nw_item : (int)(blockDim.x >> 5);
  // dynamic shared memory (sized by the launch for this C): the distances of
  // the CTA's rows [C][kAssignRows], which the last CTA reuses as the support
  // sort's scratch, then the FP32 row of the slow re-score path [R.dp]
  extern __shared__ float dyn[];
  __shared__ AssignShared sh;
  float* const dshp = dyn;
  auto dsh_at = [&](int j, int r) -> float& { return dshp[j * kAssignRows + r]; };
  float* const xs = dyn + assign_dist_words(S.C, nw);
  __shared__ float rbest[kAssignRows], rsecond[kAssignRows];
  __shared__ int rlab[kAssignRows];
  __shared__ float wsum[32];
  __shared__ unsigned flag_mask;
  __shared__ int is_last;
  __shared__ int cand[kCandCap];  // re-score pairs (row << 9 | cluster)
  __shared__ int n_cand;
  __shared__ unsigned slow_mask;
  // Everything but the partials and g_hat was written by launches that have
  // finished when this one starts (the support tables, the old labels, the
  // column ordinals, the self terms): load it before waiting for the f_hat
  // stream.
  if (I.done && *I.done) return;
  const int C = S.C;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool wact = w < nw;  // a working warp
  const float inf = __int_as_float(0x7f800000);
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    sh.nj[j] = S.n_j[j];
    sh.su[j] = S.seg_unit[j];
  }
  if (threadIdx.x == 0) sh.su[C] = S.seg_unit[C];
  __syncthreads();
  griddep_wait();
  // The next launch (the next iteration's f_hat stream) may start once every
  // CTA has triggered or exited.  With the iteration close in the last CTA
  // only that CTA triggers, after its ticket: the stream's CTAs are then
  // placed on SMs the assign has left, evenly, while the close runs.
  if (trace != 1) griddep_launch();
  // g_hat (given for an assign against a model, else formed by the f_hat
  // stream) is loaded here and used after the partial sums, so that both
  // loads are in flight together (C <= blockDim.x)
  const double gval =
      threadIdx.x < C && sh.nj[threadIdx.x] > 0 ? cluster_ghat(I, threadIdx.x, sh.nj[threadIdx.x]) : 0.0;
  // Row blocks bx * RG ... bx * RG + RG - 1 of 32 rows each, one after the
  // other: each gets exactly the work and the partial sums (omega_part[rb],
  // ...) it would get in a CTA of its own, so RG changes no result.
  const int G_rows = (Ni + kAssignRows - 1) / kAssignRows;
  for (int rg = 0; rg < RG; ++rg) {
  const int rb = bx * RG + rg;
  if (rb >= G_rows) break;  // the same in every thread
  const int i = rb * kAssignRows + lane;
  const float ks = (kself && i < Ni) ? kself[i] : 1.0f;
  const int old_u = (w == 0 && i < Ni) ? u[i] : 0;
  const int cord = (w == 0 && S.col_ord && i < Ni) ? S.col_ord[i] : -1;
  // f_hat_ij of cluster j from its unit sum f (the units of j added in
  // order); NaN for an empty cluster
  auto finish = [&](int j, float f) {
    float fh = __int_as_float(0x7fc00000);
    if (i < Ni) {
      if (sh.nj[j] > 0) fh = f / (float)sh.nj[j];
      if (fhat_out) fhat_out[(int64_t)i * C + j] = fh;
    }
    dsh_at(j, lane) = fh;
  };
  // Warp w takes the contiguous clusters [jb, je), whose units are contiguous
  // too: one flat pass over them keeps 8 loads in flight across cluster
  // boundaries (j and its end are the same in every lane).
  const int jb = wact ? (w * C) / nw : 0, je = wact ? ((w + 1) * C) / nw : 0;
  if (jb < je) {
    int j = jb;
    int jend = sh.su[j + 1];
    float f = 0.0f;
    const int E = sh.su[je];
    for (int un = sh.su[jb]; un < E; un += 8) {
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = (un + q < E && i < Ni) ? partial_at(I.partial, ldk, un + q, i) : 0.0f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (un + q < E) {
          while (un + q >= jend) {
            finish(j, f);
            f = 0.0f;
            ++j;
            jend = sh.su[j + 1];
          }
          f += v[q];
        }
      }
    }
    for (; j < je; ++j) {
      finish(j, f);
      f = 0.0f;
    }
  }
  if (threadIdx.x < C) {
    sh.gh[threadIdx.x] = sh.nj[threadIdx.x] > 0 ? gval : __longlong_as_double(0x7ff8000000000000LL);
    sh.ghf[threadIdx.x] = (float)sh.gh[threadIdx.x];
  }
  __syncthreads();
  if (rb == 0 && ghat_out)
    for (int j = threadIdx.x; j < C; j += blockDim.x) ghat_out[j] = sh.gh[j];
  // d_ij = K_ii - 2 f_hat_ij + g_hat_j for the warp's clusters (+inf when
  // n_j = 0 or past the last row)
  for (int j = jb; j < je; ++j) {
    const float fh = dsh_at(j, lane);
    dsh_at(j, lane) = (i < Ni && sh.nj[j] > 0) ? ks - 2.0f * fh + sh.ghf[j] : inf;
  }
  __syncthreads();
  if (w == 0) {
    float best = inf, second = inf;
    int bj = 0;
    bool flagged = false;
    if (i < Ni) {
      for (int j = 0; j < C; ++j) {  // lowest j on ties
        const float dj = dsh_at(j, lane);
        if (dj < best) {
          second = best;
          best = dj;
          bj = j;
        } else if (dj < second) {
          second = dj;
        }
      }
      // near tie on the scale of the terms of d (K_ii + g_hat ~ 1): the
      // low-precision error of d is absolute, so the criterion is too
      if (R.Xi && I.flag_tau > 0.0f && second < inf)
        flagged = (second - best) < I.flag_tau * fmaxf(fabsf(second), ks + sh.ghf[bj]);
    }
    rbest[lane] = best;
    rsecond[lane] = second;
    rlab[lane] = bj;
    const unsigned fm = __ballot_sync(kFull, flagged);
    if (lane == 0) flag_mask = fm;
  }
  __syncthreads();
  if (flag_mask) {
    // Candidate pairs (row r, cluster j) of the flagged rows, listed by warp 0:
    // the clusters whose low-precision distance is inside the row's window.
    if (w == 0) {
      const bool fl = (flag_mask >> lane) & 1u;
      const float b0 = rbest[lane];
      const float scale = ks + sh.ghf[rlab[lane]];
      int cnt = 0;
      if (fl)
        for (int j = 0; j < C; ++j) {
          const float dj0 = dsh_at(j, lane);
          cnt += dj0 - b0 < I.flag_tau * fmaxf(fabsf(dj0), scale);
        }
      int x = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
      }
      const int off = x - cnt;
      const bool fits = off + cnt <= kCandCap;  // rows in lane order: the fitting ones are a prefix
      if (fl && fits) {
        int k = off;
        for (int j = 0; j < C; ++j) {
          const float dj0 = dsh_at(j, lane);
          if (dj0 - b0 < I.flag_tau * fmaxf(fabsf(dj0), scale)) cand[k++] = (lane << 9) | j;
        }
      }
      int used = fits ? off + cnt : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) used = max(used, __shfl_xor_sync(kFull, used, o));
      const unsigned slow = __ballot_sync(kFull, fl && !fits);
      if (lane == 0) {
        n_cand = used;
        slow_mask = slow;
      }
    }
    __syncthreads();
    // every warp re-scores whole pairs, one landmark per lane (lane-strided
    // over the cluster's segment, then a fixed xor tree): FP32 kernel values
    // from the FP32 rows (16-byte loads; rows are padded to 8 floats)
    for (int p = w; wact && p < n_cand; p += nw) {
      const int r = cand[p] >> 9, j = cand[p] & 511;
      const int ir = rb * kAssignRows + r;
      const float4* xi = reinterpret_cast<const float4*>(R.Xi + (int64_t)ir * R.dp);
      const float ni = R.nXi[ir];
      const float ksr = kself ? kself[ir] : 1.0f;
      const int k0 = S.seg_off[j], k1 = S.seg_off[j + 1];
      float acc = 0.0f;
      if (R.K32) {  // the block's own FP32 values
        for (int kk = k0 + lane; kk < k1; kk += 32) acc += __ldg(R.K32 + (int64_t)S.perm[kk] * R.ldk32 + ir);
      }
      for (int kk = k0 + lane; !R.K32 && kk < k1; kk += 32) {
        const int k = S.perm[kk];
        const float4* xl = reinterpret_cast<const float4*>(R.XL + (int64_t)k * R.dp);
        // in chunks of 32 products (see the Gram kernel: one long FP32 sum drifts)
        float dot = 0.0f, part = 0.0f;
        for (int c = 0; c < (R.dp >> 2); ++c) {
          const float4 a = __ldg(xi + c), b = __ldg(xl + c);
          part = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, part))));
          if ((c & 7) == 7) {
            dot += part;
            part = 0.0f;
          }
        }
        dot += part;
        float kv;
        if (R.kind == DK_LINEAR) kv = dot;
        else kv = (S.L[k] == ir) ? 1.0f : exp2f(fmaxf(ni + R.nXL[k] - 2.0f * dot, 0.0f) * R.neg_scale);
        acc += kv;
      }
      acc = warp_sum_f32(acc);
      if (lane == 0) dsh_at(j, r) = k1 > k0 ? ksr - 2.0f * (acc / (float)(k1 - k0)) + sh.ghf[j] : inf;
    }
    __syncthreads();
    // rows whose candidates did not fit the list: the whole CTA per row
    for (unsigned fm = slow_mask; fm; fm &= fm - 1) {  // the same sequence in every thread
      const int r = __ffs(fm) - 1;
      const int ir = rb * kAssignRows + r;
      const float* xi = R.Xi + (int64_t)ir * R.dp;
      for (int c = threadIdx.x; c < R.dp; c += blockDim.x) xs[c] = xi[c];
      __syncthreads();
      const float ni = R.nXi[ir];
      const float ksr = kself ? kself[ir] : 1.0f;
      const float b0 = rbest[r];
      const float scale = ksr + sh.ghf[rlab[r]];
      for (int j = 0; j < C; ++j) {
        const float dj0 = dsh_at(j, r);  // low-precision value (same in every thread)
        if (!(dj0 - b0 < I.flag_tau * fmaxf(fabsf(dj0), scale))) continue;
        const int k0 = S.seg_off[j], k1 = S.seg_off[j + 1];
        float acc = 0.0f;
        for (int kk = k0 + w; wact && kk < k1; kk += nw) {
          const int k = S.perm[kk];
          float kv;
          if (R.K32) {  // the block's own FP32 values
            kv = __ldg(R.K32 + (int64_t)k * R.ldk32 + ir);
          } else {
            const float* xl = R.XL + (int64_t)k * R.dp;
            float dot = 0.0f;
            for (int c = lane; c < R.dp; c += 32) dot = fmaf(xs[c], xl[c], dot);
            dot = warp_sum_f32(dot);
            if (R.kind == DK_LINEAR) kv = dot;
            else kv = (S.L[k] == ir) ? 1.0f : exp2f(fmaxf(ni + R.nXL[k] - 2.0f * dot, 0.0f) * R.neg_scale);
          }
          acc += kv;
        }
        if (lane == 0) wsum[w] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
          float f = 0.0f;
          for (int q = 0; q < nw; ++q) f += wsum[q];
          const int n = k1 - k0;
          dsh_at(j, r) = n > 0 ? ksr - 2.0f * (f / (float)n) + sh.ghf[j] : inf;
        }
        __syncthreads();
      }
    }
    // the argmin of every flagged row over its updated distances
    if (w == 0 && ((flag_mask >> lane) & 1u)) {
      float best = inf;
      int bj = 0;
      for (int j = 0; j < C; ++j)
        if (dsh_at(j, lane) < best) {
          best = dsh_at(j, lane);
          bj = j;
        }
      rbest[lane] = best;
      rlab[lane] = bj;
    }
    __syncthreads();
  }
  if (w == 0) {
    float2 om = make_float2(0.0f, 0.0f);
    int ch = 0, lmc = 0;
    if (i < Ni) {
      const int bj = rlab[lane];
      const float best = rbest[lane];
      u[i] = bj;
      ch = (old_u != bj);
      if (cord >= 0) {
        S.lab[cord] = bj;
        lmc = ch;
      }
      if (margin) margin[i] = rsecond[lane] - best;
      if (dmin) dmin[i] = best;
      om.x = best;
    }
    om = warp_sum_df(om);
    ch = warp_sum_i32(ch);
    lmc = warp_sum_i32(lmc);
    if (lane == 0) {
      I.omega_part[rb] = om;
      I.changed_part[rb] = ch;
      if (I.lm_part) I.lm_part[rb] = lmc;
    }
  }
  __syncthreads();  // the next row block reuses the shared tiles
  }
  if (trace != 1) return;
  // The last CTA to finish (atomic ticket, no waiting) closes the iteration
  // and prepares the next one: Omega and the counts in a fixed order, the
  // trace entry, the early-stop flag, the landmark-change count; then, if a
  // landmark label changed, the support sort (every other CTA has read the
  // support tables by the time it takes its ticket).
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(I.ticket, 1u) == (unsigned)G - 1u);
  __syncthreads();
  if (!is_last) return;
  griddep_launch();
  __threadfence();
  float2 o = make_float2(0.0f, 0.0f);
  int c = 0, lm = 0;
  const int nthr = 32 * nw;
  for (int b = threadIdx.x; (int)threadIdx.x < nthr && b < G_rows; b += nthr) {
    o = df_add(o, __ldcg(I.omega_part + b));
    c += __ldcg(I.changed_part + b);
    lm += I.lm_part ? __ldcg(I.lm_part + b) : 0;
  }
  o = warp_sum_df(o);
  c = warp_sum_i32(c);
  lm = warp_sum_i32(lm);
  __shared__ float2 wo[kAssignWarps];
  __shared__ int wc[kAssignWarps], wl[kAssignWarps];
  if (lane == 0) {
    wo[w] = o;
    wc[w] = c;
    wl[w] = lm;
  }
  __syncthreads();
  if (w == 0) {
    o = lane < nw ? wo[lane] : make_float2(0.0f, 0.0f);
    c = lane < nw ? wc[lane] : 0;
    lm = lane < nw ? wl[lane] : 0;
    o = warp_sum_df(o);
    c = warp_sum_i32(c);
    lm = warp_sum_i32(lm);
    if (lane == 0) {
      const int t = *I.trace_count;
      I.trace_omega[t] = (double)o.x + (double)o.y;
      I.trace_changed[t] = c;
      *I.trace_count = t + 1;
      if (early_stop && c == 0) *I.done = 1;
      *I.ticket = 0u;
      wl[0] = lm;
    }
  }
  // every CTA has read the fixed-point numerators: zero them for the next
  // stream
  if (I.gfix)
    for (int j = threadIdx.x; j < C; j += blockDim.x) I.gfix[j] = 0ull;
  __syncthreads();
  if (wl[0] == 0 || defer_sort) return;  // same landmark labels: same supports (or sorted by a later launch)
  int* const scr = reinterpret_cast<int*>(dyn);  // every CTA is past its distances
  sort_supports_cta(S, scr, scr + C, scr + 2 * C, scr + 2 * C + nw * C);
}

__global__ void __launch_bounds__(kAssignWarps * 32, 4)
assign_kernel(int64_t ldk, int Ni, Supports S, IterState I, const float* __restrict__ kself,
              int32_t* __restrict__ u, float* __restrict__ margin, float* __restrict__ dmin,
              float* __restrict__ fhat_out, double* __restrict__ ghat_out, int early_stop,
              int trace, RescoreArgs R, int RG) {
  assign_body(ldk, Ni, S, I, kself, u, margin, dmin, fhat_out, ghat_out, early_stop, trace, R, (int)blockIdx.x,
              (int)gridDim.x, false, RG);
}

// Timing samples of the row tuner from a fit's own assign launches: events
// from a pool, read once they have completed (by a later launch).
struct SoloSample {
  long long key;
  int rows, blocks;
  cudaEvent_t a, b;
};
static std::mutex g_solo_mu;
static std::vector<SoloSample> g_solo_samples;
static std::vector<cudaEvent_t> g_solo_events;
static cudaEvent_t solo_event() {
  std::lock_guard<std::mutex> lk(g_solo_mu);
  if (!g_solo_events.empty()) {
    cudaEvent_t e = g_solo_events.back();
    g_solo_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
static void solo_samples_collect() {
  std::lock_guard<std::mutex> lk(g_solo_mu);
  for (size_t q = 0; q < g_solo_samples.size();) {
    SoloSample& m = g_solo_samples[q];
    const cudaError_t e = cudaEventQuery(m.b);
    if (e == cudaErrorNotReady) {
      ++q;
      continue;
    }
    float ms = 0.0f;
    if (e == cudaSuccess && cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess)
      assign_rows_sample(m.key, m.rows, m.blocks, ms);
    cudaGetLastError();
    g_solo_events.push_back(m.a);
    g_solo_events.push_back(m.b);
    g_solo_samples.erase(g_solo_samples.begin() + (std::ptrdiff_t)q);
  }
}

cudaError_t launch_assign(int64_t ldk, int Ni, const Supports& S, const IterState& I,
                          const float* kself, int32_t* u, float* margin, float* dmin,
                          float* fhat_out, double* ghat_out, int early_stop, int trace,
                          cudaStream_t st, const RescoreArgs& R) {
  if (Ni <= 0) return cudaSuccess;
  const int threads = 32 * std::min(S.C, kAssignWarps);
  const size_t smem = ((size_t)assign_dist_words(S.C, threads / 32) + (R.Xi ? (size_t)R.dp : 0)) * sizeof(float);
  if (smem > (size_t)kAssignMaxDynSmem) return cudaErrorInvalidValue;
  // one attribute for every launch (set once: launches from several host
  // threads never race on it)
  static const cudaError_t attr =
      cudaFuncSetAttribute(assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kAssignMaxDynSmem);
  if (attr != cudaSuccess) return attr;
  const int blocks = (int)ceil_div(Ni, kAssignRows);
  // a fit's iteration launches: rows per CTA from the tuner (timing samples
  // are events around a launch, read back by later calls)
  int RG = 1;
  bool timed = false;
  long long key = 0;
  if (trace == 1) {
    solo_samples_collect();
    key = assign_rows_key(threads / 32, blocks, /*solo=*/true);
    RG = assign_rows_choose(key, &timed);
  }
  SoloSample smp{key, RG, blocks, nullptr, nullptr};
  if (timed) {
    smp.a = solo_event();
    smp.b = solo_event();
    if (smp.a && smp.b) cudaEventRecord(smp.a, st);
  }
  const cudaError_t e = launch_pdl(assign_kernel, dim3((unsigned)ceil_div(blocks, RG)), dim3(threads), smem, st, ldk,
                                   Ni, S, I, kself, u, margin, dmin, fhat_out, ghat_out, early_stop, trace, R, RG);
  if (timed && smp.a && smp.b) {
    cudaEventRecord(smp.b, st);
    std::lock_guard<std::mutex> lk(g_solo_mu);
    g_solo_samples.push_back(smp);
  }
  return e;
}

// ------------------------------------------- inner loops as work lists
// The item whose CTA range [cta_off[k], cta_off[k + 1]) holds CTA b.
__device__ __forceinline__ int round_item_of(const RoundList& L, int b) {
  int lo = 0, hi = L.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.cta_off[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
// Copies item `slot` into shared memory (16-byte words).
__device__ __forceinline__ const LoopItem& load_item(const LoopItem* __restrict__ items, int slot,
                                                    unsigned char* sh) {
  const int4* src = reinterpret_cast<const int4*>(items + slot);
  int4* dst = reinterpret_cast<int4*>(sh);
  for (int t = threadIdx.x; t < (int)(sizeof(LoopItem) / 16); t += blockDim.x) dst[t] = src[t];
  __syncthreads();
  return *reinterpret_cast<const LoopItem*>(sh);
}

// Every CTA waits for the launch before it first (programmatic dependent
// launch), so that a launch of the work list completes only after the one
// before it has: the chain of launches stays ordered for every item.
template <typename T>
__global__ void __launch_bounds__(kStreamThreads, 8)
fhat_partial_multi_kernel(const LoopItem* __restrict__ items, RoundList L) {
  __shared__ __align__(16) unsigned char raw[sizeof(LoopItem)];
  griddep_wait();
  const int k = round_item_of(L, (int)blockIdx.x);
  const LoopItem& it = load_item(items, L.slot[k], raw);
  const int local = (int)blockIdx.x - L.cta_off[k];
  const int unit = local / it.n_strips, strip = local - unit * it.n_strips;
  fhat_partial_body<T>(static_cast<const T*>(it.KT), it.ldk, it.Ni, it.S, it.I.partial, it.I.gpart, it.n_strips,
                       it.I.done, it.I.keep_rows, it.S.col_label ? it.I.gtick : nullptr, it.I.ghat_cur,
                       it.S.col_label ? it.I.gfix : nullptr, it.gfix_scale, strip, unit);
}

__global__ void __launch_bounds__(kAssignWarps * 32, 4)
assign_multi_kernel(const LoopItem* __restrict__ items, RoundList L, int RG) {
  __shared__ __align__(16) unsigned char raw[sizeof(LoopItem)];
  griddep_wait();
  const int k = round_item_of(L, (int)blockIdx.x);
  const LoopItem& it = load_item(items, L.slot[k], raw);
  const int bx = (int)blockIdx.x - L.cta_off[k], G = L.cta_off[k + 1] - L.cta_off[k];
  assign_body(it.ldk, it.Ni, it.S, it.I, it.kself, it.u, nullptr, nullptr, nullptr, nullptr, it.early_stop,
              /*trace=*/1, it.R, bx, G, /*defer_sort=*/true, RG, it.nw);
}

// The support sort of every listed item (one CTA of kSortThreads each) whose
// landmark labels changed in the assign before it (the sum of its assign
// CTAs' change counts): in a work-list round the sort runs here with a full
// CTA, not in the item's last assign CTA.  The sort is stable, so the
// supports are those the assign would have built.
__global__ void __launch_bounds__(kSortThreads) sort_multi_kernel(const LoopItem* __restrict__ items, RoundList L) {
  __shared__ int cnt[kMaxC];
  __shared__ int base[kMaxC];
  __shared__ int wtab[32 * kMaxC];
  __shared__ int scan_sh[32];
  __shared__ int any;
  __shared__ __align__(16) unsigned char raw[sizeof(LoopItem)];
  griddep_wait();
  const LoopItem& it = load_item(items, L.slot[blockIdx.x], raw);
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int c = 0;
  if (it.I.lm_part)
    for (int b = threadIdx.x; b < it.assign_ctas; b += blockDim.x) c += __ldcg(it.I.lm_part + b);
  if (c) atomicOr(&any, 1);
  __syncthreads();
  if (!any) return;
  sort_supports_cta(it.S, cnt, base, wtab, scan_sh);
}

cudaError_t make_loop_item(const void* KT, bool half, int64_t ldk, int Ni, const Supports& S, const IterState& I,
                           const float* kself, int32_t* u, int early_stop, const RescoreArgs& R, LoopItem* out) {
  LoopItem it;
  it.KT = KT;
  it.ldk = ldk;
  it.Ni = Ni;
  it.half = half ? 1 : 0;
  it.n_strips = (int)ceil_div(ldk, half ? StreamCfg<__half>::kStrip : StreamCfg<float>::kStrip);
  if (it.n_strips > I.n_strips) return cudaErrorInvalidValue;  // gpart capacity
  it.units = S.max_units;
  it.nw = std::min(S.C, kAssignWarps);
  it.early_stop = early_stop;
  it.assign_ctas = (int)ceil_div(Ni, kAssignRows);
  const size_t smem = ((size_t)assign_dist_words(S.C, it.nw) + (R.Xi ? (size_t)R.dp : 0)) * sizeof(float);
  if (smem > (size_t)kAssignMaxDynSmem) return cudaErrorInvalidValue;
  it.assign_smem = (int)smem;
  it.gfix_scale = ldexp(1.0, I.gfix_shift);
  it.kself = kself;
  it.u = u;
  it.S = S;
  it.I = I;
  it.R = R;
  *out = it;
  return cudaSuccess;
}

cudaError_t launch_fhat_multi(const LoopItem* items, const RoundList& L, bool half, cudaStream_t st) {
  if (L.n <= 0 || L.cta_off[L.n] <= 0) return cudaSuccess;
  const dim3 grid((unsigned)L.cta_off[L.n]);
  return half ? launch_pdl(fhat_partial_multi_kernel<__half>, grid, dim3(kStreamThreads), 0, st, items, L)
              : launch_pdl(fhat_partial_multi_kernel<float>, grid, dim3(kStreamThreads), 0, st, items, L);
}

cudaError_t launch_sort_multi(const LoopItem* items, const RoundList& L, cudaStream_t st) {
  if (L.n <= 0) return cudaSuccess;
  return launch_pdl(sort_multi_kernel, dim3((unsigned)L.n), dim3(kSortThreads), 0, st, items, L);
}

cudaError_t launch_assign_multi(const LoopItem* items, const RoundList& L, int nw, int smem, int RG,
                                cudaStream_t st) {
  if (L.n <= 0 || L.cta_off[L.n] <= 0) return cudaSuccess;
  if (nw < 1 || nw > kAssignWarps || smem > kAssignMaxDynSmem || RG < 1) return cudaErrorInvalidValue;
  static const cudaError_t attr = cudaFuncSetAttribute(assign_multi_kernel,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kAssignMaxDynSmem);
  if (attr != cudaSuccess) return attr;
  return launch_pdl(assign_multi_kernel, dim3((unsigned)L.cta_off[L.n]), dim3(32 * nw), (size_t)smem, st, items, L,
                    RG);
}

// ------------------------------------------------- fused inner loop
// The inner loop of one mini-batch (Eq. 15-17, Alg. 1 lines 9-16) in one
// cooperative launch.  Every CTA owns a strip of sample columns of the block
// and streams ALL landmark rows of that strip, in the label-sorted order of
// `perm`, so the f_hat numerators of its columns are complete inside the CTA
// (no partial sums leave it).  Per iteration:
//   A  stream the strip; per-cluster g_hat shares of its landmark columns;
//   -- grid barrier 1 (arrive; e_lj = K_ll - 2 f_hat_lj while waiting);
//   B  g_hat (Eq. 16) from the shares of every CTA, the same value in every
//      CTA; d_lj = e_lj + g_hat_j, argmin (lowest j on ties), margin,
//      near-tie re-score, changed landmark labels, cost and counts;
//   -- grid barrier 2;
//   C  every CTA reads the iteration's cost and counts; CTA 0 writes the
//      trace entry; with early stop a pass without change ends the loop in
//      every CTA; if a landmark label changed, CTA 0 re-sorts the supports and
//      a third barrier publishes them.
// For the Gaussian kernels (values in [0, 1]) the shares of g_hat and of the
// cost are added as fixed-point integers (exact, so the same bits in any
// order) into accumulators that alternate between iterations; for the linear
// kernel each CTA writes its shares and every CTA adds them in CTA order.
//
// Inside a CTA: thread t takes column group g = t % gmax (16 bytes of
// columns) and row stream r = t / gmax; stream r walks the contiguous rows
// [r nL / R, (r+1) nL / R) of the sorted landmark list, keeps one running sum
// per segment it is in, and flushes it to the shared slot r + j when it
// leaves segment j.  Streams cover the rows in order, so the slots of
// different (stream, segment) pairs are distinct, and the numerator of
// segment j is the sum of its slots in stream order: every sum has a fixed
// order, results are bit-reproducible.  The rows of a thread reach shared
// memory through a ring of asynchronous copies that runs on into the next
// iteration's rows (the block and, unless the supports change, the row
// order are the same), so the loads of iteration t+1 are in flight during
// the barriers of iteration t; a support change drains and refills it.
//
// The barriers need every CTA resident at once: the kernel is launched as a
// cooperative grid of at most one CTA per SM.  Every wait is bounded; when a
// bound is hit the kernel records an error and every CTA returns.
constexpr int kFusedThreads = 512;
constexpr int kFusedWarps = kFusedThreads / 32;
constexpr int kFusedDepth = 16;         // rows in flight per thread (asynchronous copies to shared memory)
constexpr int kFusedPermCap = 8192;     // sorted landmark list staged in shared memory up to this size
constexpr int kFusedCandCap = 1024;     // re-score pairs listed per round
constexpr unsigned kFusedSpinLimit = 1u << 25;  // polls per barrier (>= ~1 s with the 32 ns back-off)
constexpr int kFusedCtaPerLane = 8;     // per-CTA values a lane loads in the cross-CTA sums (<= 256 CTAs)

// 16 bytes of a block row (FP32: 4 values, FP16: 8) added to the running
// sums, read from the thread's slot of the copy ring in shared memory.
__device__ __forceinline__ void add16(const float* p, float (&acc)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  acc[0] += v.x;
  acc[1] += v.y;
  acc[2] += v.z;
  acc[3] += v.w;
}
__device__ __forceinline__ void add16(const float* p, float (&acc)[8]) {
  const uint4 x = *reinterpret_cast<const uint4*>(p);
  const uint32_t wds[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&wds[c]));
    acc[2 * c] += f.x;
    acc[2 * c + 1] += f.y;
  }
}
// Asynchronous 16-byte copy global -> shared (cp.async, L2 eviction-priority
// policy), its commit group and the wait for all but the newest N groups.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint64_t pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// stream of row k when nL rows are cut into R contiguous streams
// [floor(r nL / R), floor((r+1) nL / R))
__host__ __device__ inline int fused_stream_of(int k, int nL, int R) {
  const int r = (int)((((int64_t)k + 1) * R - 1) / nL);
  return r < R - 1 ? r : R - 1;
}

// Offset (in 4-byte words, a multiple of 4) of the copy ring in the fused
// kernel's dynamic shared memory: after the slots and the staged landmark list.
__host__ __device__ inline size_t fused_ring_offset(int R, int C, int gmax, int NC, int perm_words) {
  return ((size_t)(R + C) * gmax * NC + (size_t)perm_words + 3) & ~(size_t)3;
}

// Grid barrier of the cooperative launch on *bar (zeroed by the host before
// the launch; it only grows during it): every CTA syncs, its thread 0 makes
// the CTA's writes visible and arrives; later it waits for `target` arrivals
// and the CTA syncs again.  The wait gives up after a bound, or at once when
// another CTA already gave up (*err), and then returns false everywhere.
__device__ __forceinline__ void fused_arrive(unsigned* bar) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
  }
}
__device__ __forceinline__ bool fused_wait(unsigned* bar, unsigned target, int* err, int* flag_sh) {
  if (threadIdx.x == 0) {
    unsigned polls = 0;
    *flag_sh = 1;
    while (ld_acquire_u32(bar) < target) {
      __nanosleep(32);
      if (++polls > kFusedSpinLimit || ld_acquire_u32(reinterpret_cast<const unsigned*>(err)) != 0) {
        atomicExch(err, 1);
        *flag_sh = 0;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *flag_sh != 0;
}

// Fixed-point accumulators of the fused loop (Gaussian kernels), two sets
// alternating between iterations: [set][C] g_hat numerators, then the cost,
// the changed-label and the changed-landmark counts of each set.
__host__ __device__ inline int fused_acc_words(int C) { return 2 * (C + 3); }

template <typename T>
__global__ void __launch_bounds__(kFusedThreads, 1)
iterate_fused_kernel(const T* __restrict__ KT, int64_t ldk, int Ni, Supports S, IterState I, FusedShape F,
                     int iters, const float* __restrict__ kself, int32_t* __restrict__ u,
                     float* __restrict__ margin, float* __restrict__ fhat_out, double* __restrict__ ghat_out,
                     int early_stop, RescoreArgs R) {
  constexpr int NC = 16 / (int)sizeof(T);
  extern __shared__ __align__(16) float fdyn[];
  __shared__ int seg_sh[kFusedMaxC + 1];
  __shared__ int nj_sh[kFusedMaxC];
  __shared__ int first_sh[kFusedMaxC];
  __shared__ int rhi_sh[kFusedMaxC];
  __shared__ int j0_sh[kFusedThreads];
  __shared__ double gh_sh[kFusedMaxC];
  __shared__ float ghf_sh[kFusedMaxC];
  __shared__ float2 wom[kFusedWarps];
  __shared__ int wch[kFusedWarps], wlm[kFusedWarps];
  __shared__ int scan_sh[32];
  __shared__ int cand[kFusedCandCap];
  __shared__ int clab_sh[kFusedThreads];
  __shared__ double tot_om;
  __shared__ int tot_ch, tot_lm, ok_sh;
  griddep_wait();
  if (I.done && *I.done) return;  // early stop: the same flag in every CTA
  const int C = S.C, nL = S.nL;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int gmax = F.gmax, RS = F.R;
  const int gb = (int)(((int64_t)blockIdx.x * F.groups) / gridDim.x);
  const int ge = (int)(((int64_t)(blockIdx.x + 1) * F.groups) / gridDim.x);
  const int ng = ge - gb;
  const int ncol = ng * NC;  // this CTA's columns: col0 + [0, ncol)
  const int col0 = gb * NC;
  const float inf = __int_as_float(0x7f800000);
  const bool fixed = I.gfix != nullptr;  // Gaussian kernel: fixed-point shares
  unsigned long long* const facc = I.facc;
  const double gscale = ldexp(1.0, I.gfix_shift), oscale = ldexp(1.0, I.fom_shift);
  float* const slots = fdyn;  // [(RS + C)][gmax][NC]
  const bool perm_in_sh = nL <= kFusedPermCap;
  int* const perm_sh = reinterpret_cast<int*>(fdyn + (size_t)(RS + C) * gmax * NC);
  // the copy ring: [kFusedDepth][kFusedThreads] 16-byte slots, 16-byte aligned
  float* const ring = fdyn + fused_ring_offset(RS, C, gmax, NC, perm_in_sh ? nL : 0);
  const int t0 = *I.trace_count;  // trace entries before this loop (written by CTA 0 only)
  unsigned bar_target = 0;

  // this thread's column in phase B (column col0 + tid): its inputs, loaded
  // once, and its label, kept in a register through the loop
  const int q = tid;
  const int l = col0 + q;
  const bool mine = q < ncol && l < Ni;
  float ks = 1.0f;
  int cur_u = 0, cord = -1;
  if (mine) {
    if (kself) ks = kself[l];
    cur_u = u[l];
    if (S.col_ord) cord = S.col_ord[l];
  }
  // this thread's stream of the block: rows [ra, re) of the sorted list,
  // column group g; the copy cursor (it_i, k_i) runs ahead of the reads
  const int g = tid % gmax, r = tid / gmax;
  const bool streams = r < RS && g < ng;
  const int ra = streams ? (int)(((int64_t)r * nL) / RS) : 0;
  const int re = streams ? (int)(((int64_t)(r + 1) * nL) / RS) : 0;
  const T* const base = KT + (int64_t)col0 + (int64_t)g * NC;
  const uint32_t ring0 = smem_u32(ring + (size_t)tid * 4);  // slot s at ring0 + s * kFusedThreads * 16
  const int keep_rows = I.keep_rows;
  uint64_t keep, strm;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(strm));
  int it_i = 0, k_i = ra, slot_i = 0;  // next copy: iteration it_i, row k_i, ring slot slot_i
  int slot_r = 0;                      // next read: ring slot
  auto issue_next = [&]() {
    if (streams && re > ra && it_i < iters) {
      // the global list is re-sorted inside the launch: read it past L1
      const int row = perm_in_sh ? perm_sh[k_i] : __ldcg(S.perm + k_i);
      cp_async16(ring0 + (uint32_t)slot_i * kFusedThreads * 16u, base + (int64_t)row * ldk,
                 row < keep_rows ? keep : strm);
      slot_i = (slot_i + 1) & (kFusedDepth - 1);
      if (++k_i == re) {
        k_i = ra;
        ++it_i;
      }
    }
    cp_async_commit();  // one group per call, empty or not
  };

  bool reload = true;  // the support tables in shared memory are stale
  int t = 0;
  for (; t < iters; ++t) {
    if (reload) {
      // the rows in flight (if any) follow the old order: drain, reload, refill
      cp_async_wait<0>();
      __syncthreads();
      for (int j = tid; j <= C; j += kFusedThreads) seg_sh[j] = __ldcg(S.seg_off + j);
      for (int j = tid; j < C; j += kFusedThreads) nj_sh[j] = __ldcg(S.n_j + j);
      if (perm_in_sh)
        for (int k = tid; k < nL; k += kFusedThreads) perm_sh[k] = __ldcg(S.perm + k);
      clab_sh[q] = (mine && S.col_label) ? __ldcg(S.col_label + l) : -1;
      __syncthreads();
      // segment of the first row of every stream (empty segments skipped);
      // each segment's first and last stream, and its whole numerator's slot
      for (int rr = tid; rr < RS; rr += kFusedThreads) {
        const int a = (int)(((int64_t)rr * nL) / RS);
        int j = 0;
        while (j < C - 1 && seg_sh[j + 1] <= a) ++j;
        j0_sh[rr] = j;
      }
      for (int j = tid; j < C; j += kFusedThreads) {
        first_sh[j] = nj_sh[j] > 0 ? fused_stream_of(seg_sh[j], nL, RS) + j : -1;
        rhi_sh[j] = nj_sh[j] > 0 ? fused_stream_of(seg_sh[j + 1] - 1, nL, RS) : -1;
      }
      __syncthreads();
      it_i = t;
      k_i = ra;
      slot_i = slot_r = 0;
#pragma unroll 1
      for (int qq = 0; qq < kFusedDepth; ++qq) issue_next();
      reload = false;
    }

    // ---- phase A: stream the strip, one running sum per (stream, segment);
    // each row is read from the ring once its copy has landed, then the copy
    // kFusedDepth rows ahead (possibly of the next iteration) takes its slot
    if (streams && ra < re) {
      int j = j0_sh[r];
      int jend = seg_sh[j + 1];
      float acc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = 0.0f;
      auto flush = [&](int jj) {
        float4* dst = reinterpret_cast<float4*>(slots + ((size_t)(r + jj) * gmax + g) * NC);
#pragma unroll
        for (int c = 0; c < NC; c += 4) dst[c / 4] = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = 0.0f;
      };
      for (int k = ra; k < re; ++k) {
        cp_async_wait<kFusedDepth - 1>();  // row k has landed
        while (k >= jend) {  // the row opens a later segment
          flush(j);
          ++j;
          jend = seg_sh[j + 1];
        }
        add16(ring + (size_t)tid * 4 + (size_t)slot_r * kFusedThreads * 4, acc);
        slot_r = (slot_r + 1) & (kFusedDepth - 1);
        issue_next();  // after the read of the slot it refills
      }
      flush(j);
    }
    __syncthreads();
    // every segment's numerator: its pieces in stream order, into its first slot
    for (int e = tid; e < C * ncol; e += kFusedThreads) {
      const int j = e / ncol, qq = e - j * ncol;
      if (nj_sh[j] == 0) continue;
      const int r0 = first_sh[j] - j, r1 = rhi_sh[j];
      const int gq = qq / NC, cq = qq - gq * NC;
      float s = 0.0f;
      for (int rr = r0; rr <= r1; ++rr) s += slots[((size_t)(rr + j) * gmax + gq) * NC + cq];
      slots[((size_t)(r0 + j) * gmax + gq) * NC + cq] = s;
    }
    __syncthreads();
    // this CTA's share of the g_hat numerators (Eq. 16): landmark columns of
    // each cluster, double-float, columns in order within a fixed lane tree
    if (S.col_label) {
      for (int j = w; j < C; j += kFusedWarps) {
        float2 gs = make_float2(0.0f, 0.0f);
        if (nj_sh[j] > 0) {
          const float* fj = slots + (size_t)first_sh[j] * gmax * NC;
          for (int qq = lane; qq < ncol; qq += 32)
            if (clab_sh[qq] == j) gs = df_add(gs, make_float2(fj[qq], 0.0f));
        }
        gs = warp_sum_df(gs);
        if (lane == 0) {
          if (fixed) {
            if (nj_sh[j] > 0)  // non-negative; the scale is a power of two
              atomicAdd(facc + (t & 1) * (C + 3) + j,
                        (unsigned long long)llrint(((double)gs.x + (double)gs.y) * gscale));
          } else {
            I.gcta[(size_t)blockIdx.x * C + j] = gs;
          }
        }
      }
    }
    // barrier 1: arrive now, wait after the work that does not need g_hat
    fused_arrive(I.bar);
    bar_target += gridDim.x;
    // e_lj = K_ll - 2 f_hat_lj for this thread's column (d_lj = e_lj + g_hat_j)
    if (mine) {
      for (int j = 0; j < C; ++j) {
        if (nj_sh[j] == 0) {
          if (fhat_out) fhat_out[(int64_t)l * C + j] = __int_as_float(0x7fc00000);
          continue;
        }
        float* fp = slots + (size_t)first_sh[j] * gmax * NC + q;
        const float fh = *fp / (float)nj_sh[j];
        if (fhat_out) fhat_out[(int64_t)l * C + j] = fh;
        *fp = ks - 2.0f * fh;
      }
    }
    if (!fused_wait(I.bar, bar_target, I.err, &ok_sh)) break;  // KKM_ETIMEOUT on the host
    // g_hat of every cluster (Eq. 16), the same value in every CTA
    if (fixed) {
      for (int j = tid; j < C; j += kFusedThreads) {
        const int n = nj_sh[j];
        double gv = __longlong_as_double(0x7ff8000000000000LL);
        if (n > 0)
          gv = I.ghat_in ? I.ghat_in[j]
                         : (double)__ldcg(facc + (t & 1) * (C + 3) + j) / gscale / ((double)n * (double)n);
        gh_sh[j] = gv;
        ghf_sh[j] = (float)gv;
      }
      // the other set's counters were last read before barrier 1: zero them
      // for the next iteration (published by barrier 2)
      if (blockIdx.x == 0)
        for (int e = tid; e < C + 3; e += kFusedThreads) facc[((t + 1) & 1) * (C + 3) + e] = 0ull;
    } else {
      // one warp per cluster: the CTA shares, lane b taking CTAs b, b + 32,
      // ... (all loads in flight at once), then a fixed xor tree
      for (int j = w; j < C; j += kFusedWarps) {
        const int n = nj_sh[j];
        float2 v[kFusedCtaPerLane];
#pragma unroll
        for (int m = 0; m < kFusedCtaPerLane; ++m) {
          const int b = lane + 32 * m;
          v[m] = (n > 0 && b < (int)gridDim.x) ? __ldcg(I.gcta + (size_t)b * C + j) : make_float2(0.0f, 0.0f);
        }
        float2 a2 = v[0];
#pragma unroll
        for (int m = 1; m < kFusedCtaPerLane; ++m) a2 = df_add(a2, v[m]);
        a2 = warp_sum_df(a2);
        if (lane == 0) {
          double gv = __longlong_as_double(0x7ff8000000000000LL);
          if (n > 0) gv = I.ghat_in ? I.ghat_in[j] : ((double)a2.x + (double)a2.y) / ((double)n * (double)n);
          gh_sh[j] = gv;
          ghf_sh[j] = (float)gv;
        }
      }
    }
    __syncthreads();
    if (blockIdx.x == 0 && ghat_out)
      for (int j = tid; j < C; j += kFusedThreads) ghat_out[j] = gh_sh[j];

    // ---- phase B: one column per thread
    float best = inf, second = inf;
    int bj = 0;
    bool flagged = false;
    if (mine) {
      for (int j = 0; j < C; ++j) {
        if (nj_sh[j] == 0) continue;
        float* fp = slots + (size_t)first_sh[j] * gmax * NC + q;
        const float dj = *fp + ghf_sh[j];
        *fp = dj;  // the slot now holds d_lj
        if (dj < best) {  // lowest j on ties
          second = best;
          best = dj;
          bj = j;
        } else if (dj < second) {
          second = dj;
        }
      }
      if (R.Xi && I.flag_tau > 0.0f && second < inf)
        flagged = (second - best) < I.flag_tau * fmaxf(fabsf(second), ks + ghf_sh[bj]);
    }
    // near-tie re-score: candidate (column, cluster) pairs of the flagged
    // columns, each re-scored by one warp from exact FP32 kernel values of
    // its support (one landmark per lane, then a fixed xor tree); pairs are
    // listed in rounds of kFusedCandCap in (column, cluster) order
    if (__syncthreads_or(flagged)) {
      const float b0 = best, scale = ks + ghf_sh[bj];
      auto is_cand = [&](int j) {
        if (nj_sh[j] == 0) return false;
        const float dj = slots[(size_t)first_sh[j] * gmax * NC + q];
        return dj - b0 < I.flag_tau * fmaxf(fabsf(dj), scale);
      };
      int cnt = 0;
      if (flagged)
        for (int j = 0; j < C; ++j) cnt += is_cand(j);
      int total;
      const int off = block_excl_scan(cnt, scan_sh, &total);
      for (int cbase = 0; cbase < total; cbase += kFusedCandCap) {
        if (flagged && off + cnt > cbase && off < cbase + kFusedCandCap) {
          int k = off;
          for (int j = 0; j < C; ++j)
            if (is_cand(j)) {
              if (k >= cbase && k < cbase + kFusedCandCap) cand[k - cbase] = (q << 8) | j;
              ++k;
            }
        }
        __syncthreads();
        const int np = min(kFusedCandCap, total - cbase);
        for (int p = w; p < np; p += kFusedWarps) {
          const int qq = cand[p] >> 8, j = cand[p] & 255;
          const int ir = col0 + qq;
          const float4* xi = reinterpret_cast<const float4*>(R.Xi + (int64_t)ir * R.dp);
          const float ni = R.nXi[ir];
          const float ksr = kself ? kself[ir] : 1.0f;
          const int k0 = seg_sh[j], k1 = seg_sh[j + 1];
          float accr = 0.0f;
          for (int kk = k0 + lane; kk < k1; kk += 32) {
            const int k = perm_in_sh ? perm_sh[kk] : __ldcg(S.perm + kk);
            const float4* xl = reinterpret_cast<const float4*>(R.XL + (int64_t)k * R.dp);
            // in chunks of 32 products (see the Gram kernel: one long FP32 sum drifts)
            float dot = 0.0f, part = 0.0f;
            for (int c = 0; c < (R.dp >> 2); ++c) {
              const float4 a4 = __ldg(xi + c), b4 = __ldg(xl + c);
              part = fmaf(a4.x, b4.x, fmaf(a4.y, b4.y, fmaf(a4.z, b4.z, fmaf(a4.w, b4.w, part))));
              if ((c & 7) == 7) {
                dot += part;
                part = 0.0f;
              }
            }
            dot += part;
            float kv;
            if (R.kind == DK_LINEAR) kv = dot;
            else kv = (S.L[k] == ir) ? 1.0f : exp2f(fmaxf(ni + R.nXL[k] - 2.0f * dot, 0.0f) * R.neg_scale);
            accr += kv;
          }
          accr = warp_sum_f32(accr);
          if (lane == 0)
            slots[(size_t)first_sh[j] * gmax * NC + qq] = ksr - 2.0f * (accr / (float)(k1 - k0)) + ghf_sh[j];
        }
        __syncthreads();
      }
      if (flagged) {  // argmin and margin over the updated distances
        best = inf;
        second = inf;
        for (int j = 0; j < C; ++j) {
          if (nj_sh[j] == 0) continue;
          const float dj = slots[(size_t)first_sh[j] * gmax * NC + q];
          if (dj < best) {
            second = best;
            best = dj;
            bj = j;
          } else if (dj < second) {
            second = dj;
          }
        }
      }
    }
    float2 om = make_float2(0.0f, 0.0f);
    int ch = 0, lmc = 0;
    if (mine) {
      ch = cur_u != bj;
      cur_u = bj;
      if (cord >= 0 && ch) {  // read by the support sort (CTA 0)
        S.lab[cord] = bj;
        lmc = 1;
      }
      if (margin) margin[l] = second - best;
      om.x = best;
    }
    // this CTA's cost and counts, in a fixed order
    om = warp_sum_df(om);
    ch = warp_sum_i32(ch);
    lmc = warp_sum_i32(lmc);
    if (lane == 0) {
      wom[w] = om;
      wch[w] = ch;
      wlm[w] = lmc;
    }
    __syncthreads();
    if (tid == 0) {
      float2 o = wom[0];
      int c = wch[0], lm = wlm[0];
      for (int k = 1; k < kFusedWarps; ++k) {
        o = df_add(o, wom[k]);
        c += wch[k];
        lm += wlm[k];
      }
      if (fixed) {
        unsigned long long* a = facc + (t & 1) * (C + 3) + C;
        // two's complement: a slightly negative share (rounding of d ~ 0) adds correctly
        atomicAdd(a, (unsigned long long)llrint(((double)o.x + (double)o.y) * oscale));
        if (c) atomicAdd(a + 1, (unsigned long long)c);
        if (lm) atomicAdd(a + 2, (unsigned long long)lm);
      } else {
        I.omega_part[blockIdx.x] = o;
        I.changed_part[blockIdx.x] = c;
        I.lm_part[blockIdx.x] = lm;
      }
    }
    fused_arrive(I.bar);
    bar_target += gridDim.x;
    if (!fused_wait(I.bar, bar_target, I.err, &ok_sh)) break;
    // ---- phase C: the iteration's cost and counts (the same in every CTA),
    // the trace, early stop, supports
    if (fixed) {
      if (tid == 0) {
        const unsigned long long* a = facc + (t & 1) * (C + 3) + C;
        tot_om = (double)(long long)__ldcg(a) / oscale;
        tot_ch = (int)__ldcg(a + 1);
        tot_lm = (int)__ldcg(a + 2);
      }
    } else if (w == 0) {
      float2 ov[kFusedCtaPerLane];
      int cv[kFusedCtaPerLane], lv[kFusedCtaPerLane];
#pragma unroll
      for (int m = 0; m < kFusedCtaPerLane; ++m) {
        const int b = lane + 32 * m;
        const bool in = b < (int)gridDim.x;
        ov[m] = in ? __ldcg(I.omega_part + b) : make_float2(0.0f, 0.0f);
        cv[m] = in ? __ldcg(I.changed_part + b) : 0;
        lv[m] = in ? __ldcg(I.lm_part + b) : 0;
      }
      float2 o = ov[0];
      int c = cv[0], lm = lv[0];
#pragma unroll
      for (int m = 1; m < kFusedCtaPerLane; ++m) {
        o = df_add(o, ov[m]);
        c += cv[m];
        lm += lv[m];
      }
      o = warp_sum_df(o);
      c = warp_sum_i32(c);
      lm = warp_sum_i32(lm);
      if (lane == 0) {
        tot_om = (double)o.x + (double)o.y;
        tot_ch = c;
        tot_lm = lm;
      }
    }
    __syncthreads();
    if (blockIdx.x == 0 && tid == 0) {
      I.trace_omega[t0 + t] = tot_om;
      I.trace_changed[t0 + t] = tot_ch;
    }
    const bool stop = early_stop && tot_ch == 0;
    const int lm_total = tot_lm;
    __syncthreads();  // every thread has read the totals before they are rewritten
    if (stop) {
      ++t;
      break;
    }
    if (lm_total > 0) {
      // a landmark label changed: CTA 0 re-sorts the supports (the copies in
      // flight follow the old order and are replaced after the reload)
      if (blockIdx.x == 0) {
        cp_async_wait<0>();
        __syncthreads();
        int* const scr = reinterpret_cast<int*>(slots);  // the slots are free now
        sort_supports_cta(S, scr, scr + C, scr + 2 * C, scr + 2 * C + kFusedWarps * C);
      }
      if (t + 1 < iters) {  // barrier 3 publishes the new supports to every CTA
        fused_arrive(I.bar);
        bar_target += gridDim.x;
        if (!fused_wait(I.bar, bar_target, I.err, &ok_sh)) break;
        reload = true;
      }
    }
  }
  cp_async_wait<0>();  // no copy is left in flight at exit
  if (mine) u[l] = cur_u;
  if (blockIdx.x == 0 && tid == 0) {
    *I.trace_count = t0 + t;
    if (early_stop && t < iters) *I.done = 1;
  }
}

// Grid and shared memory of the fused loop for a block of Ni columns of
// `esize`-byte values and nL landmark rows; false when it does not apply
// (more than kFusedMaxC clusters, or a strip wider than one column per thread
// with one CTA per SM).
bool fused_shape(int Ni, int nL, int C, int esize, int n_sms, FusedShape* F, size_t* smem) {
  if (C > kFusedMaxC || Ni < 1 || nL < 1) return false;
  const int NC = 16 / esize;
  F->groups = (int)ceil_div(Ni, NC);
  F->n_cta = std::max(1, std::min(std::min(n_sms, 32 * kFusedCtaPerLane), (int)ceil_div(F->groups, 4)));
  F->gmax = (int)ceil_div(F->groups, F->n_cta);
  if (F->gmax * NC > kFusedThreads) return false;
  F->R = std::max(1, std::min(kFusedThreads / F->gmax, nL));
  size_t words = fused_ring_offset(F->R, C, F->gmax, NC, nL <= kFusedPermCap ? nL : 0) +
                 (size_t)kFusedDepth * kFusedThreads * 4;
  const size_t sort_words = (size_t)(2 + kFusedWarps) * C + 32;
  words = std::max(words, sort_words);
  *smem = words * sizeof(float);
  return *smem <= (size_t)kFusedMaxDynSmem;
}

template <typename T>
static cudaError_t launch_iterate_t(const T* KT, int64_t ldk, int Ni, const Supports& S, const IterState& I,
                                    int iters, const float* kself, int32_t* u, float* margin, float* fhat_out,
                                    double* ghat_out, int early_stop, int n_sms, cudaStream_t st,
                                    const RescoreArgs& R) {
  if (iters <= 0) return cudaSuccess;
  FusedShape F;
  size_t smem = 0;
  if (!fused_shape(Ni, S.nL, S.C, (int)sizeof(T), n_sms, &F, &smem)) return cudaErrorInvalidValue;
  if (F.n_cta > I.fused_cap) return cudaErrorInvalidValue;  // gcta / per-CTA slot capacity
  static const cudaError_t attr = cudaFuncSetAttribute(iterate_fused_kernel<T>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       kFusedMaxDynSmem);
  if (attr != cudaSuccess) return attr;
  // the barrier counter and the fixed-point accumulators start at zero in
  // every launch
  cudaError_t e = cudaMemsetAsync(I.bar, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(I.facc, 0, sizeof(unsigned long long) * fused_acc_words(S.C), st);
  if (e != cudaSuccess) return e;
  IterState J = I;
  // cost shares as fixed point: |Omega| <= 4 Ni for the Gaussian kernels
  int b = 0;
  while (b < 40 && ((int64_t)1 << b) <= Ni) ++b;  // Ni < 2^b
  J.fom_shift = std::max(8, 60 - b);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)F.n_cta);
  cfg.blockDim = dim3(kFusedThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attrs[1];
  attrs[0].id = cudaLaunchAttributeCooperative;
  attrs[0].val.cooperative = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, iterate_fused_kernel<T>, KT, ldk, Ni, S, J, F, iters, kself, u, margin, fhat_out,
                            ghat_out, early_stop, R);
}
cudaError_t launch_iterate(const float* KT, int64_t ldk, int Ni, const Supports& S, const IterState& I, int iters,
                           const float* kself, int32_t* u, float* margin, float* fhat_out, double* ghat_out,
                           int early_stop, int n_sms, cudaStream_t st, const RescoreArgs& R) {
  return launch_iterate_t(KT, ldk, Ni, S, I, iters, kself, u, margin, fhat_out, ghat_out, early_stop, n_sms, st,
                          R);
}
cudaError_t launch_iterate(const __half* KT, int64_t ldk, int Ni, const Supports& S, const IterState& I, int iters,
                           const float* kself, int32_t* u, float* margin, float* fhat_out, double* ghat_out,
                           int early_stop, int n_sms, cudaStream_t st, const RescoreArgs& R) {
  return launch_iterate_t(KT, ldk, Ni, S, I, iters, kself, u, margin, fhat_out, ghat_out, early_stop, n_sms, st,
                          R);
}

// ----------------------------------------------------- Eq. 8 nearest medoid
__global__ void nearest_kernel(const float* __restrict__ Kt, int64_t ldk, int Ni, int C,
                               const float* __restrict__ kself, const float* __restrict__ kmm,
                               int32_t* __restrict__ u, float* __restrict__ dmin) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Ni) return;
  const float ks = kself ? kself[i] : 1.0f;
  float best = __int_as_float(0x7f800000);
  int bj = 0;
  for (int j = 0; j < C; ++j) {
    const float dj = ks - 2.0f * Kt[(int64_t)j * ldk + i] + (kmm ? kmm[j] : 1.0f);
    if (dj < best) {
      best = dj;
      bj = j;
    }
  }
  u[i] = bj;
  if (dmin) dmin[i] = best;
}

cudaError_t launch_nearest(const float* Kt, int64_t ldk, int Ni, int C, const float* kself,
                           const float* kmm, int32_t* u, float* dmin, cudaStream_t st) {
  if (Ni <= 0) return cudaSuccess;
  nearest_kernel<<<(unsigned)ceil_div(Ni, 256), 256, 0, st>>>(Kt, ldk, Ni, C, kself, kmm, u, dmin);
  return cudaGetLastError();
}

// ---------------------------------------------------- Eq. 10 medoid keys
__global__ void __launch_bounds__(kAssignThreads)
medoid_keys_kernel(int64_t ldk, int Ni, Supports S, IterState I, const float* __restrict__ kself,
                   const int32_t* __restrict__ u, unsigned long long* __restrict__ keys,
                   int32_t* __restrict__ c, double* __restrict__ ghat_out) {
  __shared__ AssignShared sh;
  __shared__ unsigned long long bkey[kMaxC];
  __shared__ int bcnt[kMaxC];
  const int C = S.C;
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    bkey[j] = ~0ull;
    bcnt[j] = 0;
  }
  load_cluster_stats(sh, S, I);
  if (blockIdx.x == 0 && ghat_out)
    for (int j = threadIdx.x; j < C; j += blockDim.x) ghat_out[j] = sh.gh[j];
  for (int i = blockIdx.x * kAssignThreads + threadIdx.x; i < Ni; i += gridDim.x * kAssignThreads) {
    const float ks = kself ? kself[i] : 1.0f;
    atomicAdd(&bcnt[u[i]], 1);
    for (int j = 0; j < C; ++j) {
      if (sh.nj[j] == 0) continue;
      const float v = ks - 2.0f * fhat_of(sh, I.partial, ldk, i, j);
      atomicMin(&bkey[j], pack_key(v, (uint32_t)i));
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    if (bkey[j] != ~0ull) atomicMin(keys + j, bkey[j]);
    if (bcnt[j]) atomicAdd(c + j, bcnt[j]);
  }
}

cudaError_t launch_medoid_keys(int64_t ldk, int Ni, const Supports& S, const IterState& I,
                               const float* kself, const int32_t* u, unsigned long long* keys,
                               int32_t* c, double* ghat_out, cudaStream_t st) {
  medoid_keys_kernel<<<I.assign_grid, kAssignThreads, 0, st>>>(ldk, Ni, S, I, kself, u, keys, c,
                                                              ghat_out);
  return cudaGetLastError();
}

// With reset, the key slot is left at ~0 for the next min-reduction (the
// Eq. 12 merge keys).
__global__ void medoid_pick_kernel(unsigned long long* __restrict__ keys, const int32_t* __restrict__ c,
                                   const int32_t* __restrict__ n_j, int C, int32_t* __restrict__ mi, int reset) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= C) return;
  const unsigned long long key = keys[j];
  mi[j] = (c[j] > 0 && n_j[j] > 0 && key != ~0ull) ? (int32_t)(key & 0xffffffffull) : -1;
  if (reset) keys[j] = ~0ull;
}

cudaError_t launch_medoid_pick(unsigned long long* keys, const int32_t* c, const int32_t* n_j, int C, int32_t* mi,
                               cudaStream_t st, bool reset_keys) {
  medoid_pick_kernel<<<(unsigned)ceil_div(C, 256), 256, 0, st>>>(keys, c, n_j, C, mi, reset_keys ? 1 : 0);
  return cudaGetLastError();
}

// ----------------------------------------------------------- Eq. 12 merge
__global__ void __launch_bounds__(256)
merge_keys_kernel(const float* __restrict__ Kt, const float* __restrict__ Kmi, int64_t ldk, int Ni,
                  int C, const float* __restrict__ kself, const int32_t* __restrict__ mi,
                  const int32_t* __restrict__ c, const int64_t* __restrict__ W,
                  unsigned long long* __restrict__ keys) {
  __shared__ unsigned long long bkey[kMaxC];
  __shared__ float alpha[kMaxC];
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    bkey[j] = ~0ull;
    alpha[j] = mi[j] >= 0 ? (float)((double)c[j] / ((double)c[j] + (double)W[j])) : 0.0f;
  }
  __syncthreads();
  // clusters in groups of 8: each thread's minimum over its samples (the
  // group's 16 loads of a sample in flight together), then the warp's (a min
  // is order-free: the same key whatever the split)
  constexpr int G = 8;
  for (int j0 = 0; j0 < C; j0 += G) {
    unsigned long long kmin[G];
#pragma unroll
    for (int q = 0; q < G; ++q) kmin[q] = ~0ull;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < Ni; l += gridDim.x * blockDim.x) {
      const float ks = kself ? kself[l] : 1.0f;
      float kt[G], km[G];
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const int j = j0 + q;
        kt[q] = j < C ? Kt[(int64_t)j * ldk + l] : 0.0f;
        km[q] = j < C ? Kmi[(int64_t)j * ldk + l] : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const int j = j0 + q;
        if (j < C && mi[j] >= 0) {
          const float a = alpha[j];
          const float v = ks - 2.0f * (1.0f - a) * kt[q] - 2.0f * a * km[q];
          const unsigned long long k = pack_key(v, (uint32_t)l);
          kmin[q] = k < kmin[q] ? k : kmin[q];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < G; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(kFull, kmin[q], o);
        kmin[q] = y < kmin[q] ? y : kmin[q];
      }
      if ((threadIdx.x & 31) == 0 && j0 + q < C && kmin[q] != ~0ull) atomicMin(&bkey[j0 + q], kmin[q]);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < C; j += blockDim.x)
    if (bkey[j] != ~0ull) atomicMin(keys + j, bkey[j]);
}

cudaError_t launch_merge_keys(const float* Kt, const float* Kmi, int64_t ldk, int Ni, int C,
                              const float* kself, const int32_t* mi, const int32_t* c,
                              const int64_t* W, unsigned long long* keys, cudaStream_t st) {
  const int grid = (int)std::min<int64_t>(ceil_div(Ni, 256), 152 * 4);
  merge_keys_kernel<<<grid, 256, 0, st>>>(Kt, Kmi, ldk, Ni, C, kself, mi, c, W, keys);
  return cudaGetLastError();
}

// prev (nullable) gets the medoids before the update.
__global__ void merge_apply_kernel(const unsigned long long* __restrict__ keys,
                                   const int32_t* __restrict__ mi, const int32_t* __restrict__ c,
                                   int C, int64_t start, int64_t step, int64_t* __restrict__ M,
                                   int64_t* __restrict__ W, int64_t* __restrict__ prev) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= C) return;
  if (prev) prev[j] = M[j];
  if (mi[j] < 0) return;
  const int64_t l = (int64_t)(keys[j] & 0xffffffffull);
  M[j] = start + l * step;
  W[j] += c[j];
}

cudaError_t launch_merge_apply(const unsigned long long* keys, const int32_t* mi, const int32_t* c,
                               int C, int64_t start, int64_t step, int64_t* M, int64_t* W,
                               cudaStream_t st, int64_t* prev) {
  merge_apply_kernel<<<(unsigned)ceil_div(C, 256), 256, 0, st>>>(keys, mi, c, C, start, step, M, W, prev);
  return cudaGetLastError();
}

// ------------------------------------------- centre displacement (Fig. 4b)
// out = mean over j of the feature-space distance between the medoid before
// (old[j]) and after (cur[j]) a mini-batch: sqrt(max(0, K(a,a) - 2K(a,b) +
// K(b,b))) from the C x C block K[a][b] = K(old_a, cur_b) (self terms 1 for
// the Gaussian kernels, the squared norms selfA/selfB for the linear one); an
// unchanged medoid contributes 0 exactly.  One CTA; a fixed-order sum.
__global__ void __launch_bounds__(256) displacement_kernel(const float* __restrict__ K, int64_t ldk, int C,
                                                          const float* __restrict__ selfA,
                                                          const float* __restrict__ selfB,
                                                          const int64_t* __restrict__ old,
                                                          const int64_t* __restrict__ cur, double* __restrict__ out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int j = threadIdx.x; j < C; j += blockDim.x) {
    if (old[j] == cur[j]) continue;
    const double ka = selfA ? (double)selfA[j] : 1.0, kb = selfB ? (double)selfB[j] : 1.0;
    const double d2 = ka - 2.0 * (double)K[(int64_t)j * ldk + j] + kb;
    s += sqrt(d2 > 0.0 ? d2 : 0.0);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s / (double)C;
}

cudaError_t launch_displacement(const float* K, int64_t ldk, int C, const float* selfA, const float* selfB,
                                const int64_t* old, const int64_t* cur, double* out, cudaStream_t st) {
  displacement_kernel<<<1, 256, 0, st>>>(K, ldk, C, selfA, selfB, old, cur, out);
  return cudaGetLastError();
}

// ------------------- Eq. 10 medoid rows, and the displacement from rows
// Per cluster j (one warp each): mi[j] = the local index of the Eq. 10
// medoid (-1 when empty), the Eq. 10 key reset to ~0 for the merge keys,
// mi_safe[j] (0 for an empty cluster), idMI[j] its global id (-1 when empty),
// and its prepared row and norm copied from the mini-batch's rows (the values
// a gather of that row would give).
__global__ void medoid_rows_kernel(unsigned long long* __restrict__ keys, const int32_t* __restrict__ c,
                                   const int32_t* __restrict__ n_j, int C, int32_t* __restrict__ mi,
                                   int32_t* __restrict__ mi_safe, const float4* __restrict__ Xi,
                                   const float* __restrict__ aux_i, int dp4, const int64_t* __restrict__ gid,
                                   float4* __restrict__ MIX, float* __restrict__ auxMI, int64_t* __restrict__ idMI) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= C) return;
  const unsigned long long key = keys[j];
  const int m = (c[j] > 0 && n_j[j] > 0 && key != ~0ull) ? (int)(key & 0xffffffffull) : -1;
  const int ms = m >= 0 ? m : 0;
  // four 16-byte loads in flight per lane before the stores
  for (int q0 = lane; q0 < dp4; q0 += 128) {
    float4 t[4];
#pragma unroll
    for (int v = 0; v < 4; ++v)
      if (q0 + 32 * v < dp4) t[v] = Xi[(int64_t)ms * dp4 + q0 + 32 * v];
#pragma unroll
    for (int v = 0; v < 4; ++v)
      if (q0 + 32 * v < dp4) MIX[(int64_t)j * dp4 + q0 + 32 * v] = t[v];
  }
  __syncwarp();
  if (lane == 0) {
    mi[j] = m;
    mi_safe[j] = ms;
    keys[j] = ~0ull;
    auxMI[j] = aux_i[ms];
    idMI[j] = m >= 0 ? gid[m] : -1;
  }
}

cudaError_t launch_medoid_rows(unsigned long long* keys, const int32_t* c, const int32_t* n_j, int C, int32_t* mi,
                               int32_t* mi_safe, const float* Xi, const float* aux_i, int dp, const int64_t* gid,
                               float* MIX, float* auxMI, int64_t* idMI, cudaStream_t st) {
  if (dp % 4 != 0) return cudaErrorInvalidValue;
  medoid_rows_kernel<<<(unsigned)ceil_div(C, 8), 256, 0, st>>>(keys, c, n_j, C, mi, mi_safe,
                                                               reinterpret_cast<const float4*>(Xi), aux_i, dp / 4,
                                                               gid, reinterpret_cast<float4*>(MIX), auxMI, idMI);
  return cudaGetLastError();
}

// The displacement of a mini-batch (as displacement_kernel) from the rows:
// the medoid before is MX[j] (global id old[j]); after the merge it is
// cur[j], the mini-batch's local row (keys[j] & 0xffffffff) when mi[j] >= 0
// and it moved.  K(a, b) = exp2(|a - b|^2 neg_scale) (Gaussian, self terms 1)
// or a.b (linear, self terms the squared norms auxM, aux_i), |a - b|^2 and
// a.b summed lane-strided over 16-byte vectors, then a fixed xor tree.  The
// next mini-batch's medoid rows are written as well: NX[j] = the row after.
// One warp per cluster (up to 32 warps; more clusters take turns), eight
// 16-byte loads in flight per lane; the launch width changes no sum (thread
// j holds cluster j's value for the block sum, the other slots are zero).
constexpr int kDispMaxWarps = 32;
__global__ void __launch_bounds__(kDispMaxWarps * 32)
displacement_rows_kernel(const float4* __restrict__ MX, const float* __restrict__ auxM,
                         const float4* __restrict__ Xi, const float* __restrict__ aux_i, int dp4, int C,
                         const unsigned long long* __restrict__ keys, const int32_t* __restrict__ mi,
                         const int64_t* __restrict__ old, const int64_t* __restrict__ cur, int linear,
                         float neg_scale, double* __restrict__ out, float4* __restrict__ NX, float* __restrict__ nauxM) {
  __shared__ double val[kMaxC];
  __shared__ double red[kDispMaxWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = w; j < C; j += nw) {
    const bool moved = mi[j] >= 0 && old[j] != cur[j];
    const int l = moved ? (int)(keys[j] & 0xffffffffull) : 0;
    const float4* a = MX + (int64_t)j * dp4;
    const float4* b = Xi + (int64_t)l * dp4;
    float acc = 0.0f;
    for (int q0 = lane; q0 < dp4; q0 += 128) {
      float4 xs[4], ys[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int q = q0 + 32 * v;
        if (q < dp4) {
          xs[v] = a[q];
          ys[v] = moved ? b[q] : xs[v];
        }
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int q = q0 + 32 * v;
        if (q < dp4) {
          const float4 x = xs[v], y = ys[v];
          NX[(int64_t)j * dp4 + q] = y;
          if (linear) {
            acc = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, acc))));
          } else {
            const float e0 = x.x - y.x, e1 = x.y - y.y, e2 = x.z - y.z, e3 = x.w - y.w;
            acc = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, acc))));
          }
        }
      }
    }
    acc = warp_sum_f32(acc);
    if (lane == 0) {
      const float kb_f = moved ? aux_i[l] : auxM[j];
      nauxM[j] = kb_f;
      double v = 0.0;
      if (moved) {
        const double k = linear ? (double)acc : (double)exp2f(acc * neg_scale);
        const double ka = linear ? (double)auxM[j] : 1.0, kb = linear ? (double)kb_f : 1.0;
        const double d2 = ka - 2.0 * k + kb;
        v = sqrt(d2 > 0.0 ? d2 : 0.0);
      }
      val[j] = v;
    }
  }
  __syncthreads();
  double s = 0.0;
  for (int j = threadIdx.x; j < C; j += blockDim.x) s += val[j];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s / (double)C;
}

cudaError_t launch_displacement_rows(const float* MX, const float* auxM, const float* Xi, const float* aux_i, int dp,
                                     int C, const unsigned long long* keys, const int32_t* mi, const int64_t* old,
                                     const int64_t* cur, bool linear, float neg_scale, double* out, float* NX,
                                     float* nauxM, cudaStream_t st) {
  if (dp % 4 != 0 || C > kMaxC) return cudaErrorInvalidValue;
  const int warps = std::min(std::max(C, 1), kDispMaxWarps);
  displacement_rows_kernel<<<1, 32 * warps, 0, st>>>(reinterpret_cast<const float4*>(MX), auxM,
                                              reinterpret_cast<const float4*>(Xi), aux_i, dp / 4, C, keys, mi, old,
                                              cur, linear ? 1 : 0, neg_scale, out, reinterpret_cast<float4*>(NX),
                                              nauxM);
  return cudaGetLastError();
}

// ------------------------------------------------------------- small utils
__global__ void scatter_labels_kernel(const int32_t* __restrict__ u, int Ni, int64_t start,
                                      int64_t step, int32_t* __restrict__ out) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < Ni) out[start + (int64_t)l * step] = u[l];
}
cudaError_t launch_scatter_labels(const int32_t* u, int Ni, int64_t start, int64_t step,
                                  int32_t* labels_out, cudaStream_t st) {
  if (Ni <= 0) return cudaSuccess;
  scatter_labels_kernel<<<(unsigned)ceil_div(Ni, 256), 256, 0, st>>>(u, Ni, start, step, labels_out);
  return cudaGetLastError();
}

template <typename T>
__global__ void fill_kernel(T* p, T v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}
cudaError_t launch_fill_u64(unsigned long long* p, unsigned long long v, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  fill_kernel<unsigned long long><<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, st>>>(p, v, n);
  return cudaGetLastError();
}
cudaError_t launch_fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  fill_kernel<int32_t><<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, st>>>(p, v, n);
  return cudaGetLastError();
}
cudaError_t launch_fill_f32(float* p, float v, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  fill_kernel<float><<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, st>>>(p, v, n);
  return cudaGetLastError();
}

__global__ void local_to_global_kernel(const int32_t* __restrict__ picks, int C, int64_t start,
                                       int64_t step, int64_t* __restrict__ M) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < C) M[j] = start + (int64_t)picks[j] * step;
}
cudaError_t launch_local_to_global(const int32_t* picks, int C, int64_t start, int64_t step,
                                   int64_t* M, cudaStream_t st) {
  local_to_global_kernel<<<(unsigned)ceil_div(C, 256), 256, 0, st>>>(picks, C, start, step, M);
  return cudaGetLastError();
}

// --------------------------------------------------------- k-means++ round
// Round r (1..C-1) of kernel k-means++:
//   kpp_update  D2 <- min(D2, max(0, K_ll - 2K(x_l, m) + K_mm)) with the
//               kernel column of the previous pick, and an FP64 inclusive
//               prefix of D2 inside each 256-row block plus the block totals;
//   kpp_pick    one CTA scans the block totals, takes target = u01 * total
//               and finds the first index whose running sum exceeds it (the
//               lowest unchosen index when the total is 0).
constexpr int kKppThreads = 256;

__global__ void __launch_bounds__(kKppThreads)
kpp_update_kernel(const float* __restrict__ Kc, int N0, const float* __restrict__ kself,
                  double* __restrict__ D2, double* __restrict__ P, double* __restrict__ bsum,
                  const int32_t* __restrict__ picks, int r) {
  __shared__ double wsum[kKppThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int l = blockIdx.x * kKppThreads + tid;
  const int m = picks[r - 1];
  const double km = kself ? (double)kself[m] : 1.0;
  double dv = 0.0;
  if (l < N0) {
    const double ks = kself ? (double)kself[l] : 1.0;
    double v = ks - 2.0 * (double)Kc[l] + km;
    v = v > 0.0 ? v : 0.0;
    dv = (r == 1) ? v : fmin(D2[l], v);
    D2[l] = dv;
  }
  double x = dv;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  double off = 0.0;
  for (int q = 0; q < w; ++q) off += wsum[q];
  if (l < N0) P[l] = off + x;
  if (tid == kKppThreads - 1) bsum[blockIdx.x] = off + x;
}

__global__ void __launch_bounds__(kKppThreads)
kpp_pick_kernel(const double* __restrict__ D2, const double* __restrict__ P,
                const double* __restrict__ bsum, int nb, int N0, int32_t* __restrict__ picks,
                const double* __restrict__ draws, int r) {
  __shared__ double base_sh, total_sh;
  __shared__ int blk;
  const int tid = threadIdx.x;
  if (tid == 0) {
    // running sum over the block totals, in block order
    double run = 0.0;
    for (int b = 0; b < nb; ++b) run += bsum[b];
    total_sh = run;
    blk = -1;
    picks[r] = -1;
    if (run > 0.0) {
      const double target = draws[r] * run;
      double acc = 0.0;
      for (int b = 0; b < nb; ++b) {
        if (acc <= target && acc + bsum[b] > target) {
          blk = b;
          base_sh = acc;
          break;
        }
        acc += bsum[b];
      }
    }
  }
  __syncthreads();
  const double total = total_sh;
  if (total > 0.0 && blk >= 0) {
    // interval [base + P[l-1], base + P[l]) of element l; neighbours share endpoints exactly
    const double target = draws[r] * total;
    const double base = base_sh;
    const int l = blk * kKppThreads + tid;
    if (l < N0) {
      const double hi = base + P[l];
      const double lo = base + (tid > 0 ? P[l - 1] : 0.0);
      if (lo <= target && hi > target) picks[r] = l;
    }
  }
  __syncthreads();
  if (tid == 0 && picks[r] < 0) {
    if (total > 0.0) {  // rounding put the target at the very end
      int l = N0 - 1;
      while (l > 0 && !(D2[l] > 0.0)) --l;
      picks[r] = l;
    } else {
      for (int l = 0; l < N0; ++l) {
        bool taken = false;
        for (int q = 0; q < r; ++q) taken |= (picks[q] == l);
        if (!taken) {
          picks[r] = l;
          break;
        }
      }
    }
  }
}

// One whole round of kernel k-means++ (Alg. 1 lines 4-6) in one launch, for
// the RBF and linear kernels on prepared rows X [N0][dp] (dp a multiple of 8).
// CTA b takes the samples [32 b, 32 b + 32), warp w four of them:
// K(x_m, x_l) against the last pick m (the RBF kernel from direct squared
// differences, the linear one from the dot product; lanes over 16-byte
// chunks of the row, a fixed xor tree), D^2(l) = min over the picks of
// K_ll - 2 K(x_l, m) + K_mm (clamped at 0, FP64) and the running sums of D^2
// within the CTA.  The last CTA to finish (atomic ticket, no waiting) draws
// the next pick: the CTA totals' running sums (a block scan per chunk of 256
// CTAs, chunks in order), target = u * (their total), the first sample whose
// interval [running sum before, running sum after) contains it; if rounding
// put the target at the very end, the last sample with D^2 > 0; if every D^2
// is 0, the lowest sample not picked yet.
constexpr int kKppSamples = 32;  // samples per CTA of the one-launch round

// inclusive scan of one double per thread over the CTA (kKppThreads); sh
// holds kKppThreads / 32 slots
__device__ __forceinline__ double kpp_block_scan(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += y;
  }
  __syncthreads();
  if (lane == 31) sh[w] = v;
  __syncthreads();
  double off = 0.0;
  for (int q = 0; q < w; ++q) off += sh[q];
  return off + v;
}

// One 32-sample group g of a round: the kernel column of the last pick m
// (its row in kpp_row), the D^2 update (from D2in into D2out; the same array
// for the one-launch-per-round kernel), the running sums P of the group and
// its total bsum[g].
__device__ __forceinline__ void kpp_group(const float* __restrict__ X, int dp, int N0, int linear, float neg_scale,
                                          const float* __restrict__ kself, const double* D2in, double* D2out,
                                          double* __restrict__ P, double* __restrict__ bsum, int m, int r, int g,
                                          const float4* kpp_row, float* kv) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int d4 = dp >> 2;
  const int l0 = g * kKppSamples;
  {
    const float4* xl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int l = l0 + 4 * w + q;
      xl[q] = l < N0 ? reinterpret_cast<const float4*>(X + (int64_t)l * dp) : nullptr;
    }
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int c0 = 0; c0 < d4; c0 += 64) {
      float4 v[4][2];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = c0 + 32 * h + lane;
          v[q][h] = (xl[q] && c < d4) ? __ldg(xl[q] + c) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = c0 + 32 * h + lane;
        const float4 b = c < d4 ? kpp_row[c] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 a = v[q][h];
          if (linear) {
            acc[q] = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc[q]))));
          } else {
            const float tx = a.x - b.x, ty = a.y - b.y, tz = a.z - b.z, tw = a.w - b.w;
            acc[q] = fmaf(tx, tx, fmaf(ty, ty, fmaf(tz, tz, fmaf(tw, tw, acc[q]))));
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float a = warp_sum_f32(acc[q]);
      if (lane == 0) {
        const int l = l0 + 4 * w + q;
        kv[4 * w + q] = linear ? a : (l == m ? 1.0f : exp2f(a * neg_scale));
      }
    }
  }
  __syncthreads();
  // D^2 update and running sums within the group (warp 0)
  if (w == 0) {
    const int l = l0 + lane;
    const double km = kself ? (double)kself[m] : 1.0;
    double dv = 0.0;
    if (l < N0) {
      const double ks = kself ? (double)kself[l] : 1.0;
      double v = ks - 2.0 * (double)kv[lane] + km;
      v = v > 0.0 ? v : 0.0;
      dv = (r == 1) ? v : fmin(D2in[l], v);
      D2out[l] = dv;
    }
    double x = dv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (l < N0) P[l] = x;
    if (lane == 31) bsum[g] = x;
  }
}

// The next pick from the groups' running sums (every thread of the CTA
// calls it; the same value in every thread): the group totals' running sums
// (a block scan per chunk of 256 groups, chunks in order), target = u * their
// total, the first sample whose interval [running sum before, running sum
// after) contains it; if rounding put the target at the very end, the last
// sample with D^2 > 0; if every D^2 is 0, the lowest sample not picked yet
// (picks[0..r) in global memory).
__device__ int kpp_pick(int N0, int nb, const double* P, const double* bsum, const double* D2, const int32_t* picks,
                        double u, int r, double* wsh, double* base_sh, double* total_sh, int* blk_sh, int* pick_sh) {
  const int tid = threadIdx.x;
  double run = 0.0;
  for (int b0 = 0; b0 < nb; b0 += kKppThreads) {
    const double v = b0 + tid < nb ? __ldcg(bsum + b0 + tid) : 0.0;
    const double incl = kpp_block_scan(v, wsh);
    if (tid == kKppThreads - 1) *total_sh = incl;
    __syncthreads();
    run += *total_sh;
    __syncthreads();
  }
  if (tid == 0) {
    *blk_sh = -1;
    *pick_sh = -1;
  }
  __syncthreads();
  const double total = run;
  if (total > 0.0) {
    const double target = u * total;
    double before = 0.0;  // running sum of the earlier chunks
    for (int b0 = 0; b0 < nb; b0 += kKppThreads) {
      const double v = b0 + tid < nb ? __ldcg(bsum + b0 + tid) : 0.0;
      const double incl = before + kpp_block_scan(v, wsh);
      const double excl = incl - v;
      if (b0 + tid < nb && excl <= target && incl > target) {
        *blk_sh = b0 + tid;
        *base_sh = excl;
      }
      if (tid == kKppThreads - 1) *total_sh = incl;
      __syncthreads();
      before = *total_sh;
      const bool found = *blk_sh >= 0;
      __syncthreads();
      if (found) break;
    }
    const int blk = *blk_sh;
    if (blk >= 0 && tid < kKppSamples) {
      // interval [base + P[l-1], base + P[l]) of sample l; neighbours share endpoints exactly
      const double base = *base_sh;
      const int l = blk * kKppSamples + tid;
      if (l < N0) {
        const double hi = base + __ldcg(P + l);
        const double lo = base + (tid > 0 ? __ldcg(P + l - 1) : 0.0);
        if (lo <= target && hi > target) *pick_sh = l;
      }
    }
  }
  __syncthreads();
  if (tid == 0 && *pick_sh < 0) {
    if (total > 0.0) {  // rounding put the target at the very end
      int l = N0 - 1;
      while (l > 0 && !(__ldcg(D2 + l) > 0.0)) --l;
      *pick_sh = l;
    } else {
      for (int l = 0; l < N0; ++l) {
        bool taken = false;
        for (int q = 0; q < r; ++q) taken |= (__ldcg(picks + q) == l);
        if (!taken) {
          *pick_sh = l;
          break;
        }
      }
    }
  }
  __syncthreads();
  return *pick_sh;
}

__global__ void __launch_bounds__(kKppThreads)
kpp_fused_round_kernel(const float* __restrict__ X, int dp, int N0, int linear, float neg_scale,
                       const float* __restrict__ kself, double* __restrict__ D2, double* __restrict__ P,
                       double* __restrict__ bsum, int32_t* __restrict__ picks, const double* __restrict__ draws,
                       int r, uint32_t* __restrict__ ticket) {
  extern __shared__ float4 kpp_row[];  // [dp / 4]: the row of the last pick
  __shared__ float kv[kKppSamples];
  __shared__ double wsh[kKppThreads / 32];
  __shared__ double base_sh, total_sh;
  __shared__ int blk_sh, last_sh, pick_sh;
  const int tid = threadIdx.x;
  const int m = picks[r - 1];
  const float4* xm_g = reinterpret_cast<const float4*>(X + (int64_t)m * dp);
  for (int c = tid; c < (dp >> 2); c += kKppThreads) kpp_row[c] = __ldg(xm_g + c);
  __syncthreads();
  kpp_group(X, dp, N0, linear, neg_scale, kself, D2, D2, P, bsum, m, r, (int)blockIdx.x, kpp_row, kv);
  // the last CTA draws the next pick
  __threadfence();
  __syncthreads();
  if (tid == 0) last_sh = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last_sh) return;
  __threadfence();
  const int pick = kpp_pick(N0, (int)gridDim.x, P, bsum, D2, picks, draws[r], r, wsh, &base_sh, &total_sh, &blk_sh,
                            &pick_sh);
  if (tid == 0) {
    picks[r] = pick;
    *ticket = 0u;
  }
}

cudaError_t launch_kpp_fused_round(const float* X, int dp, int N0, bool linear, float neg_scale, const float* kself,
                                   double* D2, double* P, double* bsum, int32_t* picks, const double* draws, int r,
                                   uint32_t* ticket, cudaStream_t st) {
  if ((dp & 7) != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0) return cudaErrorInvalidValue;
  const int nb = (int)ceil_div(N0, kKppSamples);
  const size_t smem = (size_t)dp * sizeof(float);
  if (smem > 48 * 1024) {
    static const cudaError_t e = cudaFuncSetAttribute(kpp_fused_round_kernel,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
  }
  kpp_fused_round_kernel<<<nb, kKppThreads, smem, st>>>(X, dp, N0, linear ? 1 : 0, neg_scale, kself, D2, P, bsum,
                                                        picks, draws, r, ticket);
  return cudaGetLastError();
}

cudaError_t launch_kpp_round(const float* Kc, int N0, const float* kself, double* D2, double* P,
                             double* bsum, int32_t* picks, const double* draws, int r, cudaStream_t st) {
  const int nb = (int)ceil_div(N0, kKppThreads);
  kpp_update_kernel<<<nb, kKppThreads, 0, st>>>(Kc, N0, kself, D2, P, bsum, picks, r);
  kpp_pick_kernel<<<1, kKppThreads, 0, st>>>(D2, P, bsum, nb, N0, picks, draws, r);
  prof_more_launches(1);
  return cudaGetLastError();
}

// -------------------------------------------------------- fixed-order sums
__global__ void sum_partial_kernel(const float* __restrict__ v, int64_t n, double* __restrict__ part) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += (double)v[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
__global__ void sum_final_kernel(const double* __restrict__ part, int parts, double* __restrict__ out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int b = threadIdx.x; b < parts; b += blockDim.x) s += part[b];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}
cudaError_t launch_sum_f32_to_f64(const float* v, int64_t n, double* part, int parts, double* out,
                                  cudaStream_t st) {
  sum_partial_kernel<<<parts, 256, 0, st>>>(v, n, part);
  sum_final_kernel<<<1, 256, 0, st>>>(part, parts, out);
  prof_more_launches(1);
  return cudaGetLastError();
}

}  // namespace kkm
