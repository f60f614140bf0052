// Kernel-block evaluation for feature vectors (Alg. 1 line 3, Section 3.2):
// out[a][b] = kappa(A_a, B_b) with kappa the Gaussian RBF, the linear kernel
// or the plain Euclidean distance (for the bandwidth rule).
//
// The contraction A.B^T runs as an FP32 FFMA register-tiled product (128x128
// CTA tile, 8x8 outputs per thread, double-buffered shared memory) and the
// epilogue forms ||a||^2 + ||b||^2 - 2 a.b, clamps it at 0 and applies the
// exponential.  Squared norms are accumulated in double-float (FP32 pairs)
// once per row by the gather kernels.  A "skinny" kernel covers <= 32 reference rows (medoid
// columns, k-means++ columns) with one warp per sample row.
#include <cuda_fp16.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace kkm {

// ------------------------------------------------------------------ gathers
__global__ void gather_rows_kernel(const float* __restrict__ X, int64_t d, int64_t start,
                                   int64_t step, int64_t n, float* __restrict__ out, int dp,
                                   float* __restrict__ normsq) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const float* src = X + (start + row * step) * d;
  float* dst = out + row * (int64_t)dp;
  float2 acc = make_float2(0.0f, 0.0f);
  for (int c = lane; c < dp; c += 32) {
    float v = c < d ? src[c] : 0.0f;
    dst[c] = v;
    acc = df_add_sq(acc, v);
  }
  acc = warp_sum_df(acc);
  if (normsq && lane == 0) normsq[row] = df_to_float(acc);
}

// One row with 16-byte vectors: d4 source vectors, zero padded to dp4; each
// lane issues up to 8 loads before its first store, and accumulates the
// squared norm of its vectors in column order (double-float), then the warp
// adds the lanes in a fixed order.
__device__ __forceinline__ void copy_row4(const float4* __restrict__ src, int64_t d4, float4* __restrict__ dst,
                                          int dp4, int lane, float* normsq) {
  float2 acc = make_float2(0.0f, 0.0f);
  for (int c0 = 0; c0 < dp4; c0 += 32 * 8) {
    float4 v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int c = c0 + t * 32 + lane;
      v[t] = c < d4 ? __ldg(src + c) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int c = c0 + t * 32 + lane;
      if (c < dp4) {
        dst[c] = v[t];
        acc = df_add_sq(df_add_sq(df_add_sq(df_add_sq(acc, v[t].x), v[t].y), v[t].z), v[t].w);
      }
    }
  }
  acc = warp_sum_df(acc);
  if (normsq && lane == 0) *normsq = df_to_float(acc);
}

// Rows start + l*step with 16-byte vectors (d a multiple of 4, X 16-byte
// aligned): one warp per row.
__global__ void gather_rows4_kernel(const float4* __restrict__ X, int64_t d4, int64_t start,
                                    int64_t step, int64_t n, float4* __restrict__ out, int dp4,
                                    float* __restrict__ normsq) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  copy_row4(X + (start + row * step) * d4, d4, out + row * (int64_t)dp4, dp4, lane, normsq ? normsq + row : nullptr);
}

// Rows X[idx[l]] with 16-byte vectors (row pitch and length multiples of 4,
// X 16-byte aligned): one warp per row.
template <typename IDX>
__global__ void gather_idx4_kernel(const float4* __restrict__ X, int64_t ld4, int64_t d4,
                                   const IDX* __restrict__ idx, int64_t n, float4* __restrict__ out, int dp4,
                                   float* __restrict__ normsq) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  copy_row4(X + (int64_t)idx[row] * ld4, d4, out + row * (int64_t)dp4, dp4, lane, normsq ? normsq + row : nullptr);
}

template <typename IDX>
__global__ void gather_idx_kernel(const float* __restrict__ X, int64_t ld_in, int64_t d,
                                  const IDX* __restrict__ idx, int64_t n, float* __restrict__ out,
                                  int dp, float* __restrict__ normsq) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const int64_t g = (int64_t)idx[row];
  const float* src = X + g * ld_in;
  float* dst = out + row * (int64_t)dp;
  float2 acc = make_float2(0.0f, 0.0f);
  for (int c = lane; c < dp; c += 32) {
    float v = c < d ? src[c] : 0.0f;
    dst[c] = v;
    acc = df_add_sq(acc, v);
  }
  acc = warp_sum_df(acc);
  if (normsq && lane == 0) normsq[row] = df_to_float(acc);
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

cudaError_t launch_gather_rows(const float* X, int64_t d, int64_t start, int64_t step, int64_t n,
                               float* out, int dp, float* normsq, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (d % 4 == 0 && dp % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
      (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
    gather_rows4_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(
        reinterpret_cast<const float4*>(X), d / 4, start, step, n, reinterpret_cast<float4*>(out), dp / 4,
        normsq);
  } else {
    gather_rows_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(X, d, start, step, n, out, dp, normsq);
  }
  return cudaGetLastError();
}
cudaError_t launch_gather_idx64(const float* X, int64_t d, const int64_t* idx, int64_t n,
                                float* out, int dp, float* normsq, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (d % 4 == 0 && dp % 4 == 0 && aligned16(X) && aligned16(out))
    gather_idx4_kernel<int64_t><<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(
        reinterpret_cast<const float4*>(X), d / 4, d / 4, idx, n, reinterpret_cast<float4*>(out), dp / 4, normsq);
  else
    gather_idx_kernel<int64_t><<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(X, d, d, idx, n, out, dp, normsq);
  return cudaGetLastError();
}
cudaError_t launch_gather_idx32(const float* Xp, int dp_in, const int32_t* idx, int64_t n,
                                float* out, int dp, float* normsq, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (dp_in % 4 == 0 && dp % 4 == 0 && aligned16(Xp) && aligned16(out))
    gather_idx4_kernel<int32_t><<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(
        reinterpret_cast<const float4*>(Xp), dp_in / 4, dp_in / 4, idx, n, reinterpret_cast<float4*>(out), dp / 4,
        normsq);
  else
    gather_idx_kernel<int32_t><<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(Xp, dp_in, dp_in, idx, n, out, dp,
                                                                      normsq);
  return cudaGetLastError();
}

__global__ void check_finite_kernel(const float* __restrict__ X, int64_t n, int* flag) {
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(X[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}
// dst[i] = src[i] for i < n and *flag = 1 if any value is NaN or Inf, in one
// pass: src is host memory the GPU reads directly (pinned), so the copy is
// pulled by the SMs with many 16-byte requests in flight rather than pushed
// by a copy engine.  n4 16-byte vectors, then `tail` (< 4) single floats.
__global__ void __launch_bounds__(256)
copy_check_kernel(const float4* src, float4* __restrict__ dst, int64_t n4, const float* src_tail,
                  float* __restrict__ dst_tail, int tail, int* flag) {
  int bad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n4; i0 += 4 * stride) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + u * stride;
      v[u] = i < n4 ? src[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + u * stride;
      if (i < n4) {
        dst[i] = v[u];
        bad |= !isfinite(v[u].x) | !isfinite(v[u].y) | !isfinite(v[u].z) | !isfinite(v[u].w);
      }
    }
  }
  if (blockIdx.x == 0 && (int)threadIdx.x < tail) {
    const float x = src_tail[threadIdx.x];
    dst_tail[threadIdx.x] = x;
    bad |= !isfinite(x);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}
cudaError_t launch_copy_check(const float* src, float* dst, int64_t n, int* flag, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(src) & 15) || (reinterpret_cast<uintptr_t>(dst) & 15)) return cudaErrorInvalidValue;
  const int64_t n4 = n / 4;
  const int tail = (int)(n - 4 * n4);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n4, 256 * 4), 152 * 8));
  copy_check_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const float4*>(src), reinterpret_cast<float4*>(dst), n4,
                                          src + 4 * n4, dst + 4 * n4, tail, flag);
  return cudaGetLastError();
}

// Rows start + l*step of pinned host memory, fetched by the copy engine (a
// strided 2-D copy into rows of dp floats), then one pass over the fetched
// rows: the padding columns zeroed, the squared norms (the arithmetic of
// gather_rows4_kernel, so the rows are those of a device-memory gather bit
// for bit) and *bad set when a value is NaN or Inf.  A fit whose X stays on
// the host so checks every row as its mini-batch is fetched, and the fetch of
// the next mini-batch crosses the link while the current one iterates; the
// copy engine leaves the SMs (and their memory pipes) to the loop beside it.
__global__ void rows_norm_check_kernel(float4* __restrict__ rows, int64_t d4, int dp4, int64_t n,
                                       float* __restrict__ normsq, int* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  float4* r = rows + row * (int64_t)dp4;
  float2 acc = make_float2(0.0f, 0.0f);
  int nonfinite = 0;
  for (int c0 = 0; c0 < dp4; c0 += 32 * 8) {
    float4 v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int c = c0 + t * 32 + lane;
      v[t] = c < d4 ? r[c] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int c = c0 + t * 32 + lane;
      if (c < dp4) {
        if (c >= d4) r[c] = v[t];
        nonfinite |= !isfinite(v[t].x) | !isfinite(v[t].y) | !isfinite(v[t].z) | !isfinite(v[t].w);
        acc = df_add_sq(df_add_sq(df_add_sq(df_add_sq(acc, v[t].x), v[t].y), v[t].z), v[t].w);
      }
    }
  }
  acc = warp_sum_df(acc);
  if (normsq && lane == 0) normsq[row] = df_to_float(acc);
  if (__any_sync(kFull, nonfinite) && lane == 0) atomicOr(bad, 1);
}
cudaError_t launch_gather_rows_pull(const float* X, int64_t d, int64_t start, int64_t step, int64_t n, float* out,
                                    int dp, float* normsq, int* bad, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (d % 4 != 0 || dp % 4 != 0 || !aligned16(X) || !aligned16(out)) return cudaErrorInvalidValue;
  const cudaError_t e = cudaMemcpy2DAsync(out, (size_t)dp * 4, X + start * d, (size_t)(step * d) * 4, (size_t)d * 4,
                                          (size_t)n, cudaMemcpyDefault, st);
  if (e != cudaSuccess) return e;
  rows_norm_check_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(reinterpret_cast<float4*>(out), d / 4, dp / 4, n,
                                                                   normsq, bad);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const float* X, int64_t n, int* flag, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
  check_finite_kernel<<<grid, 256, 0, st>>>(X, n, flag);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- epilogue
template <int KIND>
__device__ __forceinline__ float gram_epilogue(float dot, float na, float nb, bool same,
                                               float neg_scale) {
  if (KIND == DK_LINEAR || KIND == DK_RAW) return dot;
  float d2 = fmaxf(na + nb - 2.0f * dot, 0.0f);
  if (KIND == DK_DIST) return same ? 0.0f : sqrtf(d2);
  return same ? 1.0f : exp2f(d2 * neg_scale);
}

// ------------------------------------------------------- tiled FP32 product
constexpr int TB_M = 128, TB_N = 128, TB_K = 8;
// Kernel values (RBF, linear) accumulate the dot product in chunks: every
// kGramChunkTiles k-tiles (32 terms) the thread's 64 running sums are added
// into a second set kept in shared memory and restart from zero.  One FP32
// running sum over all of K drifts: adding small positive products to an
// ever larger sum rounds them with a bias (measured on k/255-quantised
// rows: about 1e-5 on the squared distance of near pairs, 7e-8 relative on
// their kernel values), which moves the cost Omega by 1e-6 relative where
// d = K_ii - 2 f_hat + g_hat cancels.  Short chunks keep each partial sum
// small; the cost is one shared-memory add per output every 32 products.
constexpr int kGramChunkTiles = 4;
constexpr size_t kGramChunkSmem = sizeof(float) * 64 * 256;   // [64 outputs][256 threads]
template <int KIND>
constexpr bool gram_chunked() { return KIND == DK_RBF || KIND == DK_LINEAR; }

// OutT: float, or __half for a Gaussian block stored in FP16 (values in [0, 1]).
template <int KIND, typename OutT>
__global__ void __launch_bounds__(256, 2)
gram_tiled_kernel(const float* __restrict__ A, int nA, const float* __restrict__ Bm, int nB,
                  int dp, const float* __restrict__ normA, const float* __restrict__ normB,
                  const int64_t* __restrict__ idA, const int64_t* __restrict__ idB,
                  float neg_scale, OutT* __restrict__ out, int64_t ldo, int vec_ok, int upper_only,
                  float* __restrict__ out32) {
  __shared__ __align__(16) float As[2][TB_K][TB_M];
  __shared__ __align__(16) float Bs[2][TB_K][TB_N];
  const int tid = threadIdx.x;
  const int a0 = blockIdx.y * TB_M, b0 = blockIdx.x * TB_N;
  // only the strict upper triangle (b > a) is wanted: tiles wholly at or
  // below the diagonal are skipped (their outputs are left unwritten)
  if (upper_only && b0 + TB_N - 1 <= a0) return;
  // split K (DK_RAW): slice z of gridDim.z takes its share of the k-tiles and
  // stores raw products in out + z * nA * ldo
  const int nk_all = dp / TB_K;
  const int kt0 = (int)((int64_t)nk_all * blockIdx.z / gridDim.z);
  const int nk = (int)((int64_t)nk_all * (blockIdx.z + 1) / gridDim.z) - kt0;
  if (KIND == DK_RAW) out += (int64_t)blockIdx.z * nA * ldo;
  const int lr = tid >> 1, lk = (tid & 1) << 2;
  // Rows past the end re-read the last valid row; their outputs are dropped.
  const float* pa = A + (int64_t)min(a0 + lr, nA - 1) * dp + lk + kt0 * TB_K;
  const float* pb = Bm + (int64_t)min(b0 + lr, nB - 1) * dp + lk + kt0 * TB_K;
  float4 ga = __ldg(reinterpret_cast<const float4*>(pa));
  float4 gb = __ldg(reinterpret_cast<const float4*>(pb));
  As[0][lk + 0][lr] = ga.x; As[0][lk + 1][lr] = ga.y; As[0][lk + 2][lr] = ga.z; As[0][lk + 3][lr] = ga.w;
  Bs[0][lk + 0][lr] = gb.x; Bs[0][lk + 1][lr] = gb.y; Bs[0][lk + 2][lr] = gb.z; Bs[0][lk + 3][lr] = gb.w;
  __syncthreads();

  const int tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  extern __shared__ float chunk_sum[];  // [64][256] when gram_chunked<KIND>()
  bool have_chunk = false;

  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) {
      ga = __ldg(reinterpret_cast<const float4*>(pa + (kt + 1) * TB_K));
      gb = __ldg(reinterpret_cast<const float4*>(pb + (kt + 1) * TB_K));
    }
#pragma unroll
    for (int k = 0; k < TB_K; ++k) {
      const float4 al = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
      const float4 ah = *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]);
      const float4 bl = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
      const float4 bh = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
      const float a[8] = {al.x, al.y, al.z, al.w, ah.x, ah.y, ah.z, ah.w};
      const float b[8] = {bl.x, bl.y, bl.z, bl.w, bh.x, bh.y, bh.z, bh.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nk) {
      const int nx = cur ^ 1;
      As[nx][lk + 0][lr] = ga.x; As[nx][lk + 1][lr] = ga.y; As[nx][lk + 2][lr] = ga.z; As[nx][lk + 3][lr] = ga.w;
      Bs[nx][lk + 0][lr] = gb.x; Bs[nx][lk + 1][lr] = gb.y; Bs[nx][lk + 2][lr] = gb.z; Bs[nx][lk + 3][lr] = gb.w;
    }
    if constexpr (gram_chunked<KIND>()) {
      if ((kt + 1) % kGramChunkTiles == 0 && kt + 1 < nk) {  // close a chunk (not the last one)
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float* p = chunk_sum + (i * 8 + j) * 256 + tid;
            *p = have_chunk ? *p + acc[i][j] : acc[i][j];
            acc[i][j] = 0.0f;
          }
        have_chunk = true;
      }
    }
    __syncthreads();
  }
  if constexpr (gram_chunked<KIND>()) {
    if (have_chunk) {  // the open chunk joins the closed ones
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] += chunk_sum[(i * 8 + j) * 256 + tid];
    }
  }

  // Epilogue: rows a0 + {ty*4+i, 64+ty*4+i}, columns b0 + {tx*4+j, 64+tx*4+j}.
  float nb[8];
  int64_t ib[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int b = b0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
    nb[j] = (KIND != DK_LINEAR && b < nB) ? normB[b] : 0.0f;
    ib[j] = (idB && b < nB) ? idB[b] : -1;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int a = a0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (a >= nA) continue;
    const float na = KIND != DK_LINEAR ? normA[a] : 0.0f;
    const int64_t ia = idA ? idA[a] : -2;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = gram_epilogue<KIND>(acc[i][j], na, nb[j], ia == ib[j], neg_scale);
    OutT* orow = out + (int64_t)a * ldo;
    if constexpr (sizeof(OutT) == 2) {
      // the FP32 values too (the re-score of the FP16-stored block reads them)
      if (out32) {
        float* o32 = out32 + (int64_t)a * ldo;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int b = b0 + h * 64 + tx * 4;
          if (vec_ok && b + 3 < nB) {
            *reinterpret_cast<float4*>(o32 + b) = make_float4(v[h * 4], v[h * 4 + 1], v[h * 4 + 2], v[h * 4 + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (b + q < nB) o32[b + q] = v[h * 4 + q];
          }
        }
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int b = b0 + h * 64 + tx * 4;
      if constexpr (sizeof(OutT) == 4) {
        if (vec_ok && b + 3 < nB) {
          *reinterpret_cast<float4*>(orow + b) = make_float4(v[h * 4], v[h * 4 + 1], v[h * 4 + 2], v[h * 4 + 3]);
          continue;
        }
      } else {
        if (vec_ok && b + 3 < nB) {  // 8-byte store of four FP16 values
          const __half2 lo = __floats2half2_rn(v[h * 4], v[h * 4 + 1]);
          const __half2 hi = __floats2half2_rn(v[h * 4 + 2], v[h * 4 + 3]);
          uint2 u;
          u.x = *reinterpret_cast<const uint32_t*>(&lo);
          u.y = *reinterpret_cast<const uint32_t*>(&hi);
          *reinterpret_cast<uint2*>(orow + b) = u;
          continue;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (b + q < nB) orow[b + q] = OutT(v[h * 4 + q]);
    }
  }
}

// ------------------------------------------------ skinny (<= 32 reference rows)
// Sum over the warp of NA values per lane (NA a power of two <= 32), as a
// reduce-scatter: at each of the first log2(NA) xor steps a lane keeps half
// of its values and adds its partner's copy of them, so NA - 1 + 5 - log2(NA)
// shuffles replace NA full reductions.  Afterwards lane l holds the warp sum
// of value (l >> (5 - log2(NA))).
template <int NA>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[NA], int lane) {
  int o = 16;
#pragma unroll
  for (int m = NA; m > 1; m >>= 1, o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < m / 2; ++i) {
      const float keep = upper ? v[i + m / 2] : v[i];
      const float send = upper ? v[i] : v[i + m / 2];
      v[i] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  float t = v[0];
  for (; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
  return t;
}
template <int NA>
__host__ __device__ constexpr int scatter_shift() {
  return NA >= 32 ? 0 : NA >= 16 ? 1 : NA >= 8 ? 2 : NA >= 4 ? 3 : NA >= 2 ? 4 : 5;
}

// K(A_a, B_b) for nA <= NA reference rows held in shared memory and many
// sample rows.  One warp takes skinny_rows<NA>() sample rows at a time; a
// lane handles the 16-byte vectors q = lane, lane + 32, ... of a row, in that
// order whatever the row count, so the sums do not depend on it.  The kernel
// is bound by instruction issue, not memory (16 warps per SM, the FP32 work
// of nA references per sample value), so:
//  - the FP32 work runs on the paired (float2) instructions: two reference
//    rows per instruction, each half the same IEEE operation on its own
//    values as the scalar form (a - b as a + (-b), which rounds identically),
//    so the sums are those of the scalar form bit for bit;
//  - the reference rows sit in shared memory as pairs, interleaved by
//    component ((a.x, b.x, a.y, b.y), (a.z, b.z, a.w, b.w) per vector;
//    negated for the distance kinds), so one pair load feeds both halves;
//  - the sample vectors reach shared memory by cp.async, two stages per warp,
//    the next step's copies in flight while the current step computes.
// The Gaussian and distance kinds sum the squared differences directly: the
// squared distance does not cancel as |x|^2 + |y|^2 - 2 x.y does for rows far
// from the origin.
// 16-byte asynchronous copy global -> shared (cp.async, L2 only) and its
// group commit / wait (per thread: a thread's wait covers its own copies).
__device__ __forceinline__ void skinny_cp16(float4* dst, const float4* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void skinny_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void skinny_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int NA>
__host__ __device__ constexpr int skinny_rows() {
  return NA <= 16 ? 4 : 2;
}
constexpr int kSkinnyLoadsInFlight = 8;  // 16-byte loads per lane, over the warp's rows
constexpr size_t kSkinnyStageBytes = (size_t)8 * 2 * kSkinnyLoadsInFlight * 32 * 16;  // 8 warps, 2 stages
// shared memory of the reference pairs (an odd count padded with a zero row)
inline size_t skinny_ref_bytes(int64_t nA, int dp) { return (size_t)((nA + 1) / 2) * 2 * dp * sizeof(float); }

template <int KIND, int NA>
__global__ void __launch_bounds__(256)
gram_skinny_kernel(const float* __restrict__ A, int nA, const float* __restrict__ Bm, int nB,
                   int dp, const float* __restrict__ normA, const float* __restrict__ normB,
                   const int64_t* __restrict__ idA, const int64_t* __restrict__ idB,
                   float neg_scale, float* __restrict__ out, int64_t ldo) {
  constexpr int R = skinny_rows<NA>(), QB = kSkinnyLoadsInFlight / R;
  constexpr int NP = NA >= 2 ? NA / 2 : 1;  // reference pairs per lane's accumulators
  constexpr bool kDiff = KIND == DK_RBF || KIND == DK_DIST;
  extern __shared__ float4 As4[];  // [(nA + 1) / 2][dp / 4][2] reference pairs, then the warps' stages
  const int dq = dp >> 2;
  const int np = (nA + 1) / 2;
  const float4* A4 = reinterpret_cast<const float4*>(A);
  {
    // four vector pairs per thread in flight before any store
    const int n2 = np * dq;
    for (int e0 = threadIdx.x; e0 < n2; e0 += 4 * blockDim.x) {
      float4 ra[4], rb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * blockDim.x;
        ra[u] = rb[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (e < n2) {
          const int pr = e / dq, q = e - pr * dq;
          ra[u] = __ldg(A4 + (int64_t)(2 * pr) * dq + q);
          if (2 * pr + 1 < nA) rb[u] = __ldg(A4 + (int64_t)(2 * pr + 1) * dq + q);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < n2) {
          const float sg = kDiff ? -1.0f : 1.0f;  // exact
          As4[2 * e] = make_float4(sg * ra[u].x, sg * rb[u].x, sg * ra[u].y, sg * rb[u].y);
          As4[2 * e + 1] = make_float4(sg * ra[u].z, sg * rb[u].z, sg * ra[u].w, sg * rb[u].w);
        }
      }
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nwarp = blockDim.x >> 5;
  const int a_mine = lane >> scatter_shift<NA>();
  const bool writer = (lane & ((1 << scatter_shift<NA>()) - 1)) == 0 && a_mine < nA;
  // The warp's work is a sequence of items (row group, step of 32 * QB
  // vectors); the sample vectors of item k + 1 are copied to the warp's
  // shared-memory stage (k + 1) & 1 while item k is computed from stage k & 1.
  // Each lane copies and reads only its own 16-byte slots, so the lane's
  // cp.async group wait is the only synchronisation.
  const int warp = threadIdx.x >> 5;
  float4* const stage = As4 + (size_t)np * dq * 2 + (size_t)warp * 2 * R * QB * 32;  // [2][R][QB][32]
  const int first = (blockIdx.x * nwarp + warp) * R, stride = gridDim.x * nwarp * R;
  const int steps = (dq + 32 * QB - 1) / (32 * QB);
  const int groups = first < nB ? (nB - first + stride - 1) / stride : 0;
  const int n_items = groups * steps;
  auto issue = [&](int item) {
    const int b0 = first + (item / steps) * stride, q0 = (item % steps) * 32 * QB;
    float4* st = stage + (item & 1) * R * QB * 32;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4* pb = reinterpret_cast<const float4*>(Bm + (int64_t)min(b0 + r, nB - 1) * dp);
#pragma unroll
      for (int t = 0; t < QB; ++t) {
        const int q = q0 + t * 32 + lane;
        if (q < dq) skinny_cp16(st + (r * QB + t) * 32 + lane, pb + q);
      }
    }
    skinny_commit();
  };
  // acc[r][p] = (sum for reference 2p, sum for reference 2p + 1) of row r
  float2 acc[R][NP];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[r][p] = make_float2(0.0f, 0.0f);
  if (n_items > 0) issue(0);
  for (int item = 0; item < n_items; ++item) {
    if (item + 1 < n_items) {
      issue(item + 1);
      skinny_wait<1>();  // item's copies have landed
    } else {
      skinny_wait<0>();
    }
    const int b0 = first + (item / steps) * stride, q0 = (item % steps) * 32 * QB;
    const float4* st = stage + (item & 1) * R * QB * 32;
#pragma unroll
    for (int t = 0; t < QB; ++t) {
      const int q = q0 + t * 32 + lane;
      if (q >= dq) break;
      float4 x[R];
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = st[(r * QB + t) * 32 + lane];
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        if (2 * p < nA) {
          const float4 y0 = As4[2 * (p * dq + q)], y1 = As4[2 * (p * dq + q) + 1];
          const float2 yx = make_float2(y0.x, y0.y), yy = make_float2(y0.z, y0.w);
          const float2 yz = make_float2(y1.x, y1.y), yw = make_float2(y1.z, y1.w);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            // components w, z, y, x in that order, as the scalar form's fma nest
            if constexpr (kDiff) {
              const float2 ew = __fadd2_rn(make_float2(x[r].w, x[r].w), yw);
              const float2 ez = __fadd2_rn(make_float2(x[r].z, x[r].z), yz);
              const float2 ey = __fadd2_rn(make_float2(x[r].y, x[r].y), yy);
              const float2 ex = __fadd2_rn(make_float2(x[r].x, x[r].x), yx);
              acc[r][p] = __ffma2_rn(ew, ew, acc[r][p]);
              acc[r][p] = __ffma2_rn(ez, ez, acc[r][p]);
              acc[r][p] = __ffma2_rn(ey, ey, acc[r][p]);
              acc[r][p] = __ffma2_rn(ex, ex, acc[r][p]);
            } else {
              acc[r][p] = __ffma2_rn(make_float2(x[r].w, x[r].w), yw, acc[r][p]);
              acc[r][p] = __ffma2_rn(make_float2(x[r].z, x[r].z), yz, acc[r][p]);
              acc[r][p] = __ffma2_rn(make_float2(x[r].y, x[r].y), yy, acc[r][p]);
              acc[r][p] = __ffma2_rn(make_float2(x[r].x, x[r].x), yx, acc[r][p]);
            }
          }
        }
      }
    }
    if (item % steps == steps - 1) {  // the group's last step: its rows are complete
#pragma unroll
      for (int r = 0; r < R; ++r) {
        // x.y, or |x - y|^2, of reference a_mine
        const float sum = warp_reduce_scatter<NA>(reinterpret_cast<float(&)[NA]>(acc[r][0]), lane);
        const int b = b0 + r;
        if (writer && b < nB) {
          const bool same = idA && idB && idA[a_mine] == idB[b];
          float v;
          if constexpr (KIND == DK_RBF) v = same ? 1.0f : exp2f(sum * neg_scale);
          else if constexpr (KIND == DK_DIST) v = same ? 0.0f : sqrtf(sum);
          else v = gram_epilogue<KIND>(sum, 0.0f, 0.0f, same, neg_scale);
          out[(int64_t)a_mine * ldo + b] = v;
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) acc[r][p] = make_float2(0.0f, 0.0f);
      }
    }
  }
}

template <int KIND>
static cudaError_t gram_dispatch(const float* A, int64_t nA, const float* Bm, int64_t nB, int dp,
                                 const float* normA, const float* normB, const int64_t* idA,
                                 const int64_t* idB, float neg_scale, float* out, int64_t ldo,
                                 cudaStream_t st) {
  const size_t skinny_smem = skinny_ref_bytes(nA, dp);
  if (nA <= 32 && skinny_smem <= 96 * 1024) {
    // every CTA first copies the reference rows to shared memory: few CTAs,
    // many sample rows each; behind the reference rows, each warp's two
    // stages of sample vectors (8 warps x 2 x 8 x 32 x 16 B = 64 KB)
    const size_t smem = skinny_smem + kSkinnyStageBytes;
    const int per_sm = smem + 1024 <= 113 * 1024 ? 2 : 1;  // 228 KB of shared memory per SM
    cudaError_t e;
#define KKM_SKINNY(NAV)                                                                 \
  e = cudaFuncSetAttribute(gram_skinny_kernel<KIND, NAV>,                               \
                           cudaFuncAttributeMaxDynamicSharedMemorySize,                 \
                           96 * 1024 + (int)kSkinnyStageBytes);                         \
  if (e != cudaSuccess) return e;                                                       \
  gram_skinny_kernel<KIND, NAV><<<(int)std::min<int64_t>(ceil_div(nB, 8 * skinny_rows<NAV>()), 152 * per_sm), \
                                  256, smem, st>>>(                                     \
      A, (int)nA, Bm, (int)nB, dp, normA, normB, idA, idB, neg_scale, out, ldo);
    if (nA <= 1) { KKM_SKINNY(1) }
    else if (nA <= 4) { KKM_SKINNY(4) }
    else if (nA <= 16) { KKM_SKINNY(16) }
    else { KKM_SKINNY(32) }
#undef KKM_SKINNY
    return cudaGetLastError();
  }
  dim3 grid((unsigned)ceil_div(nB, TB_N), (unsigned)ceil_div(nA, TB_M));
  const int vec_ok = (ldo % 4 == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
  const size_t smem = gram_chunked<KIND>() ? kGramChunkSmem : 0;
  if (smem) {
    static const cudaError_t attr =
        cudaFuncSetAttribute(gram_tiled_kernel<KIND, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
  }
  gram_tiled_kernel<KIND, float><<<grid, 256, smem, st>>>(A, (int)nA, Bm, (int)nB, dp, normA, normB, idA, idB,
                                                          neg_scale, out, ldo, vec_ok, 0, nullptr);
  return cudaGetLastError();
}

// dist[a][b] = sqrt(max(|x_a|^2 + |x_b|^2 - 2 sum_z part[z][a][b], 0)) for
// b > a (the slices added in order), 0 for equal ids.
__global__ void dist_from_parts_kernel(const float* __restrict__ part, int nsplit, int n, int64_t ldo,
                                       const float* __restrict__ norm, const int64_t* __restrict__ ids,
                                       float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int a = (int)(e / n), b = (int)(e % n);
  if (b <= a) return;
  const int64_t o = (int64_t)a * ldo + b;
  float dot = 0.0f;
  for (int z = 0; z < nsplit; ++z) dot += part[(int64_t)z * n * ldo + o];
  out[o] = gram_epilogue<DK_DIST>(dot, norm[a], norm[b], ids && ids[a] == ids[b], 0.0f);
}

cudaError_t launch_gram_dist_upper(const float* A, int64_t n, int dp, const float* normA, const int64_t* idA,
                                   float* out, int64_t ldo, float* scratch, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (dp < kDistSplitMinDp) {
    dim3 grid((unsigned)ceil_div(n, TB_N), (unsigned)ceil_div(n, TB_M));
    const int vec_ok = (ldo % 4 == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
    gram_tiled_kernel<DK_DIST, float><<<grid, 256, 0, st>>>(A, (int)n, A, (int)n, dp, normA, normA, idA, idA, 0.0f,
                                                            out, ldo, vec_ok, 1, nullptr);
    return cudaGetLastError();
  }
  // a few hundred tiles at most: K is split kDistSplit ways so that every SM
  // has work, the raw products go to scratch and a second pass adds them
  dim3 grid((unsigned)ceil_div(n, TB_N), (unsigned)ceil_div(n, TB_M), kDistSplit);
  const int vec_ok = (ldo % 4 == 0) && ((reinterpret_cast<uintptr_t>(scratch) & 15) == 0);
  gram_tiled_kernel<DK_RAW, float><<<grid, 256, 0, st>>>(A, (int)n, A, (int)n, dp, normA, normA, nullptr, nullptr,
                                                         0.0f, scratch, ldo, vec_ok, 1, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dist_from_parts_kernel<<<(unsigned)ceil_div(n * n, 256), 256, 0, st>>>(scratch, kDistSplit, (int)n, ldo, normA,
                                                                         idA, out);
  prof_more_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gram_rbf_half(const float* A, int64_t nA, const float* Bm, int64_t nB, int dp, const float* normA,
                                 const float* normB, const int64_t* idA, const int64_t* idB, float neg_scale,
                                 __half* out, int64_t ldo, cudaStream_t st, float* out32) {
  if (nA <= 0 || nB <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(nB, TB_N), (unsigned)ceil_div(nA, TB_M));
  const int vec_ok = (ldo % 4 == 0) && ((reinterpret_cast<uintptr_t>(out) & 7) == 0) &&
                     ((reinterpret_cast<uintptr_t>(out32) & 15) == 0);
  static const cudaError_t attr = cudaFuncSetAttribute(
      gram_tiled_kernel<DK_RBF, __half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGramChunkSmem);
  if (attr != cudaSuccess) return attr;
  gram_tiled_kernel<DK_RBF, __half><<<grid, 256, kGramChunkSmem, st>>>(A, (int)nA, Bm, (int)nB, dp, normA, normB,
                                                                       idA, idB, neg_scale, out, ldo, vec_ok, 0, out32);
  return cudaGetLastError();
}

cudaError_t launch_gram(int kind, const float* A, int64_t nA, const float* Bm, int64_t nB, int dp,
                        const float* normA, const float* normB, const int64_t* idA,
                        const int64_t* idB, float neg_scale, float* out, int64_t ldo,
                        cudaStream_t st) {
  if (nA <= 0 || nB <= 0) return cudaSuccess;
  switch (kind) {
    case DK_RBF:
      return gram_dispatch<DK_RBF>(A, nA, Bm, nB, dp, normA, normB, idA, idB, neg_scale, out, ldo, st);
    case DK_LINEAR:
      return gram_dispatch<DK_LINEAR>(A, nA, Bm, nB, dp, normA, normB, idA, idB, neg_scale, out, ldo, st);
    default:
      return gram_dispatch<DK_DIST>(A, nA, Bm, nB, dp, normA, normB, idA, idB, neg_scale, out, ldo, st);
  }
}

}  // namespace kkm
