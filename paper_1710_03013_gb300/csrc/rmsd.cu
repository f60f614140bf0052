// MD kernel: K(x, y) = exp(-rmsd^2 / (2 sigma^2)) with rmsd the minimum RMSD
// of two frames after optimal proper superposition.  The paper asks for a
// roto-translation invariant similarity for MD frames without writing one
// down; the minimum RMSD is the standard choice.
//
// Frames are prepared once as centred structure-of-arrays rows [3][ap]
// (x, y, z planes of ap = n_atoms rounded up to 8, zero padded) with their
// squared radius G = sum |x_a|^2.
//
// rmsd_gram computes a CTA tile of 32 (or, for few references, 8) reference
// frames x 64 sample frames, 8 pairs per thread, in two passes over the atoms:
//   pass 1  the 3x3 correlation H = sum_a x_a y_a^T of each pair (FP32 FFMA,
//           72 accumulators per thread, double-buffered shared-memory tiles of
//           8 atoms);  then per pair the QCP root: the largest eigenvalue of
//           Horn's 4x4 quaternion matrix as the largest root of its
//           characteristic polynomial lambda^4 + c2 lambda^2 + c1 lambda + c0
//           (c2 = -2 |S|_F^2, c1 = -8 det S, c0 = det N; Theobald 2005), found
//           by Newton's method from the upper bound (G_x + G_y)/2, and the
//           rotation from the quaternion eigenvector (a cofactor row of
//           N - lambda I).
//   pass 2  for pairs whose kernel value is not negligible, the residual
//           sum_a |R x_a - y_a|^2 evaluated directly at that rotation.
// Why two passes: rmsd^2 = (G_x + G_y - 2 lambda)/n cancels catastrophically
// (G ~ 1e5 A^2 against n rmsd^2 ~ 1e2 for similar frames), so FP32 rounding of
// H and G alone moves K by ~1e-4.  The direct residual has no cancellation,
// and since the residual is stationary at the optimal rotation, the rotation's
// own FP32 error enters only at second order.  No FP64 is needed.  Pass 2
// runs only in warps holding a pair with a non-negligible kernel value.
#include <cuda_bf16.h>
#include <limits.h>

#include "device_common.cuh"
#include "internal.h"
#include "qcp.cuh"

namespace kkm {

// ------------------------------------------------------------------ prep
__global__ void rmsd_prep_kernel(const float* __restrict__ X, int n_atoms, int64_t start, int64_t step,
                                 const int64_t* __restrict__ idx, int64_t n, float* __restrict__ out,
                                 int ap, float* __restrict__ gsq) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const int64_t g = idx ? idx[row] : start + row * step;
  const float* src = X + g * 3 * (int64_t)n_atoms;
  // FP32 is ample here: a centring error of ~1e-6 A changes rmsd^2 by ~1e-12
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int a = lane; a < n_atoms; a += 32) {
    sx += src[3 * a];
    sy += src[3 * a + 1];
    sz += src[3 * a + 2];
  }
  const float inv_n = 1.0f / (float)n_atoms;
  sx = warp_sum_f32(sx) * inv_n;
  sy = warp_sum_f32(sy) * inv_n;
  sz = warp_sum_f32(sz) * inv_n;
  float* dst = out + row * 3 * (int64_t)ap;
  float gg = 0.f;
  for (int a = lane; a < ap; a += 32) {
    float cx = 0.f, cy = 0.f, cz = 0.f;
    if (a < n_atoms) {
      cx = src[3 * a] - sx;
      cy = src[3 * a + 1] - sy;
      cz = src[3 * a + 2] - sz;
    }
    dst[a] = cx;
    dst[ap + a] = cy;
    dst[2 * ap + a] = cz;
    gg = fmaf(cx, cx, fmaf(cy, cy, fmaf(cz, cz, gg)));
  }
  gg = warp_sum_f32(gg);
  if (lane == 0) gsq[row] = gg;
}

cudaError_t launch_rmsd_prep_rows(const float* X, int n_atoms, int64_t start, int64_t step, int64_t n,
                                  float* out, int ap, float* gsq, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  rmsd_prep_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(X, n_atoms, start, step, nullptr, n, out, ap, gsq);
  return cudaGetLastError();
}
cudaError_t launch_rmsd_prep_idx64(const float* X, int n_atoms, const int64_t* idx, int64_t n, float* out,
                                   int ap, float* gsq, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  rmsd_prep_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(X, n_atoms, 0, 0, idx, n, out, ap, gsq);
  return cudaGetLastError();
}

// SoA FP32 frames -> BF16 planes for the tensor-core correlation: one warp per
// frame, row [4 planes][3 kp].  Each coordinate is split v = hi + lo (hi =
// bf16(v), lo = bf16(v - hi)) and the three kp-long segments of a row are
// (hi, lo, hi) on the reference side and (hi, hi, lo) on the sample side, so
// one GEMM over 3 kp sums hi.hi + lo.hi + hi.lo: the correlation to about 16
// significant bits (the lo.lo term, ~2^-16 relative, is dropped).
__global__ void rmsd_to_bf16_kernel(const float* __restrict__ src, int64_t n, int ap, int n_atoms,
                                    __nv_bfloat16* __restrict__ dst, int kp, int side) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const float* s = src + row * 3 * (int64_t)ap;
  __nv_bfloat16* d = dst + row * 4 * (int64_t)(3 * kp);
  for (int c = 0; c < 4; ++c)
    for (int k = lane; k < kp; k += 32) {
      const float v = (c < 3 && k < n_atoms) ? s[c * ap + k] : 0.0f;
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
      __nv_bfloat16* r = d + (int64_t)c * 3 * kp + k;
      r[0] = hi;
      r[kp] = side == 0 ? lo : hi;
      r[2 * kp] = side == 0 ? hi : lo;
    }
}

cudaError_t launch_rmsd_to_bf16(const float* src, int64_t n, int ap, int n_atoms, __nv_bfloat16* dst, int kp,
                                int side, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  rmsd_to_bf16_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(src, n, ap, n_atoms, dst, kp, side);
  return cudaGetLastError();
}

// ------------------------------------------------- refine-tile ordering
// After the tensor-core estimate, the exact kernel recomputes only tiles of
// 32 reference frames x 64 samples holding a pair above kRmsdRefine.  Samples
// are in trajectory order, so a sample tile is mostly one conformational
// state; the references are reordered so that a reference tile is too: key
// = the first sample whose estimate exceeds the threshold (references of one
// state share it; references near nothing sort last), ties by index.
__global__ void rmsd_near_key_kernel(const float* __restrict__ est, int64_t ldo, int nA, int nB,
                                     int* __restrict__ key) {
  const int lane = threadIdx.x & 31;
  const int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (a >= nA) return;
  const float* row = est + (int64_t)a * ldo;
  int first = INT_MAX;
  for (int b0 = 0; b0 < nB && first == INT_MAX; b0 += 32 * 8) {
    int f = INT_MAX;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int b = b0 + q * 32 + lane;
      if (b < nB && row[b] > kRmsdRefine) f = min(f, b);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f = min(f, __shfl_xor_sync(kFull, f, o));
    first = f;
  }
  if (lane == 0) key[a] = first;
}

// order[rank(a)] = a, rank by (key, index); keys staged in shared memory
// when they fit (else read from global memory, the same in every lane).
template <bool SMEM>
__global__ void rmsd_rank_kernel(const int* __restrict__ key, int nA, int* __restrict__ order) {
  extern __shared__ int ks[];
  if (SMEM) {
    for (int i = threadIdx.x; i < nA; i += blockDim.x) ks[i] = key[i];
    __syncthreads();
  }
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nA) return;
  const int* kk = SMEM ? ks : key;
  const int ka = kk[a];
  int rank = 0;
  for (int i = 0; i < nA; ++i) {
    const int ki = kk[i];
    rank += (ki < ka) || (ki == ka && i < a);
  }
  order[rank] = a;
}

// flag[t][u] = 1 if reference tile t (of the order) and sample tile u hold a
// pair above the threshold; one CTA per (sample tile, reference tile).
__global__ void rmsd_tile_flag_kernel(const float* __restrict__ est, int64_t ldo, int nA, int nB,
                                      const int* __restrict__ order, int* __restrict__ flag) {
  const int u = blockIdx.x, t = blockIdx.y;
  const int b = u * 64 + (threadIdx.x & 63);
  int hit = 0;
  for (int r = threadIdx.x >> 6; r < 32; r += blockDim.x >> 6) {
    const int ar = t * 32 + r;
    if (ar < nA && b < nB) hit |= est[(int64_t)order[ar] * ldo + b] > kRmsdRefine;
  }
  hit = __syncthreads_or(hit);
  if (threadIdx.x == 0) flag[(int64_t)t * gridDim.x + u] = hit;
}

cudaError_t launch_rmsd_refine_plan(const float* est, int64_t ldo, int nA, int nB, int* key, int* order, int* flag,
                                    cudaStream_t st) {
  if (nA <= 0 || nB <= 0) return cudaSuccess;
  rmsd_near_key_kernel<<<(unsigned)ceil_div(nA, 8), 256, 0, st>>>(est, ldo, nA, nB, key);
  if ((size_t)nA * sizeof(int) <= 48 * 1024)
    rmsd_rank_kernel<true><<<(unsigned)ceil_div(nA, 256), 256, (size_t)nA * sizeof(int), st>>>(key, nA, order);
  else
    rmsd_rank_kernel<false><<<(unsigned)ceil_div(nA, 256), 256, 0, st>>>(key, nA, order);
  rmsd_tile_flag_kernel<<<dim3((unsigned)ceil_div(nB, 64), (unsigned)ceil_div(nA, 32)), 256, 0, st>>>(est, ldo, nA, nB,
                                                                                                   order, flag);
  prof_more_launches(2);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- QCP
// H = sum_a x_a y_a^T (row-major 3x3) of centred frames x (reference) and y
// (sample) with squared radii Gx, Gy.  Returns the estimate G_x + G_y -
// 2 lambda_max (>= 0) and the rotation R (row-major) with R x ~ y.
__device__ __forceinline__ float qcp_rotation(const float H[9], float Gx, float Gy, float R[9]) {
  float q[4];
  const float est = qcp_quaternion(H, Gx, Gy, q);
  quat_to_rot(q, R);
  return est;
}

// --------------------------------------------------------------- pair tile
// Tile: TA reference frames x 64 sample frames, 8 atoms per shared-memory
// stage, 2 references x 4 samples per thread (16 x TA/2 threads).  TA = 32
// for kernel blocks, TA = 8 for the few-reference calls (medoid columns,
// k-means++ columns).
constexpr int RT_B = 64, RT_K = 8;

template <int TA>
struct RmsdCfg {
  static constexpr int NT = 16 * (TA / 2);           // threads
  static constexpr int A4 = TA * 6;                   // float4 per A stage
  static constexpr int B4 = RT_B * 6;                 // float4 per B stage
  static constexpr int PA = (A4 + NT - 1) / NT;
  static constexpr int PB = (B4 + NT - 1) / NT;
};

template <int TA>
struct RmsdTiles {
  float As[2][RT_K][3][TA];
  float Bs[2][RT_K][3][RT_B];
};



template <int TA>
struct RmsdPrefetch {
  float4 a[RmsdCfg<TA>::PA];
  float4 b[RmsdCfg<TA>::PB];
};

// element e of a stage: frame f = e % rows, coordinate plane c, half h of the 8 atoms
template <int TA>
__device__ __forceinline__ void rmsd_fetch(const float* __restrict__ A, int nA, const float* __restrict__ Bm,
                                           int nB, int ap, int a0, int b0, int k0, RmsdPrefetch<TA>& p,
                                           const int* __restrict__ arow) {
  using Cf = RmsdCfg<TA>;
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < Cf::PA; ++q) {
    const int e = tid + q * Cf::NT;
    if (e < Cf::A4) {
      const int f = e % TA, rest = e / TA, c = rest >> 1, h = rest & 1;
      const int ar = min(a0 + f, nA - 1);
      p.a[q] = __ldg(reinterpret_cast<const float4*>(A + (int64_t)(arow ? arow[ar] : ar) * 3 * ap + c * ap + k0 + h * 4));
    }
  }
#pragma unroll
  for (int q = 0; q < Cf::PB; ++q) {
    const int e = tid + q * Cf::NT;
    if (e < Cf::B4) {
      const int f = e % RT_B, rest = e / RT_B, c = rest >> 1, h = rest & 1;
      p.b[q] = __ldg(reinterpret_cast<const float4*>(Bm + (int64_t)min(b0 + f, nB - 1) * 3 * ap + c * ap + k0 + h * 4));
    }
  }
}

template <int TA>
__device__ __forceinline__ void rmsd_store(RmsdTiles<TA>& t, int buf, const RmsdPrefetch<TA>& p) {
  using Cf = RmsdCfg<TA>;
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < Cf::PA; ++q) {
    const int e = tid + q * Cf::NT;
    if (e < Cf::A4) {
      const int f = e % TA, rest = e / TA, c = rest >> 1, h = rest & 1;
      t.As[buf][h * 4 + 0][c][f] = p.a[q].x;
      t.As[buf][h * 4 + 1][c][f] = p.a[q].y;
      t.As[buf][h * 4 + 2][c][f] = p.a[q].z;
      t.As[buf][h * 4 + 3][c][f] = p.a[q].w;
    }
  }
#pragma unroll
  for (int q = 0; q < Cf::PB; ++q) {
    const int e = tid + q * Cf::NT;
    if (e < Cf::B4) {
      const int f = e % RT_B, rest = e / RT_B, c = rest >> 1, h = rest & 1;
      t.Bs[buf][h * 4 + 0][c][f] = p.b[q].x;
      t.Bs[buf][h * 4 + 1][c][f] = p.b[q].y;
      t.Bs[buf][h * 4 + 2][c][f] = p.b[q].z;
      t.Bs[buf][h * 4 + 3][c][f] = p.b[q].w;
    }
  }
}

template <int KIND, int TA>
__global__ void __launch_bounds__(RmsdCfg<TA>::NT, (TA == 32) ? 2 : 4)
rmsd_gram_kernel(const float* __restrict__ A, int nA, const float* __restrict__ Bm, int nB, int ap,
                 int n_atoms, const float* __restrict__ gA, const float* __restrict__ gB,
                 const int64_t* __restrict__ idA, const int64_t* __restrict__ idB, float neg_scale,
                 float* __restrict__ out, int64_t ldo, int vec_ok, const int* __restrict__ tile_flag,
                 const int* __restrict__ arow, const float4* __restrict__ quat) {
  __shared__ __align__(16) RmsdTiles<TA> t;
  if (tile_flag && !tile_flag[(int64_t)blockIdx.y * gridDim.x + blockIdx.x]) return;  // estimate stands
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int a0 = blockIdx.y * TA, b0 = blockIdx.x * RT_B;
  const int nk = ap / RT_K;

  float h[2][4][9];
  float r2[2][4];
  unsigned need = 0u;
  const float inv_n = 1.0f / (float)n_atoms;
  RmsdPrefetch<TA> pf;
  if (quat) {
    // ---- after the tensor-core screen: the rotations of the pairs it did
    // not certify far come from its correlation (accurate to ~1e-5); only
    // pass 2 runs
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int ar = min(a0 + ty * 2 + r, nA - 1);
      const int a = arow ? arow[ar] : ar;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int b = min(b0 + tx * 4 + q, nB - 1);
        r2[r][q] = 0.0f;
        const bool live = a0 + ty * 2 + r < nA && b0 + tx * 4 + q < nB;
        float qq[4] = {1.f, 0.f, 0.f, 0.f};
        if (live && out[(int64_t)a * ldo + b] != 0.0f) {
          need |= 1u << (r * 4 + q);
          const float4 v = quat[(int64_t)a * ldo + b];
          qq[0] = v.x;
          qq[1] = v.y;
          qq[2] = v.z;
          qq[3] = v.w;
        }
        quat_to_rot(qq, h[r][q]);
      }
    }
  } else {
  // ---- pass 1: correlation matrices
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int e = 0; e < 9; ++e) h[r][q][e] = 0.f;
  rmsd_fetch<TA>(A, nA, Bm, nB, ap, a0, b0, 0, pf, arow);
  rmsd_store<TA>(t, 0, pf);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) rmsd_fetch<TA>(A, nA, Bm, nB, ap, a0, b0, (kt + 1) * RT_K, pf, arow);
#pragma unroll
    for (int k = 0; k < RT_K; ++k) {
      float2 av[3];
      float4 bv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        av[c] = *reinterpret_cast<const float2*>(&t.As[cur][k][c][ty * 2]);
        bv[c] = *reinterpret_cast<const float4*>(&t.Bs[cur][k][c][tx * 4]);
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const float x[3] = {r ? av[0].y : av[0].x, r ? av[1].y : av[1].x, r ? av[2].y : av[2].x};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float y[3] = {q == 0 ? bv[0].x : q == 1 ? bv[0].y : q == 2 ? bv[0].z : bv[0].w,
                              q == 0 ? bv[1].x : q == 1 ? bv[1].y : q == 2 ? bv[1].z : bv[1].w,
                              q == 0 ? bv[2].x : q == 1 ? bv[2].y : q == 2 ? bv[2].z : bv[2].w};
#pragma unroll
          for (int c1 = 0; c1 < 3; ++c1)
#pragma unroll
            for (int c2 = 0; c2 < 3; ++c2) h[r][q][c1 * 3 + c2] = fmaf(x[c1], y[c2], h[r][q][c1 * 3 + c2]);
        }
      }
    }
    if (kt + 1 < nk) rmsd_store<TA>(t, cur ^ 1, pf);
    __syncthreads();
  }

  // ---- QCP estimates and rotations (h is overwritten by R)
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int a = arow ? arow[min(a0 + ty * 2 + r, nA - 1)] : min(a0 + ty * 2 + r, nA - 1);
    const float ga = gA[a];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int b = min(b0 + tx * 4 + q, nB - 1);
      float Rm[9];
      const float est = qcp_rotation(h[r][q], ga, gB[b], Rm) * inv_n;
#pragma unroll
      for (int e = 0; e < 9; ++e) h[r][q][e] = Rm[e];
      r2[r][q] = est;
      const bool refine = (KIND == DK_DIST) || (exp2f(est * neg_scale) > 1e-4f);
      if (refine) need |= 1u << (r * 4 + q);
    }
  }

  }

  // ---- pass 2: direct residuals at the QCP rotation, for the warps holding
  // a pair that needs one (the stage loads stay CTA-wide)
  if (__syncthreads_or(need != 0u)) {
    const bool warp_need = __any_sync(kFull, need != 0u);
    float res[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) res[r][q] = 0.f;
    rmsd_fetch<TA>(A, nA, Bm, nB, ap, a0, b0, 0, pf, arow);
    rmsd_store<TA>(t, 0, pf);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
      const int cur = kt & 1;
      if (kt + 1 < nk) rmsd_fetch<TA>(A, nA, Bm, nB, ap, a0, b0, (kt + 1) * RT_K, pf, arow);
      if (warp_need) {
#pragma unroll
        for (int k = 0; k < RT_K; ++k) {
          float2 av[3];
          float4 bv[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            av[c] = *reinterpret_cast<const float2*>(&t.As[cur][k][c][ty * 2]);
            bv[c] = *reinterpret_cast<const float4*>(&t.Bs[cur][k][c][tx * 4]);
          }
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const float x0 = r ? av[0].y : av[0].x, x1 = r ? av[1].y : av[1].x, x2 = r ? av[2].y : av[2].x;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float y0 = q == 0 ? bv[0].x : q == 1 ? bv[0].y : q == 2 ? bv[0].z : bv[0].w;
              const float y1 = q == 0 ? bv[1].x : q == 1 ? bv[1].y : q == 2 ? bv[1].z : bv[1].w;
              const float y2 = q == 0 ? bv[2].x : q == 1 ? bv[2].y : q == 2 ? bv[2].z : bv[2].w;
              const float* Rm = h[r][q];
              const float e0 = fmaf(Rm[0], x0, fmaf(Rm[1], x1, fmaf(Rm[2], x2, -y0)));
              const float e1 = fmaf(Rm[3], x0, fmaf(Rm[4], x1, fmaf(Rm[5], x2, -y1)));
              const float e2 = fmaf(Rm[6], x0, fmaf(Rm[7], x1, fmaf(Rm[8], x2, -y2)));
              res[r][q] = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, res[r][q])));
            }
          }
        }
      }
      if (kt + 1 < nk) rmsd_store<TA>(t, cur ^ 1, pf);
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (need & (1u << (r * 4 + q))) r2[r][q] = res[r][q] * inv_n;
  }

  // ---- epilogue
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if (a0 + ty * 2 + r >= nA) continue;
    const int a = arow ? arow[a0 + ty * 2 + r] : a0 + ty * 2 + r;
    const int64_t ia = idA ? idA[a] : -2;
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int b = b0 + tx * 4 + q;
      const bool same = idB && b < nB && idB[b] == ia;
      const float rr = fmaxf(r2[r][q], 0.0f);
      if (KIND == DK_DIST) v[q] = same ? 0.0f : sqrtf(rr);
      else v[q] = same ? 1.0f : exp2f(rr * neg_scale);
    }
    float* orow = out + (int64_t)a * ldo;
    const int b = b0 + tx * 4;
    if (tile_flag) {
      // after the tensor-core screen: a pair it certified far keeps its 0,
      // so every pair's value depends on the pair alone, not on its tile
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (b + q < nB && orow[b + q] == 0.0f) v[q] = 0.0f;
    }
    if (vec_ok && b + 3 < nB) {
      *reinterpret_cast<float4*>(orow + b) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (b + q < nB) orow[b + q] = v[q];
    }
  }
}

cudaError_t launch_rmsd_gram(int kind, const float* A, int64_t nA, const float* Bm, int64_t nB, int ap,
                             int n_atoms, const float* gA, const float* gB, const int64_t* idA,
                             const int64_t* idB, float neg_scale, float* out, int64_t ldo, cudaStream_t st,
                             const int* tile_flag, const int* arow, const float4* quat) {
  if (nA <= 0 || nB <= 0) return cudaSuccess;
  if ((tile_flag || quat) && nA <= 8) return cudaErrorInvalidValue;  // laid out for 32-frame A tiles
  const int vec_ok = (ldo % 4 == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
#define KKM_RMSD_LAUNCH(K, TA)                                                                       \
  rmsd_gram_kernel<K, TA><<<dim3((unsigned)ceil_div(nB, RT_B), (unsigned)ceil_div(nA, TA)),          \
                            RmsdCfg<TA>::NT, 0, st>>>(A, (int)nA, Bm, (int)nB, ap, n_atoms, gA, gB, idA, \
                                                      idB, neg_scale, out, ldo, vec_ok, tile_flag, arow, quat)
  if (nA <= 8) {
    if (kind == DK_DIST) KKM_RMSD_LAUNCH(DK_DIST, 8); else KKM_RMSD_LAUNCH(DK_RBF, 8);
  } else {
    if (kind == DK_DIST) KKM_RMSD_LAUNCH(DK_DIST, 32); else KKM_RMSD_LAUNCH(DK_RBF, 32);
  }
#undef KKM_RMSD_LAUNCH
  return cudaGetLastError();
}

}  // namespace kkm
