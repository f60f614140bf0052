// Kernel-block evaluation on the 5th-generation tensor cores (tcgen05) in
// BF16 (the precision option KKM_BF16) or FP8 e4m3 with a scale per row
// (KKM_FP8), with FP32 accumulation.
//
//   out[n][m] = kappa(P_n, Q_m),  kappa = exp(-max(0, |p|^2 + |q|^2 - 2 p.q) / (2 sigma^2))
//
// with P the reference rows (landmarks) and Q the sample rows, both BF16 and
// K-major in HBM.  The product Q P^T runs as tcgen05.mma kind::f16 (M = 128
// sample rows, N = 256 reference rows, K = 16 per instruction) from
// shared-memory tiles that TMA fills with the 128-byte swizzle, into an FP32
// accumulator in tensor memory.  The epilogue reads the accumulator with
// tcgen05.ld (thread = sample row, so every column is a coalesced 128-byte
// store of the transposed block) and applies the norms and the exponential.
//
// The squared norms passed in are those of the BF16-rounded rows, so
// |p|^2 + |q|^2 - 2 p.q is the squared distance of the rounded vectors up to
// FP32 accumulation: its error scales with |p - q|, not with the norms, and
// near-duplicate pairs do not cancel catastrophically.
//
// FP8: row r is stored as e4m3 codes of x / s_r, s_r = max_c |x_rc| / 448
// (the largest finite e4m3 value), so each row uses the whole e4m3 range;
// the MMA (kind::f8f6f4, K = 32 per instruction) sums the products of the
// codes exactly in FP32 and the epilogue multiplies by s_p s_q.  A stage
// holds 128 e4m3 values per row: the same 128-byte swizzle rows and byte
// offsets as the BF16 stage of 64 values.
//
// Structure: persistent CTAs (one per SM), 10 warps:
//   warp 0      TMA producer (one elected lane), 4-stage ring of 48 KB stages
//   warp 1      TMEM owner (allocates all 512 columns) and MMA issuer
//   warps 2..9  epilogue: warp w reads TMEM lane quarter w % 4 (the lanes a
//               warp may access) and half (w - 2) / 4 of the 256 columns
// Two accumulators of 256 columns let the epilogue of one tile overlap the
// MMAs of the next.  Every mbarrier wait is bounded: on timeout the kernel
// records an error code, stops issuing work, and still frees its tensor
// memory before returning.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "device_common.cuh"
#include "internal.h"
#include "qcp.cuh"
#include "tc_common.cuh"

namespace kkm {

constexpr int TC_M = 128;          // sample rows per tile (UMMA M)
constexpr int TC_N = 256;          // reference rows per tile (UMMA N)
constexpr int TC_K = 64;           // K elements per stage (one 128-byte swizzle row)
constexpr int TC_STAGES = 4;
constexpr int TC_A_BYTES = TC_M * TC_K * 2;   // 16 KB
constexpr int TC_B_BYTES = TC_N * TC_K * 2;   // 32 KB
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr int TC_THREADS = 320;   // 2 + 8 warps
constexpr int TC_TMEM_COLS = 512;
constexpr size_t TC_SMEM = (size_t)TC_STAGES * TC_STAGE_BYTES + 2048;
// The MD estimate's epilogue also stages each warp's accumulator chunk in
// shared memory, 32 lanes x 16 columns at a time (8 warps x 2 KB), to regroup
// the 3 x 3 blocks (static + dynamic shared memory stays within 227 KB).
constexpr int TC_RMSD_WARP_FLOATS = 512;
constexpr size_t TC_SMEM_RMSD = TC_SMEM + 8 * TC_RMSD_WARP_FLOATS * sizeof(float);

// 2^x with the hardware approximation (ex2.approx, ~2 ulp); its error is far
// below the BF16 rounding of the inputs.
__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = TC_N, M = TC_M.
__host__ __device__ constexpr uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}
// The same for kind::f8f6f4 with e4m3 A and B (format code 0).
__host__ __device__ constexpr uint32_t tc_idesc_e4m3() {
  return (1u << 4) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

struct TcShared {
  uint64_t full[TC_STAGES];
  uint64_t empty[TC_STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint32_t tmem_base;
  int abort_flag;
  float nP[8][TC_N / 2];    // reference norms of the current tile, per epilogue warp
  float sP[8][TC_N / 2];    // FP8: reference row scales of the current tile
};

__device__ __forceinline__ void store_out(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_out(__half* p, float v) { *p = __float2half_rn(v); }

// OutT: float, or __half for a Gaussian kernel block (values in [0, 1]).
//
// KIND == DK_RMSD_EST (the MD kernel's estimate): P and Q rows are the x, y,
// z and zero planes of frames (row 4f + c), so the accumulator holds, for
// sample frame s (rows 4s..4s+3) and reference frame l (columns 4l..4l+3),
// the 3 x 3 correlation of the pair in its top-left corner.  Each epilogue
// warp stages a 32 x 32 chunk (8 samples x 8 references) in shared memory,
// then every lane takes one pair and writes out[l * ldo + s] = 0 if the
// correlation (split-BF16 operands, see the prep) and the frames' squared
// radii (normQ / normP per frame) certify rmsd^2 beyond the refine threshold
// (a sign test of the QCP characteristic polynomial and its derivatives, no
// root iteration); else 1 and the QCP rotation (a unit quaternion) to
// quat[l * ldo + s] for the exact residual pass.
template <int KIND, typename OutT, bool FP8 = false>
__global__ void __launch_bounds__(TC_THREADS, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap mapQ, const __grid_constant__ CUtensorMap mapP,
               int nQ, int nP, int dk, const float* __restrict__ normQ, const float* __restrict__ normP,
               float neg_scale, OutT* __restrict__ out, int64_t ldo, int* __restrict__ err, float inv_n,
               float4* __restrict__ quat, const float* __restrict__ scaleQ = nullptr,
               const float* __restrict__ scaleP = nullptr) {
  constexpr int EK = FP8 ? 2 * TC_K : TC_K;  // K elements per stage (128 bytes per row either way)
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // stages must start on a 1024-byte boundary (swizzle atom)
  uint8_t* stages = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ TcShared sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  static_assert(TC_THREADS == 320, "two control warps and eight epilogue warps");
  const int tiles_m = (nQ + TC_M - 1) / TC_M, tiles_n = (nP + TC_N - 1) / TC_N;
  const int n_tiles = tiles_m * tiles_n;
  const int nk = (dk + EK - 1) / EK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.tfull[b], 1);
      mbar_init(&sh.tempty[b], 8);
    }
    sh.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(&sh.tmem_base, TC_TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const int tm = t % tiles_m, tn = t / tiles_m;
        for (int kb = 0; kb < nk; ++kb) {
          if (!mbar_wait(&sh.empty[s], ph ^ 1u, &sh.abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* a = stages + (size_t)s * TC_STAGE_BYTES;
          uint8_t* b = a + TC_A_BYTES;
          mbar_expect_tx(&sh.full[s], TC_STAGE_BYTES);
          tma_load_2d(&mapQ, &sh.full[s], a, kb * EK, tm * TC_M);
          tma_load_2d(&mapP, &sh.full[s], b, kb * EK, tn * TC_N);
          if (++s == TC_STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      if (!ok) {
        atomicExch(err, 1);
        sh.abort_flag = 1;
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      int lt = 0;
      const uint32_t idesc = FP8 ? tc_idesc_e4m3() : tc_idesc();
      for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++lt) {
        const int buf = lt & 1;
        const uint32_t tph = (uint32_t)(lt >> 1) & 1u;
        if (!mbar_wait(&sh.tempty[buf], tph ^ 1u, &sh.abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem + (uint32_t)(buf * TC_N);
        for (int kb = 0; kb < nk; ++kb) {
          if (!mbar_wait(&sh.full[s], ph, &sh.abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a = smem_u32(stages + (size_t)s * TC_STAGE_BYTES);
          const uint32_t b = a + TC_A_BYTES;
          // 4 instructions of 32 bytes per row: K = 16 BF16 or K = 32 e4m3 values each
#pragma unroll
          for (int k = 0; k < TC_K / 16; ++k) {
            if constexpr (FP8)
              umma_fp8(d_tmem, sw128_desc(a + k * 32), sw128_desc(b + k * 32), idesc, (kb | k) != 0);
            else
              umma_bf16(d_tmem, sw128_desc(a + k * 32), sw128_desc(b + k * 32), idesc, (kb | k) != 0);
          }
          umma_commit(&sh.empty[s]);
          if (++s == TC_STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (ok) umma_commit(&sh.tfull[buf]);
      }
      if (!ok) {
        atomicExch(err, 2);
        sh.abort_flag = 1;
      }
    }
  } else {
    // ---------------- epilogue (warps 2..9)
    const int q = warp & 3;             // TMEM lane quarter of this warp
    const int ew = warp - 2;            // epilogue warp index 0..7
    const int half = ew >> 2;           // column half 0..1
    int lt = 0;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++lt) {
      const int tm = t % tiles_m, tn = t / tiles_m;
      const int buf = lt & 1;
      const uint32_t tph = (uint32_t)(lt >> 1) & 1u;
      const int n0 = tn * TC_N + half * (TC_N / 2);   // first reference row of this warp
      if constexpr (KIND != DK_RMSD_EST) {  // (the MD estimate reads its radii per frame)
        for (int c = lane; c < TC_N / 2; c += 32) {
          const int n = n0 + c;
          sh.nP[ew][c] = n < nP ? normP[n] : 0.0f;
          if constexpr (FP8) sh.sP[ew][c] = n < nP ? scaleP[n] : 0.0f;
        }
      }
      __syncwarp();
      bool ok = true;
      if (lane == 0) ok = mbar_wait(&sh.tfull[buf], tph, &sh.abort_flag);
      ok = __shfl_sync(kFull, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        if (lane == 0) {
          atomicExch(err, 3);
          sh.abort_flag = 1;
        }
        break;
      }
      tc_fence_after();
      if constexpr (KIND == DK_RMSD_EST) {
        float* sb = reinterpret_cast<float*>(stages + (size_t)TC_STAGES * TC_STAGE_BYTES) + ew * TC_RMSD_WARP_FLOATS;
        const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * TC_N + half * (TC_N / 2));
        const int nSf = nQ >> 2, nLf = nP >> 2;
        // n rmsd^2 at which the kernel value falls to kRmsdRefine
        const float n_r2_far = (log2f(kRmsdRefine) / neg_scale) / inv_n;
#pragma unroll 1
        for (int c0 = 0; c0 < TC_N / 2; c0 += 32) {
          uint32_t r[32];
          tmem_ld32(tb + (uint32_t)c0, r);
          // lane = (sample lane / 4, sample coordinate lane % 4); column 4 l + j
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            float4* row = reinterpret_cast<float4*>(sb + lane * 16);
#pragma unroll
            for (int l4 = 0; l4 < 4; ++l4)
              row[l4] = make_float4(__uint_as_float(r[hh * 16 + 4 * l4]), __uint_as_float(r[hh * 16 + 4 * l4 + 1]),
                                    __uint_as_float(r[hh * 16 + 4 * l4 + 2]),
                                    __uint_as_float(r[hh * 16 + 4 * l4 + 3]));
            __syncwarp();
            // one pair per lane: sample ps (of 8), reference pl (of 4)
            const int ps = lane >> 2, pl = lane & 3;
            const int sf = tm * (TC_M / 4) + q * 8 + ps;
            const int lf = tn * (TC_N / 4) + half * (TC_N / 8) + (c0 >> 2) + hh * 4 + pl;
            if (sf < nSf && lf < nLf) {
              float H[9];  // H[c1][c2] = sum_a x_a[c1] y_a[c2], x the reference frame
#pragma unroll
              for (int c1 = 0; c1 < 3; ++c1)
#pragma unroll
                for (int c2 = 0; c2 < 3; ++c2) H[c1 * 3 + c2] = sb[(ps * 4 + c2) * 16 + pl * 4 + c1];
              // 0 for a pair certainly beyond the refine threshold (its true
              // value is below 1e-5); else 1, and the QCP rotation for the
              // exact pass (which then only evaluates the residual)
              const float gx = normP[lf], gy = normQ[sf];
              const bool far = qcp_certainly_far(H, gx, gy, n_r2_far);
              store_out(out + (int64_t)lf * ldo + sf, far ? 0.0f : 1.0f);
              if (!far) {
                float qv[4];
                qcp_quaternion(H, gx, gy, qv);
                quat[(int64_t)lf * ldo + sf] = make_float4(qv[0], qv[1], qv[2], qv[3]);
              }
            }
            __syncwarp();
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.tempty[buf]);
        continue;
      }
      const int m = tm * TC_M + q * 32 + lane;
      const bool mvalid = m < nQ;
      const float nq = mvalid ? normQ[m] : 0.0f;
      const float sq = (FP8 && mvalid) ? scaleQ[m] : 1.0f;
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * TC_N + half * (TC_N / 2));
      const int ncols = min(TC_N / 2, nP - n0);  // valid reference rows of this warp (may be <= 0)
      OutT* orow = out + (int64_t)n0 * ldo + m;
#pragma unroll 1
      for (int c0 = 0; c0 < TC_N / 2; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tbase + (uint32_t)c0, r);
        if (mvalid) {
          if (c0 + 32 <= ncols) {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              const float dot = FP8 ? __uint_as_float(r[c]) * (sq * sh.sP[ew][c0 + c]) : __uint_as_float(r[c]);
              float v;
              if (KIND == DK_LINEAR) {
                v = dot;
              } else {
                const float d2 = fmaxf(fmaf(-2.0f, dot, nq + sh.nP[ew][c0 + c]), 0.0f);
                if (KIND == DK_DIST) v = sqrtf(d2);
                else v = fast_exp2(d2 * neg_scale);
              }
              store_out(orow + (int64_t)(c0 + c) * ldo, v);
            }
          } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              if (c0 + c < ncols) {
                const float dot = FP8 ? __uint_as_float(r[c]) * (sq * sh.sP[ew][c0 + c]) : __uint_as_float(r[c]);
                float v;
                if (KIND == DK_LINEAR) {
                  v = dot;
                } else {
                  const float d2 = fmaxf(fmaf(-2.0f, dot, nq + sh.nP[ew][c0 + c]), 0.0f);
                  if (KIND == DK_DIST) v = sqrtf(d2);
                  else v = fast_exp2(d2 * neg_scale);
                }
                store_out(orow + (int64_t)(c0 + c) * ldo, v);
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.tempty[buf]);
    }
  }
  // teardown: every role is done issuing; the TMEM owner frees tensor memory
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TC_TMEM_COLS);
  }
}

// ------------------------------------------------------------ host side
// 2-D map of a row-major BF16 (or e4m3) matrix [rows][ld] (ld elements per
// row, a multiple of 16 bytes), box = box_rows x 128 bytes, 128-byte
// swizzle, zero fill past the cols valid values.
static bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                     bool fp8 = false) {
  auto enc = get_encode();
  if (!enc) return false;
  const int esize = fp8 ? 1 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esize), (cuuint32_t)box_rows};  // 128-byte rows
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <typename OutT>
static cudaError_t launch_gram_tc_t(int kind, const CUtensorMap& mq, const CUtensorMap& mp, int nQ, int nP, int dk,
                                    const float* normP, const float* normQ, float neg_scale, OutT* out,
                                    int64_t ldo, int* err, int grid, cudaStream_t st) {
  cudaError_t e;
#define KKM_TC_LAUNCH(K)                                                                                  \
  e = cudaFuncSetAttribute(gram_tc_kernel<K, OutT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM); \
  if (e != cudaSuccess) return e;                                                                         \
  gram_tc_kernel<K, OutT><<<grid, TC_THREADS, TC_SMEM, st>>>(mq, mp, nQ, nP, dk, normQ, normP, neg_scale, out, \
                                                             ldo, err, 0.0f, nullptr);
  if (kind == DK_DIST) {
    KKM_TC_LAUNCH(DK_DIST)
  } else if (kind == DK_LINEAR) {
    KKM_TC_LAUNCH(DK_LINEAR)
  } else {
    KKM_TC_LAUNCH(DK_RBF)
  }
#undef KKM_TC_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_gram_tc(int kind, const __nv_bfloat16* P, int64_t nP, const __nv_bfloat16* Q, int64_t nQ,
                           int dk, int ldb, const float* normP, const float* normQ, float neg_scale, void* out,
                           bool out_half, int64_t ldo, int* err, int n_sms, cudaStream_t st) {
  if (nP <= 0 || nQ <= 0) return cudaSuccess;
  if ((ldb * 2) % 16 != 0 || (reinterpret_cast<uintptr_t>(P) & 15) || (reinterpret_cast<uintptr_t>(Q) & 15))
    return cudaErrorInvalidValue;
  if (out_half && kind != DK_RBF) return cudaErrorInvalidValue;  // FP16 holds values in [0, 1] only
  alignas(64) CUtensorMap mq, mp;
  if (!make_map(&mq, Q, nQ, dk, ldb, TC_M) || !make_map(&mp, P, nP, dk, ldb, TC_N)) return cudaErrorInvalidValue;
  const int64_t tiles = ceil_div(nQ, TC_M) * ceil_div(nP, TC_N);
  const int grid = (int)std::min<int64_t>(tiles, std::max(n_sms, 1));
  if (out_half)
    return launch_gram_tc_t(kind, mq, mp, (int)nQ, (int)nP, dk, normP, normQ, neg_scale,
                            static_cast<__half*>(out), ldo, err, grid, st);
  return launch_gram_tc_t(kind, mq, mp, (int)nQ, (int)nP, dk, normP, normQ, neg_scale, static_cast<float*>(out),
                          ldo, err, grid, st);
}

cudaError_t launch_gram_tc_fp8(int kind, const uint8_t* P, int64_t nP, const uint8_t* Q, int64_t nQ, int dk, int ld8,
                               const float* normP, const float* normQ, const float* scaleP, const float* scaleQ,
                               float neg_scale, void* out, bool out_half, int64_t ldo, int* err, int n_sms,
                               cudaStream_t st) {
  if (nP <= 0 || nQ <= 0) return cudaSuccess;
  if (ld8 % 16 != 0 || (reinterpret_cast<uintptr_t>(P) & 15) || (reinterpret_cast<uintptr_t>(Q) & 15))
    return cudaErrorInvalidValue;
  if (out_half && kind != DK_RBF) return cudaErrorInvalidValue;
  if (kind != DK_RBF && kind != DK_LINEAR) return cudaErrorInvalidValue;
  alignas(64) CUtensorMap mq, mp;
  if (!make_map(&mq, Q, nQ, dk, ld8, TC_M, true) || !make_map(&mp, P, nP, dk, ld8, TC_N, true))
    return cudaErrorInvalidValue;
  const int64_t tiles = ceil_div(nQ, TC_M) * ceil_div(nP, TC_N);
  const int grid = (int)std::min<int64_t>(tiles, std::max(n_sms, 1));
  cudaError_t e;
#define KKM_TC8(K, OT)                                                                                            \
  e = cudaFuncSetAttribute(gram_tc_kernel<K, OT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM); \
  if (e != cudaSuccess) return e;                                                                                 \
  gram_tc_kernel<K, OT, true><<<grid, TC_THREADS, TC_SMEM, st>>>(mq, mp, (int)nQ, (int)nP, dk, normQ, normP,        \
                                                                 neg_scale, static_cast<OT*>(out), ldo, err, 0.0f, \
                                                                 nullptr, scaleQ, scaleP);
  if (kind == DK_LINEAR) {
    KKM_TC8(DK_LINEAR, float)
  } else if (out_half) {
    KKM_TC8(DK_RBF, __half)
  } else {
    KKM_TC8(DK_RBF, float)
  }
#undef KKM_TC8
  return cudaGetLastError();
}

cudaError_t launch_rmsd_tc_estimate(const __nv_bfloat16* P, int64_t nP, const __nv_bfloat16* Q, int64_t nQ, int kp,
                                    const float* gP, const float* gQ, int n_atoms, float neg_scale, float* out,
                                    float4* quat, int64_t ldo, int* err, int n_sms, cudaStream_t st) {
  if (nP <= 0 || nQ <= 0) return cudaSuccess;
  if (kp % TC_K != 0 || (reinterpret_cast<uintptr_t>(P) & 15) || (reinterpret_cast<uintptr_t>(Q) & 15) ||
      n_atoms <= 0 || !quat)
    return cudaErrorInvalidValue;
  alignas(64) CUtensorMap mq, mp;
  if (!make_map(&mq, Q, 4 * nQ, kp, kp, TC_M) || !make_map(&mp, P, 4 * nP, kp, kp, TC_N))
    return cudaErrorInvalidValue;
  const int64_t tiles = ceil_div(4 * nQ, TC_M) * ceil_div(4 * nP, TC_N);
  const int grid = (int)std::min<int64_t>(tiles, std::max(n_sms, 1));
  cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel<DK_RMSD_EST, float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_RMSD);
  if (e != cudaSuccess) return e;
  gram_tc_kernel<DK_RMSD_EST, float><<<grid, TC_THREADS, TC_SMEM_RMSD, st>>>(
      mq, mp, (int)(4 * nQ), (int)(4 * nP), kp, gQ, gP, neg_scale, out, ldo, err, 1.0f / (float)n_atoms, quat);
  return cudaGetLastError();
}

// K = 1 on the diagonal of the block: out[k][L[k]] for landmark ordinals k.
template <typename T>
__global__ void set_diag_kernel(T* __restrict__ out, int64_t ldo, const int32_t* __restrict__ L, int nL) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nL) out[(int64_t)k * ldo + L[k]] = T(1.0f);
}
cudaError_t launch_set_diag(void* out, bool out_half, int64_t ldo, const int32_t* L, int nL, cudaStream_t st) {
  if (nL <= 0) return cudaSuccess;
  if (out_half)
    set_diag_kernel<__half><<<(unsigned)ceil_div(nL, 256), 256, 0, st>>>(static_cast<__half*>(out), ldo, L, nL);
  else
    set_diag_kernel<float><<<(unsigned)ceil_div(nL, 256), 256, 0, st>>>(static_cast<float*>(out), ldo, L, nL);
  return cudaGetLastError();
}

// ------------------------------------------------ FP32 rows -> BF16 rows
// dst[r][c] = bf16(src[r][c]) for c < dp, and the squared norm of the rounded
// row (double-float accumulation, rounded to FP32) in normsq.
__global__ void to_bf16_kernel(const float* __restrict__ src, int64_t n, int dp, __nv_bfloat16* __restrict__ dst,
                               float* __restrict__ normsq) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const float* s = src + row * dp;
  __nv_bfloat16* d = dst + row * dp;
  float2 acc = make_float2(0.0f, 0.0f);
  for (int c = lane; c < dp; c += 32) {
    const __nv_bfloat16 b = __float2bfloat16_rn(s[c]);
    d[c] = b;
    acc = df_add_sq(acc, __bfloat162float(b));
  }
  acc = warp_sum_df(acc);
  if (normsq && lane == 0) normsq[row] = df_to_float(acc);
}

// ------------------------------------------- FP32 rows -> e4m3 rows + scale
// One warp per row: s = max_c |x_c| / 448 (1 for an all-zero row), dst[c] =
// e4m3(clamp(x_c / s, -448, 448)) (round to nearest even) for c < dp and 0 up
// to ld8, scale[row] = s, normsq[row] = the squared norm of the decoded row
// s * e4m3 (double-float accumulation, rounded to FP32).
__global__ void to_fp8_kernel(const float* __restrict__ src, int64_t n, int dp, int ld8, uint8_t* __restrict__ dst,
                              float* __restrict__ scale, float* __restrict__ normsq) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const float* s = src + row * dp;
  uint8_t* d = dst + row * ld8;
  float m = 0.0f;
  for (int c = lane; c < dp; c += 32) m = fmaxf(m, fabsf(s[c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
  const float sc = m > 0.0f ? m / 448.0f : 1.0f;
  float2 acc = make_float2(0.0f, 0.0f);
  for (int c = lane; c < ld8; c += 32) {
    uint8_t code = 0;
    if (c < dp) {
      const float v = fminf(fmaxf(s[c] / sc, -448.0f), 448.0f);
      const __nv_fp8_e4m3 q(v);
      code = q.__x;
      acc = df_add_sq(acc, (float)q * sc);
    }
    d[c] = code;
  }
  acc = warp_sum_df(acc);
  if (lane == 0) {
    scale[row] = sc;
    normsq[row] = df_to_float(acc);
  }
}

cudaError_t launch_to_fp8(const float* src, int64_t n, int dp, int ld8, uint8_t* dst, float* scale, float* normsq,
                          cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  to_fp8_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(src, n, dp, ld8, dst, scale, normsq);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* src, int64_t n, int dp, __nv_bfloat16* dst, float* normsq, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  to_bf16_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(src, n, dp, dst, normsq);
  return cudaGetLastError();
}

}  // namespace kkm
