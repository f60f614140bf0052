// The inner loop of one mini-batch (Alg. 1 lines 9-16) as one cooperative
// launch, with the f_hat numerators of Eq. 17 formed on the tensor cores.
//
// For sample x_i and cluster j, n_j f_hat_ij = sum of K(x_i, l_k) over the
// landmarks l_k with label j: the product of the kernel block with the
// one-hot label matrix Z (Z_kj = 1 when landmark k has label j).  The block
// is the FP16 landmark-major K^T [nL][ldk] of the reduced-precision Gaussian
// path; a CTA owns one tile of 128 samples and streams its 128 columns in
// landmark order, 64 landmarks (16 KB) per step, through TMA into shared
// memory, where they are the MN-major A operand of tcgen05.mma kind::f16
// (M = 128 samples, N = 16 clusters, K = 16 landmarks per instruction).  Z is
// built once in shared memory as K-major B tiles of 64 landmarks (values 0
// and 1, exact in FP16) and patched when landmark labels change; the
// products accumulate in FP32 in tensor memory.  The sum runs over every
// landmark in index order whatever the labels, so the stream needs no
// gather and no per-iteration sort.
//
// Two rings of TMA stages per CTA, each with its own producer thread, MMA
// issuer thread and tensor-memory accumulator (their sums are added in a
// fixed order): one ring's request-completion round trip limits a CTA to
// about 6 TB/s over the GPU, two reach the L2 read rate.
//
// Per iteration: the epilogue (four warps, one thread per sample) reads the
// accumulators, adds the tile's g_hat numerators (Eq. 16: the landmark rows'
// f_hat numerators of their own cluster) as fixed-point integers (exact and
// order-free), and every CTA meets at grid barrier A; then g_hat, the
// distances d_ij = K_ii - 2 f_hat_ij + g_hat_j, argmin (lowest j on ties),
// the FP32 re-score of near ties, Omega and the number of changed labels
// (fixed point again), the new landmark labels (written to the support table
// and appended to a change list), and grid barrier B.  After B every CTA
// reads the totals (trace, early stop) and applies the change list to its Z
// and cluster sizes; the MMA issuers then start the next iteration, while the
// producers have already filled the rings with its first tiles (the block
// does not change between iterations).
//
// The barriers need every CTA resident: a cooperative launch of one CTA per
// 128-sample tile, at most one per SM.  Every wait is bounded; a grid
// barrier that gives up sets the error word and every CTA winds down (the
// host reports KKM_ETIMEOUT); the TMA copies in flight are waited for and the
// tensor memory is freed before the CTA exits.
#include <cuda.h>
#include <cuda_fp16.h>

#include "device_common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace kkm {

constexpr int kTcRings = 2;
constexpr int kTcMaxStages = 4;      // stages per ring
constexpr int kTcStage = 16384;      // 64 landmark rows x 128 samples of FP16: two 64-column TMA boxes
constexpr int kTcZTile = 2048;       // 16 clusters x 64 landmarks of FP16
constexpr int kTcN = 16;             // clusters per MMA (N)
constexpr int kTcEpiWarps = 4;       // one thread per sample of the tile
constexpr int kTcThreads = 32 * (2 * kTcRings + kTcEpiWarps);
constexpr int kTcTmemCols = 64;      // two sets (iteration parity) of kTcRings accumulators of kTcN columns
constexpr unsigned kTcBarSpin = 1u << 25;  // polls per grid barrier (>= ~1 s)
constexpr size_t kTcMaxDynSmem = 227 * 1024 - 1280;  // leaves room for the static shared memory

// kind::f16 instruction descriptor: FP32 accumulator, F16 A (MN-major) and
// F16 B (K-major), N = 16, M = 128.
__host__ __device__ constexpr uint32_t tc_iter_idesc() {
  return (1u << 4) | (1u << 15) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// What the epilogue tells the MMA issuers after an iteration: the landmark
// labels did not change (the pass of the next iteration already made with the
// same Z stands), they changed (Z was patched: the pass is made again), or the
// loop ended.
constexpr int kVerdictSame = 0, kVerdictChanged = 1, kVerdictStop = 2;
// the loop ended and the last iteration moved landmark labels: one more pass
// with the patched Z gives f_hat and g_hat of the final supports (Eq. 10)
constexpr int kVerdictFinal = 3;

struct TcIterShared {
  uint64_t full[kTcRings][kTcMaxStages];
  uint64_t empty[kTcRings][kTcMaxStages];
  uint64_t acc_done[2];        // iteration parity: every active ring's MMAs of the iteration are complete
  uint64_t zready;             // Z and the cluster sizes of the first iteration are built
  uint64_t vready;             // the verdict of an iteration is posted (one phase per iteration)
  uint64_t mma_idle[kTcRings]; // the ring's last MMAs are complete (teardown)
  int verdict;
  uint32_t tmem;
  int abort_flag;
  int stop;
  int never;  // stays 0
  int consumed[kTcRings];
  int nj[kTcN];
  float ghf[kTcN];
  double gh[kTcN];
  unsigned long long gsum[kTcN];
  unsigned long long osum_w[kTcEpiWarps];
  int chsum_w[kTcEpiWarps];
  unsigned long long kbest[kTcN];  // Eq. 10 keys of this tile
  int kcnt[kTcN];
  double tot_om;
  int tot_ch, tot_lm;
  int ok;
};

static_assert(sizeof(TcIterShared) <= 1280, "static shared memory beside the dynamic share");

// Barrier of the epilogue warps only (named barrier 1), after the warp has
// reconverged.
__device__ __forceinline__ void epi_sync() {
  __syncwarp();
  asm volatile("barrier.sync 1, %0;" ::"n"(kTcEpiWarps * 32) : "memory");
}

__device__ __forceinline__ unsigned tc_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Waits until *bar reaches target; false after the bound or when another CTA
// already gave up (*err).
__device__ bool tc_grid_wait(const unsigned* bar, unsigned target, int* err) {
  for (unsigned polls = 0; polls < kTcBarSpin; ++polls) {
    if (tc_ld_acquire(bar) >= target) return true;
    if ((polls & 63u) == 63u && *reinterpret_cast<volatile int*>(err) != 0) break;
    if (polls > 256) __nanosleep(20);
  }
  atomicExch(err, 1);
  return false;
}

// Arrival at a grid barrier: a release add (the CTA's earlier writes, ordered
// before it by the CTA barrier, become visible to the threads that see the
// count).
__device__ __forceinline__ void tc_grid_arrive(unsigned* bar) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
}

// Byte offset of Z's element (cluster n, landmark k): K-major tiles of 64
// landmarks, 128-byte rows with the 128-byte swizzle.
__device__ __forceinline__ uint32_t z_offset(int k, int n) {
  const int kk = k & 63;
  return (uint32_t)((k >> 6) * kTcZTile + (n >> 3) * 1024 + (n & 7) * 128 + ((((kk >> 3) ^ (n & 7))) << 4) +
                    (kk & 7) * 2);
}

__global__ void __launch_bounds__(kTcThreads, 1)
iterate_tc_kernel(const __grid_constant__ CUtensorMap map, int Ni, Supports S, IterState I, int iters, int nstages,
                  int32_t* __restrict__ u, float* __restrict__ margin, float* __restrict__ fhat_out,
                  double* __restrict__ ghat_out, int early_stop, RescoreArgs R, unsigned long long* __restrict__ keys,
                  int32_t* __restrict__ kcount, double* __restrict__ ghat_final) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  uint8_t* const base =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ TcIterShared sh;
  griddep_wait();
  if (I.done && *I.done) return;  // early stop: the same flag in every CTA
  const int C = S.C, nL = S.nL;
  const int nKT = (nL + 63) / 64;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * 128;
  const int active = nKT < kTcRings ? nKT : kTcRings;  // rings with at least one tile
  uint8_t* const ring0 = base;
  uint8_t* const Z = base + (size_t)kTcRings * nstages * kTcStage;
  const int t0 = *I.trace_count;

  if (threadIdx.x == 0) {
    for (int r = 0; r < kTcRings; ++r) {
      for (int s = 0; s < nstages; ++s) {
        mbar_init(&sh.full[r][s], 1);
        mbar_init(&sh.empty[r][s], 1);
      }
      mbar_init(&sh.mma_idle[r], 1);
    }
    mbar_init(&sh.acc_done[0], (uint32_t)active);
    mbar_init(&sh.acc_done[1], (uint32_t)active);
    mbar_init(&sh.zready, 1);
    mbar_init(&sh.vready, 1);
    sh.verdict = kVerdictSame;
    sh.abort_flag = 0;
    sh.stop = 0;
    sh.never = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < kTcN) {
    sh.nj[threadIdx.x] = 0;
    sh.gsum[threadIdx.x] = 0ull;
    sh.kbest[threadIdx.x] = ~0ull;
    sh.kcnt[threadIdx.x] = 0;
  }
  if (threadIdx.x < kTcRings) sh.consumed[threadIdx.x] = 0;
  if (warp == kTcRings) {  // the first MMA warp owns the tensor memory
    tmem_alloc(&sh.tmem, kTcTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;
  volatile int* const abort_flag = &sh.abort_flag;
  volatile int* const stop_flag = &sh.stop;
  int issued = 0;  // producers: stages issued

  if (warp < kTcRings) {
    // ---------------- TMA producer of ring r: its tiles kt = r, r + R, ...
    // pass after pass (the block is the same in every iteration, so a pass of
    // copies serves whichever pass of the MMA issuer consumes it) until the
    // loop ends
    const int r = warp;
    if (lane == 0 && r < active) {
      uint64_t pol;
      asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
      int s = 0;
      uint32_t ph = 0;
      const int passes = 2 * iters + 1;  // every iteration at most twice (a speculation made again)
      bool go = true;
      for (int pass = 0; pass < passes && go; ++pass) {
        for (int kt = r; kt < nKT; kt += kTcRings) {
          bool got = false;
          // (the flags are read every few polls: a try_wait that finds the
          // slot still busy may suspend the thread for a while, and at the
          // end of the loop the slot is never released)
          for (uint32_t it = 0; it < kTcSpinLimit; ++it) {
            if (mbar_try_wait(&sh.empty[r][s], ph ^ 1u)) {
              got = true;
              break;
            }
            if ((it & 7u) == 7u && (*stop_flag || *abort_flag)) break;
          }
          if (!got || *stop_flag || *abort_flag) {
            if (!got && !*stop_flag && !*abort_flag) {
              atomicExch(I.err, 2);
              *abort_flag = 1;
            }
            go = false;
            break;
          }
          uint8_t* a = ring0 + ((size_t)r * nstages + s) * kTcStage;
          mbar_expect_tx(&sh.full[r][s], kTcStage);
          tma_load_2d_hint(&map, &sh.full[r][s], a, i0, kt * 64, pol);
          tma_load_2d_hint(&map, &sh.full[r][s], a + kTcStage / 2, i0 + 64, kt * 64, pol);
          ++issued;
          if (++s == nstages) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
    }
  } else if (warp < 2 * kTcRings) {
    // ---------------- MMA issuer of ring r: D_r = A (block tiles) x Z tiles.
    // The pass of iteration t + 1 starts as soon as that of t is issued, with
    // the Z of iteration t: when the verdict of t says the landmark labels did
    // not change it stands, else it is made again with the patched Z.
    const int r = warp - kTcRings;
    if (lane == 0 && r < active) {
      int s = 0, consumed = 0;
      uint32_t ph = 0;
      const uint32_t idesc = tc_iter_idesc();
      // one pass over the ring's tiles into the accumulator of parity p;
      // false on abort
      auto run_pass = [&](int p) -> bool {
        const uint32_t d_tmem = tmem + (uint32_t)((p * kTcRings + r) * kTcN);
        bool first = true;
        for (int kt = r; kt < nKT; kt += kTcRings) {
          if (!mbar_wait(&sh.full[r][s], ph, abort_flag)) {
            if (!*abort_flag) atomicExch(I.err, 4);
            *abort_flag = 1;
            return false;
          }
          tc_fence_after();
          const uint32_t a = smem_u32(ring0 + ((size_t)r * nstages + s) * kTcStage);
          const uint32_t b = smem_u32(Z + (size_t)kt * kTcZTile);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)  // 16 landmarks (two 8-row K atoms) per instruction
            umma_f16(d_tmem, sw128_mn_desc(a + ks * 2048, kTcStage / 2, 1024), sw128_desc(b + ks * 32), idesc,
                     (first && ks == 0) ? 0u : 1u);
          first = false;
          umma_commit(&sh.empty[r][s]);
          ++consumed;
          if (++s == nstages) {
            s = 0;
            ph ^= 1u;
          }
        }
        return true;
      };
      bool ok = mbar_wait(&sh.zready, 0u, abort_flag);  // the first iteration's Z
      if (!ok && !*abort_flag) {
        atomicExch(I.err, 3);
        *abort_flag = 1;
      }
      if (ok) {
        tc_fence_after();
        ok = run_pass(0);
        if (ok) umma_commit(&sh.acc_done[0]);
      }
      bool ended = false;  // a verdict ended the loop (or a wait gave up)
      for (int t = 0; ok && t + 1 < iters; ++t) {
        const int p = (t + 1) & 1;
        if (!run_pass(p)) {  // iteration t + 1 with the Z of iteration t
          ended = true;
          break;
        }
        if (!mbar_wait(&sh.vready, (uint32_t)t & 1u, abort_flag)) {
          if (!*abort_flag) atomicExch(I.err, 3);
          *abort_flag = 1;
          ended = true;
          break;
        }
        tc_fence_after();  // the epilogue's reads of the other accumulator set are ordered before what follows
        const int v = *reinterpret_cast<volatile int*>(&sh.verdict);
        if (v == kVerdictStop || *abort_flag) {
          ended = true;
          break;
        }
        if ((v == kVerdictChanged || v == kVerdictFinal) && !run_pass(p)) {  // Z was patched: the pass again
          ended = true;
          break;
        }
        umma_commit(&sh.acc_done[p]);
        if (v == kVerdictFinal) {
          ended = true;
          break;
        }
      }
      if (ok && !ended) {
        // the last iteration's verdict may ask for the final pass
        if (mbar_wait(&sh.vready, (uint32_t)(iters - 1) & 1u, abort_flag)) {
          tc_fence_after();
          const int v = *reinterpret_cast<volatile int*>(&sh.verdict);
          if (v == kVerdictFinal && !*abort_flag && run_pass(iters & 1)) umma_commit(&sh.acc_done[iters & 1]);
        } else {
          if (!*abort_flag) atomicExch(I.err, 3);
          *abort_flag = 1;
        }
      }
      sh.consumed[r] = consumed;
      if (consumed > 0) umma_commit(&sh.mma_idle[r]);
    }
  } else {
    // ---------------- epilogue: one thread per sample of the tile
    const int q = warp & 3;  // tensor-memory lane quarter of this warp
    const int et = threadIdx.x - 2 * kTcRings * 32;
    const int row = q * 32 + lane;
    const int i = i0 + row;
    const bool valid = i < Ni;
    int cur = valid ? u[i] : 0;
    const int cord = (valid && S.col_ord) ? S.col_ord[i] : -1;
    const float ks = 1.0f;  // K_ii of a Gaussian kernel
    const float inf = __int_as_float(0x7f800000);
    unsigned long long* const facc = I.facc;
    const double gscale = ldexp(1.0, I.gfix_shift), oscale = ldexp(1.0, I.fom_shift);
    const float tau = I.flag_tau;
    const bool rescore = R.Xi != nullptr && tau > 0.0f;

    // Z and the cluster sizes from the landmark labels: Z zeroed, then a one
    // (0x3C00) at (label, landmark) for every landmark, the labels of eight
    // landmarks per thread loaded together; the sizes by one shared atomic per
    // distinct label in a warp
    {
      uint4* const z4 = reinterpret_cast<uint4*>(Z);
      for (int e = et; e < nKT * (kTcZTile / 16); e += kTcEpiWarps * 32) z4[e] = make_uint4(0u, 0u, 0u, 0u);
      epi_sync();
      // the trip count depends on the warp only (every lane takes part in
      // each match; lanes past nL carry no label)
      constexpr int kZPre = 8;
      const int wbase = et & ~31;
      for (int kb = wbase; kb < nL; kb += kZPre * kTcEpiWarps * 32) {
        int lab[kZPre];
#pragma unroll
        for (int p = 0; p < kZPre; ++p) {
          const int k = kb + p * kTcEpiWarps * 32 + lane;
          lab[p] = k < nL ? __ldcg(S.lab + k) : -1;
        }
#pragma unroll
        for (int p = 0; p < kZPre; ++p) {
          const int k = kb + p * kTcEpiWarps * 32 + lane;
          const int l = lab[p];
          const unsigned peers = __match_any_sync(kFull, l);
          if (l >= 0 && l < kTcN) {
            *reinterpret_cast<unsigned short*>(Z + z_offset(k, l)) = 0x3C00;
            if (lane == __ffs(peers) - 1) atomicAdd(&sh.nj[l], __popc(peers));
          }
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // Z is read by the tensor cores
    epi_sync();
    if (et == 0) mbar_arrive(&sh.zready);

    unsigned target = 0;
    int t = 0;
    bool failed = false;
    for (; t < iters; ++t) {
      // 1. this tile's f_hat numerators (the rings' accumulators, added in order)
      bool ok = true;
      if (lane == 0) ok = mbar_wait(&sh.acc_done[t & 1], (uint32_t)(t >> 1) & 1u, abort_flag);
      ok = __shfl_sync(kFull, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        if (lane == 0) {
          if (!*abort_flag) atomicExch(I.err, 5);
          *abort_flag = 1;
        }
        failed = true;
        break;
      }
      tc_fence_after();
      float D[kTcN];
#pragma unroll
      for (int j = 0; j < kTcN; ++j) D[j] = 0.0f;
      for (int r = 0; r < active; ++r) {
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(((t & 1) * kTcRings + r) * kTcN), v);
#pragma unroll
        for (int j = 0; j < kTcN; ++j) D[j] += __uint_as_float(v[j]);
      }
      tc_fence_before();
      // 2. g_hat numerators (Eq. 16): a landmark row's numerator of its own
      // cluster, as a fixed-point integer (value * 2^gfix_shift), added in
      // shared memory (integer sums: exact in any order)
      if (valid && cord >= 0) {
        float dl = 0.0f;
#pragma unroll
        for (int j = 0; j < kTcN; ++j)
          if (j == cur) dl = D[j];
        atomicAdd(&sh.gsum[cur], (unsigned long long)llrint((double)dl * gscale));
      }
      epi_sync();
      if (et < C) {
        const unsigned long long g = sh.gsum[et];
        if (g) atomicAdd(facc + (t & 1) * (C + 3) + et, g);
        sh.gsum[et] = 0ull;
      }
      epi_sync();
      if (et == 0) tc_grid_arrive(I.bar);  // grid barrier A: arrive now, wait after the work that needs no g_hat
      target += gridDim.x;
      // e_ij = K_ii - 2 f_hat_ij (Eq. 15 without g_hat)
      float e[kTcN];
#pragma unroll
      for (int j = 0; j < kTcN; ++j) {
        const int n = j < C ? sh.nj[j] : 0;
        const float fh = n > 0 ? D[j] / (float)n : __int_as_float(0x7fc00000);
        e[j] = n > 0 ? ks - 2.0f * fh : inf;
        if (fhat_out && valid && j < C) fhat_out[(int64_t)i * C + j] = fh;
      }
      if (et == 0) sh.ok = tc_grid_wait(I.bar, target, I.err) ? 1 : 0;
      epi_sync();
      if (!sh.ok) {
        failed = true;
        break;
      }
      // 3. g_hat of every cluster, the same in every CTA
      if (et < C) {
        const int n = sh.nj[et];
        double gv = __longlong_as_double(0x7ff8000000000000LL);
        if (n > 0)
          gv = I.ghat_in ? I.ghat_in[et]
                         : (double)__ldcg(facc + (t & 1) * (C + 3) + et) / gscale / ((double)n * (double)n);
        sh.gh[et] = gv;
        sh.ghf[et] = (float)gv;
      }
      // the other set was last read before this barrier: zero it for the
      // next iteration (published by barrier B)
      if (blockIdx.x == 0 && et < C + 3) facc[((t + 1) & 1) * (C + 3) + et] = 0ull;
      epi_sync();
      if (blockIdx.x == 0 && ghat_out && et < C) ghat_out[et] = sh.gh[et];
      // 4. distances and argmin (lowest j on ties)
      float d[kTcN];
      float best = inf, second = inf;
      int bj = 0;
#pragma unroll
      for (int j = 0; j < kTcN; ++j) {
        d[j] = e[j] < inf ? e[j] + sh.ghf[j < C ? j : 0] : inf;
        if (d[j] < best) {
          second = best;
          best = d[j];
          bj = j;
        } else if (d[j] < second) {
          second = d[j];
        }
      }
      const float scale = ks + sh.ghf[bj];
      const bool flagged = valid && rescore && second < inf && (second - best) < tau * fmaxf(fabsf(second), scale);
      // 5. near-tie re-score: every candidate cluster of a flagged row gets
      // f_hat from exact FP32 kernel values of its support (one landmark per
      // lane in index order, dot products in chunks of 32 products, then a
      // fixed xor tree); one flagged row at a time per warp
      unsigned fm = __ballot_sync(kFull, flagged);
      while (fm) {
        const int L = __ffs(fm) - 1;
        fm &= fm - 1;
        const float bL = __shfl_sync(kFull, best, L), sL = __shfl_sync(kFull, scale, L);
        const int iL = i0 + q * 32 + L;
        const float4* xi = reinterpret_cast<const float4*>(R.Xi + (int64_t)iL * R.dp);
        const float ni = R.nXi[iL];
        unsigned cmask = 0;  // the row's candidate clusters
#pragma unroll
        for (int j = 0; j < kTcN; ++j) {
          const float dj = __shfl_sync(kFull, d[j], L);
          if (j < C && sh.nj[j] > 0 && dj - bL < tau * fmaxf(fabsf(dj), sL)) cmask |= 1u << j;
        }
        while (cmask) {
          const int j = __ffs(cmask) - 1;
          cmask &= cmask - 1;
          float accr = 0.0f;
          for (int k = lane; k < nL; k += 32) {
            if (*reinterpret_cast<const unsigned short*>(Z + z_offset(k, j)) == 0) continue;
            if (R.K32) {  // the block's own FP32 values
              accr += __ldg(R.K32 + (int64_t)k * R.ldk32 + iL);
              continue;
            }
            const float4* xl = reinterpret_cast<const float4*>(R.XL + (int64_t)k * R.dp);
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
            accr += (S.L[k] == iL) ? 1.0f : exp2f(fmaxf(ni + R.nXL[k] - 2.0f * dot, 0.0f) * R.neg_scale);
          }
          accr = warp_sum_f32(accr);
          const float dn = ks - 2.0f * (accr / (float)sh.nj[j]) + sh.ghf[j];
#pragma unroll
          for (int jj = 0; jj < kTcN; ++jj)
            if (jj == j && lane == L) d[jj] = dn;
        }
      }
      if (flagged) {
        best = inf;
        second = inf;
        bj = 0;
#pragma unroll
        for (int j = 0; j < kTcN; ++j) {
          if (d[j] < best) {
            second = best;
            best = d[j];
            bj = j;
          } else if (d[j] < second) {
            second = d[j];
          }
        }
      }
      // 6. labels, the changed landmarks, cost and counts
      const bool ch = valid && bj != cur;
      if (ch && cord >= 0) {
        S.lab[cord] = bj;
        const int idx = (int)atomicAdd(facc + (t & 1) * (C + 3) + C + 2, 1ull);
        I.lm_list[(size_t)(t & 1) * nL + idx] = (cord << 8) | (cur << 4) | bj;
      }
      // the cost share as a fixed-point integer (two's complement: a slightly
      // negative d near 0 adds correctly), summed per warp, then per CTA
      unsigned long long om = 0ull;
      if (valid) {
        cur = bj;
        if (margin) margin[i] = second - best;
        if (best < inf) om = (unsigned long long)llrint((double)best * oscale);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) om += __shfl_xor_sync(kFull, om, o);
      const int chw = (int)__reduce_add_sync(kFull, ch ? 1u : 0u);
      if (lane == 0) {
        sh.osum_w[warp - 2 * kTcRings] = om;
        sh.chsum_w[warp - 2 * kTcRings] = chw;
      }
      epi_sync();
      if (et == 0) {  // grid barrier B
        unsigned long long o = 0ull;
        int c = 0;
        for (int w = 0; w < kTcEpiWarps; ++w) {
          o += sh.osum_w[w];
          c += sh.chsum_w[w];
        }
        unsigned long long* a = facc + (t & 1) * (C + 3) + C;
        atomicAdd(a, o);
        if (c) atomicAdd(a + 1, (unsigned long long)c);
        tc_grid_arrive(I.bar);
      }
      target += gridDim.x;
      if (et == 0) {
        sh.ok = tc_grid_wait(I.bar, target, I.err) ? 1 : 0;
        if (sh.ok) {
          const unsigned long long* a = facc + (t & 1) * (C + 3) + C;
          sh.tot_om = (double)(long long)__ldcg(a) / oscale;
          sh.tot_ch = (int)__ldcg(a + 1);
          sh.tot_lm = (int)__ldcg(a + 2);
        }
      }
      epi_sync();
      if (!sh.ok) {
        failed = true;
        break;
      }
      // 7. the trace, early stop, and the next iteration's Z and sizes
      if (blockIdx.x == 0 && et == 0) {
        I.trace_omega[t0 + t] = sh.tot_om;
        I.trace_changed[t0 + t] = sh.tot_ch;
      }
      const bool stop = (early_stop && sh.tot_ch == 0) || t + 1 == iters;
      const int lm = sh.tot_lm;
      const bool final_pass = stop && lm > 0 && keys != nullptr;
      if ((!stop || final_pass) && lm > 0) {
        for (int c = et; c < lm; c += kTcEpiWarps * 32) {
          const int v = __ldcg(I.lm_list + (size_t)(t & 1) * nL + c);
          const int k = v >> 8, from = (v >> 4) & 15, to = v & 15;
          *reinterpret_cast<unsigned short*>(Z + z_offset(k, from)) = 0;
          *reinterpret_cast<unsigned short*>(Z + z_offset(k, to)) = 0x3C00;
          atomicSub(&sh.nj[from], 1);
          atomicAdd(&sh.nj[to], 1);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      epi_sync();
      if (et == 0) {
        if (stop && !final_pass) *stop_flag = 1;
        sh.verdict = final_pass ? kVerdictFinal
                                : (stop ? kVerdictStop : (lm > 0 ? kVerdictChanged : kVerdictSame));
        mbar_arrive(&sh.vready);
      }
      if (stop) {
        ++t;
        if (keys) {
          // Eq. 10 on the final supports: the keys (K_ii - 2 f_hat_ij, sample)
          // of every cluster, the member counts and g_hat
          if (final_pass) {
            // the pass with the patched Z: f_hat and g_hat of the final labels
            bool okf = true;
            if (lane == 0) okf = mbar_wait(&sh.acc_done[t & 1], (uint32_t)(t >> 1) & 1u, abort_flag);
            okf = __shfl_sync(kFull, okf ? 1 : 0, 0) != 0;
            if (!okf) {
              if (lane == 0) {
                if (!*abort_flag) atomicExch(I.err, 5);
                *abort_flag = 1;
              }
              failed = true;
              break;
            }
            tc_fence_after();
            float Df[kTcN];
#pragma unroll
            for (int j = 0; j < kTcN; ++j) Df[j] = 0.0f;
            for (int r = 0; r < active; ++r) {
              uint32_t v[16];
              tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(((t & 1) * kTcRings + r) * kTcN), v);
#pragma unroll
              for (int j = 0; j < kTcN; ++j) Df[j] += __uint_as_float(v[j]);
            }
            tc_fence_before();
            epi_sync();
            if (et == 0) *stop_flag = 1;  // the producers may wind down
            if (valid && cord >= 0) {
              float dl = 0.0f;
#pragma unroll
              for (int j = 0; j < kTcN; ++j)
                if (j == cur) dl = Df[j];
              atomicAdd(&sh.gsum[cur], (unsigned long long)llrint((double)dl * gscale));
            }
            epi_sync();
            if (et < C) {
              const unsigned long long g = sh.gsum[et];
              if (g) atomicAdd(facc + (t & 1) * (C + 3) + et, g);
              sh.gsum[et] = 0ull;
            }
            epi_sync();
            if (et == 0) tc_grid_arrive(I.bar);
            target += gridDim.x;
#pragma unroll
            for (int j = 0; j < kTcN; ++j) {
              const int n = j < C ? sh.nj[j] : 0;
              e[j] = n > 0 ? ks - 2.0f * (Df[j] / (float)n) : inf;
            }
            if (et == 0) sh.ok = tc_grid_wait(I.bar, target, I.err) ? 1 : 0;
            epi_sync();
            if (!sh.ok) {
              failed = true;
              break;
            }
            if (et < C) {
              const int n = sh.nj[et];
              sh.gh[et] = n > 0 ? (double)__ldcg(facc + (t & 1) * (C + 3) + et) / gscale / ((double)n * (double)n)
                                : __longlong_as_double(0x7ff8000000000000LL);
            }
            epi_sync();
          }
          if (valid) {
#pragma unroll
            for (int j = 0; j < kTcN; ++j)
              if (j < C && sh.nj[j] > 0) atomicMin(&sh.kbest[j], pack_key(e[j], (uint32_t)i));
            atomicAdd(&sh.kcnt[cur], 1);
          }
          epi_sync();
          if (et < C) {
            if (sh.kbest[et] != ~0ull) atomicMin(keys + et, sh.kbest[et]);
            if (sh.kcnt[et]) atomicAdd(kcount + et, sh.kcnt[et]);
            if (blockIdx.x == 0) {
              if (ghat_final) ghat_final[et] = sh.gh[et];
              S.n_j[et] = sh.nj[et];
            }
          }
        }
        break;
      }
    }
    if (failed && et == 0) {
      *abort_flag = 1;
      *stop_flag = 1;
      sh.verdict = kVerdictStop;
      mbar_arrive(&sh.vready);  // wakes the MMA issuers, which then see the flags
    }
    if (valid) u[i] = cur;
    if (blockIdx.x == 0 && et == 0) {
      *I.trace_count = t0 + t;
      if (early_stop && t < iters && !failed) *I.done = 1;
    }
  }

  // ---------------- teardown: the copies in flight land, the MMAs complete,
  // the tensor memory is freed
  __syncwarp();
  __syncthreads();
  volatile int* const never = &sh.never;  // drain waits do not give up on an abort
  if (warp < kTcRings && lane == 0) {
    const int r = warp;
    for (int seq = sh.consumed[r]; seq < issued; ++seq)
      if (!mbar_wait(&sh.full[r][seq % nstages], (uint32_t)(seq / nstages) & 1u, never)) atomicExch(I.err, 6);
  } else if (warp >= kTcRings && warp < 2 * kTcRings && lane == 0) {
    if (sh.consumed[warp - kTcRings] > 0 && !mbar_wait(&sh.mma_idle[warp - kTcRings], 0u, never))
      atomicExch(I.err, 7);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kTcRings) {
    tc_fence_after();
    tmem_dealloc(tmem, kTcTmemCols);
  }
}

// Stages per ring and dynamic shared memory of the tensor-core loop for a
// block of Ni samples and nL landmarks; false when it does not apply (more
// than 16 clusters, more 128-sample tiles than SMs, or Z does not fit).
bool tc_iter_shape(int Ni, int nL, int C, int n_sms, int* nstages, size_t* smem) {
  if (C < 1 || C > kTcN || Ni < 1 || nL < 1 || nL >= (1 << 23)) return false;
  if (ceil_div(Ni, 128) > n_sms) return false;
  const size_t zbytes = (size_t)ceil_div(nL, 64) * kTcZTile;
  for (int s = kTcMaxStages; s >= 2; --s) {
    const size_t bytes = 1024 + (size_t)kTcRings * s * kTcStage + zbytes;
    if (bytes <= kTcMaxDynSmem) {
      *nstages = s;
      *smem = bytes;
      return true;
    }
  }
  return false;
}

cudaError_t launch_iterate_tc(const __half* KT, int64_t ldk, int Ni, const Supports& S, const IterState& I, int iters,
                              int32_t* u, float* margin, float* fhat_out, double* ghat_out, int early_stop,
                              int n_sms, cudaStream_t st, const RescoreArgs& R, unsigned long long* keys,
                              int32_t* kcount, double* ghat_final) {
  if (iters <= 0) return cudaSuccess;
  int nstages = 0;
  size_t smem = 0;
  if (!tc_iter_shape(Ni, S.nL, S.C, n_sms, &nstages, &smem)) return cudaErrorInvalidValue;
  if (!I.facc || !I.lm_list || !I.bar || !I.err || (ldk * 2) % 16 != 0 ||
      (reinterpret_cast<uintptr_t>(KT) & 15) != 0)
    return cudaErrorInvalidValue;
  auto enc = get_encode();
  if (!enc) return cudaErrorInvalidValue;
  alignas(64) CUtensorMap map;
  cuuint64_t dims[2] = {(cuuint64_t)Ni, (cuuint64_t)S.nL};
  cuuint64_t strides[1] = {(cuuint64_t)(ldk * 2)};
  cuuint32_t box[2] = {64, 64};
  cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half*>(KT), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  static const cudaError_t attr =
      cudaFuncSetAttribute(iterate_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcMaxDynSmem);
  if (attr != cudaSuccess) return attr;
  // the barrier counter and the fixed-point accumulators start at zero
  cudaError_t e = cudaMemsetAsync(I.bar, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(I.facc, 0, sizeof(unsigned long long) * 2 * (S.C + 3), st);
  if (e != cudaSuccess) return e;
  IterState J = I;
  // cost shares as fixed point: |Omega| <= 4 Ni for the Gaussian kernels
  int b = 0;
  while (b < 40 && ((int64_t)1 << b) <= Ni) ++b;  // Ni < 2^b
  J.fom_shift = std::max(8, 60 - b);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ceil_div(Ni, 128));
  cfg.blockDim = dim3(kTcThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attrs[1];
  attrs[0].id = cudaLaunchAttributeCooperative;
  attrs[0].val.cooperative = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, iterate_tc_kernel, map, Ni, S, J, iters, nstages, u, margin, fhat_out, ghat_out,
                            early_stop, R, keys, kcount, ghat_final);
}

}  // namespace kkm
