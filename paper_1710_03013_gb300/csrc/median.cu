// Bandwidth rule: the k-th smallest entry of the strict upper triangle of a
// distance matrix, found by a 4-pass radix select on the float bit patterns
// (non-negative floats order like their unsigned bit patterns).
#include "device_common.cuh"
#include "internal.h"

namespace kkm {

struct SelectState {
  uint32_t prefix;
  uint32_t mask;
  uint32_t k;
  uint32_t pad;
  uint32_t hist[256];
};

__global__ void select_init_kernel(SelectState* s, uint32_t k) {
  if (threadIdx.x == 0) {
    s->prefix = 0;
    s->mask = 0;
    s->k = k;
  }
  s->hist[threadIdx.x] = 0;
}

// Histogram of byte `shift` of the keys that match the prefix so far, over
// the strict upper triangle: one CTA per row at a time, threads over the
// columns right of the diagonal.
__global__ void __launch_bounds__(256)
select_hist_kernel(const float* __restrict__ D, int M, int64_t ld, SelectState* s, int shift) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t prefix = s->prefix, mask = s->mask;
  for (int i = blockIdx.x; i < M; i += gridDim.x) {
    const float* row = D + (int64_t)i * ld;
    for (int j = i + 1 + threadIdx.x; j < M; j += blockDim.x) {
      const uint32_t key = __float_as_uint(row[j]);
      if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
    }
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&s->hist[threadIdx.x], h[threadIdx.x]);
}

// One warp: the bin holding the k-th key (lanes own 8 bins each; a warp
// prefix sum finds the lane, the lane its bin), then the next byte's state.
__global__ void select_pick_kernel(SelectState* s, int shift, float* out, int last) {
  const int lane = threadIdx.x;
  const uint32_t k = s->k;
  uint32_t v[8], own = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    v[q] = s->hist[lane * 8 + q];
    own += v[q];
  }
  uint32_t incl = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t excl = incl - own;
  // the lane whose range [excl, incl) holds k (the last lane if k is past
  // every key, which cannot happen for a valid k)
  const unsigned hit = __ballot_sync(kFull, k >= excl && k < incl);
  const int owner = hit ? __ffs(hit) - 1 : 31;
  if (lane == owner) {
    uint32_t cum = excl;
    int b = lane * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (k < cum + v[q]) {
        b = lane * 8 + q;
        break;
      }
      cum += v[q];
      b = lane * 8 + q;
    }
    s->k = k - cum;
    s->prefix |= (uint32_t)b << shift;
    s->mask |= 255u << shift;
    if (last) *out = __uint_as_float(s->prefix);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 8; ++q) s->hist[lane * 8 + q] = 0;
}

cudaError_t launch_select_upper(const float* D, int M, int64_t ld, int64_t k, uint32_t* scratch,
                                float* out, cudaStream_t st) {
  SelectState* s = reinterpret_cast<SelectState*>(scratch);
  select_init_kernel<<<1, 256, 0, st>>>(s, (uint32_t)k);
  const int grid = std::min(M, 152 * 8);
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    select_hist_kernel<<<grid, 256, 0, st>>>(D, M, ld, s, shift);
    select_pick_kernel<<<1, 32, 0, st>>>(s, shift, out, pass == 3);
  }
  prof_more_launches(8);
  return cudaGetLastError();
}

}  // namespace kkm
