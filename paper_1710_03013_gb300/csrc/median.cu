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

__global__ void __launch_bounds__(256)
select_hist_kernel(const float* __restrict__ D, int M, int64_t ld, SelectState* s, int shift) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t prefix = s->prefix, mask = s->mask;
  const int64_t total = (int64_t)M * M;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / M), j = (int)(e % M);
    if (j <= i) continue;
    const uint32_t key = __float_as_uint(D[(int64_t)i * ld + j]);
    if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255u], 1u);
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&s->hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void select_pick_kernel(SelectState* s, int shift, float* out, int last) {
  if (threadIdx.x != 0) return;
  uint32_t cum = 0, k = s->k;
  int b = 0;
  for (; b < 256; ++b) {
    if (k < cum + s->hist[b]) break;
    cum += s->hist[b];
  }
  if (b > 255) b = 255;
  s->k = k - cum;
  s->prefix |= (uint32_t)b << shift;
  s->mask |= 255u << shift;
  for (int q = 0; q < 256; ++q) s->hist[q] = 0;
  if (last) *out = __uint_as_float(s->prefix);
}

cudaError_t launch_select_upper(const float* D, int M, int64_t ld, int64_t k, uint32_t* scratch,
                                float* out, cudaStream_t st) {
  SelectState* s = reinterpret_cast<SelectState*>(scratch);
  select_init_kernel<<<1, 256, 0, st>>>(s, (uint32_t)k);
  const int grid = (int)std::min<int64_t>(ceil_div((int64_t)M * M, 256), 152 * 8);
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    select_hist_kernel<<<grid, 256, 0, st>>>(D, M, ld, s, shift);
    select_pick_kernel<<<1, 32, 0, st>>>(s, shift, out, pass == 3);
  }
  return cudaGetLastError();
}

}  // namespace kkm
