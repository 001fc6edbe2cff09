// Block reductions in FP64 and the last-block-done pattern: every block
// writes its partial, and the last block of an instance to finish (counted
// with an atomic, no waiting) sums the partials in a fixed order.
#pragma once
#include <cuda_runtime.h>

namespace gsm {

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// Returns true in every thread of the last block; out[b] then holds the sum.
__device__ __forceinline__ bool last_block_sum(double v, double *red, double *partial, unsigned *counter,
                                               double *out, int b, int nblk, int blk) {
  __shared__ int am_last;
  double s = block_sum(v, red);
  if (threadIdx.x == 0) {
    partial[(long long)b * nblk + blk] = s;
    __threadfence();
    unsigned t = atomicAdd(&counter[b], 1u);
    am_last = (t == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  double acc = 0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += __ldcg(&partial[(long long)b * nblk + i]);
  double tot = block_sum(acc, red);
  if (threadIdx.x == 0) {
    out[b] = tot;
    counter[b] = 0;
  }
  __syncthreads();
  return true;
}

}  // namespace gsm
