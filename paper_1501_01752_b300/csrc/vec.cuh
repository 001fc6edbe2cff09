// Vector I/O helpers of the Krylov kernels: every thread moves EPT
// consecutive values of a vector whose stored length Us is a multiple of 64,
// with 16-byte loads and stores, and warp-level sums.
#pragma once
#include "common.cuh"

namespace gsm {

constexpr int KT = 256;  // threads per block of the vector kernels

// Vectors are stored with a stride Us (the length U rounded up to 64
// complex values, pads held at zero), so each thread moves EPT consecutive
// values with 16-byte loads: a tile is KT * EPT values.
template <typename R> struct Ept { static constexpr int v = sizeof(R) == 4 ? 8 : 4; };

template <typename C, int EPT> __device__ __forceinline__ void load_ept(C (&d)[EPT], const C *src) {
  if constexpr (sizeof(C) == 8) {
    const float4 *q = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int k = 0; k < EPT / 2; ++k) {
      const float4 t = q[k];
      d[2 * k] = mk(t.x, t.y);
      d[2 * k + 1] = mk(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < EPT; ++k) d[k] = src[k];
  }
}

template <typename C, int EPT> __device__ __forceinline__ void store_ept(C *dst, const C (&d)[EPT]) {
  if constexpr (sizeof(C) == 8) {
    float4 *q = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int k = 0; k < EPT / 2; ++k) q[k] = make_float4(d[2 * k].x, d[2 * k].y, d[2 * k + 1].x, d[2 * k + 1].y);
  } else {
#pragma unroll
    for (int k = 0; k < EPT; ++k) dst[k] = d[k];
  }
}

template <typename R> __device__ __forceinline__ R warp_sum(R v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace gsm
