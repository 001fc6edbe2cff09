// Register-resident FFTs of L = 8 Q points (Q = 4 or 8) held by one thread.
//
// With j = t + 8 a (t < 8, a < Q) and q = p + Q s (p < Q, s < 8),
//   X[q] = sum_j x[j] w_L^{S j q}
//        = sum_t w_8^{S t s} w_L^{S t p} sum_a x[t + 8 a] w_Q^{S a p}.
// forward(): natural input order -> Q-point DFTs over a (one per t), twiddles
//   w_L^{S t p}, 8-point DFTs over t (one per p).  X[q] ends at register
//   pos(q) = 8 (q mod Q) + q / Q ("permuted" order): every stage writes its
//   outputs where its inputs were, so nothing moves between stages.
// inverse(): the same DFT for data in permuted order, producing natural
//   order (8-point DFTs over s, twiddles, Q-point DFTs over p).
// A forward transform followed by a pointwise product and an inverse
// transform therefore never needs the permutation undone.  All indices are
// compile-time; twiddles come from the 256-entry table in shared memory.
#pragma once
#include "fft.cuh"

namespace gsm {

template <int L> struct RegFFT {
  static_assert(L == 32 || L == 64, "register FFT sizes are 32 and 64");
  static constexpr int Q = L / 8;
  static constexpr int TS = TWN / L;  // table stride for w_L
  __host__ __device__ static constexpr int pos(int q) { return 8 * (q % Q) + q / Q; }
  __host__ __device__ static constexpr int freq(int i) { return i / 8 + Q * (i % 8); }

  template <int S, typename C> __device__ static __forceinline__ C tw(const C *t, int k) {
    C w = t[k * TS];
    if (S < 0) w.y = -w.y;
    return w;
  }

  template <int S, typename C> __device__ static __forceinline__ void dftQ(C *u) {
    if constexpr (Q == 8) dft8<S>(u);
    else dft4<S>(u);
  }

  template <int S, typename C> __device__ static __forceinline__ void forward(C (&v)[L], const C *twt) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      C u[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) u[a] = v[t + 8 * a];
      dftQ<S>(u);
#pragma unroll
      for (int p = 0; p < Q; ++p) v[t + 8 * p] = (t * p) ? cmul(u[p], tw<S>(twt, t * p)) : u[p];
    }
#pragma unroll
    for (int p = 0; p < Q; ++p) {
      C u[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) u[t] = v[8 * p + t];
      dft8<S>(u);
#pragma unroll
      for (int s = 0; s < 8; ++s) v[8 * p + s] = u[s];
    }
  }

  template <int S, typename C> __device__ static __forceinline__ void inverse(C (&v)[L], const C *twt) {
#pragma unroll
    for (int p = 0; p < Q; ++p) {
      C u[8];
#pragma unroll
      for (int s = 0; s < 8; ++s) u[s] = v[8 * p + s];
      dft8<S>(u);
#pragma unroll
      for (int t = 0; t < 8; ++t) v[8 * p + t] = (t * p) ? cmul(u[t], tw<S>(twt, t * p)) : u[t];
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      C u[Q];
#pragma unroll
      for (int p = 0; p < Q; ++p) u[p] = v[8 * p + t];
      dftQ<S>(u);
#pragma unroll
      for (int a = 0; a < Q; ++a) v[t + 8 * a] = u[a];
    }
  }
};

}  // namespace gsm
