// FFTs of L = 8 TS points (TS = 4 or 8) by a team of TS lanes that each
// hold 8 values in registers, with one shared-memory transpose per transform.
//
// With j = t + TS a (t < TS, a < 8) and q = p + 8 s (p < 8, s < TS):
//   X[q] = sum_t w_TS^{S t s} w_L^{S t p} sum_a x[t + TS a] w_8^{S a p}.
// forward(): lane t holds x[t + TS a] in register a ("natural" layout;
//   registers 2..5 must be zero, which harmonic inputs with L >= 2N - 1 are);
//   8-point DFT over a, twiddle w_L^{S t p}, transpose through the team
//   buffer, TS-point DFTs over t.  Result: X[p + 8 s] in lane p (TS = 8,
//   register s) or in lane p mod 4, register 4 (p / 4) + s (TS = 4)
//   ("spectral" layout).
// inverse(): the same DFT from the spectral layout back to the natural one
//   (TS-point DFTs over s, twiddle, transpose, 8-point DFTs over p).
// The team buffer holds 8 x 9 complex values (row pitch 9 keeps the
// transpose free of bank conflicts).  Each lane keeps its own twiddles
// w_L^{lane k}, k < 8, in registers, read once from the global table.
#pragma once
#include "fft.cuh"

namespace gsm {

template <int L> struct Team8 {
  static_assert(L == 32 || L == 64, "team FFT sizes are 32 and 64");
  static constexpr int TS = L / 8;
  static constexpr int BUF = 8 * 9;    // complex values per team buffer
  // spectral layout: frequency of (lane, register)
  __host__ __device__ static constexpr int freq(int lane, int r) {
    return TS == 8 ? lane + 8 * r : (lane + 4 * (r / 4)) + 8 * (r % 4);
  }

  // lane twiddles w_L^{lane k} (k < 8) from the 256-entry table in global
  // memory (2 or 4 KB: it stays in L1 after the first warps touch it)
  template <typename C> __device__ static __forceinline__ void twiddles(C (&w)[8], int lane, const C *tw) {
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = ldg_c(&tw[((lane * k) % L) * (TWN / L)]);
  }

  template <int S, typename C> __device__ static __forceinline__ C tmul(C v, C w) {
    if (S < 0) w.y = -w.y;
    return cmul(v, w);
  }

  // 8-point DFT of inputs whose registers 2..5 are zero: a transform of
  // harmonics m in [-n, n] placed at m mod L with L >= 4 n + 4 has nonzero
  // inputs only at t + TS a for a in {0, 1, 6, 7}.
  template <int S, typename C> __device__ static __forceinline__ void dft8_in0167(C *v) {
    const C e0 = cadd(v[0], v[6]), e2 = csub(v[0], v[6]);
    const C r6 = mul_si<S>(v[6]);
    const C e1 = csub(v[0], r6), e3 = cadd(v[0], r6);
    const C o0 = cadd(v[1], v[7]), o2 = csub(v[1], v[7]);
    const C r7 = mul_si<S>(v[7]);
    const C o1 = csub(v[1], r7), o3 = cadd(v[1], r7);
    using R = decltype(o0.x);
    const R h = (R)0.70710678118654752440;
    const C t1 = mk((o1.x - S * o1.y) * h, (o1.y + S * o1.x) * h);
    const C t2 = mul_si<S>(o2);
    const C t3 = mk((-o3.x - S * o3.y) * h, (-o3.y + S * o3.x) * h);
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, t1);
    v[5] = csub(e1, t1);
    v[2] = cadd(e2, t2);
    v[6] = csub(e2, t2);
    v[3] = cadd(e3, t3);
    v[7] = csub(e3, t3);
  }

  template <int S, typename C>
  __device__ static __forceinline__ void forward(C (&v)[8], int lane, const C (&w)[8], C *buf, unsigned mask) {
    dft8_in0167<S>(v);                              // Y[t = lane][p], p = register
#pragma unroll
    for (int p = 1; p < 8; ++p) v[p] = tmul<S>(v[p], w[p]);
#pragma unroll
    for (int p = 0; p < 8; ++p) buf[lane * 9 + p] = v[p];
    __syncwarp(mask);
    if constexpr (TS == 8) {
#pragma unroll
      for (int t = 0; t < 8; ++t) v[t] = buf[t * 9 + lane];   // Y[t][p = lane]
      dft8<S>(v);                                             // X[lane + 8 s], s = register
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int t = 0; t < 4; ++t) v[4 * h + t] = buf[t * 9 + lane + 4 * h];   // Y[t][p = lane + 4h]
      dft4<S>(v);
      dft4<S>(v + 4);                                          // X[p + 8 s] at 4h + s
    }
    __syncwarp(mask);
  }

  template <int S, typename C>
  __device__ static __forceinline__ void inverse(C (&v)[8], int lane, const C (&w)[8], C *buf, unsigned mask) {
    if constexpr (TS == 8) {
      dft8<S>(v);                                             // W[p = lane][t], t = register
#pragma unroll
      for (int t = 1; t < 8; ++t) v[t] = tmul<S>(v[t], w[t]);   // w_L^{t p}, p = lane
#pragma unroll
      for (int t = 0; t < 8; ++t) buf[lane * 9 + t] = v[t];
      __syncwarp(mask);
#pragma unroll
      for (int p = 0; p < 8; ++p) v[p] = buf[p * 9 + lane];   // W[p][t = lane]
    } else {
      dft4<S>(v);
      dft4<S>(v + 4);                                         // W[p][t], p = lane + 4h, t = register
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = lane + 4 * h;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          C wv = w[t];                                        // w_32^{t lane}
          if (h) {                                            // times w_32^{4 t} = w_8^{t}
            const C e = w8pow<C>(t);
            wv = cmul(wv, e);
          }
          buf[p * 9 + t] = t ? tmul<S>(v[4 * h + t], wv) : v[4 * h + t];
        }
      }
      __syncwarp(mask);
#pragma unroll
      for (int p = 0; p < 8; ++p) v[p] = buf[p * 9 + lane];   // W[p][t = lane]
    }
    dft8<S>(v);                                               // x[lane + TS a], a = register
    __syncwarp(mask);
  }

  // exp(+2 pi i t / 8) for t < 4
  template <typename C> __device__ static __forceinline__ C w8pow(int t) {
    using R = decltype(C{}.x);
    const R h = (R)0.70710678118654752440;
    return t == 0 ? mk((R)1, (R)0) : (t == 1 ? mk(h, h) : (t == 2 ? mk((R)0, (R)1) : mk(-h, h)));
  }
};

}  // namespace gsm
