// FFTs of L = 8 TS points (TS = 4, 8 or 16) by a team of TS lanes that each
// hold 8 values in registers, with one shared-memory transpose per transform.
//
// With j = t + TS a (t < TS, a < 8) and q = p + 8 s (p < 8, s < TS):
//   X[q] = sum_t w_TS^{S t s} w_L^{S t p} sum_a x[t + TS a] w_8^{S a p}.
// forward(): lane t holds x[t + TS a] in register a ("natural" layout;
//   registers 2..5 must be zero, which harmonic inputs with L >= 4n + 4 are);
//   8-point DFT over a, twiddle w_L^{S t p}, transpose through the team
//   buffer, TS-point DFTs over t.  Result: X[p + 8 s] in lane p (TS = 8,
//   register s), in lane p mod 4, register 4 (p / 4) + s (TS = 4), or, for
//   TS = 16, in lane 2 p + (s >= 8), register s mod 8 ("spectral" layout):
//   the 16-point DFT over t is split t = t1 + 2 t2 between the two lanes of
//   a pair (an 8-point DFT over t2 in registers, the twiddle w_16^{S t1 s},
//   and one radix-2 butterfly across the pair by a lane shuffle).
// inverse(): the same DFT from the spectral layout back to the natural one
//   (the steps in reverse order, with the conjugate-direction twiddles).
// The team buffer holds 8 x 9 (16 x 9 for TS = 16) complex values: the row
// pitch 9 keeps the transposes nearly free of bank conflicts.  Each lane
// keeps its twiddles in registers, read once from the global table: w_L^{lane
// k} for k < 8, and for TS = 16 also w_L^{(lane / 2)(lane mod 2 + 2 k)} for
// the inverse.
#pragma once
#include "fft.cuh"

namespace gsm {

template <int L> struct Team8 {
  static_assert(L == 32 || L == 64 || L == 128, "team FFT sizes are 32, 64 and 128");
  static constexpr int TS = L / 8;
  static constexpr int NTW = TS == 16 ? 16 : 8;                // lane twiddles
  static constexpr int BUF = (TS == 16 ? 16 : 8) * 9;          // complex values per team buffer
  // spectral layout: frequency of (lane, register)
  __host__ __device__ static constexpr int freq(int lane, int r) {
    return TS == 16 ? (lane >> 1) + 8 * (r + 8 * (lane & 1))
                    : (TS == 8 ? lane + 8 * r : (lane + 4 * (r / 4)) + 8 * (r % 4));
  }

  // freq(lane, r) - freq(lane, 0): the same for every lane, so the stores of
  // one lane's spectral values are one base address plus constant offsets
  __host__ __device__ static constexpr int fstep(int r) {
    return TS == 4 ? 4 * (r / 4) + 8 * (r % 4) : 8 * r;
  }
  __host__ __device__ static constexpr bool fstep_ok() {
    for (int l = 0; l < TS; ++l)
      for (int r = 0; r < 8; ++r)
        if (freq(l, r) - freq(l, 0) != fstep(r)) return false;
    return true;
  }

  // lane twiddles w_L^{lane k} (k < 8; for TS = 16 also the inverse set)
  // from the TWN-entry table in global memory (6 or 12 KB: it stays in L1
  // after the first warps touch it)
  template <typename C> __device__ static __forceinline__ void twiddles(C (&w)[NTW], int lane, const C *tw) {
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = ldg_c(&tw[((lane * k) % L) * (TWN / L)]);
    if constexpr (TS == 16) {
#pragma unroll
      for (int k = 0; k < 8; ++k) w[8 + k] = ldg_c(&tw[(((lane >> 1) * ((lane & 1) + 2 * k)) % L) * (TWN / L)]);
    }
  }

  // exp(+2 pi i s / 16) for s < 8: the twiddles of the split 16-point DFT
  template <typename C> __device__ static __forceinline__ C w16pow(int s) {
    using R = decltype(C{}.x);
    const double c[8] = {1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173,
                         0.0, -0.38268343236508977173, -0.70710678118654752440, -0.92387953251128675613};
    const double sn[8] = {0.0, 0.38268343236508977173, 0.70710678118654752440, 0.92387953251128675613,
                          1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173};
    return mk((R)c[s], (R)sn[s]);
  }

  // the radix-2 butterfly across the lane pair of the split 16-point DFT:
  // lane t1 = 0 keeps mine + other, lane t1 = 1 keeps other - mine
  template <typename C>
  __device__ static __forceinline__ void pair_butterfly(C (&v)[8], int t1, unsigned mask) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const C o = shfl_xor1(v[r], mask);
      v[r] = t1 ? csub(o, v[r]) : cadd(v[r], o);
    }
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
    const C t1 = rot8<S>(o1);
    const C t2 = mul_si<S>(o2);
    const C t3 = rot8_3<S>(o3);
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
  __device__ static __forceinline__ void forward(C (&v)[8], int lane, const C (&w)[NTW], C *buf, unsigned mask) {
    dft8_in0167<S>(v);                              // Y[t = lane][p], p = register
#pragma unroll
    for (int p = 1; p < 8; ++p) v[p] = tmul<S>(v[p], w[p]);
    if constexpr (TS == 16) {
#pragma unroll
      for (int p = 0; p < 8; ++p) buf[lane * 9 + p] = v[p];
      __syncwarp(mask);
      const int p = lane >> 1, t1 = lane & 1;
#pragma unroll
      for (int t2 = 0; t2 < 8; ++t2) v[t2] = buf[(t1 + 2 * t2) * 9 + p];
      dft8<S>(v);                                   // U_t1[s'], s' = register
#pragma unroll
      for (int s = 1; s < 8; ++s) {
        const C m = tmul<S>(v[s], w16pow<C>(s));
        v[s] = t1 ? m : v[s];
      }
      pair_butterfly(v, t1, mask);                  // X[p + 8 (s' + 8 t1)]
      __syncwarp(mask);
      return;
    }
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

  // OUT0167: only the natural positions lane + TS a with a in {0, 1, 6, 7}
  // are computed (every harmonic position of a grid with L >= 4 n + 4)
  template <int S, bool OUT0167 = false, typename C>
  __device__ static __forceinline__ void inverse(C (&v)[8], int lane, const C (&w)[NTW], C *buf, unsigned mask) {
    if constexpr (TS == 16) {
      const int p = lane >> 1, t1 = lane & 1;
      pair_butterfly(v, t1, mask);                  // R[s'][t_lo = t1]
#pragma unroll
      for (int s = 1; s < 8; ++s) {
        const C m = tmul<S>(v[s], w16pow<C>(s));
        v[s] = t1 ? m : v[s];
      }
      dft8<S>(v);                                   // G[p][t1 + 2 t_hi], t_hi = register
#pragma unroll
      for (int th = 0; th < 8; ++th) v[th] = tmul<S>(v[th], w[8 + th]);   // w_L^{S p (t1 + 2 t_hi)}
#pragma unroll
      for (int th = 0; th < 8; ++th) buf[(t1 + 2 * th) * 9 + p] = v[th];
      __syncwarp(mask);
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = buf[lane * 9 + q];   // G'[q][t = lane]
      if (OUT0167) dft8_out0167<S>(v);
      else dft8<S>(v);                              // x[lane + 16 a], a = register
      __syncwarp(mask);
      return;
    }
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
    if (OUT0167) dft8_out0167<S>(v);
    else dft8<S>(v);                                          // x[lane + TS a], a = register
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
