// 64-point lane-team FFTs of two complex64 transforms at once, with the
// packed FP32 instructions of sm_100+ (add/sub/mul/fma .f32x2).
//
// A value pair CP holds the same entry of two independent transforms a, b as
// re = (Re a, Re b), im = (Im a, Im b).  Every complex addition is then two
// packed instructions for both transforms, a multiplication by +-i is only a
// swap of the re/im halves, and a twiddle product costs five packed
// instructions for both transforms (instead of four scalar ones for each).
// The decomposition is the one of Team8<64> (fft_team8.cuh): lane t < 8
// holds x[t + 8 a] in register a; 8-point DFT over a, twiddle w_64^{S t p},
// transpose through the team buffer, 8-point DFT over t.  Forward inputs
// with registers 2..5 zero (harmonics placed at m mod 64 with 64 >= 4n + 4)
// take the pruned first stage.
//
// The team buffer holds 8 x 8 value pairs with a row pitch of 9: the
// row-wise writes (lane = row) and the column-wise reads (lane = column) of
// eight lanes then fall on distinct 16-byte bank groups, and every access
// is a per-lane base address plus a compile-time offset.
#pragma once
#include "fft.cuh"

namespace gsm {

struct CP {
  float2 re, im;
};


__device__ __forceinline__ CP cp_add(CP a, CP b) { return {f2::add(a.re, b.re), f2::add(a.im, b.im)}; }
__device__ __forceinline__ CP cp_sub(CP a, CP b) { return {f2::sub(a.re, b.re), f2::sub(a.im, b.im)}; }
// a + S i b
template <int S> __device__ __forceinline__ CP cp_add_si(CP a, CP b) {
  if (S > 0) return {f2::sub(a.re, b.im), f2::add(a.im, b.re)};
  return {f2::add(a.re, b.im), f2::sub(a.im, b.re)};
}
// a - S i b
template <int S> __device__ __forceinline__ CP cp_sub_si(CP a, CP b) {
  if (S > 0) return {f2::add(a.re, b.im), f2::sub(a.im, b.re)};
  return {f2::sub(a.re, b.im), f2::add(a.im, b.re)};
}

// twiddle w = (cos, sin) broadcast to both halves
struct WP {
  float2 c, s;
};

// v * w (S > 0) or v * conj(w) (S < 0)
template <int S> __device__ __forceinline__ CP cp_twiddle(CP v, WP w) {
  if (S > 0) return {f2::sub(f2::mul(v.re, w.c), f2::mul(v.im, w.s)), f2::fma(v.re, w.s, f2::mul(v.im, w.c))};
  return {f2::fma(v.re, w.c, f2::mul(v.im, w.s)), f2::sub(f2::mul(v.im, w.c), f2::mul(v.re, w.s))};
}

struct Team8x2 {
  static constexpr int L = 64;
  static constexpr int BUF = 72;   // value pairs per team buffer (8 rows, pitch 9)
  // spectral layout of the forward output: frequency lane + 8 r in register r
  __host__ __device__ static constexpr int freq(int lane, int r) { return lane + 8 * r; }

  __device__ static __forceinline__ void twiddles(WP (&w)[8], int lane, const float2 *tw) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float2 t = __ldg(&tw[((lane * k) % L) * (TWN / L)]);
      w[k].c = make_float2(t.x, t.x);
      w[k].s = make_float2(t.y, t.y);
    }
  }

  // the closing butterflies of an 8-point DFT, shared by the full and the
  // pruned first stage: E = DFT4 of the even inputs, O = DFT4 of the odd
  // ones, v[k] = E[k] + w_8^{S k} O[k], v[k + 4] = E[k] - w_8^{S k} O[k]
  template <int S> __device__ static __forceinline__ void close8(CP *v, CP E0, CP E1, CP E2, CP E3, CP O0, CP O1,
                                                                 CP O2, CP O3) {
    const float h = 0.70710678118654752440f;
    const float2 H = make_float2(h, h), NH = make_float2(-h, -h);
    v[0] = cp_add(E0, O0);
    v[4] = cp_sub(E0, O0);
    v[2] = cp_add_si<S>(E2, O2);
    v[6] = cp_sub_si<S>(E2, O2);
    // w_8^S O1 = h (1 + S i) O1 = h (O1.re - S O1.im, O1.im + S O1.re)
    const float2 xr = S > 0 ? f2::sub(O1.re, O1.im) : f2::add(O1.re, O1.im);
    const float2 xi = S > 0 ? f2::add(O1.im, O1.re) : f2::sub(O1.im, O1.re);
    v[1] = {f2::fma(xr, H, E1.re), f2::fma(xi, H, E1.im)};
    v[5] = {f2::fma(xr, NH, E1.re), f2::fma(xi, NH, E1.im)};
    // w_8^{3S} O3 = h (-1 + S i) O3 = h (-O3.re - S O3.im, -O3.im + S O3.re)
    //   S > 0: (-h (O3.re + O3.im), h (O3.re - O3.im))
    //   S < 0: ( h (O3.im - O3.re), -h (O3.re + O3.im))
    if (S > 0) {
      const float2 yr = f2::add(O3.re, O3.im), yi = f2::sub(O3.re, O3.im);
      v[3] = {f2::fma(yr, NH, E3.re), f2::fma(yi, H, E3.im)};
      v[7] = {f2::fma(yr, H, E3.re), f2::fma(yi, NH, E3.im)};
    } else {
      const float2 yr = f2::sub(O3.im, O3.re), yi = f2::add(O3.re, O3.im);
      v[3] = {f2::fma(yr, H, E3.re), f2::fma(yi, NH, E3.im)};
      v[7] = {f2::fma(yr, NH, E3.re), f2::fma(yi, H, E3.im)};
    }
  }

  // 4-point DFT of (a, b, c, d) with sign S
  template <int S> __device__ static __forceinline__ void dft4(CP &a, CP &b, CP &c, CP &d) {
    const CP t0 = cp_add(a, c), t1 = cp_sub(a, c), t2 = cp_add(b, d), t3 = cp_sub(b, d);
    a = cp_add(t0, t2);
    c = cp_sub(t0, t2);
    b = cp_add_si<S>(t1, t3);
    d = cp_sub_si<S>(t1, t3);
  }

  template <int S> __device__ static __forceinline__ void dft8(CP *v) {
    CP e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    CP o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<S>(e0, e1, e2, e3);
    dft4<S>(o0, o1, o2, o3);
    close8<S>(v, e0, e1, e2, e3, o0, o1, o2, o3);
  }

  // 8-point DFT of inputs whose registers 2..5 are zero
  template <int S> __device__ static __forceinline__ void dft8_in0167(CP *v) {
    // even inputs (v0, 0, 0, v6): DFT4 = (v0 + v6, v0 - S i v6, v0 - v6, v0 + S i v6)
    const CP E0 = cp_add(v[0], v[6]), E2 = cp_sub(v[0], v[6]);
    const CP E1 = cp_sub_si<S>(v[0], v[6]), E3 = cp_add_si<S>(v[0], v[6]);
    // odd inputs (v1, 0, 0, v7)
    const CP O0 = cp_add(v[1], v[7]), O2 = cp_sub(v[1], v[7]);
    const CP O1 = cp_sub_si<S>(v[1], v[7]), O3 = cp_add_si<S>(v[1], v[7]);
    close8<S>(v, E0, E1, E2, E3, O0, O1, O2, O3);
  }

  // outputs 0, 1, 6, 7 of an 8-point DFT (the others are left undefined):
  // the last stage of an inverse transform whose outputs outside the
  // harmonic box are not kept
  template <int S> __device__ static __forceinline__ void dft8_out0167(CP *v) {
    CP e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    CP o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<S>(e0, e1, e2, e3);
    dft4<S>(o0, o1, o2, o3);
    const float h = 0.70710678118654752440f;
    const float2 H = make_float2(h, h), NH = make_float2(-h, -h);
    v[0] = cp_add(e0, o0);
    v[6] = cp_sub_si<S>(e2, o2);
    const float2 xr = S > 0 ? f2::sub(o1.re, o1.im) : f2::add(o1.re, o1.im);
    const float2 xi = S > 0 ? f2::add(o1.im, o1.re) : f2::sub(o1.im, o1.re);
    v[1] = {f2::fma(xr, H, e1.re), f2::fma(xi, H, e1.im)};
    if (S > 0) {
      const float2 yr = f2::add(o3.re, o3.im), yi = f2::sub(o3.re, o3.im);
      v[7] = {f2::fma(yr, H, e3.re), f2::fma(yi, NH, e3.im)};
    } else {
      const float2 yr = f2::sub(o3.im, o3.re), yi = f2::add(o3.re, o3.im);
      v[7] = {f2::fma(yr, NH, e3.re), f2::fma(yi, H, e3.im)};
    }
  }

  template <int S>
  __device__ static __forceinline__ void forward(CP (&v)[8], int lane, const WP (&w)[8], CP *buf, unsigned mask) {
    dft8_in0167<S>(v);                          // Y[t = lane][p], p = register
#pragma unroll
    for (int p = 1; p < 8; ++p) v[p] = cp_twiddle<S>(v[p], w[p]);
    CP *row = buf + lane * 9;
#pragma unroll
    for (int p = 0; p < 8; ++p) row[p] = v[p];
    __syncwarp(mask);
    const CP *col = buf + lane;
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = col[t * 9];   // Y[t][p = lane]
    dft8<S>(v);                                      // X[lane + 8 s], s = register
    __syncwarp(mask);
  }

  // inverse from the spectral layout; OUT0167 computes only the natural
  // positions lane + 8 a with a in {0, 1, 6, 7}
  template <int S, bool OUT0167 = false>
  __device__ static __forceinline__ void inverse(CP (&v)[8], int lane, const WP (&w)[8], CP *buf, unsigned mask) {
    dft8<S>(v);                                                  // W[p = lane][t], t = register
#pragma unroll
    for (int t = 1; t < 8; ++t) v[t] = cp_twiddle<S>(v[t], w[t]);   // w_64^{S t p}, p = lane
    CP *row = buf + lane * 9;
#pragma unroll
    for (int t = 0; t < 8; ++t) row[t] = v[t];
    __syncwarp(mask);
    const CP *col = buf + lane;
#pragma unroll
    for (int p = 0; p < 8; ++p) v[p] = col[p * 9];               // W[p][t = lane]
    if (OUT0167) dft8_out0167<S>(v);
    else dft8<S>(v);                                             // x[lane + 8 a], a = register
    __syncwarp(mask);
  }
};

}  // namespace gsm
