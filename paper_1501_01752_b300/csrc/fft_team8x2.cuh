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

namespace gsm {

// The same 64-point transforms of two planes at once, with the transpose
// between the two radix-8 stages done by lane shuffles instead of the team
// buffer.  With w = exp(S 2 pi i / 64), w8 = w^8 and X[p + 8 s] =
// sum_t w^{t p} w8^{t s} Y[t][p], Y[t][p] = sum_a x[t + 8 a] w8^{a p}:
//
// forward<S> (lane t holds x[t + 8 a] in register a):
//   1. u[a] = x[t + 8 a] w8^{a t}; the DFT over a then gives register r the
//      value Y[t][(r + t) mod 8] (a rotation by the lane index);
//   2. twiddle register r by w^{t ((r + t) mod 8)};
//   3. round k = 1..7: register k takes register k of lane (t - k) mod 8,
//      which holds Y'[(t - k) mod 8][t]: one shuffle per round, the same
//      register on both sides (register 0 keeps Y'[t][t]);
//   4. X[t + 8 s] = w8^{t s} sum_k w8^{-k s} R[k]: a DFT of sign -S over k.
//      The factor w8^{t s} is NOT applied: register s returns
//      Z[s] = X[t + 8 s] w8^{-t s} ("phase-deferred" spectral layout).
// inverse<S'> (lane p holds, in register s, X[p + 8 s] w8'^{p s} with
// w8' = exp(S' 2 pi i / 8)): a DFT of sign S' over s gives W[p][(r + p) mod 8]
// directly (the modulation is the input's), twiddle w'^{p ((r + p) mod 8)},
// the same seven shuffle rounds, a DFT of sign -S' over k, and x[t + 8 a] =
// w8'^{a t} Q[a] for the kept outputs a in {0, 1, 6, 7}.
//
// For S' = -S the phase-deferred output of forward<S> is exactly the input
// inverse<S'> expects: a pointwise real multiplier between them (D along z)
// and any factor constant along a transform (the y phases are constant
// along each z column, which the z convolution carries linearly) leave the
// pair forward<+1> ... inverse<-1> equal to the plain transforms.
struct Team8x2R {
  static constexpr int L = 64;

  // per lane t: tw[r] = w^{t ((r + t) mod 8)} (r < 8), from the
  // positive-sign table
  __device__ static __forceinline__ void constants(WP (&tw)[8], int t, const float2 *twg) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const float2 x = __ldg(&twg[((t * ((r + t) & 7)) & 63) * (TWN / L)]);
      tw[r].c = make_float2(x.x, x.x);
      tw[r].s = make_float2(x.y, x.y);
    }
  }
  // the same and md[j] = w8^{a t} for a = 1, 6, 7 (j = 0, 1, 2)
  __device__ static __forceinline__ void constants(WP (&tw)[8], WP (&md)[3], int t, const float2 *twg) {
    constants(tw, t, twg);
    const int as[3] = {1, 6, 7};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float2 x = __ldg(&twg[((8 * as[j] * t) & 63) * (TWN / L)]);
      md[j].c = make_float2(x.x, x.x);
      md[j].s = make_float2(x.y, x.y);
    }
  }

  // register k <- register k of team lane (t - k) mod 8, k = 1..7
  __device__ static __forceinline__ void rotate_exchange(CP (&v)[8], int t, unsigned mask) {
    const int base = (threadIdx.x & 31) & ~7;
#pragma unroll
    for (int k = 1; k < 8; ++k) {
      const int src = base | ((t - k) & 7);
      v[k].re.x = __shfl_sync(mask, v[k].re.x, src);
      v[k].re.y = __shfl_sync(mask, v[k].re.y, src);
      v[k].im.x = __shfl_sync(mask, v[k].im.x, src);
      v[k].im.y = __shfl_sync(mask, v[k].im.y, src);
    }
  }

  // forward of inputs whose registers 2..5 are zero; phase-deferred output.
  // MOD = false: the caller has already multiplied x[t + 8 a] by w8^{S a t}
  // (md is not read)
  template <int S, bool MOD = true>
  __device__ static __forceinline__ void forward(CP (&v)[8], int t, const WP (&tw)[8], const WP *md,
                                                 unsigned mask) {
    if constexpr (MOD) {
      v[1] = cp_twiddle<S>(v[1], md[0]);
      v[6] = cp_twiddle<S>(v[6], md[1]);
      v[7] = cp_twiddle<S>(v[7], md[2]);
    }
    Team8x2::dft8_in0167<S>(v);
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = cp_twiddle<S>(v[r], tw[r]);
    rotate_exchange(v, t, mask);
    Team8x2::dft8<-S>(v);
  }

  // inverse of a phase-deferred input; natural outputs at a in {0, 1, 6, 7}
  // only (the others are left undefined).  MOD = false leaves the factor
  // w8^{S a t} of output x[t + 8 a] to the caller (md is not read).
  template <int S, bool MOD = true>
  __device__ static __forceinline__ void inverse(CP (&v)[8], int t, const WP (&tw)[8], const WP *md,
                                                 unsigned mask) {
    Team8x2::dft8<S>(v);
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = cp_twiddle<S>(v[r], tw[r]);
    rotate_exchange(v, t, mask);
    Team8x2::dft8_out0167<-S>(v);
    if constexpr (MOD) {
      v[1] = cp_twiddle<S>(v[1], md[0]);
      v[6] = cp_twiddle<S>(v[6], md[1]);
      v[7] = cp_twiddle<S>(v[7], md[2]);
    }
  }
};

}  // namespace gsm
