// Shared-memory FFT building blocks for the pruned 3D convolution.
//
// A line of L complex values in shared memory, L = 2^p or L = 3 * 2^p with
// p >= 3 (mixed radix: 24, 48, 96, 192), is transformed in place by a team of
// ts = max(1, L/8) lanes of one warp.  Teams never straddle a warp: a warp
// holds floor(32 / ts) teams and its remaining lanes stay idle, so every team
// synchronises with __syncwarp on its own mask.  The transform is a Stockham
// autosort decomposition: radix-8 stages while the remaining length has a
// factor 8, then one radix-4 or radix-2 stage, and a final radix-3 stage
// when L has a factor 3; every stage reads R values per group into
// registers, synchronises, applies the twiddles exp(S 2 pi i k r / (Ns R))
// (k = g mod Ns, Ns the product of the radices already applied), an R-point
// DFT, and writes the R outputs to their natural-order positions.  Output is
// in natural order.
//
//   S = +1:  X[q] = sum_j x[j] exp(+2 pi i j q / L)   (harmonics -> grid)
//   S = -1:  X[q] = sum_j x[j] exp(-2 pi i j q / L)   (grid -> harmonics)
//
// Twiddles come from a 768-entry table tw[j] = exp(+2 pi i j / 768) built on
// the host in FP64 (768 = 3 * 256 holds every root of unity of the supported
// sizes); S = -1 uses its conjugate.
#pragma once
#include "common.cuh"

namespace gsm {

constexpr int TWN = 768;     // table resolution: every supported L divides it

template <int S, typename C> __device__ __forceinline__ C mul_si(C a) {  // a * (S i)
  return S > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

// The w_8 and w_8^3 rotations of the radix-8 DFT: (1 + S i) h a and
// (-1 + S i) h a with h = 1/sqrt(2) (dfloat.cuh has packed versions for dcx)
template <int S, typename C> __device__ __forceinline__ C rot8(C a) {
  using R = decltype(a.x);
  const R h = (R)0.70710678118654752440;
  return mk((a.x - S * a.y) * h, (a.y + S * a.x) * h);
}
template <int S, typename C> __device__ __forceinline__ C rot8_3(C a) {
  using R = decltype(a.x);
  const R h = (R)0.70710678118654752440;
  return mk((-a.x - S * a.y) * h, (-a.y + S * a.x) * h);
}

template <int S, typename C> __device__ __forceinline__ void dft2(C* v) {
  C t = v[0];
  v[0] = cadd(t, v[1]);
  v[1] = csub(t, v[1]);
}

template <int S, typename C> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  C t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), t3 = mul_si<S>(csub(v1, v3));
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  v1 = cadd(t1, t3);
  v3 = csub(t1, t3);
}

template <int S, typename C> __device__ __forceinline__ void dft4(C* v) { dft4<S>(v[0], v[1], v[2], v[3]); }

template <int S, typename C> __device__ __forceinline__ void dft8(C* v) {
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<S>(e0, e1, e2, e3);
  dft4<S>(o0, o1, o2, o3);
  // w = exp(S i pi / 4): w o1 = (1 + S i) h o1, w^2 o2 = S i o2, w^3 o3 = (-1 + S i) h o3
  C t1 = rot8<S>(o1);
  C t2 = mul_si<S>(o2);
  C t3 = rot8_3<S>(o3);
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1);
  v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2);
  v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3);
  v[7] = csub(e3, t3);
}

// outputs 0, 1, 6, 7 of the 8-point DFT above (the others are left
// undefined): the last stage of an inverse lane-team transform, whose
// outputs outside the harmonic box are not kept
template <int S, typename C> __device__ __forceinline__ void dft8_out0167(C* v) {
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<S>(e0, e1, e2, e3);
  dft4<S>(o0, o1, o2, o3);
  v[0] = cadd(e0, o0);
  v[1] = cadd(e1, rot8<S>(o1));
  v[6] = csub(e2, mul_si<S>(o2));
  v[7] = csub(e3, rot8_3<S>(o3));
}

// 3-point DFT: with w = exp(S 2 pi i / 3) = -1/2 + S i sqrt(3)/2,
// X0 = v0 + v1 + v2, X1,2 = v0 - (v1 + v2)/2 +- S i (sqrt(3)/2) (v1 - v2)
template <int S, typename C> __device__ __forceinline__ void dft3(C* v) {
  using R = decltype(v[0].x);
  const R h = (R)0.86602540378443864676;
  const C t1 = cadd(v[1], v[2]);
  const C t2 = mk(v[0].x - (R)0.5 * t1.x, v[0].y - (R)0.5 * t1.y);
  const C d = csub(v[1], v[2]);
  const C t3 = mul_si<S>(mk(h * d.x, h * d.y));
  v[0] = cadd(v[0], t1);
  v[1] = cadd(t2, t3);
  v[2] = csub(t2, t3);
}

template <int R, int S, typename C> __device__ __forceinline__ void dft_r(C* v) {
  if constexpr (R == 8) dft8<S>(v);
  else if constexpr (R == 4) dft4<S>(v);
  else if constexpr (R == 3) dft3<S>(v);
  else dft2<S>(v);
}

// One Stockham stage of radix R on a line of L points; Ns is the product of
// the radices already applied.  ts = max(1, L / 8) lanes share the L / R
// groups, at most ceil(8 / R) per lane.
template <int R, int S, typename C>
__device__ __forceinline__ void fft_stage(C* line, int L, int Ns, int lane, int ts, unsigned mask, const C* tw) {
  constexpr int MAXG = (8 + R - 1) / R;
  const int ngroups = L / R;
  C v[MAXG][R];
#pragma unroll
  for (int q = 0; q < MAXG; ++q) {
    int g = lane + q * ts;
    if (g < ngroups) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = line[g + r * ngroups];
    }
  }
  __syncwarp(mask);
  const int step = TWN / (Ns * R);   // table stride of exp(2 pi i / (Ns R))
#pragma unroll
  for (int q = 0; q < MAXG; ++q) {
    int g = lane + q * ts;
    if (g < ngroups) {
      const int k = g % Ns;
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = tw[k * r * step];
          if (S < 0) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      dft_r<R, S>(v[q]);
      const int base = (g - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) line[base + r * Ns] = v[q][r];
    }
  }
  __syncwarp(mask);
}

// In-place FFT of one line of L points (2^p or 3 * 2^p) by a team of ts
// lanes: radix-8 stages over the power-of-two part, one radix-4 or radix-2
// stage for what remains of it, then a radix-3 stage when 3 divides L.
template <int S, typename C>
__device__ __forceinline__ void team_fft(C* line, int L, int lane, int ts, unsigned mask, const C* tw) {
  const bool three = L % 3 == 0;
  int rem = three ? L / 3 : L, Ns = 1;
  while (rem >= 8) {
    fft_stage<8, S>(line, L, Ns, lane, ts, mask, tw);
    Ns *= 8;
    rem /= 8;
  }
  if (rem == 4) {
    fft_stage<4, S>(line, L, Ns, lane, ts, mask, tw);
    Ns *= 4;
  } else if (rem == 2) {
    fft_stage<2, S>(line, L, Ns, lane, ts, mask, tw);
    Ns *= 2;
  }
  if (three) fft_stage<3, S>(line, L, Ns, lane, ts, mask, tw);
}

// Team geometry for lines of L points: ts = max(1, L / 8) lanes per team,
// floor(32 / ts) teams per warp (a team never straddles a warp).  When ts
// does not divide 32 the last lanes of each warp are idle: their id is
// IDLE (beyond any loop bound), so every "for (x = id; x < bound; x +=
// count)" loop skips them and they never take part in a team's __syncwarp;
// nothing may be computed from id outside such a loop.  blockDim.x is a
// multiple of 32.
struct Team {
  static constexpr int IDLE = 1 << 30;
  int ts, lane, id, count;
  unsigned mask;
  __device__ __forceinline__ Team(int L) {
    ts = L >= 8 ? L / 8 : 1;
    const int per = 32 / ts, wl = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = wl / ts;
    count = (blockDim.x >> 5) * per;
    lane = wl - t * ts;
    id = t < per ? w * per + t : IDLE;
    const unsigned m = ts == 32 ? 0xffffffffu : ((1u << ts) - 1u);
    mask = t < per ? m << (wl - lane) : 0u;
  }
};

template <typename C> __device__ __forceinline__ void load_twiddles(C* tw_s, const C* tw_g) {
  for (int i = threadIdx.x; i < TWN; i += blockDim.x) tw_s[i] = tw_g[i];
}

}  // namespace gsm
