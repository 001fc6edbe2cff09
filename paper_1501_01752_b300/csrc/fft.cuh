// Shared-memory FFT building blocks for the pruned 3D convolution.
//
// A line of L = 2^p complex values in shared memory is transformed in place
// by a team of ts = max(1, L/8) consecutive lanes of one warp (the team never
// straddles a warp, so it synchronises with __syncwarp on its own mask).
// The transform is a Stockham autosort decomposition: radix-8 stages while at
// least three bits remain, then one radix-4 or radix-2 stage; every stage
// reads R values per group into registers, synchronises, applies the
// twiddles exp(S 2 pi i k r / (Ns R)), an R-point DFT, and writes the R
// outputs to their natural-order positions.  Output is in natural order.
//
//   S = +1:  X[q] = sum_j x[j] exp(+2 pi i j q / L)   (harmonics -> grid)
//   S = -1:  X[q] = sum_j x[j] exp(-2 pi i j q / L)   (grid -> harmonics)
//
// Twiddles come from a 256-entry table tw[j] = exp(+2 pi i j / 256) built on
// the host in FP64 and staged in shared memory; S = -1 uses its conjugate.
#pragma once
#include "common.cuh"

namespace gsm {

constexpr int TWN = 256;     // table resolution = largest supported L
constexpr int LG_TWN = 8;

template <int S, typename C> __device__ __forceinline__ C mul_si(C a) {  // a * (S i)
  return S > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
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
  using R = decltype(o0.x);
  const R h = (R)0.70710678118654752440;
  // w = exp(S i pi / 4): w o1 = (1 + S i) h o1, w^2 o2 = S i o2, w^3 o3 = (-1 + S i) h o3
  C t1 = mk((o1.x - S * o1.y) * h, (o1.y + S * o1.x) * h);
  C t2 = mul_si<S>(o2);
  C t3 = mk((-o3.x - S * o3.y) * h, (-o3.y + S * o3.x) * h);
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1);
  v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2);
  v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3);
  v[7] = csub(e3, t3);
}

template <int LR, int S, typename C> __device__ __forceinline__ void dft_r(C* v) {
  if constexpr (LR == 3) dft8<S>(v);
  else if constexpr (LR == 2) dft4<S>(v);
  else dft2<S>(v);
}

// One Stockham stage of radix R = 2^LR on a line of 2^lgL points; Ns = 2^lgNs
// is the product of the radices already applied.
template <int LR, int S, typename C>
__device__ __forceinline__ void fft_stage(C* line, int lgL, int lgNs, int lane, int ts, unsigned mask,
                                          const C* tw) {
  constexpr int R = 1 << LR;
  constexpr int MAXG = 8 / R;   // groups per lane: ts = max(1, L/8) => L/(R ts) <= 8/R
  const int ngroups = 1 << (lgL - LR);
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
  const int Ns = 1 << lgNs;
  const int sh = LG_TWN - lgNs - LR;
#pragma unroll
  for (int q = 0; q < MAXG; ++q) {
    int g = lane + q * ts;
    if (g < ngroups) {
      const int k = g & (Ns - 1);
      if (lgNs > 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = tw[(k * r) << sh];
          if (S < 0) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      dft_r<LR, S>(v[q]);
      const int base = ((g - k) << LR) + k;
#pragma unroll
      for (int r = 0; r < R; ++r) line[base + (r << lgNs)] = v[q][r];
    }
  }
  __syncwarp(mask);
}

// In-place FFT of one line of 2^lgL points by a team of ts lanes.
template <int S, typename C>
__device__ __forceinline__ void team_fft(C* line, int lgL, int lane, int ts, unsigned mask, const C* tw) {
  int lgNs = 0, rem = lgL;
  while (rem >= 3) {
    fft_stage<3, S>(line, lgL, lgNs, lane, ts, mask, tw);
    lgNs += 3;
    rem -= 3;
  }
  if (rem == 2) fft_stage<2, S>(line, lgL, lgNs, lane, ts, mask, tw);
  else if (rem == 1) fft_stage<1, S>(line, lgL, lgNs, lane, ts, mask, tw);
}

// Team geometry for lines of 2^lgL points: team size, lane, team index, mask.
struct Team {
  int ts, lane, id, count;
  unsigned mask;
  __device__ __forceinline__ Team(int lgL) {
    ts = lgL >= 3 ? (1 << (lgL - 3)) : 1;
    lane = threadIdx.x % ts;
    id = threadIdx.x / ts;
    count = blockDim.x / ts;
    unsigned m = ts == 32 ? 0xffffffffu : ((1u << ts) - 1u);
    mask = m << ((threadIdx.x & 31) - lane);
  }
};

template <typename C> __device__ __forceinline__ void load_twiddles(C* tw_s, const C* tw_g) {
  for (int i = threadIdx.x; i < TWN; i += blockDim.x) tw_s[i] = tw_g[i];
}

}  // namespace gsm
