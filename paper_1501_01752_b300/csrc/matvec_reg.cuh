// Lane-team path of the Eq. 4 operator (complex64 and complex128) for FFT sizes 32 and 64 per
// axis: the same three passes as matvec.cu, with every 1D transform done by
// a team of L/8 lanes holding 8 values each (fft_team8.cuh): one radix-8 DFT
// in registers, one bank-conflict-free transpose through a team buffer, the
// second radix in registers.  Loads come straight from global memory into
// the natural layout and stores leave from the spectral layout, so the
// only shared-memory staging is the y-z plane of pass 2 and the three
// components of pass 3.
//
//   pass 1  k_fwd_x_t8 : team per x-row (c, m_z, m_y): N_x -> L_x
//   pass 2  k_yz_t8    : per (r_x, c) plane, team per row (y forward), team
//                        per column (z forward, x D, z inverse), team per
//                        row (y inverse)
//   pass 3  k_inv_x_t8 : team per (c, row): L_x -> N_x, then per harmonic
//                        the Green tensor and y = x - G u (or the residual)
//
// complex64 on 64-point y and z grids runs pass 2 as k_yz_t8x2r (two x
// frequencies per block in packed FP32 pairs, lane-shuffle transposes), which
// leaves an 8th-root factor per (m_z, m_y) row of the intermediate that pass 1
// applies (yz_phase_index) and pass 3 removes (k_inv_x_t8c).
#pragma once
#include "fft_team8.cuh"
#include "fft_team8x2.cuh"
#include "kernels.h"
#include "reduce.cuh"

#include <type_traits>

namespace gsm {

// harmonic index (0..N-1) held at natural grid position k, or -1
__device__ __forceinline__ int harm_at(int k, int n, int L) {
  if (k <= n) return k + n;
  if (k >= L - n) return k - L + n;
  return -1;
}

// Index k of the factor w8^k = exp(2 pi i k / 8) that the shuffle yz pass
// (k_yz_t8x2r) leaves to passes 1 and 3 for the T row of harmonic indices
// (hy, hz) on the 64-point y and z grids: with grid positions p = (h - n) mod
// 64 = t + 8 a, k = (a_y t_y + a_z t_z) mod 8 (the rotation's input
// modulations along y and z; its inverses take the conjugate).
__device__ __forceinline__ int yz_phase_index(int hy, int ny, int hz, int nz) {
  const int py = (hy - ny) & 63, pz = (hz - nz) & 63;
  return ((py >> 3) * (py & 7) + (pz >> 3) * (pz & 7)) & 7;
}

constexpr int TB_DEFAULT = 256;  // threads per block unless the autotuner picks another

struct Lanes {
  int team, lane;
  unsigned mask;
  __device__ __forceinline__ Lanes(int ts) {
    team = threadIdx.x / ts;
    lane = threadIdx.x % ts;
    const unsigned m = ts == 32 ? 0xffffffffu : ((1u << ts) - 1u);
    mask = m << ((threadIdx.x & 31) - lane);
  }
};

// q = r / d and rem = r - q d for 0 <= r < 2^22, 0 < d <= 256, with rd the
// FP32 reciprocal of d: the truncated estimate r rd is within one of q
// (relative error below 2^-23 on a quotient below 2^22 / d) and is corrected
// once, in place of an integer division.
__device__ __forceinline__ int divmod_small(int r, int d, float rd, int &rem) {
  int q = __float2int_rz((float)r * rd);
  int m = r - q * d;
  if (m < 0) {
    --q;
    m += d;
  } else if (m >= d) {
    ++q;
    m -= d;
  }
  rem = m;
  return q;
}

// Harmonic offsets of a lane's natural positions k = lane + TS a.  Harmonics
// m in [-n, n] sit at m mod L with L >= 4 n + 4 (every lane-team grid: L is
// a multiple of 4 and >= 2 N - 1 = 4 n + 1), so only a in {0, 1, 6, 7} can
// hold one: slot j = 0..3 stands for a = 0, 1, 6, 7, and off[j] is the
// harmonic index (0..N-1) there or -1.
template <int L, int TS> struct HarmSlots {
  int off[4];
  __device__ __forceinline__ HarmSlots(int lane, int n) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = lane + TS * (j < 2 ? j : j + 4);
      off[j] = j < 2 ? (k <= n ? k + n : -1) : (k >= L - n ? k - L + n : -1);
    }
  }
  __host__ __device__ static constexpr int slot(int a) { return a < 2 ? a : (a >= 6 ? a - 4 : -1); }
};

// Each team transforms RPT rows (RB rows apart), issuing the loads of all of
// them before the first transform, so that more reads are in flight per
// thread.  Row indices are 32-bit (3 N1 N2 < 2^22 rows per instance).
template <typename R, int L0, int TT, int RPT>
__global__ void __launch_bounds__(TT) k_fwd_x_t8(Geo g, const typename Io<R>::T *__restrict__ X, long long xstride,
                                                 typename Cx<R>::T *__restrict__ T, const R *__restrict__ scale,
                                                 const int *__restrict__ act,
                                                 const typename Cx<R>::T *__restrict__ twg, const int *__restrict__ jdev,
                                                 long long jstride, int ph) {
  using C = typename Cx<R>::T;
  using IO = typename Io<R>::T;
  using F = Team8<L0>;
  static_assert(F::fstep_ok(), "spectral layout must be a lane base plus constant steps");
  if (jdev) X += (long long)(*jdev) * jstride;
  constexpr int TS = F::TS, RB = TT / TS;
  __shared__ C bufs[RB * F::BUF];
  const int b = blockIdx.y;
  if (act && !act[b]) return;
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const int P = N2 * N1, nrows = 3 * P;
  const float rN1 = 1.0f / (float)N1, rN2 = 1.0f / (float)N2;
  const Lanes ln(TS);
  C w[F::NTW];
  F::twiddles(w, ln.lane, twg);
  const HarmSlots<L0, TS> hs(ln.lane, g.n[0]);
  const int rbase = blockIdx.x * RB * RPT + ln.team;
  const R s = scale ? scale[b] : (R)1;
  const IO *Xb = X + b * xstride;
  C v[RPT][8];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int r = rbase + i * RB;
    const bool valid = r < nrows;
    const IO *Xr = Xb + r * N0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      v[i][a] = mk((R)0, (R)0);
      const int j = HarmSlots<L0, TS>::slot(a);
      if (j >= 0 && valid && hs.off[j] >= 0) v[i][a] = io_in<C>(Xr[hs.off[j]]);
    }
  }
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int r = rbase + i * RB;
    const bool valid = r < nrows;
    int my, mz;
    const int plane = divmod_small(r, N1, rN1, my);
    const int c = divmod_small(plane, N2, rN2, mz);
    if (ph) {   // the scale times the row's factor for the shuffle yz pass
      const C wk = ldg_c(&twg[yz_phase_index(my, g.n[1], mz, g.n[2]) * (TWN / 8)]);
      const C sw = mk(wk.x * s, wk.y * s);
#pragma unroll
      for (int a = 0; a < 8; ++a)
        if (HarmSlots<L0, TS>::slot(a) >= 0) v[i][a] = cmul(v[i][a], sw);
    } else {
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        v[i][a].x *= s;
        v[i][a].y *= s;
      }
    }
    F::template forward<+1>(v[i], ln.lane, w, bufs + ln.team * F::BUF, ln.mask);
    if (!valid) continue;
    C *Tq = T + b * g.Tst + ((3 * F::freq(ln.lane, 0) + c) * P + mz * N1 + my);
#pragma unroll
    for (int q = 0; q < 8; ++q) Tq[F::fstep(q) * 3 * P] = v[i][q];
  }
}

// Pass 1 with a per-harmonic 3 x 3 map applied before the x transforms, one
// team per (m_z, m_y) row holding all three components of the row, so that
// the scaled write-back of a Krylov vector and the map read and write only
// the team's own values.  op 0: k_m x x (H-field form, Eq. 5); op 1: M^{-1} x
// (right preconditioner of Inst, Eq. 4; iden = 1/(k_m^2 - k_b^2)); op 2:
// G(m) x (the adjoint of Eq. 4, A^H v = v - T (G v): G is real and symmetric
// for real k and k_b, and T Hermitian for real eps).
template <typename R, int L0, int TT>
__global__ void __launch_bounds__(TT) k_fwd_x_t8h(Geo g, const typename Io<R>::T *__restrict__ X, long long xstride,
                                                  typename Cx<R>::T *__restrict__ T, const R *__restrict__ scale,
                                                  const int *__restrict__ act,
                                                  const Inst *__restrict__ inst,
                                                  const typename Cx<R>::T *__restrict__ twg, const int *__restrict__ jdev,
                                                  long long jstride, int op, const R *__restrict__ iden, int ph) {
  using C = typename Cx<R>::T;
  using IO = typename Io<R>::T;
  using F = Team8<L0>;
  if (jdev) X += (long long)(*jdev) * jstride;
  constexpr int TS = F::TS, RB = TT / TS;
  __shared__ C bufs[RB * F::BUF];
  const int b = blockIdx.y;
  if (act && !act[b]) return;
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const int Nh = (int)g.Nh, P = N2 * N1;
  const Lanes ln(TS);
  C w[F::NTW];
  F::twiddles(w, ln.lane, twg);
  const HarmSlots<L0, TS> hs(ln.lane, g.n[0]);
  const int r = blockIdx.x * RB + ln.team;
  const bool valid = r < P;
  const R s = scale ? scale[b] : (R)1;
  int my;
  const int mz = divmod_small(r, N1, 1.0f / (float)N1, my);
  const R ky = (R)(inst[b].kinc[1] + (my - g.n[1]) * g.K[1]);
  const R kz = (R)(inst[b].kinc[2] + (mz - g.n[2]) * g.K[2]);
  const IO *Xr = X + b * xstride + r * N0;
  const R *idr = iden ? iden + (long long)b * g.ist + r * N0 : nullptr;
  const R pcc = (R)inst[b].pc_c, pcb = (R)inst[b].pc_beta;
  C v[3][8];
  R idv[4];   // 1/(k_m^2 - k_b^2) of the four harmonic slots, loaded with x (op 1, 2)
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int j = HarmSlots<L0, TS>::slot(a);
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c][a] = mk((R)0, (R)0);
    if (j >= 0) idv[j] = (R)0;
    if (j >= 0 && valid && hs.off[j] >= 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][a] = io_in<C>(Xr[c * Nh + hs.off[j]]);
      if (op == 1 || op == 2) idv[j] = idr[hs.off[j]];
    }
  }
  if (ph) {
    // the row's factor for the shuffle yz pass: a complex constant per row
    // commutes with every per-harmonic map below
    const C wk = ldg_c(&twg[yz_phase_index(my, g.n[1], mz, g.n[2]) * (TWN / 8)]);
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (HarmSlots<L0, TS>::slot(a) >= 0)
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c][a] = cmul(v[c][a], wk);
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int j = HarmSlots<L0, TS>::slot(a);
    if (j < 0) continue;   // no harmonic here: v = 0 and so is k x v
    const int h = hs.off[j];
    const R kx = (R)(inst[b].kinc[0] + (h - g.n[0]) * g.K[0]);
    C u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = mk(v[c][a].x * s, v[c][a].y * s);
    if constexpr (!std::is_same<R, dfl>::value) {
      if (op == 1) {
        // M^{-1} u = alpha u + (beta - alpha) k (k . u) / k^2 (zero where no harmonic sits)
        if (!valid || h < 0) continue;
        const R al = rcp((R)1 - pcc * idv[j]);
        const R k2 = kx * kx + ky * ky + kz * kz;
        const R f = k2 > (R)0 ? (pcb - al) * rcp(k2) : (R)0;
        const C ku = mk(kx * u[0].x + ky * u[1].x + kz * u[2].x, kx * u[0].y + ky * u[1].y + kz * u[2].y);
        v[0][a] = mk(al * u[0].x + f * kx * ku.x, al * u[0].y + f * kx * ku.y);
        v[1][a] = mk(al * u[1].x + f * ky * ku.x, al * u[1].y + f * ky * ku.y);
        v[2][a] = mk(al * u[2].x + f * kz * ku.x, al * u[2].y + f * kz * ku.y);
        continue;
      }
      if (op == 2) {
        // G u = (k_b^2 u - k (k . u)) / (k_m^2 - k_b^2) (zero where no harmonic sits)
        if (!valid || h < 0) continue;
        const R id = idv[j], kb2 = (R)inst[b].kb2;
        const C ku = mk(kx * u[0].x + ky * u[1].x + kz * u[2].x, kx * u[0].y + ky * u[1].y + kz * u[2].y);
        v[0][a] = mk(id * (kb2 * u[0].x - kx * ku.x), id * (kb2 * u[0].y - kx * ku.y));
        v[1][a] = mk(id * (kb2 * u[1].x - ky * ku.x), id * (kb2 * u[1].y - ky * ku.y));
        v[2][a] = mk(id * (kb2 * u[2].x - kz * ku.x), id * (kb2 * u[2].y - kz * ku.y));
        continue;
      }
    }
    // (k x u), zero where no harmonic sits (u = 0 there)
    v[0][a] = csub(cscale(u[2], ky), cscale(u[1], kz));
    v[1][a] = csub(cscale(u[0], kz), cscale(u[2], kx));
    v[2][a] = csub(cscale(u[1], kx), cscale(u[0], ky));
  }
  C *Tq = T + b * g.Tst + (3 * F::freq(ln.lane, 0) * P + mz * N1 + my);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    F::template forward<+1>(v[c], ln.lane, w, bufs + ln.team * F::BUF, ln.mask);
    if (valid)
#pragma unroll
      for (int q = 0; q < 8; ++q) Tq[(F::fstep(q) * 3 + c) * P] = v[c][q];
  }
}

// Plane buffer of pass 2: row r (a z harmonic), column c (a y frequency) at
// r LY + (c XOR sw(r)), sw(r) = 8 (r & 1) + (r & 6).  Row passes touch 4
// consecutive rows x 8 consecutive columns per warp, column passes 8
// consecutive rows x 4 consecutive columns: with the swizzle both spread a
// warp's 8-byte accesses evenly over the 32 banks (two wavefronts, the
// minimum), where a padded pitch fixes only one of the two patterns.
template <int LY> __device__ __forceinline__ int yz_at(int r, int c) {
  return r * LY + (c ^ (((r & 1) << 3) | (r & 6)));
}

template <typename R, int LY, int LZ, int TT>
__global__ void __launch_bounds__(TT) k_yz_t8(Geo g, typename Cx<R>::T *__restrict__ T, const R *__restrict__ D,
                                              const int *__restrict__ act, const typename Cx<R>::T *__restrict__ twg) {
  using C = typename Cx<R>::T;
  using FY = Team8<LY>;
  using FZ = Team8<LZ>;
  constexpr int NTY = TT / FY::TS, NTZ = TT / FZ::TS, NT = NTY > NTZ ? NTY : NTZ;
  __shared__ C bufs[NT * FY::BUF];
  extern __shared__ __align__(16) unsigned char sm_dyn[];
  C *A = reinterpret_cast<C *>(sm_dyn);   // [N2][LY], column index swizzled per row (yz_at)
  const int rx = blockIdx.x, c = blockIdx.y, b = blockIdx.z;
  if (act && !act[b]) return;
  const int N1 = g.N[1], N2 = g.N[2];
  C *Tp = T + b * g.Tst + ((long long)rx * 3 + c) * N2 * N1;   // [m_z][m_y] block
  // y forward: team per m_z row, straight from global memory
  {
    const Lanes ln(FY::TS);
    C w[FY::NTW];
    FY::twiddles(w, ln.lane, twg);
    for (int r0 = 0; r0 < N2; r0 += NTY) {
      const int mz = r0 + ln.team;
      const bool valid = mz < N2;
      C v[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int h = harm_at(ln.lane + FY::TS * a, g.n[1], LY);
        v[a] = (valid && h >= 0) ? Tp[mz * N1 + h] : mk((R)0, (R)0);
      }
      FY::template forward<+1>(v, ln.lane, w, bufs + ln.team * FY::BUF, ln.mask);
      if (valid)
#pragma unroll
        for (int q = 0; q < 8; ++q) A[yz_at<LY>(mz, FY::freq(ln.lane, q))] = v[q];
    }
  }
  __syncthreads();
  // z forward, times D, z inverse: team per y-frequency column
  {
    const Lanes ln(FZ::TS);
    C w[FZ::NTW];
    FZ::twiddles(w, ln.lane, twg);
    const R *Dx = D + (long long)rx * LY * LZ;
    for (int c0 = 0; c0 < LY; c0 += NTZ) {
      const int ry = c0 + ln.team;
      const bool valid = ry < LY;
      C v[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int h = harm_at(ln.lane + FZ::TS * a, g.n[2], LZ);
        v[a] = (valid && h >= 0) ? A[yz_at<LY>(h, ry)] : mk((R)0, (R)0);
      }
      C *bf = bufs + ln.team * FZ::BUF;
      FZ::template forward<+1>(v, ln.lane, w, bf, ln.mask);
      if (valid) {
        const R *Dc = Dx + (long long)ry * LZ;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          v[q] = cscale(v[q], Dc[FZ::freq(ln.lane, q)]);
        }
      }
      FZ::template inverse<-1, true>(v, ln.lane, w, bf, ln.mask);
      if (valid)
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int h = harm_at(ln.lane + FZ::TS * a, g.n[2], LZ);
          if (h >= 0) A[yz_at<LY>(h, ry)] = v[a];
        }
    }
  }
  __syncthreads();
  // y inverse: team per row, straight to global memory
  {
    const Lanes ln(FY::TS);
    C w[FY::NTW];
    FY::twiddles(w, ln.lane, twg);
    for (int r0 = 0; r0 < N2; r0 += NTY) {
      const int mz = r0 + ln.team;
      const bool valid = mz < N2;
      C v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = valid ? A[yz_at<LY>(mz, FY::freq(ln.lane, q))] : mk((R)0, (R)0);
      FY::template inverse<-1, true>(v, ln.lane, w, bufs + ln.team * FY::BUF, ln.mask);
      if (valid)
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int h = harm_at(ln.lane + FY::TS * a, g.n[1], LY);
          if (h >= 0) Tp[mz * N1 + h] = v[a];
        }
    }
  }
}

// Row pitch of the pass-3 buffer: 8 mod 16 complex values, so the four
// teams of a warp (consecutive rows, 8 consecutive columns each) cover the
// 32 banks evenly.
__host__ __device__ __forceinline__ int p3_pitch(int N0) { return (N0 + 15) / 16 * 16 + 8; }

// (component, row) items per lane team in pass 3, all loads issued before the
// first transform: for 32/64-point teams three with 8-byte values (complex64:
// a team then holds the three components of one row; 330 against 367 us per
// launch with two and 390 with four, at batch 512) and two with 16-byte values (complex128 and
// double-float, whose registers would grow past 170 with three); one for the
// 128-point teams, whose registers are already taken by the longer transforms
template <int L0, typename R> __host__ __device__ constexpr int p3_items() {
  return L0 <= 64 ? (sizeof(typename Cx<R>::T) == 8 ? 3 : 2) : 1;
}

// Pass 2 for complex64 with 64-point y and z transforms, two x frequencies
// (r_x, r_x + 1) per block: every lane runs the transforms of both planes at
// once in packed FP32 pairs (Team8x2).  The plane buffer holds value pairs
// [m_z][r_y] with a row pitch of 65 pairs: a team writing a row segment (8
// consecutive columns) and a team reading a column segment (8 consecutive
// rows, 1040 bytes apart) both hit 8 distinct 16-byte bank groups, and
// every access is a per-lane base plus a compile-time or loop offset.  D
// comes as plane pairs Dp[r_x / 2][r_y][r_z] = (D(r_x, ...), D(r_x + 1, ...)).
// Inputs at lane + 8 a exist only for a in {0, 1, 6, 7} (64 >= 4 n + 4),
// which is also where the inverse transforms' kept outputs lie.
constexpr int YZP = 65;   // row pitch (value pairs) of the pass-2 plane buffer

__host__ __device__ constexpr int reg0167(int k) { return k < 2 ? k : k + 4; }

template <int TT>
__global__ void __launch_bounds__(TT) k_yz_t8x2(Geo g, float2 *__restrict__ T, const float2 *__restrict__ Dp,
                                                const int *__restrict__ act, const float2 *__restrict__ twg) {
  using F = Team8x2;
  constexpr int NT = TT / 8;
  extern __shared__ __align__(16) unsigned char sm_dyn[];
  CP *bufs = reinterpret_cast<CP *>(sm_dyn);   // [NT][F::BUF]: team transposes
  CP *A = bufs + NT * F::BUF;                  // [N2][YZP] value pairs
  const int N1 = g.N[1], N2 = g.N[2];
  const int xp = blockIdx.x, c = blockIdx.y, b = blockIdx.z;
  if (act && !act[b]) return;
  float2 *Ta = T + b * g.Tst + ((long long)(2 * xp) * 3 + c) * N2 * N1;   // [m_z][m_y] block of r_x = 2 xp
  float2 *Tb = Ta + 3LL * N2 * N1;                                         // and of r_x = 2 xp + 1
  const int team = threadIdx.x >> 3, lane = threadIdx.x & 7;
  const unsigned mask = 0xffu << (threadIdx.x & 24);
  CP *bf = bufs + team * F::BUF;
  WP w[8];
  F::twiddles(w, lane, twg);
  int hy[4], hz[4];   // harmonic held by register reg0167(k) of this lane along y / z, or -1
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    hy[k] = harm_at(lane + 8 * reg0167(k), g.n[1], 64);
    hz[k] = harm_at(lane + 8 * reg0167(k), g.n[2], 64);
  }
  const CP zero = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  // y forward: team per m_z row of both planes, straight from global memory
  for (int r0 = 0; r0 < N2; r0 += NT) {
    const int mz = r0 + team;
    const bool valid = mz < N2;
    const float2 *ra = Ta + mz * N1, *rb = Tb + mz * N1;
    CP v[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) v[a] = zero;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (valid && hy[k] >= 0) {
        const float2 xa = ra[hy[k]], xb = rb[hy[k]];
        v[reg0167(k)] = {make_float2(xa.x, xb.x), make_float2(xa.y, xb.y)};
      }
    F::forward<+1>(v, lane, w, bf, mask);
    if (valid) {
      CP *Ar = A + mz * YZP + lane;
#pragma unroll
      for (int q = 0; q < 8; ++q) Ar[8 * q] = v[q];
    }
  }
  __syncthreads();
  // z forward, times D, z inverse: team per y-frequency column
  const float2 *Dx = Dp + (long long)xp * 64 * 64;
  for (int c0 = 0; c0 < 64; c0 += NT) {
    const int ry = c0 + team;
    CP v[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) v[a] = zero;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (hz[k] >= 0) v[reg0167(k)] = A[hz[k] * YZP + ry];
    F::forward<+1>(v, lane, w, bf, mask);
    const float2 *Dc = Dx + ry * 64 + lane;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float2 d = __ldg(&Dc[8 * q]);
      v[q].re = f2::mul(v[q].re, d);
      v[q].im = f2::mul(v[q].im, d);
    }
    F::inverse<-1, true>(v, lane, w, bf, mask);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (hz[k] >= 0) A[hz[k] * YZP + ry] = v[reg0167(k)];
  }
  __syncthreads();
  // y inverse: team per row, straight to global memory
  for (int r0 = 0; r0 < N2; r0 += NT) {
    const int mz = r0 + team;
    const bool valid = mz < N2;
    CP v[8];
    const CP *Ar = A + mz * YZP + lane;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = valid ? Ar[8 * q] : zero;
    F::inverse<-1, true>(v, lane, w, bf, mask);
    if (valid) {
      float2 *ra = Ta + mz * N1, *rb = Tb + mz * N1;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (hy[k] >= 0) {
          const CP x = v[reg0167(k)];
          ra[hy[k]] = make_float2(x.re.x, x.im.x);
          rb[hy[k]] = make_float2(x.re.y, x.im.y);
        }
    }
  }
}



// Pass 2 as k_yz_t8x2 with the transposes inside each 64-point transform done
// by lane shuffles (Team8x2R) instead of team buffers: shared memory holds
// only the plane.  The y forward leaves its rows phase-deferred (frequency
// r_y carries the factor w8^{-(r_y mod 8)(r_y / 8)}, constant along each z
// column); the z forward, x D, z inverse of a column keep that factor, and
// the y inverse consumes it.  The rotation's input modulations w8^{a t} (y
// position t + 8 a) and w8^{a' t'} (z position t' + 8 a') are a factor per
// (m_z, m_y) row of T, which pass 1 applies to its output (yz_phase_index)
// and pass 3 removes from its input, and so are the conjugate output
// modulations of the inverses: T between the passes is the plain
// intermediate times that factor, and this kernel never applies it.
template <int TT>
__global__ void __launch_bounds__(TT) k_yz_t8x2r(Geo g, float2 *__restrict__ T, const float2 *__restrict__ Dp,
                                                 const int *__restrict__ act, const float2 *__restrict__ twg) {
  using F = Team8x2R;
  constexpr int NT = TT / 8;
  extern __shared__ __align__(16) unsigned char sm_dyn[];
  CP *A = reinterpret_cast<CP *>(sm_dyn);   // [N2][YZP] value pairs
  const int N1 = g.N[1], N2 = g.N[2];
  const int xp = blockIdx.x, c = blockIdx.y, b = blockIdx.z;
  if (act && !act[b]) return;
  float2 *Ta = T + b * g.Tst + ((long long)(2 * xp) * 3 + c) * N2 * N1;   // [m_z][m_y] block of r_x = 2 xp
  float2 *Tb = Ta + 3LL * N2 * N1;                                         // and of r_x = 2 xp + 1
  const int team = threadIdx.x >> 3, lane = threadIdx.x & 7;
  const unsigned mask = 0xffu << (threadIdx.x & 24);
  WP tw[8];
  F::constants(tw, lane, twg);
  int hy[4], hz[4];   // harmonic held by register reg0167(k) of this lane along y / z, or -1
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    hy[k] = harm_at(lane + 8 * reg0167(k), g.n[1], 64);
    hz[k] = harm_at(lane + 8 * reg0167(k), g.n[2], 64);
  }
  const CP zero = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  // y forward: team per m_z row of both planes, straight from global memory
  for (int r0 = 0; r0 < N2; r0 += NT) {
    const int mz = r0 + team;
    const bool valid = mz < N2;
    const float2 *ra = Ta + mz * N1, *rb = Tb + mz * N1;
    CP v[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) v[a] = zero;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (valid && hy[k] >= 0) {
        const float2 xa = ra[hy[k]], xb = rb[hy[k]];
        v[reg0167(k)] = {make_float2(xa.x, xb.x), make_float2(xa.y, xb.y)};
      }
    F::forward<+1, false>(v, lane, tw, nullptr, mask);
    if (valid) {
      CP *Ar = A + mz * YZP + lane;
#pragma unroll
      for (int q = 0; q < 8; ++q) Ar[8 * q] = v[q];
    }
  }
  __syncthreads();
  // z forward, times D, z inverse: team per y-frequency column
  const float2 *Dx = Dp + (long long)xp * 64 * 64;
  for (int c0 = 0; c0 < 64; c0 += NT) {
    const int ry = c0 + team;
    CP v[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) v[a] = zero;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (hz[k] >= 0) v[reg0167(k)] = A[hz[k] * YZP + ry];
    F::forward<+1, false>(v, lane, tw, nullptr, mask);
    const float2 *Dc = Dx + ry * 64 + lane;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float2 d = __ldg(&Dc[8 * q]);
      v[q].re = f2::mul(v[q].re, d);
      v[q].im = f2::mul(v[q].im, d);
    }
    F::inverse<-1, false>(v, lane, tw, nullptr, mask);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (hz[k] >= 0) A[hz[k] * YZP + ry] = v[reg0167(k)];
  }
  __syncthreads();
  // y inverse: team per row, straight to global memory
  for (int r0 = 0; r0 < N2; r0 += NT) {
    const int mz = r0 + team;
    const bool valid = mz < N2;
    CP v[8];
    const CP *Ar = A + mz * YZP + lane;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = valid ? Ar[8 * q] : zero;
    F::inverse<-1, false>(v, lane, tw, nullptr, mask);
    if (valid) {
      float2 *ra = Ta + mz * N1, *rb = Tb + mz * N1;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (hy[k] >= 0) {
          const CP x = v[reg0167(k)];
          ra[hy[k]] = make_float2(x.re.x, x.im.x);
          rb[hy[k]] = make_float2(x.re.y, x.im.y);
        }
    }
  }
}

// MODE 0: Y = X - G u; MODE 1: Y = b - (X - G u); HF = 1 (Eq. 5): G u is
// replaced by k_m x u / (k_m^2 - k_b^2).  nog = 1 (adjoint of Eq. 4, G
// already applied in pass 1): G u is replaced by u.
// (the body of the pass-3 kernels below)
template <typename R, int L0, int MODE, int TT, int HF>
__device__ __forceinline__ void inv_x_t8(Geo g, const typename Cx<R>::T *__restrict__ T,
                                         const typename Io<R>::T *__restrict__ X, long long xstride,
                                         typename Io<R>::T *__restrict__ Y, long long ystride,
                                         const int *__restrict__ act, const Inst *__restrict__ inst,
                                         const R *__restrict__ iden, const typename Cx<R>::T *__restrict__ twg,
                                         int rows, double *partial, unsigned *counter, double *norm_out,
                                         const int *__restrict__ jdev, long long jstride, int pc, int nog,
                                         const R *__restrict__ scale, int ph) {
  using C = typename Cx<R>::T;
  using IO = typename Io<R>::T;
  using F = Team8<L0>;
  if (jdev) {
    X += (long long)(*jdev) * jstride;
    Y += (long long)(*jdev) * jstride;
  }
  constexpr int TS = F::TS, NTM = TT / TS, IPT = p3_items<L0, R>();
  __shared__ C bufs[NTM * F::BUF];
  __shared__ double red[32];
  extern __shared__ __align__(16) unsigned char sm_dyn[];
  C *S3 = reinterpret_cast<C *>(sm_dyn);   // [3][rows][P], then phase[rows], kx[N0], ky[rows], kz[rows]
  const int b = blockIdx.y;
  if (act && !act[b]) return;
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2], P = p3_pitch(N0);
  const int Nh = (int)g.Nh, P2 = N1 * N2;   // 32-bit offsets: 3 Nh < 2^22
  const int r0 = blockIdx.x * rows;
  const int nr = min(rows, P2 - r0);
  C *phs = S3 + 3 * rows * P;   // per row: the conjugate of the shuffle yz pass's factor (ph)
  R *kxs = reinterpret_cast<R *>(phs + rows);
  R *kys = kxs + N0, *kzs = kys + rows;
  // epilogue mapping: warp per row (rows warp, warp + NW, ...), lane per
  // x harmonic mx = lane + 32 m, m < MXN (2 N0 - 1 <= L0, so N0 <= 32 MXN).
  // The first PF rows' inputs are fetched now, so their loads overlap the
  // transforms below.
  constexpr int NW = TT / 32, PF = 2, MXN = L0 > 64 ? 2 : 1;
  const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
  const IO *Xb = X + b * xstride;
  C px[PF][MXN][3];
  R pid[PF][MXN];
#pragma unroll
  for (int i = 0; i < PF; ++i)
#pragma unroll
    for (int m = 0; m < MXN; ++m) {
      const int row = warp + i * NW, mx = wl + 32 * m;
      px[i][m][0] = px[i][m][1] = px[i][m][2] = mk((R)0, (R)0);
      pid[i][m] = 0;
      if (mx < N0 && row < nr) {
        const int h = (r0 + row) * N0 + mx;
        px[i][m][0] = io_in<C>(Xb[h]);
        px[i][m][1] = io_in<C>(Xb[Nh + h]);
        px[i][m][2] = io_in<C>(Xb[2 * Nh + h]);
        pid[i][m] = iden[(long long)b * g.ist + h];
      }
    }
  for (int i = threadIdx.x; i < N0; i += blockDim.x) kxs[i] = (R)(inst[b].kinc[0] + (i - g.n[0]) * g.K[0]);
  for (int i = threadIdx.x; i < nr; i += blockDim.x) {
    int my;
    const int mz = divmod_small(r0 + i, N1, 1.0f / (float)N1, my);
    kys[i] = (R)(inst[b].kinc[1] + (my - g.n[1]) * g.K[1]);
    kzs[i] = (R)(inst[b].kinc[2] + (mz - g.n[2]) * g.K[2]);
    if constexpr (sizeof(R) == 4) {
      if (ph) {
        const C wk = ldg_c(&twg[yz_phase_index(my, g.n[1], mz, g.n[2]) * (TWN / 8)]);
        phs[i] = mk(wk.x, -wk.y);
      }
    }
  }
  {
    // team items (c, row) = divmod(team + i NTM, rows), i < IPT: the loads of
    // all of a team's items are issued before its first transform
    const Lanes ln(TS);
    C w[F::NTW];
    F::twiddles(w, ln.lane, twg);
    C v[IPT][8];
    int it_c[IPT], it_row[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const int item = ln.team + i * NTM;
      const int c = item / rows, row = item - c * rows;
      it_c[i] = c;
      it_row[i] = row;
      const bool valid = c < 3 && row < nr;
      const C *Tq = T + b * g.Tst + ((3 * F::freq(ln.lane, 0) + c) * P2 + r0 + row);
#pragma unroll
      for (int q = 0; q < 8; ++q) v[i][q] = valid ? Tq[F::fstep(q) * 3 * P2] : mk((R)0, (R)0);
    }
    const HarmSlots<L0, TS> hs(ln.lane, g.n[0]);
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      F::template inverse<-1, true>(v[i], ln.lane, w, bufs + ln.team * F::BUF, ln.mask);
      if (it_c[i] < 3 && it_row[i] < nr) {
        C *Sr = S3 + (it_c[i] * rows + it_row[i]) * P;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int j = HarmSlots<L0, TS>::slot(a);
          if (j >= 0 && hs.off[j] >= 0) Sr[hs.off[j]] = v[i][a];
        }
      }
    }
  }
  __syncthreads();
  const R kb2 = (R)inst[b].kb2, pcc = (R)inst[b].pc_c, pcb = (R)inst[b].pc_beta;
  const int h0 = (g.n[2] * N1 + g.n[1]) * N0 + g.n[0];
  IO *Yb = Y + b * ystride;
  R acc = 0;   // this thread's share of ||y||^2 (a few harmonics), widened once
  // the identity term takes the input as pass 1 did: scaled by 1 / ||v_j||
  // (the stored Krylov vector is unnormalised)
  const bool sc = scale != nullptr;
  const R sx = sc ? scale[b] : (R)1;
  auto body = [&](int row, int mx, C y0, C y1, C y2, R id) {
    if (sc) {
      y0 = cscale(y0, sx);
      y1 = cscale(y1, sx);
      y2 = cscale(y2, sx);
    }
    const int h = (r0 + row) * N0 + mx;
    C u0 = S3[(0 * rows + row) * P + mx], u1 = S3[(1 * rows + row) * P + mx], u2 = S3[(2 * rows + row) * P + mx];
    if constexpr (sizeof(R) == 4) {   // only the complex64 shuffle pass leaves a row factor
      if (ph) {
        const C pw = phs[row];
        u0 = cmul(u0, pw);
        u1 = cmul(u1, pw);
        u2 = cmul(u2, pw);
      }
    }
    const R kx = kxs[mx], ky = kys[row], kz = kzs[row];
    if (HF) {
      y0 = csub(y0, cscale(csub(cscale(u2, ky), cscale(u1, kz)), id));
      y1 = csub(y1, cscale(csub(cscale(u0, kz), cscale(u2, kx)), id));
      y2 = csub(y2, cscale(csub(cscale(u1, kx), cscale(u0, ky)), id));
    } else if (nog) {
      y0 = csub(y0, u0);
      y1 = csub(y1, u1);
      y2 = csub(y2, u2);
    } else {
      if constexpr (!std::is_same<R, dfl>::value) {
        if (pc) {
          // identity term of A M^{-1} x: x <- M^{-1} x = alpha x + (beta - alpha) k (k . x) / k^2
          const R al = rcp((R)1 - pcc * id);
          const R k2 = kx * kx + ky * ky + kz * kz;
          const R f = k2 > (R)0 ? (pcb - al) * rcp(k2) : (R)0;
          const R kxr = kx * y0.x + ky * y1.x + kz * y2.x, kxi = kx * y0.y + ky * y1.y + kz * y2.y;
          y0 = mk(al * y0.x + f * kx * kxr, al * y0.y + f * kx * kxi);
          y1 = mk(al * y1.x + f * ky * kxr, al * y1.y + f * ky * kxi);
          y2 = mk(al * y2.x + f * kz * kxr, al * y2.y + f * kz * kxi);
        }
      }
      const R kux = kx * u0.x + ky * u1.x + kz * u2.x, kuy = kx * u0.y + ky * u1.y + kz * u2.y;
      y0.x -= id * (kb2 * u0.x - kx * kux);
      y0.y -= id * (kb2 * u0.y - kx * kuy);
      y1.x -= id * (kb2 * u1.x - ky * kux);
      y1.y -= id * (kb2 * u1.y - ky * kuy);
      y2.x -= id * (kb2 * u2.x - kz * kux);
      y2.y -= id * (kb2 * u2.y - kz * kuy);
    }
    if (MODE == 1) {
      C a0 = mk((R)0, (R)0), a1 = a0, a2 = a0;
      if (h == h0) {
        a0 = mk((R)inst[b].a[0], (R)inst[b].a[1]);
        a1 = mk((R)inst[b].a[2], (R)inst[b].a[3]);
        a2 = mk((R)inst[b].a[4], (R)inst[b].a[5]);
      }
      y0 = mk(a0.x - y0.x, a0.y - y0.y);
      y1 = mk(a1.x - y1.x, a1.y - y1.y);
      y2 = mk(a2.x - y2.x, a2.y - y2.y);
    }
    if (norm_out) acc += y0.x * y0.x + y0.y * y0.y + y1.x * y1.x + y1.y * y1.y + y2.x * y2.x + y2.y * y2.y;
    Yb[h] = io_out<IO>(y0);
    Yb[Nh + h] = io_out<IO>(y1);
    Yb[2 * Nh + h] = io_out<IO>(y2);
  };
#pragma unroll
  for (int i = 0; i < PF; ++i)
#pragma unroll
    for (int m = 0; m < MXN; ++m) {
      const int row = warp + i * NW, mx = wl + 32 * m;
      if (row < nr && mx < N0) body(row, mx, px[i][m][0], px[i][m][1], px[i][m][2], pid[i][m]);
    }
  for (int row = warp + PF * NW; row < nr; row += NW)
#pragma unroll
    for (int m = 0; m < MXN; ++m) {
      const int mx = wl + 32 * m;
      if (mx < N0) {
        const int h = (r0 + row) * N0 + mx;
        body(row, mx, io_in<C>(Xb[h]), io_in<C>(Xb[Nh + h]), io_in<C>(Xb[2 * Nh + h]), iden[(long long)b * g.ist + h]);
      }
    }
  if (norm_out) last_block_sum((double)acc, red, partial, counter, norm_out, b, gridDim.x, blockIdx.x);
}

#define GSM_P3_PARAMS                                                                                       \
  Geo g, const typename Cx<R>::T *__restrict__ T, const typename Io<R>::T *__restrict__ X, long long xstride, \
      typename Io<R>::T *__restrict__ Y, long long ystride, const int *__restrict__ act,                     \
      const Inst *__restrict__ inst, const R *__restrict__ iden, const typename Cx<R>::T *__restrict__ twg,  \
      int rows, double *partial, unsigned *counter, double *norm_out, const int *__restrict__ jdev,          \
      long long jstride, int pc, int nog, const R *__restrict__ scale, int ph
#define GSM_P3_ARGS g, T, X, xstride, Y, ystride, act, inst, iden, twg, rows, partial, counter, norm_out, jdev, \
                    jstride, pc, nog, scale, ph
template <typename R, int L0, int MODE, int TT, int HF>
__global__ void __launch_bounds__(TT) k_inv_x_t8(GSM_P3_PARAMS) {
  inv_x_t8<R, L0, MODE, TT, HF>(GSM_P3_ARGS);
}
// complex64: compiled for five 128-thread blocks per SM (96 registers; the
// epilogue's row factor for the shuffle yz pass would otherwise take 108 and
// leave four)
template <typename R, int L0, int MODE, int TT, int HF>
__global__ void __launch_bounds__(TT, 640 / TT) k_inv_x_t8c(GSM_P3_PARAMS) {
  inv_x_t8<R, L0, MODE, TT, HF>(GSM_P3_ARGS);
}
#undef GSM_P3_PARAMS
#undef GSM_P3_ARGS
template <typename R, int L0, int MODE, int TT, int HF> constexpr auto p3_kernel() {
  if constexpr (sizeof(R) == 4) return &k_inv_x_t8c<R, L0, MODE, TT, HF>;
  else return &k_inv_x_t8<R, L0, MODE, TT, HF>;
}


template <typename R>
static int p3_rows(const Geo &g, int tb) {
  const int items = (tb / (g.L[0] / 8)) * (g.L[0] <= 64 ? p3_items<64, R>() : p3_items<128, R>());
  return items / 3;
}


constexpr int P1_RPT = 2;   // rows per team in pass 1

// whether pass 2 is the complex64 shuffle kernel, which leaves its rows'
// 8th-root factors to passes 1 and 3 (the same test as pass2's)
template <typename R> static int yz_phase(const MatvecArgs<R> &a) {
  if constexpr (sizeof(R) == 4) return (a.Dp && packed_yz_ok(a.g) && a.yzv == 1) ? 1 : 0;
  else return 0;
}

// Threads per block of the 128-point kernels: their static team buffers
// (TT / 16 teams x 144 values) stay under 48 KB for 16-byte values only up
// to 256 threads.
template <typename R, int TT>
constexpr int tt128() { return (sizeof(typename Cx<R>::T) > 8 && TT > 256) ? 256 : TT; }

template <typename R, int TT>
static void pass1(const MatvecArgs<R> &a, cudaStream_t st) {
  const Geo &g = a.g;
  if (g.L[0] == 128) {
    constexpr int TX = tt128<R, TT>();
    if (a.form || a.pc || a.mode >= 2) {
      dim3 gridh((int)(((long long)g.N[2] * g.N[1] + TX / 16 - 1) / (TX / 16)), a.B);
      k_fwd_x_t8h<R, 128, TX><<<gridh, TX, 0, st>>>(g, a.X, a.xstride, a.T, a.scale, a.act, a.inst,
                                                    a.tw, a.jdev, a.jstride, a.form ? 0 : (a.mode >= 2 ? 2 : 1),
                                                    a.iden, yz_phase(a));
    } else {
      const int RB = TX / 16 * P1_RPT;
      dim3 grid((int)((3LL * g.N[2] * g.N[1] + RB - 1) / RB), a.B);
      k_fwd_x_t8<R, 128, TX, P1_RPT><<<grid, TX, 0, st>>>(g, a.X, a.xstride, a.T, a.scale, a.act,
                                                          a.tw, a.jdev, a.jstride, yz_phase(a));
    }
    return;
  }
  const int RB = TT / (g.L[0] / 8) * P1_RPT;
  dim3 grid((int)((3LL * g.N[2] * g.N[1] + RB - 1) / RB), a.B);
  if (a.form || a.pc || a.mode >= 2) {
    const int RBH = TT / (g.L[0] / 8);
    const int op = a.form ? 0 : (a.mode >= 2 ? 2 : 1);
    dim3 gridh((int)(((long long)g.N[2] * g.N[1] + RBH - 1) / RBH), a.B);
    if (g.L[0] == 64)
      k_fwd_x_t8h<R, 64, TT><<<gridh, TT, 0, st>>>(g, a.X, a.xstride, a.T, a.scale, a.act, a.inst,
                                                   a.tw, a.jdev, a.jstride, op, a.iden, yz_phase(a));
    else
      k_fwd_x_t8h<R, 32, TT><<<gridh, TT, 0, st>>>(g, a.X, a.xstride, a.T, a.scale, a.act, a.inst,
                                                   a.tw, a.jdev, a.jstride, op, a.iden, yz_phase(a));
    return;
  }
  if (g.L[0] == 64)
    k_fwd_x_t8<R, 64, TT, P1_RPT><<<grid, TT, 0, st>>>(g, a.X, a.xstride, a.T, a.scale, a.act, a.tw,
                                                       a.jdev, a.jstride, yz_phase(a));
  else
    k_fwd_x_t8<R, 32, TT, P1_RPT><<<grid, TT, 0, st>>>(g, a.X, a.xstride, a.T, a.scale, a.act, a.tw,
                                                       a.jdev, a.jstride, yz_phase(a));
}

template <typename R, int TT>
static void pass2(const MatvecArgs<R> &a, cudaStream_t st) {
  using C = typename Cx<R>::T;
  const Geo &g = a.g;
  if constexpr (sizeof(R) == 4) {
    if (a.Dp && packed_yz_ok(g) && a.yzv == 1) {
      const size_t smem2 = sizeof(CP) * (size_t)g.N[2] * YZP;
      dim3 grid2(g.L[0] / 2, 3, a.B);
      cudaFuncSetAttribute(k_yz_t8x2r<TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
      k_yz_t8x2r<TT><<<grid2, TT, smem2, st>>>(g, a.T, a.Dp, a.act, a.tw);
      return;
    }
    if (a.Dp && packed_yz_ok(g)) {
      const size_t smem2 = sizeof(CP) * ((size_t)g.N[2] * YZP + (TT / 8) * Team8x2::BUF);
      dim3 grid2(g.L[0] / 2, 3, a.B);
      cudaFuncSetAttribute(k_yz_t8x2<TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
      k_yz_t8x2<TT><<<grid2, TT, smem2, st>>>(g, a.T, a.Dp, a.act, a.tw);
      return;
    }
  }
  const size_t smem = sizeof(C) * (size_t)g.N[2] * g.L[1];
  dim3 grid(g.L[0], 3, a.B);
  if (g.L[1] == 128 && g.L[2] == 128) {
    constexpr int TX = tt128<R, TT>();
    cudaFuncSetAttribute(k_yz_t8<R, 128, 128, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_yz_t8<R, 128, 128, TX><<<grid, TX, smem, st>>>(g, a.T, a.D, a.act, a.tw);
    return;
  }
#define GSM_YZ(LY, LZ)                                                                                      \
  cudaFuncSetAttribute(k_yz_t8<R, LY, LZ, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
  k_yz_t8<R, LY, LZ, TT><<<grid, TT, smem, st>>>(g, a.T, a.D, a.act, a.tw)
  if (g.L[1] == 64 && g.L[2] == 64) { GSM_YZ(64, 64); }
  else if (g.L[1] == 64) { GSM_YZ(64, 32); }
  else if (g.L[2] == 64) { GSM_YZ(32, 64); }
  else { GSM_YZ(32, 32); }
#undef GSM_YZ
}

template <typename R, int TT>
static void pass3(const MatvecArgs<R> &a, cudaStream_t st) {
  using C = typename Cx<R>::T;
  const Geo &g = a.g;
  if (g.L[0] == 128) {
    constexpr int TX = tt128<R, TT>();
    const int rows = p3_rows<R>(g, TX);
    const size_t smem = sizeof(C) * (3 * (size_t)rows * p3_pitch(g.N[0]) + rows) + sizeof(R) * (g.N[0] + 2 * rows) + 16;
    dim3 grid((int)(((long long)g.N[1] * g.N[2] + rows - 1) / rows), a.B);
#define GSM_P3X(M, HF)                                                                                           \
  cudaFuncSetAttribute(p3_kernel<R, 128, M, TX, HF>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
  p3_kernel<R, 128, M, TX, HF>()<<<grid, TX, smem, st>>>(g, a.T, a.X, a.xstride, a.Y, a.ystride, a.act, a.inst,   \
                                                        a.iden, a.tw, rows, a.partial, a.counter, a.norm_out,     \
                                                        a.jdev, a.jstride, a.pc, a.mode >= 2, a.scale, yz_phase(a))
    if (a.form) { if (a.mode & 1) { GSM_P3X(1, 1); } else { GSM_P3X(0, 1); } }
    else { if (a.mode & 1) { GSM_P3X(1, 0); } else { GSM_P3X(0, 0); } }
#undef GSM_P3X
    return;
  }
  const int rows = p3_rows<R>(g, TT);
  const size_t smem = sizeof(C) * (3 * (size_t)rows * p3_pitch(g.N[0]) + rows) + sizeof(R) * (g.N[0] + 2 * rows) + 16;
  dim3 grid((int)(((long long)g.N[1] * g.N[2] + rows - 1) / rows), a.B);
#define GSM_P3(L0, M, HF)                                                                                         \
  cudaFuncSetAttribute(p3_kernel<R, L0, M, TT, HF>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);   \
  p3_kernel<R, L0, M, TT, HF>()<<<grid, TT, smem, st>>>(g, a.T, a.X, a.xstride, a.Y, a.ystride, a.act, a.inst,     \
                                                       a.iden, a.tw, rows, a.partial, a.counter, a.norm_out, a.jdev, \
                                                       a.jstride, a.pc, a.mode >= 2, a.scale, yz_phase(a))
  if (g.L[0] == 64) {
    if (a.form) { if (a.mode & 1) { GSM_P3(64, 1, 1); } else { GSM_P3(64, 0, 1); } }
    else { if (a.mode & 1) { GSM_P3(64, 1, 0); } else { GSM_P3(64, 0, 0); } }
  } else {
    if (a.form) { if (a.mode & 1) { GSM_P3(32, 1, 1); } else { GSM_P3(32, 0, 1); } }
    else { if (a.mode & 1) { GSM_P3(32, 1, 0); } else { GSM_P3(32, 0, 0); } }
  }
#undef GSM_P3
}

template <typename R, template <typename, int> class F>
static cudaError_t dispatch_tb(int tb, const MatvecArgs<R> &a, cudaStream_t st) {
  if constexpr (std::is_same<R, dfl>::value) {   // the double-float product runs with 256 threads only
    F<R, 256>::run(a, st);
    return cudaGetLastError();
  }
  if (tb == 128) F<R, 128>::run(a, st);
  else if (tb == 512) F<R, 512>::run(a, st);
  else F<R, 256>::run(a, st);
  return cudaGetLastError();
}
template <typename R, int TT> struct P1 { static void run(const MatvecArgs<R> &a, cudaStream_t st) { pass1<R, TT>(a, st); } };
template <typename R, int TT> struct P2 { static void run(const MatvecArgs<R> &a, cudaStream_t st) { pass2<R, TT>(a, st); } };
template <typename R, int TT> struct P3 { static void run(const MatvecArgs<R> &a, cudaStream_t st) { pass3<R, TT>(a, st); } };

// One pass of the lane-team product with a given block size.  Each
// (precision, pass) pair is instantiated in a translation unit of its own
// (matvec_reg_<precision>_p<pass>.cu), so that the passes compile in
// parallel; the units that instantiate launch_reg_pass declare them extern.
template <typename R, int PASS>
cudaError_t reg_pass(int tb, const MatvecArgs<R> &a, cudaStream_t st) {
  if constexpr (PASS == 1) return dispatch_tb<R, P1>(tb, a, st);
  else if constexpr (PASS == 2) return dispatch_tb<R, P2>(tb, a, st);
  else return dispatch_tb<R, P3>(tb, a, st);
}

#define GSM_EXTERN_REG_PASSES(R)                                                          \
  extern template cudaError_t reg_pass<R, 1>(int, const MatvecArgs<R> &, cudaStream_t);  \
  extern template cudaError_t reg_pass<R, 2>(int, const MatvecArgs<R> &, cudaStream_t);  \
  extern template cudaError_t reg_pass<R, 3>(int, const MatvecArgs<R> &, cudaStream_t);

// One pass of the lane-team product with a given block size (autotuner).
template <typename R>
cudaError_t launch_reg_pass(int pass, int tb, const MatvecArgs<R> &a, cudaStream_t st) {
  if (pass == 1) return reg_pass<R, 1>(tb, a, st);
  if (pass == 2) return reg_pass<R, 2>(tb, a, st);
  return reg_pass<R, 3>(tb, a, st);
}

template <typename R>
cudaError_t launch_matvec_reg(const MatvecArgs<R> &a, cudaStream_t st, Profiler *prof, const int *tb) {
  using C = typename Cx<R>::T;
  const Geo &g = a.g;
  const double cs = sizeof(C);
  const int t1 = tb ? tb[0] : TB_DEFAULT, t2 = tb ? tb[1] : TB_DEFAULT, t3 = tb ? tb[2] : TB_DEFAULT;
  cudaError_t e;
  if (prof) prof->begin(KIND_FWD_X, st);
  if ((e = launch_reg_pass<R>(1, t1, a, st)) != cudaSuccess) return e;
  // bytes this layout moves per launch, for the instances still active: pass 1
  // reads x and writes T (plus the scaled x written back inside solves and,
  // in the three-component variant, the per-harmonic denominators)
  const double nb = a.nact > 0 ? a.nact : a.B;
  const bool p1h = a.form || a.pc || a.mode >= 2;
  if (prof)
    prof->end(KIND_FWD_X, st,
              nb * (cs * (double)(g.U + g.Tsz) + (p1h ? sizeof(R) * (double)g.Nh : 0.0)));
  if (prof) prof->begin(KIND_YZ, st);
  if ((e = launch_reg_pass<R>(2, t2, a, st)) != cudaSuccess) return e;
  if (prof) prof->end(KIND_YZ, st, nb * 2.0 * cs * (double)g.Tsz + sizeof(R) * (double)g.L[0] * g.L[1] * g.L[2]);
  if (prof) prof->begin(KIND_INV_X, st);
  if ((e = launch_reg_pass<R>(3, t3, a, st)) != cudaSuccess) return e;
  if (prof) prof->end(KIND_INV_X, st, nb * (cs * (double)(g.Tsz + 2 * g.U) + sizeof(R) * (double)g.Nh));
  return cudaGetLastError();
}

}  // namespace gsm
