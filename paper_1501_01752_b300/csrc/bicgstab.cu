// Batched BiCGSTAB (van der Vorst) for the Eq. 4 system, the alternative
// Krylov method the paper names beside GMRES ("Calculation details").
//
// Each instance b owns seven vectors V[b][slot][Us] in the working precision
// (slots below); scalars and dot accumulations are FP64.  One iteration is
//
//   k_bicg_p       p = r + beta (p - omega v),  beta = (rho / rho_old)(alpha / omega)
//                  (p = r in the first iteration)
//   product        v = A p
//   k_bicg_alpha   alpha = rho / <r^, v>
//   k_bicg_s       s = r - alpha v
//   product        t = A s
//   k_bicg_omega   omega = <t, s> / <t, t>
//   k_bicg_update  d += alpha p + omega s,  r = s - omega t,
//                  rho_old = rho, rho = <r^, r>, ||r||^2, stop test
//
// with r^ = r_0 (the shadow residual), x0 = 0 and d the correction of the
// cycle.  Reductions use the last-block-done pattern (an atomic counter per
// instance, no waiting); the last block of a reduction computes the scalar
// and may deactivate its instance (convergence, iteration cap, breakdown
// <r^, v> = 0, rho = 0 or omega = 0).  Inactive instances skip every kernel,
// so all blocks of an instance take part in a reduction or none do.
#include "kernels.h"
#include "reduce.cuh"
#include "vec.cuh"

namespace gsm {

namespace {

constexpr int BT = 256;  // threads per block

// Sum K values per thread over the instance's blocks; true in every thread
// of the instance's last block, where tot[] holds the sums.
template <int K>
__device__ bool last_block_sums(double (&v)[K], double *partial, unsigned *counter, int b, int nblk, int blk,
                                double (&tot)[K]) {
  __shared__ double red[K][32];
  __shared__ int am_last;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double s = warp_sum(v[k]);
    if (l == 0) red[k][w] = s;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0;
    for (int q = 0; q < nw; ++q) s += red[threadIdx.x][q];
    partial[((long long)b * nblk + blk) * K + threadIdx.x] = s;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(&counter[b], 1u) == (unsigned)nblk - 1;
  __syncthreads();
  if (!am_last) return false;
  if (threadIdx.x < K) {
    double s = 0;
    for (int q = 0; q < nblk; ++q) s += __ldcg(&partial[((long long)b * nblk + q) * K + threadIdx.x]);
    red[threadIdx.x][0] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = red[k][0];
  if (threadIdx.x == 0) counter[b] = 0;
  return true;
}

__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// per-instance scalar block: sc[4 b + {0, 1, 2, 3}] = rho, rho_old, alpha, omega
enum { SC_RHO = 0, SC_RHO_OLD = 1, SC_ALPHA = 2, SC_OMEGA = 3 };

template <typename R> __device__ __forceinline__ typename Cx<R>::T narrow(double2 z) { return mk((R)z.x, (R)z.y); }

// Thread t of block blk handles EPT consecutive values per tile, tiles blk,
// blk + nblk, ...; Us is a multiple of 64, so a thread's EPT values are all
// in range or all out.
__device__ __forceinline__ long long tiles_of(long long Us, int ept) { return (Us + (long long)BT * ept - 1) / ((long long)BT * ept); }

template <typename R>
__global__ void __launch_bounds__(BT) k_bicg_init(BicgPtrs bp, typename Cx<R>::T *V, long long vinst) {
  using C = typename Cx<R>::T;
  constexpr int EPT = Ept<R>::v;
  const int b = blockIdx.y;
  if (!bp.act[b]) return;
  C *Vb = V + b * vinst;
  double acc[1] = {0};
  for (long long tile = blockIdx.x; tile < tiles_of(bp.Us, EPT); tile += gridDim.x) {
    const long long e0 = tile * BT * EPT + (long long)threadIdx.x * EPT;
    if (e0 >= bp.Us) continue;
    C r[EPT], z[EPT];
    load_ept<C, EPT>(r, Vb + BS_R * bp.Us + e0);
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      z[k] = mk((R)0, (R)0);
      acc[0] += (double)(r[k].x * r[k].x + r[k].y * r[k].y);
    }
    store_ept<C, EPT>(Vb + BS_RH * bp.Us + e0, r);
    store_ept<C, EPT>(Vb + BS_D * bp.Us + e0, z);
  }
  double tot[1];
  if (last_block_sums<1>(acc, bp.partial, bp.counter, b, gridDim.x, blockIdx.x, tot) && threadIdx.x == 0) {
    double2 *sc = bp.sc + 4 * b;
    sc[SC_RHO] = make_double2(tot[0], 0.0);
    sc[SC_RHO_OLD] = sc[SC_ALPHA] = sc[SC_OMEGA] = make_double2(1.0, 0.0);
    bp.rn2[b] = tot[0];
    bp.it[b] = 0;
    if (!(tot[0] > bp.thresh2[b])) bp.act[b] = 0;   // already below the threshold (or zero)
  }
}

template <typename R>
__global__ void __launch_bounds__(BT) k_bicg_p(BicgPtrs bp, typename Cx<R>::T *V, long long vinst) {
  using C = typename Cx<R>::T;
  constexpr int EPT = Ept<R>::v;
  const int b = blockIdx.y;
  if (!bp.act[b]) return;
  C *Vb = V + b * vinst;
  const double2 *sc = bp.sc + 4 * b;
  const bool first = bp.it[b] == 0;
  const double2 beta = first ? make_double2(0.0, 0.0)
                             : zmul(zdiv(sc[SC_RHO], sc[SC_RHO_OLD]), zdiv(sc[SC_ALPHA], sc[SC_OMEGA]));
  const C be = narrow<R>(beta), om = narrow<R>(sc[SC_OMEGA]);
  for (long long tile = blockIdx.x; tile < tiles_of(bp.Us, EPT); tile += gridDim.x) {
    const long long e0 = tile * BT * EPT + (long long)threadIdx.x * EPT;
    if (e0 >= bp.Us) continue;
    C r[EPT], p[EPT], v[EPT];
    load_ept<C, EPT>(r, Vb + BS_R * bp.Us + e0);
    if (!first) {
      load_ept<C, EPT>(p, Vb + BS_P * bp.Us + e0);
      load_ept<C, EPT>(v, Vb + BS_V * bp.Us + e0);
#pragma unroll
      for (int k = 0; k < EPT; ++k) r[k] = cadd(r[k], cmul(be, csub(p[k], cmul(om, v[k]))));
    }
    store_ept<C, EPT>(Vb + BS_P * bp.Us + e0, r);
  }
}

template <typename R>
__global__ void __launch_bounds__(BT) k_bicg_alpha(BicgPtrs bp, const typename Cx<R>::T *V, long long vinst) {
  using C = typename Cx<R>::T;
  constexpr int EPT = Ept<R>::v;
  const int b = blockIdx.y;
  if (!bp.act[b]) return;
  const C *Vb = V + b * vinst;
  double acc[2] = {0, 0};   // <r^, v>
  for (long long tile = blockIdx.x; tile < tiles_of(bp.Us, EPT); tile += gridDim.x) {
    const long long e0 = tile * BT * EPT + (long long)threadIdx.x * EPT;
    if (e0 >= bp.Us) continue;
    C h[EPT], v[EPT];
    load_ept<C, EPT>(h, Vb + BS_RH * bp.Us + e0);
    load_ept<C, EPT>(v, Vb + BS_V * bp.Us + e0);
    R sr = 0, si = 0;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      sr += h[k].x * v[k].x + h[k].y * v[k].y;
      si += h[k].x * v[k].y - h[k].y * v[k].x;
    }
    acc[0] += (double)sr;
    acc[1] += (double)si;
  }
  double tot[2];
  if (last_block_sums<2>(acc, bp.partial, bp.counter, b, gridDim.x, blockIdx.x, tot) && threadIdx.x == 0) {
    double2 *sc = bp.sc + 4 * b;
    const double2 hv = make_double2(tot[0], tot[1]);
    if (hv.x == 0.0 && hv.y == 0.0) bp.act[b] = 0;   // breakdown: keep the correction so far
    else sc[SC_ALPHA] = zdiv(sc[SC_RHO], hv);
  }
}

template <typename R>
__global__ void __launch_bounds__(BT) k_bicg_s(BicgPtrs bp, typename Cx<R>::T *V, long long vinst) {
  using C = typename Cx<R>::T;
  constexpr int EPT = Ept<R>::v;
  const int b = blockIdx.y;
  if (!bp.act[b]) return;
  C *Vb = V + b * vinst;
  const C al = narrow<R>(bp.sc[4 * b + SC_ALPHA]);
  for (long long tile = blockIdx.x; tile < tiles_of(bp.Us, EPT); tile += gridDim.x) {
    const long long e0 = tile * BT * EPT + (long long)threadIdx.x * EPT;
    if (e0 >= bp.Us) continue;
    C r[EPT], v[EPT];
    load_ept<C, EPT>(r, Vb + BS_R * bp.Us + e0);
    load_ept<C, EPT>(v, Vb + BS_V * bp.Us + e0);
#pragma unroll
    for (int k = 0; k < EPT; ++k) r[k] = csub(r[k], cmul(al, v[k]));
    store_ept<C, EPT>(Vb + BS_S * bp.Us + e0, r);
  }
}

template <typename R>
__global__ void __launch_bounds__(BT) k_bicg_omega(BicgPtrs bp, const typename Cx<R>::T *V, long long vinst) {
  using C = typename Cx<R>::T;
  constexpr int EPT = Ept<R>::v;
  const int b = blockIdx.y;
  if (!bp.act[b]) return;
  const C *Vb = V + b * vinst;
  double acc[3] = {0, 0, 0};   // <t, s>, <t, t>
  for (long long tile = blockIdx.x; tile < tiles_of(bp.Us, EPT); tile += gridDim.x) {
    const long long e0 = tile * BT * EPT + (long long)threadIdx.x * EPT;
    if (e0 >= bp.Us) continue;
    C t[EPT], s[EPT];
    load_ept<C, EPT>(t, Vb + BS_T * bp.Us + e0);
    load_ept<C, EPT>(s, Vb + BS_S * bp.Us + e0);
    R sr = 0, si = 0, tt = 0;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      sr += t[k].x * s[k].x + t[k].y * s[k].y;
      si += t[k].x * s[k].y - t[k].y * s[k].x;
      tt += t[k].x * t[k].x + t[k].y * t[k].y;
    }
    acc[0] += (double)sr;
    acc[1] += (double)si;
    acc[2] += (double)tt;
  }
  double tot[3];
  if (last_block_sums<3>(acc, bp.partial, bp.counter, b, gridDim.x, blockIdx.x, tot) && threadIdx.x == 0)
    bp.sc[4 * b + SC_OMEGA] = tot[2] > 0 ? make_double2(tot[0] / tot[2], tot[1] / tot[2]) : make_double2(0.0, 0.0);
}

template <typename R>
__global__ void __launch_bounds__(BT) k_bicg_update(BicgPtrs bp, typename Cx<R>::T *V, long long vinst) {
  using C = typename Cx<R>::T;
  constexpr int EPT = Ept<R>::v;
  const int b = blockIdx.y;
  if (!bp.act[b]) return;
  C *Vb = V + b * vinst;
  const double2 *sc = bp.sc + 4 * b;
  const C al = narrow<R>(sc[SC_ALPHA]), om = narrow<R>(sc[SC_OMEGA]);
  double acc[3] = {0, 0, 0};   // <r^, r>, ||r||^2
  for (long long tile = blockIdx.x; tile < tiles_of(bp.Us, EPT); tile += gridDim.x) {
    const long long e0 = tile * BT * EPT + (long long)threadIdx.x * EPT;
    if (e0 >= bp.Us) continue;
    C d[EPT], p[EPT], s[EPT], t[EPT], h[EPT];
    load_ept<C, EPT>(d, Vb + BS_D * bp.Us + e0);
    load_ept<C, EPT>(p, Vb + BS_P * bp.Us + e0);
    load_ept<C, EPT>(s, Vb + BS_S * bp.Us + e0);
    load_ept<C, EPT>(t, Vb + BS_T * bp.Us + e0);
    load_ept<C, EPT>(h, Vb + BS_RH * bp.Us + e0);
    R sr = 0, si = 0, rr = 0;
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      d[k] = cadd(d[k], cadd(cmul(al, p[k]), cmul(om, s[k])));
      const C r = csub(s[k], cmul(om, t[k]));
      s[k] = r;
      sr += h[k].x * r.x + h[k].y * r.y;
      si += h[k].x * r.y - h[k].y * r.x;
      rr += r.x * r.x + r.y * r.y;
    }
    store_ept<C, EPT>(Vb + BS_D * bp.Us + e0, d);
    store_ept<C, EPT>(Vb + BS_R * bp.Us + e0, s);
    acc[0] += (double)sr;
    acc[1] += (double)si;
    acc[2] += (double)rr;
  }
  double tot[3];
  if (last_block_sums<3>(acc, bp.partial, bp.counter, b, gridDim.x, blockIdx.x, tot) && threadIdx.x == 0) {
    double2 *scw = bp.sc + 4 * b;
    const double2 om2 = scw[SC_OMEGA];
    scw[SC_RHO_OLD] = scw[SC_RHO];
    scw[SC_RHO] = make_double2(tot[0], tot[1]);
    bp.rn2[b] = tot[2];
    const int it = bp.it[b] + 1;
    bp.it[b] = it;
    if (tot[2] <= bp.thresh2[b] || it >= bp.max_it || (tot[0] == 0.0 && tot[1] == 0.0) ||
        (om2.x == 0.0 && om2.y == 0.0))
      bp.act[b] = 0;
  }
}

// x += d (x in FP64, the correction in the working precision)
template <typename R>
__global__ void __launch_bounds__(BT) k_bicg_sol(double2 *__restrict__ x64, long long xinst,
                                                 const typename Cx<R>::T *__restrict__ V, long long vinst, long long U,
                                                 long long Us, const int *__restrict__ need, double *partial,
                                                 unsigned *counter, double *dnorm2) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  if (!need[b]) return;
  const typename Cx<R>::T *d = V + b * vinst + BS_D * Us;
  double2 *xb = x64 + b * xinst;
  double acc = 0;   // ||d||^2: bounds the rounding error of a later r -= A d
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < U; e += (long long)gridDim.x * blockDim.x) {
    const double2 x = xb[e];
    const double dx = (double)d[e].x, dy = (double)d[e].y;
    xb[e] = make_double2(x.x + dx, x.y + dy);
    acc += dx * dx + dy * dy;
  }
  last_block_sum(acc, red, partial, counter, dnorm2, b, gridDim.x, blockIdx.x);
}

// WHILE condition of the captured iteration loop: any instance still active
__global__ void k_bicg_advance(const int *__restrict__ act, int B, cudaGraphConditionalHandle h) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x)
    if (act[b]) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

}  // namespace

template <typename R>
cudaError_t launch_bicg_step(int which, const BicgPtrs &bp, typename Cx<R>::T *V, long long vinst, cudaStream_t st) {
  dim3 grid(bp.nblk, bp.B);
  switch (which) {
    case BICG_INIT: k_bicg_init<R><<<grid, BT, 0, st>>>(bp, V, vinst); break;
    case BICG_P: k_bicg_p<R><<<grid, BT, 0, st>>>(bp, V, vinst); break;
    case BICG_ALPHA: k_bicg_alpha<R><<<grid, BT, 0, st>>>(bp, V, vinst); break;
    case BICG_S: k_bicg_s<R><<<grid, BT, 0, st>>>(bp, V, vinst); break;
    case BICG_OMEGA: k_bicg_omega<R><<<grid, BT, 0, st>>>(bp, V, vinst); break;
    case BICG_UPDATE: k_bicg_update<R><<<grid, BT, 0, st>>>(bp, V, vinst); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_bicg_sol(double2 *x64, long long xinst, const typename Cx<R>::T *V, long long vinst,
                            const BicgPtrs &bp, const int *need, cudaStream_t st) {
  dim3 grid(bp.nblk, bp.B);
  k_bicg_sol<R><<<grid, BT, 0, st>>>(x64, xinst, V, vinst, bp.U, bp.Us, need, bp.dpartial, bp.dcounter, bp.dnorm2);
  return cudaGetLastError();
}

cudaError_t launch_bicg_advance(const BicgPtrs &bp, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_bicg_advance<<<1, 256, 0, st>>>(bp.act, bp.B, h);
  return cudaGetLastError();
}

template cudaError_t launch_bicg_step<float>(int, const BicgPtrs &, float2 *, long long, cudaStream_t);
template cudaError_t launch_bicg_step<double>(int, const BicgPtrs &, double2 *, long long, cudaStream_t);
template cudaError_t launch_bicg_sol<float>(double2 *, long long, const float2 *, long long, const BicgPtrs &,
                                            const int *, cudaStream_t);
template cudaError_t launch_bicg_sol<double>(double2 *, long long, const double2 *, long long, const BicgPtrs &,
                                             const int *, cudaStream_t);

}  // namespace gsm
