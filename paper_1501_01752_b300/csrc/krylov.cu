// Batched GMRES kernels ("Calculation details": GMRES in Saad's form).
//
// Each instance b of a batch owns a Krylov basis V[b][0..m] of U complex
// values per vector.  One Arnoldi step j, after the matrix-vector product
// w = A v_j has been written to V[b][j+1], is
//
//   k_dots(0)    h   = V_j^H w, ||w||^2       (one pass over v_0..v_j and w)
//   k_update(0)  w  -= V_j h, ||w||^2         (one pass; decides reorthogonalisation)
//   k_dots(1)    h'  = V_j^H w                (only if ||w_new|| < ||w_old|| / sqrt 2)
//   k_update(1)  w  -= V_j h'
//   k_finish     column j of H, Givens rotations, residual estimate |g_{j+1}|
//
// i.e. classical Gram-Schmidt with the Daniel-Gragg-Kaufman-Stewart
// reorthogonalisation test instead of the paper's modified Gram-Schmidt: the
// j sequential dot/axpy pairs of MGS become two fused passes (four when the
// test fires), with orthogonality at least as good as MGS.  The test can be
// forced on or off per solve (force 1 / 2), or replaced by a second pass at
// every 2^(force - 2)-th step (force >= 3; a power of two, so that the test
// costs the kernel no registers): complex64 inner solves of Eq. 4, which
// stop at 1e-4 relative, skip the second pass.  Dots of FP32 vectors sum
// FP32 products in each thread's registers and across a warp, and the warp
// sums in FP64; Hessenberg, rotations and residual estimates are FP64.
// Reductions across blocks use the last-block-done pattern (atomic counter,
// no waiting).
#include "kernels.h"
#include "reduce.cuh"
#include "vec.cuh"

namespace gsm {

constexpr int MAXM = 128;

// h_i = <v_i, w> for i < nv and ||w||^2: w is held in registers per tile,
// every basis vector streamed once.  Each block takes a group of GV basis
// vectors over a strided set of tiles; every thread accumulates its products
// in registers (basis precision) over all of its tiles, and the block reduces
// once at the end (warp tree, then FP64 across warps and blocks).
constexpr int GV = 8;  // basis vectors per block of k_dots (grid.x = tile blocks x vector groups)
// values per thread and vector in k_dots: 32 bytes, so that four vectors in
// flight fit in few registers
template <typename R> struct EptDots { static constexpr int v = sizeof(R) == 4 ? 4 : 2; };

template <typename R>
__global__ void __launch_bounds__(KT) k_dots(const typename Cx<R>::T *__restrict__ V, long long vinst, long long Us,
                                             int nv, int wi, const int *__restrict__ act,
                                             const int *__restrict__ gate, double *partial, unsigned *counter,
                                             double *out, int ostride, int nblk, const int *__restrict__ jdev,
                                             const int *__restrict__ alist, int bcap,
                                             const double *__restrict__ svec, int sstride,
                                             const long long *__restrict__ ulen) {
  using C = typename Cx<R>::T;
  constexpr int EPT = EptDots<R>::v, NW = KT / 32, CH = 4, NA = 2 * GV + 1;
  __shared__ double wsum[NA][NW];
  __shared__ int am_last;
  // the active instances share the grid's blocks: slot a = blockIdx.x / nblk
  const int nact = alist[0];
  if (nact == 0) return;
  nblk = min(bcap, max(nblk, (int)(gridDim.x / nact)));
  const int a = blockIdx.x / nblk, blk = blockIdx.x % nblk, grp = blockIdx.y;
  if (a >= nact) return;
  const int b = alist[1 + a];
  (void)act;
  if (gate && !gate[b]) return;
  if (jdev) {                        // graph mode: the step comes from the device counter
    nv = *jdev + 1;
    wi = nv;
  }
  const int K = 2 * nv + 1, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = grp * GV, i1 = min(nv, i0 + GV), ng = max(0, i1 - i0);   // groups past nv only count in
  const C *Vb = V + b * vinst;
  const C *W = Vb + (long long)wi * Us;
  const C *V0 = Vb + (long long)i0 * Us;
  const long long Ub = ulen ? ulen[b] : Us;   // this instance's stored length (vectors stay Us apart)
  const long long ntiles = (Ub + KT * EPT - 1) / (KT * EPT);
  R acc[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) acc[k] = 0;
  for (long long t = blk; ng > 0 && t < ntiles; t += nblk) {
    const long long e0 = t * (KT * EPT) + (long long)threadIdx.x * EPT;
    if (e0 >= Ub) continue;          // Ub is a multiple of 64: a thread's EPT values are all in range
    C w[EPT];
    load_ept<C, EPT>(w, W + e0);
    if (grp == 0)
#pragma unroll
      for (int k = 0; k < EPT; ++k) acc[2 * GV] += w[k].x * w[k].x + w[k].y * w[k].y;
#pragma unroll
    for (int c0 = 0; c0 < GV; c0 += CH) {
      if (c0 < ng) {
        C v[CH][EPT];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          if (c0 + u < ng) load_ept<C, EPT>(v[u], V0 + (long long)(c0 + u) * Us + e0);
          else
#pragma unroll
            for (int k = 0; k < EPT; ++k) v[u][k] = mk((R)0, (R)0);
        }
#pragma unroll
        for (int u = 0; u < CH; ++u)
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            acc[2 * (c0 + u)] += v[u][k].x * w[k].x + v[u][k].y * w[k].y;       // conj(v) w
            acc[2 * (c0 + u) + 1] += v[u][k].x * w[k].y - v[u][k].y * w[k].x;
          }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NA; ++k) {
    const R sk = warp_sum(acc[k]);
    if (lane == 0) wsum[k][warp] = (double)sk;
  }
  __syncthreads();
  // this block's share: dots i0..i1-1 (and ||w||^2 from group 0).  The
  // partials of one value lie together ([instance][value][block]), so that
  // the last block reads each value's partials with coalesced loads.
  double *pb = partial + (long long)a * nblk * ostride + blk;
  for (int k = threadIdx.x; k < 2 * ng + (grp == 0); k += blockDim.x) {
    const int src = k < 2 * ng ? k : 2 * GV;
    double s = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) s += wsum[src][q];
    pb[(long long)(k < 2 * ng ? 2 * i0 + k : 2 * nv) * nblk] = s;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(&counter[b], 1u);
    am_last = (t == (unsigned)(nblk * gridDim.y) - 1);
  }
  __syncthreads();
  if (!am_last) return;
  const double *pin = partial + (long long)a * nblk * ostride;
  if (nblk <= 16) {
    // few blocks per instance (large batches): one thread per value
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      const double *pk = pin + (long long)k * nblk;
      double s = 0;
      for (int q = 0; q < nblk; ++q) s += __ldcg(pk + q);
      if (svec && k < 2 * nv) s *= svec[(long long)b * sstride + (k >> 1)];   // <v_i, w> = s_i <V_i, w>
      out[(long long)b * ostride + k] = s;
    }
  } else {
    // hundreds of blocks per instance (small batches): one warp per value,
    // the lanes across the partials (lane-strided sums, then the shuffle
    // tree; a fixed order either way)
    for (int k = warp; k < K; k += NW) {
      const double *pk = pin + (long long)k * nblk;
      double s = 0;
      for (int q = lane; q < nblk; q += 32) s += __ldcg(pk + q);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (svec && k < 2 * nv) s *= svec[(long long)b * sstride + (k >> 1)];
      if (lane == 0) out[(long long)b * ostride + k] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) counter[b] = 0;
}

// w -= sum_i h_i v_i over the tile held in registers, and ||w||^2.
template <typename R>
__global__ void __launch_bounds__(KT) k_update(typename Cx<R>::T *__restrict__ V, long long vinst, long long Us,
                                               int nv, int wi, const double *__restrict__ h, int hstride,
                                               const int *__restrict__ act, const int *__restrict__ gate,
                                               double *partial, unsigned *counter, double *wn_out,
                                               int *gate_out, int force, const int *__restrict__ jdev,
                                               const int *__restrict__ alist, int nblk, int bcap,
                                               const double *__restrict__ svec, int sstride,
                                               const long long *__restrict__ ulen) {
  using C = typename Cx<R>::T;
  constexpr int EPT = Ept<R>::v;
  if (jdev) {
    nv = *jdev + 1;
    wi = nv;
  }
  __shared__ C hs[MAXM + 1];
  __shared__ double red[32];
  // the active instances share the grid's blocks, as in k_dots
  const int nact = alist[0];
  if (nact == 0) return;
  nblk = min(bcap, max(nblk, (int)(gridDim.x / nact)));
  const int a = blockIdx.x / nblk, blk = blockIdx.x % nblk;
  if (a >= nact) return;
  const int b = alist[1 + a];
  (void)act;
  if (gate && !gate[b]) return;
  // the coefficient of the stored (unnormalised) V_i is h_i s_i
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const double si = svec ? svec[(long long)b * sstride + i] : 1.0;
    hs[i] = mk((R)(h[(long long)b * hstride + 2 * i] * si), (R)(h[(long long)b * hstride + 2 * i + 1] * si));
  }
  __syncthreads();
  C *Vb = V + b * vinst;
  C *W = Vb + (long long)wi * Us;
  const long long Ub = ulen ? ulen[b] : Us;
  const long long ntiles = (Ub + KT * EPT - 1) / (KT * EPT);
  double acc = 0;
  for (long long t = blk; t < ntiles; t += nblk) {
    const long long e0 = t * (KT * EPT) + (long long)threadIdx.x * EPT;
    if (e0 >= Ub) continue;
    C w[EPT];
    load_ept<C, EPT>(w, W + e0);
    int i = 0;
    for (; i + 4 <= nv; i += 4) {
      C v[4][EPT];
#pragma unroll
      for (int u = 0; u < 4; ++u) load_ept<C, EPT>(v[u], Vb + (long long)(i + u) * Us + e0);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const C hi = hs[i + u];
#pragma unroll
        for (int k = 0; k < EPT; ++k) w[k] = csub(w[k], cmul(hi, v[u][k]));
      }
    }
    for (; i < nv; ++i) {
      C v[EPT];
      load_ept<C, EPT>(v, Vb + (long long)i * Us + e0);
      const C hi = hs[i];
#pragma unroll
      for (int k = 0; k < EPT; ++k) w[k] = csub(w[k], cmul(hi, v[k]));
    }
    store_ept<C, EPT>(W + e0, w);
    R n2 = 0;
#pragma unroll
    for (int k = 0; k < EPT; ++k) n2 += w[k].x * w[k].x + w[k].y * w[k].y;
    acc += (double)n2;
  }
  if (last_block_sum(acc, red, partial + (long long)a * nblk, counter + b, wn_out + b, 0, nblk, blk)) {
    if (gate_out && threadIdx.x == 0) {
      const double before = h[(long long)b * hstride + 2 * nv];
      gate_out[b] = (force == 1 || (force == 0 && wn_out[b] < 0.5 * before) ||
                     (force >= 3 && (nv & ((1 << (force - 2)) - 1)) == 0)) ? 1 : 0;
    }
  }
}

// Column j of the Hessenberg matrix, Givens rotations, residual estimate
// (Saad's GMRES with complex rotations).  One warp per instance: the lanes
// fetch the column and the earlier rotations into shared memory in
// parallel, lane 0 applies the rotations in order, and the lanes write the
// rotated column back.
constexpr int FIN_W = 4;  // instances (warps) per block of k_finish
__global__ void __launch_bounds__(32 * FIN_W) k_finish(KrylovPtrs k, int j) {
  __shared__ double2 col_s[FIN_W][MAXM + 1];
  __shared__ double cs_s[FIN_W][MAXM];
  __shared__ double2 sn_s[FIN_W][MAXM];
  if (k.jdev) j = *k.jdev;
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * FIN_W + wi;
  if (b >= k.B || !k.act[b]) return;   // uniform over the warp
  const int m = k.m, hs = 2 * (m + 1) + 1;
  const bool re = k.gate[b] != 0;
  const double *h0 = k.hdot0 + (long long)b * hs, *h1 = k.hdot1 + (long long)b * hs;
  double *cs = k.cs + (long long)b * m;
  double2 *sn = k.sn + (long long)b * m;
  double2 *col = col_s[wi];
  for (int i = lane; i <= j; i += 32)
    col[i] = mk(h0[2 * i] + (re ? h1[2 * i] : 0.0), h0[2 * i + 1] + (re ? h1[2 * i + 1] : 0.0));
  for (int i = lane; i < j; i += 32) {
    cs_s[wi][i] = cs[i];
    sn_s[wi][i] = sn[i];
  }
  __syncwarp();
  if (lane == 0) {
    const double hn = sqrt(fmax(re ? k.wn1[b] : k.wn0[b], 0.0));
    double2 *g = k.gv + (long long)b * (m + 1);
    double2 a = col[0];
    for (int i = 0; i < j; ++i) {
      const double2 c2 = col[i + 1];
      const double c = cs_s[wi][i];
      const double2 s = sn_s[wi][i];
      col[i] = mk(c * a.x + s.x * c2.x - s.y * c2.y, c * a.y + s.x * c2.y + s.y * c2.x);
      // -conj(s) a + c c2
      a = mk(-(s.x * a.x + s.y * a.y) + c * c2.x, -(s.x * a.y - s.y * a.x) + c * c2.y);
    }
    const double na = hypot(a.x, a.y);
    const double rho = hypot(na, hn);
    double c;
    double2 s;
    if (na == 0.0) {
      c = 0.0;
      s = mk(1.0, 0.0);
    } else {
      c = na / rho;
      s = mk(a.x / na * hn / rho, a.y / na * hn / rho);
    }
    col[j] = mk(c * a.x + s.x * hn, c * a.y + s.y * hn);
    const double2 gj = g[j];
    g[j + 1] = mk(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    g[j] = mk(c * gj.x, c * gj.y);
    cs[j] = c;
    sn[j] = s;
    k.kcount[b] = j + 1;
    k.scale32[b] = hn > 0 ? (float)(1.0 / hn) : 0.f;
    k.scale64[b] = hn > 0 ? 1.0 / hn : 0.0;
    k.svec[(long long)b * (m + 1) + j + 1] = hn > 0 ? 1.0 / hn : 0.0;
    const double r = hypot(g[j + 1].x, g[j + 1].y);
    k.resid[b] = r;
    if (r <= k.thresh[b] || hn == 0.0 || j + 1 >= m) k.act[b] = 0;
  }
  __syncwarp();
  double2 *Hc = k.H + ((long long)b * m + j) * (m + 1);
  for (int i = lane; i <= j; i += 32) Hc[i] = col[i];
}

// y = R^-1 g over the kcount[b] rotated columns (back substitution).  One
// block per instance: all threads stage the upper triangle (column l at
// l (l + 1) / 2) in shared memory, then warp 0 substitutes column by
// column, every lane updating its rows of the right-hand side.
constexpr int BSOLVE_T = 256;
__global__ void __launch_bounds__(BSOLVE_T) k_backsolve(KrylovPtrs k) {
  extern __shared__ __align__(16) unsigned char bs_dyn[];
  double2 *Rs = reinterpret_cast<double2 *>(bs_dyn);   // m (m + 1) / 2 entries
  __shared__ double2 s_s[MAXM];
  const int b = blockIdx.x;
  const int m = k.m, n = k.kcount[b];
  const double2 *Hb = k.H + (long long)b * m * (m + 1);
  const long long tri = (long long)n * (n + 1) / 2;
  for (long long e = threadIdx.x; e < tri; e += blockDim.x) {
    // column l holds rows 0..l: e = l (l + 1) / 2 + i
    int l = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
    while ((long long)l * (l + 1) / 2 > e) --l;
    while ((long long)(l + 1) * (l + 2) / 2 <= e) ++l;
    const int i = (int)(e - (long long)l * (l + 1) / 2);
    Rs[e] = Hb[(long long)l * (m + 1) + i];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) s_s[i] = k.gv[(long long)b * (m + 1) + i];
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double2 *y = k.y + (long long)b * m;
  for (int l = n - 1; l >= 0; --l) {
    const double2 d = Rs[(long long)l * (l + 1) / 2 + l];
    const double dd = d.x * d.x + d.y * d.y;
    const double2 s = s_s[l];
    const double2 yl = dd > 0 ? mk((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd) : mk(0.0, 0.0);
    if (lane == 0) y[l] = yl;
    const double2 *Rc = Rs + (long long)l * (l + 1) / 2;
    for (int i = lane; i < l; i += 32) s_s[i] = csub(s_s[i], cmul(Rc[i], yl));
    __syncwarp();
  }
}

// x += V y (FP64 x; the combination in the basis precision).
template <typename R>
__global__ void __launch_bounds__(KT) k_sol_update(double2 *__restrict__ x64, long long xinst,
                                                   typename Cx<R>::T *__restrict__ V, long long vinst,
                                                   long long U, long long Us, const double2 *__restrict__ y, int m,
                                                   const int *__restrict__ kcount, const int *__restrict__ need,
                                                   int dslot, const double *__restrict__ svec, double *partial,
                                                   unsigned *counter, double *dnorm2) {
  using C = typename Cx<R>::T;
  __shared__ C ys[MAXM];
  __shared__ double red[32];
  const int b = blockIdx.y;
  if (!need[b]) return;
  const int n = kcount[b];
  if (n == 0) return;
  // V y over the normalised basis = sum_i (y_i s_i) V_i over the stored one
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double si = svec[(long long)b * (m + 1) + i];
    ys[i] = mk((R)(y[(long long)b * m + i].x * si), (R)(y[(long long)b * m + i].y * si));
  }
  __syncthreads();
  C *Vb = V + b * vinst;
  double2 *xb = x64 + b * xinst;
  C *dv = dslot >= 0 ? Vb + (long long)dslot * Us : nullptr;   // keeps the correction d for r -= A d
  // ||d||^2: bounds the rounding error of a later r -= A d (a few digits
  // suffice: summed in the basis precision per thread, FP64 across threads)
  R acc = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < U; e += (long long)gridDim.x * blockDim.x) {
    const double2 xv = xb[e];   // fetched first: its load overlaps the basis loads
    C d = mk((R)0, (R)0);
#pragma unroll 4
    for (int i = 0; i < n; ++i) d = cadd(d, cmul(ys[i], Vb[(long long)i * Us + e]));
    xb[e] = mk(xv.x + (double)d.x, xv.y + (double)d.y);
    if (dv) dv[e] = d;
    acc += d.x * d.x + d.y * d.y;
  }
  last_block_sum((double)acc, red, partial, counter, dnorm2, b, gridDim.x, blockIdx.x);
}

// Right-preconditioned Krylov cycles solve A M^{-1} u = r, so the
// correction is M^{-1} u.  One thread per harmonic forms the three
// components of u = V y (GMRES, src < 0; kept in slot dslot for
// r -= (A M^{-1}) u when dslot >= 0) or reads them from slot src (BiCGSTAB's
// accumulated iterate), maps them by M^{-1} = alpha P_T + beta P_L with the
// same arithmetic as the product's pass 1, and adds the result to the FP64 x.
template <typename R>
__global__ void __launch_bounds__(KT) k_sol_update_pc(Geo g, const Inst *__restrict__ inst, const R *__restrict__ iden,
                                                      double2 *__restrict__ x64, long long xinst,
                                                      typename Cx<R>::T *__restrict__ V, long long vinst, long long Us,
                                                      const double2 *__restrict__ y, int m,
                                                      const int *__restrict__ kcount, const int *__restrict__ need,
                                                      int dslot, int src, const double *__restrict__ svec,
                                                      double *partial, unsigned *counter, double *dnorm2) {
  using C = typename Cx<R>::T;
  __shared__ C ys[MAXM];
  __shared__ double red[32];
  const int b = blockIdx.y;
  if (!need[b]) return;
  const int n = src >= 0 ? 1 : kcount[b];
  if (n == 0) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double si = src >= 0 ? 1.0 : svec[(long long)b * (m + 1) + i];   // GMRES: unnormalised basis
    ys[i] = src >= 0 ? mk((R)1, (R)0) : mk((R)(y[(long long)b * m + i].x * si), (R)(y[(long long)b * m + i].y * si));
  }
  __syncthreads();
  C *Vb = V + b * vinst;
  double2 *xb = x64 + b * xinst;
  C *dv = dslot >= 0 ? Vb + (long long)dslot * Us : nullptr;
  const C *V0 = Vb + (src >= 0 ? (long long)src * Us : 0);
  const long long Nh = g.Nh;
  const R pcc = (R)inst[b].pc_c, pcb = (R)inst[b].pc_beta;
  // ||M^{-1} u||^2, the correction added to x: summed in FP32 per thread (it
  // bounds the rounding of recursive residual updates, with a factor 10 to
  // spare) and in FP64 across threads
  float acc = 0.f;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < Nh; e += (long long)gridDim.x * blockDim.x) {
    double2 xv[3];   // the iterate, fetched before the basis so that its loads overlap theirs
#pragma unroll
    for (int c = 0; c < 3; ++c) xv[c] = xb[c * Nh + e];
    C d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) d[c] = mk((R)0, (R)0);
    int i = 0;
    for (; i + 4 <= n; i += 4) {       // twelve independent loads in flight
      C vv[4][3];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) vv[u][c] = V0[(long long)(i + u) * Us + c * Nh + e];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) d[c] = cadd(d[c], cmul(ys[i + u], vv[u][c]));
    }
    for (; i < n; ++i) {
      const C *Vi = V0 + (long long)i * Us + e;
#pragma unroll
      for (int c = 0; c < 3; ++c) d[c] = cadd(d[c], cmul(ys[i], Vi[c * Nh]));
    }
    if (dv)
#pragma unroll
      for (int c = 0; c < 3; ++c) dv[c * Nh + e] = d[c];
    const int ei = (int)e;   // Nh < 2^31
    const int row = ei / g.N[0], mx = ei - row * g.N[0];
    const int mz = row / g.N[1], my = row - mz * g.N[1];
    const R kx = (R)(inst[b].kinc[0] + (mx - g.n[0]) * g.K[0]);
    const R ky = (R)(inst[b].kinc[1] + (my - g.n[1]) * g.K[1]);
    const R kz = (R)(inst[b].kinc[2] + (mz - g.n[2]) * g.K[2]);
    const R al = rcp((R)1 - pcc * iden[(long long)b * g.ist + e]);
    const R k2 = kx * kx + ky * ky + kz * kz;
    const R f = k2 > (R)0 ? (pcb - al) * rcp(k2) : (R)0;
    const R kr = kx * d[0].x + ky * d[1].x + kz * d[2].x, ki = kx * d[0].y + ky * d[1].y + kz * d[2].y;
    const R kc[3] = {kx, ky, kz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R cx = al * d[c].x + f * kc[c] * kr, cy = al * d[c].y + f * kc[c] * ki;
      xb[c * Nh + e] = mk(xv[c].x + (double)cx, xv[c].y + (double)cy);
      acc += (float)(cx * cx + cy * cy);
    }
  }
  last_block_sum((double)acc, red, partial, counter, dnorm2, b, gridDim.x, blockIdx.x);
}

// r -= A d with A d from the complex64 product, and ||r||^2 (last block).
__global__ void __launch_bounds__(KT) k_resid_sub(double2 *__restrict__ r64, long long rinst,
                                                  const float2 *__restrict__ Ad, long long ainst, long long U,
                                                  const int *__restrict__ need, double *partial, unsigned *counter,
                                                  double *norm_out) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  if (!need[b]) return;
  double2 *rb = r64 + b * rinst;
  const float2 *ab = Ad + b * ainst;
  double acc = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < U; e += (long long)gridDim.x * blockDim.x) {
    const float2 a = ab[e];
    double2 r = rb[e];
    r.x -= (double)a.x;
    r.y -= (double)a.y;
    rb[e] = r;
    acc += r.x * r.x + r.y * r.y;
  }
  last_block_sum(acc, red, partial, counter, norm_out, b, gridDim.x, blockIdx.x);
}

cudaError_t launch_resid_sub(double2 *r64, long long rinst, const float2 *Ad, long long ainst, long long U, int B,
                             int nblk, const int *need, double *partial, unsigned *counter, double *norm_out,
                             cudaStream_t st) {
  dim3 grid(nblk, B);
  k_resid_sub<<<grid, KT, 0, st>>>(r64, rinst, Ad, ainst, U, need, partial, counter, norm_out);
  return cudaGetLastError();
}

// V_b[0] = r_b in the basis precision, for every instance that starts a cycle
template <typename C>
__global__ void __launch_bounds__(KT) k_start_basis(const double2 *__restrict__ r64, long long rinst, C *__restrict__ V,
                                                    long long vinst, long long U, const int *__restrict__ need) {
  const int b = blockIdx.y;
  if (!need[b]) return;
  const double2 *rb = r64 + b * rinst;
  C *vb = V + b * vinst;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < U; e += (long long)gridDim.x * blockDim.x) {
    const double2 r = rb[e];
    vb[e] = mk((decltype(vb[0].x))r.x, (decltype(vb[0].x))r.y);
  }
}

template <typename C>
cudaError_t launch_start_basis(const double2 *r64, long long rinst, C *V, long long vinst, long long U, int B,
                               int nblk, const int *need, cudaStream_t st) {
  dim3 grid(nblk, B);
  k_start_basis<C><<<grid, KT, 0, st>>>(r64, rinst, V, vinst, U, need);
  return cudaGetLastError();
}
template cudaError_t launch_start_basis<float2>(const double2 *, long long, float2 *, long long, long long, int, int,
                                                const int *, cudaStream_t);
template cudaError_t launch_start_basis<double2>(const double2 *, long long, double2 *, long long, long long, int, int,
                                                 const int *, cudaStream_t);

// zero the padding (U..Us) of every stored Krylov vector
template <typename C>
__global__ void k_zero_pads(C *V, long long nvec, long long U, long long Us) {
  const long long pad = Us - U, tot = nvec * pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long v = e / pad;
    V[v * Us + U + (e - v * pad)] = mk((decltype(V[0].x))0, (decltype(V[0].x))0);
  }
}

template <typename C>
cudaError_t launch_zero_pads(C *V, long long nvec, long long U, long long Us, cudaStream_t st) {
  if (Us == U || nvec == 0) return cudaSuccess;
  const long long tot = nvec * (Us - U);
  k_zero_pads<<<(int)std::min<long long>((tot + 255) / 256, 1184), 256, 0, st>>>(V, nvec, U, Us);
  return cudaGetLastError();
}
template cudaError_t launch_zero_pads<float2>(float2 *, long long, long long, long long, cudaStream_t);
template cudaError_t launch_zero_pads<double2>(double2 *, long long, long long, long long, cudaStream_t);

__global__ void k_set_rhs(double2 *r64, long long xinst, Geo g, const Inst *inst, int B) {
  const long long tot = (long long)B * g.U;
  const long long h0 = ((long long)g.n[2] * g.N[1] + g.n[1]) * g.N[0] + g.n[0];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / g.U);
    const long long r = e - (long long)b * g.U;
    const int c = (int)(r / g.Nh);
    const long long h = r - (long long)c * g.Nh;
    r64[b * xinst + r] = h == h0 ? mk(inst[b].a[2 * c], inst[b].a[2 * c + 1]) : mk(0.0, 0.0);
  }
}

__global__ void k_extract_e0(const double2 *x64, long long xinst, Geo g, int B, double2 *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * B) return;
  const int b = t / 3, c = t % 3;
  const long long h0 = ((long long)g.n[2] * g.N[1] + g.n[1]) * g.N[0] + g.n[0];
  out[t] = x64[b * xinst + c * g.Nh + h0];
}

// The active instances in increasing order: alist[0] = count, alist[1 + a]
// = index of the a-th active instance.  One block, chunks of its width.
__global__ void k_active_list(const int *__restrict__ act, int B, int *alist) {
  __shared__ int wc[32];
  __shared__ int base;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < B; c0 += blockDim.x) {
    const int b = c0 + threadIdx.x;
    const bool on = b < B && act[b] != 0;
    const unsigned msk = __ballot_sync(0xffffffffu, on);
    if (lane == 0) wc[w] = __popc(msk);
    __syncthreads();
    int off = base;
    for (int q = 0; q < w; ++q) off += wc[q];
    if (on) alist[1 + off + __popc(msk & ((1u << lane) - 1u))] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int q = 0; q < nw; ++q) t += wc[q];
      base += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) alist[0] = base;
}

// ------------------------------------------------------------ launchers
template <typename R>
cudaError_t launch_arnoldi_ortho(const KrylovPtrs &k, typename Cx<R>::T *V, long long vinst, int j, cudaStream_t st,
                                 Profiler *prof) {
  const int nv = j + 1, wi = j + 1, hs = 2 * (k.m + 1) + 1;
  // nblk * B blocks, spread over the instances still iterating (at least
  // nblk each, at most bcap): a step where few instances remain streams
  // their basis with as many blocks as a full batch
  k_active_list<<<1, 1024, 0, st>>>(k.act, k.B, k.alist);
  dim3 grid(k.nblk * k.B);
  // graph mode sizes the dots grid for the longest basis; blocks past the
  // current step only take part in the completion count
  const int ngroups = k.jdev ? (k.m + GV - 1) / GV : (nv + GV - 1) / GV;
  dim3 gdots(k.nblk * k.B, ngroups);
  // logical bytes per vector over the instances still iterating
  const double vb = (double)sizeof(typename Cx<R>::T) * k.U * (k.nact > 0 ? k.nact : k.B);
  if (prof) prof->begin(KIND_DOTS, st);
  k_dots<R><<<gdots, KT, 0, st>>>(V, vinst, k.Us, nv, wi, k.act, nullptr, k.partial, k.counter, k.hdot0, hs, k.nblk, k.jdev,
                                    k.alist, k.bcap, k.svec, k.m + 1, k.ulen);
  if (prof) prof->end(KIND_DOTS, st, vb * (nv + 1));
  if (prof) prof->begin(KIND_UPDATE, st);
  k_update<R><<<grid, KT, 0, st>>>(V, vinst, k.Us, nv, wi, k.hdot0, hs, k.act, nullptr, k.partial, k.counter, k.wn0,
                                   k.gate, k.force_reorth, k.jdev, k.alist, k.nblk, k.bcap, k.svec, k.m + 1, k.ulen);
  if (prof) prof->end(KIND_UPDATE, st, vb * (nv + 2));
  if (k.force_reorth == 2) return cudaGetLastError();   // no second pass: gate was cleared
  if (prof) prof->begin(KIND_DOTS, st);
  k_dots<R><<<gdots, KT, 0, st>>>(V, vinst, k.Us, nv, wi, k.act, k.gate, k.partial, k.counter, k.hdot1, hs, k.nblk, k.jdev,
                                    k.alist, k.bcap, k.svec, k.m + 1, k.ulen);
  if (prof) prof->end(KIND_DOTS, st, vb * (nv + 1));
  if (prof) prof->begin(KIND_UPDATE, st);
  k_update<R><<<grid, KT, 0, st>>>(V, vinst, k.Us, nv, wi, k.hdot1, hs, k.act, k.gate, k.partial, k.counter, k.wn1,
                                   nullptr, 0, k.jdev, k.alist, k.nblk, k.bcap, k.svec, k.m + 1, k.ulen);
  if (prof) prof->end(KIND_UPDATE, st, vb * (nv + 2));
  return cudaGetLastError();
}

cudaError_t launch_finish(const KrylovPtrs &k, int j, cudaStream_t st) {
  k_finish<<<(k.B + FIN_W - 1) / FIN_W, 32 * FIN_W, 0, st>>>(k, j);
  return cudaGetLastError();
}

// j += 1; the WHILE node goes on while some instance is active and j < m
__global__ void k_advance(int *jdev, const int *__restrict__ act, int B, int m, cudaGraphConditionalHandle h) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x)
    if (act[b]) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int j = *jdev + 1;
    *jdev = j;
    cudaGraphSetConditional(h, (any && j < m) ? 1u : 0u);
  }
}

cudaError_t launch_advance(const KrylovPtrs &k, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_advance<<<1, 256, 0, st>>>(k.jdev, k.act, k.B, k.m, h);
  return cudaGetLastError();
}

cudaError_t launch_backsolve(const KrylovPtrs &k, cudaStream_t st) {
  const size_t smem = sizeof(double2) * (size_t)k.m * (k.m + 1) / 2;
  cudaFuncSetAttribute(k_backsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_backsolve<<<k.B, BSOLVE_T, smem, st>>>(k);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sol_update(const KrylovPtrs &k, double2 *x64, long long xinst, typename Cx<R>::T *V,
                              long long vinst, const int *need, int dslot, cudaStream_t st, Profiler *prof) {
  dim3 grid(k.nblk, k.B);
  if (prof) prof->begin(KIND_OTHER, st);
  k_sol_update<R><<<grid, KT, 0, st>>>(x64, xinst, V, vinst, k.U, k.Us, k.y, k.m, k.kcount, need, dslot, k.svec,
                                       k.dpartial, k.dcounter, k.dnorm2);
  if (prof) prof->end(KIND_OTHER, st, 0.0);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sol_update_pc(const KrylovPtrs &k, const Geo &g, const Inst *inst, const R *iden, double2 *x64,
                                 long long xinst, typename Cx<R>::T *V, long long vinst, const int *need, int dslot,
                                 int src, cudaStream_t st, Profiler *prof) {
  dim3 grid(k.nblk, k.B);
  if (prof) prof->begin(KIND_OTHER, st);
  k_sol_update_pc<R><<<grid, KT, 0, st>>>(g, inst, iden, x64, xinst, V, vinst, k.Us, k.y, k.m, k.kcount, need, dslot,
                                          src, k.svec, k.dpartial, k.dcounter, k.dnorm2);
  if (prof) prof->end(KIND_OTHER, st, 0.0);
  return cudaGetLastError();
}
template cudaError_t launch_sol_update_pc<float>(const KrylovPtrs &, const Geo &, const Inst *, const float *, double2 *,
                                                 long long, float2 *, long long, const int *, int, int, cudaStream_t,
                                                 Profiler *);
template cudaError_t launch_sol_update_pc<double>(const KrylovPtrs &, const Geo &, const Inst *, const double *,
                                                  double2 *, long long, double2 *, long long, const int *, int, int,
                                                  cudaStream_t, Profiler *);

cudaError_t launch_set_rhs(double2 *r64, long long xinst, const Geo &g, const Inst *inst, int B, cudaStream_t st) {
  const long long tot = (long long)B * g.U;
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 148 * 8);
  k_set_rhs<<<blocks, 256, 0, st>>>(r64, xinst, g, inst, B);
  return cudaGetLastError();
}

cudaError_t launch_extract_e0(const double2 *x64, long long xinst, const Geo &g, int B, double2 *out,
                              cudaStream_t st) {
  k_extract_e0<<<(3 * B + 127) / 128, 128, 0, st>>>(x64, xinst, g, B, out);
  return cudaGetLastError();
}

template cudaError_t launch_arnoldi_ortho<float>(const KrylovPtrs &, float2 *, long long, int, cudaStream_t, Profiler *);
template cudaError_t launch_arnoldi_ortho<double>(const KrylovPtrs &, double2 *, long long, int, cudaStream_t, Profiler *);
template cudaError_t launch_sol_update<float>(const KrylovPtrs &, double2 *, long long, float2 *, long long,
                                              const int *, int, cudaStream_t, Profiler *);
template cudaError_t launch_sol_update<double>(const KrylovPtrs &, double2 *, long long, double2 *, long long,
                                               const int *, int, cudaStream_t, Profiler *);

}  // namespace gsm
