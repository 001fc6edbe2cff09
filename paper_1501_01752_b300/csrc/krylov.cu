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
// test fires), with orthogonality at least as good as MGS.  Dots of FP32
// vectors sum FP32 products in runs of 8 and accumulate the runs in FP64;
// Hessenberg, rotations and residual estimates are FP64.  Reductions across
// blocks use the last-block-done pattern (atomic counter, no waiting).
#include "kernels.h"
#include "reduce.cuh"

namespace gsm {

constexpr int KT = 256;  // threads per block of the vector kernels
constexpr int MAXM = 128;

// Reduce K doubles per thread over the block; thread k < K gets total k in out[k].
template <int K>
__device__ __forceinline__ void block_reduce_k(double (&v)[K], double *red, double *out) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double t = v[k];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (l == 0) red[k * 32 + w] = t;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0;
    for (int i = 0; i < nw; ++i) s += red[threadIdx.x * 32 + i];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(KT) k_dots(const typename Cx<R>::T *__restrict__ V, long long vinst, long long U,
                                             int nv, int wi, const int *__restrict__ act,
                                             const int *__restrict__ gate, double *partial, unsigned *counter,
                                             double *out, int ostride) {
  using C = typename Cx<R>::T;
  __shared__ double red[9 * 32];
  __shared__ double tot[9];
  __shared__ int am_last;
  const int b = blockIdx.y, blk = blockIdx.x, nblk = gridDim.x;
  if (!act[b]) return;
  if (gate && !gate[b]) return;
  const C *Vb = V + b * vinst;
  const C *W = Vb + (long long)wi * U;
  const long long chunk = (U + nblk - 1) / nblk;
  const long long e0 = blk * chunk, e1 = min(U, e0 + chunk);
  const int K = 2 * nv + 1;
  double *pb = partial + ((long long)b * nblk + blk) * K;
  for (int i0 = 0; i0 < nv; i0 += 4) {
    double acc[9];
    R run[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) { acc[k] = 0; run[k] = 0; }
    int cnt = 0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const C w = W[e];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (i0 + k < nv) {
          const C v = Vb[(long long)(i0 + k) * U + e];
          run[2 * k] += v.x * w.x + v.y * w.y;      // conj(v) w
          run[2 * k + 1] += v.x * w.y - v.y * w.x;
        }
      }
      if (i0 == 0) run[8] += w.x * w.x + w.y * w.y;
      if (++cnt == 8) {
#pragma unroll
        for (int k = 0; k < 9; ++k) { acc[k] += (double)run[k]; run[k] = 0; }
        cnt = 0;
      }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] += (double)run[k];
    block_reduce_k<9>(acc, red, tot);
    if (threadIdx.x < 8 && i0 + threadIdx.x / 2 < nv) pb[2 * i0 + threadIdx.x] = tot[threadIdx.x];
    if (threadIdx.x == 8 && i0 == 0) pb[2 * nv] = tot[8];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(&counter[b], 1u);
    am_last = (t == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (!am_last) return;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double s = 0;
    for (int q = 0; q < nblk; ++q) s += __ldcg(&partial[((long long)b * nblk + q) * K + k]);
    out[(long long)b * ostride + k] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) counter[b] = 0;
}

template <typename R>
__global__ void __launch_bounds__(KT) k_update(typename Cx<R>::T *__restrict__ V, long long vinst, long long U,
                                               int nv, int wi, const double *__restrict__ h, int hstride,
                                               const int *__restrict__ act, const int *__restrict__ gate,
                                               double *partial, unsigned *counter, double *wn_out,
                                               int *gate_out, int force) {
  using C = typename Cx<R>::T;
  __shared__ C hs[MAXM + 1];
  __shared__ double red[32];
  const int b = blockIdx.y, blk = blockIdx.x, nblk = gridDim.x;
  if (!act[b]) return;
  if (gate && !gate[b]) return;
  for (int i = threadIdx.x; i < nv; i += blockDim.x)
    hs[i] = mk((R)h[(long long)b * hstride + 2 * i], (R)h[(long long)b * hstride + 2 * i + 1]);
  __syncthreads();
  C *Vb = V + b * vinst;
  C *W = Vb + (long long)wi * U;
  const long long chunk = (U + nblk - 1) / nblk;
  const long long e0 = blk * chunk, e1 = min(U, e0 + chunk);
  double acc = 0;
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    C w = W[e];
    int i = 0;
    for (; i + 4 <= nv; i += 4) {
      C v0 = Vb[(long long)i * U + e], v1 = Vb[(long long)(i + 1) * U + e];
      C v2 = Vb[(long long)(i + 2) * U + e], v3 = Vb[(long long)(i + 3) * U + e];
      w = csub(w, cmul(hs[i], v0));
      w = csub(w, cmul(hs[i + 1], v1));
      w = csub(w, cmul(hs[i + 2], v2));
      w = csub(w, cmul(hs[i + 3], v3));
    }
    for (; i < nv; ++i) w = csub(w, cmul(hs[i], Vb[(long long)i * U + e]));
    W[e] = w;
    acc += (double)w.x * w.x + (double)w.y * w.y;
  }
  if (last_block_sum(acc, red, partial, counter, wn_out, b, nblk, blk)) {
    if (gate_out && threadIdx.x == 0) {
      const double before = h[(long long)b * hstride + 2 * nv];
      gate_out[b] = (force || wn_out[b] < 0.5 * before) ? 1 : 0;
    }
  }
}

// Column j of the Hessenberg matrix, Givens rotations, residual estimate
// (one thread per instance; Saad's GMRES with complex rotations).
__global__ void k_finish(KrylovPtrs k, int j) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= k.B || !k.act[b]) return;
  const int m = k.m, hs = 2 * (m + 1) + 1;
  double2 col[MAXM + 1];
  const bool re = k.gate[b] != 0;
  const double *h0 = k.hdot0 + (long long)b * hs, *h1 = k.hdot1 + (long long)b * hs;
  for (int i = 0; i <= j; ++i) {
    col[i].x = h0[2 * i] + (re ? h1[2 * i] : 0.0);
    col[i].y = h0[2 * i + 1] + (re ? h1[2 * i + 1] : 0.0);
  }
  const double hn = sqrt(fmax(re ? k.wn1[b] : k.wn0[b], 0.0));
  double *cs = k.cs + (long long)b * m;
  double2 *sn = k.sn + (long long)b * m;
  double2 *g = k.gv + (long long)b * (m + 1);
  for (int i = 0; i < j; ++i) {
    const double2 a = col[i], c2 = col[i + 1];
    const double c = cs[i];
    const double2 s = sn[i];
    col[i] = mk(c * a.x + s.x * c2.x - s.y * c2.y, c * a.y + s.x * c2.y + s.y * c2.x);
    // -conj(s) a + c c2
    col[i + 1] = mk(-(s.x * a.x + s.y * a.y) + c * c2.x, -(s.x * a.y - s.y * a.x) + c * c2.y);
  }
  const double2 a = col[j];
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
  double2 *Hc = k.H + ((long long)b * m + j) * (m + 1);
  for (int i = 0; i <= j; ++i) Hc[i] = col[i];
  k.kcount[b] = j + 1;
  k.scale32[b] = hn > 0 ? (float)(1.0 / hn) : 0.f;
  k.scale64[b] = hn > 0 ? 1.0 / hn : 0.0;
  const double r = hypot(g[j + 1].x, g[j + 1].y);
  k.resid[b] = r;
  if (r <= k.thresh[b] || hn == 0.0 || j + 1 >= m) k.act[b] = 0;
}

// y = R^-1 g over the kcount[b] rotated columns (back substitution).
__global__ void k_backsolve(KrylovPtrs k) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= k.B) return;
  const int m = k.m, n = k.kcount[b];
  const double2 *g = k.gv + (long long)b * (m + 1);
  double2 *y = k.y + (long long)b * m;
  for (int i = n - 1; i >= 0; --i) {
    double2 s = g[i];
    for (int l = i + 1; l < n; ++l) {
      const double2 r = k.H[((long long)b * m + l) * (m + 1) + i];
      s = csub(s, cmul(r, y[l]));
    }
    const double2 d = k.H[((long long)b * m + i) * (m + 1) + i];
    const double dd = d.x * d.x + d.y * d.y;
    y[i] = dd > 0 ? mk((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd) : mk(0.0, 0.0);
  }
}

// x += V y (FP64 x; the combination in the basis precision).
template <typename R>
__global__ void __launch_bounds__(KT) k_sol_update(double2 *__restrict__ x64, long long xinst,
                                                   const typename Cx<R>::T *__restrict__ V, long long vinst,
                                                   long long U, const double2 *__restrict__ y, int m,
                                                   const int *__restrict__ kcount, const int *__restrict__ need) {
  using C = typename Cx<R>::T;
  __shared__ C ys[MAXM];
  const int b = blockIdx.y;
  if (!need[b]) return;
  const int n = kcount[b];
  if (n == 0) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) ys[i] = mk((R)y[(long long)b * m + i].x, (R)y[(long long)b * m + i].y);
  __syncthreads();
  const C *Vb = V + b * vinst;
  double2 *xb = x64 + b * xinst;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < U; e += (long long)gridDim.x * blockDim.x) {
    C d = mk((R)0, (R)0);
    for (int i = 0; i < n; ++i) d = cadd(d, cmul(ys[i], Vb[(long long)i * U + e]));
    double2 xv = xb[e];
    xb[e] = mk(xv.x + (double)d.x, xv.y + (double)d.y);
  }
}

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

// ------------------------------------------------------------ launchers
template <typename R>
cudaError_t launch_arnoldi_ortho(const KrylovPtrs &k, typename Cx<R>::T *V, long long vinst, int j, cudaStream_t st,
                                 Profiler *prof) {
  const int nv = j + 1, wi = j + 1, hs = 2 * (k.m + 1) + 1;
  dim3 grid(k.nblk, k.B);
  const double vb = (double)sizeof(typename Cx<R>::T) * k.U * k.B;
  if (prof) prof->begin(KIND_DOTS, st);
  k_dots<R><<<grid, KT, 0, st>>>(V, vinst, k.U, nv, wi, k.act, nullptr, k.partial, k.counter, k.hdot0, hs);
  if (prof) prof->end(KIND_DOTS, st, vb * (nv + 1));
  if (prof) prof->begin(KIND_UPDATE, st);
  k_update<R><<<grid, KT, 0, st>>>(V, vinst, k.U, nv, wi, k.hdot0, hs, k.act, nullptr, k.partial, k.counter, k.wn0,
                                   k.gate, k.force_reorth);
  if (prof) prof->end(KIND_UPDATE, st, vb * (nv + 2));
  if (prof) prof->begin(KIND_DOTS, st);
  k_dots<R><<<grid, KT, 0, st>>>(V, vinst, k.U, nv, wi, k.act, k.gate, k.partial, k.counter, k.hdot1, hs);
  if (prof) prof->end(KIND_DOTS, st, 0.0);
  if (prof) prof->begin(KIND_UPDATE, st);
  k_update<R><<<grid, KT, 0, st>>>(V, vinst, k.U, nv, wi, k.hdot1, hs, k.act, k.gate, k.partial, k.counter, k.wn1,
                                   nullptr, 0);
  if (prof) prof->end(KIND_UPDATE, st, 0.0);
  return cudaGetLastError();
}

cudaError_t launch_finish(const KrylovPtrs &k, int j, cudaStream_t st) {
  k_finish<<<(k.B + 31) / 32, 32, 0, st>>>(k, j);
  return cudaGetLastError();
}

cudaError_t launch_backsolve(const KrylovPtrs &k, cudaStream_t st) {
  k_backsolve<<<(k.B + 31) / 32, 32, 0, st>>>(k);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_sol_update(const KrylovPtrs &k, double2 *x64, long long xinst, const typename Cx<R>::T *V,
                              long long vinst, const int *need, cudaStream_t st, Profiler *prof) {
  dim3 grid(k.nblk, k.B);
  if (prof) prof->begin(KIND_OTHER, st);
  k_sol_update<R><<<grid, KT, 0, st>>>(x64, xinst, V, vinst, k.U, k.y, k.m, k.kcount, need);
  if (prof) prof->end(KIND_OTHER, st, 0.0);
  return cudaGetLastError();
}

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
template cudaError_t launch_sol_update<float>(const KrylovPtrs &, double2 *, long long, const float2 *, long long,
                                              const int *, cudaStream_t, Profiler *);
template cudaError_t launch_sol_update<double>(const KrylovPtrs &, double2 *, long long, const double2 *, long long,
                                               const int *, cudaStream_t, Profiler *);

}  // namespace gsm
