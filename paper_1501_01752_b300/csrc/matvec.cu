// The Eq. 4 operator y = A x = x - G (Delta/eps_b * x) as three fused passes
// over HBM (GSM section, truncation paragraph: the Toeplitz product is done by
// FFT).  Per instance the field is 3 planar components of N_z x N_y x N_x
// complex values, x fastest.  The cyclic convolution runs on an
// L_x x L_y x L_z grid, L_a >= 2 N_a - 1, which makes it equal to the
// truncated Toeplitz product (every offset m - m' in [-2n, 2n] has its own
// residue mod L).
//
//   pass 1  k_fwd_x : scatter each x-row into L_x points, FFT along x (S=+1)
//                     -> T[b][r_x][c][m_z][m_y]            (3 L_x N_y N_z)
//   pass 2  k_yz    : per (r_x, c): FFT along y on the N_z rows, FFT along z
//                     on every column, times D(r), inverse along z keeping
//                     the N_z harmonics, inverse along y keeping N_y; in place
//   pass 3  k_inv_x : inverse FFT along x keeping N_x harmonics, then per
//                     harmonic y = x - G(m) u (or the residual b - A x, or the
//                     adjoint form x - u) with G from k_m and 1/(k_m^2 - k_b^2)
//
// D(r) holds sum_d Delta_d exp(2 pi i d.r / L) / (L_x L_y L_z), so the
// inverse transforms need no further scaling.  The pruned loads only touch
// the N_a harmonics; pruned stores only write them.
#include "fft.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace gsm {

template <typename C> __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }

// ---------------------------------------------------------------- pass 1
// PRE 0: the input as it is (Eq. 4); PRE 1: G(m) x first (adjoint of Eq. 4);
// PRE 2: k_m x x first (Eq. 5, H-field formulation)
template <typename R, int PRE>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_fwd_x(Geo g, const typename Cx<R>::T *__restrict__ X, long long xstride,
                        typename Cx<R>::T *__restrict__ T, const R *__restrict__ scale,
                        const int *__restrict__ act, const Inst *__restrict__ inst,
                        const R *__restrict__ iden, const typename Cx<R>::T *__restrict__ twg, int rows,
                        int nchunk, const int *__restrict__ jdev, long long jstride) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C *tw = reinterpret_cast<C *>(sm_raw);
  C *S = tw + TWN;
  if (jdev) X += (long long)(*jdev) * jstride;
  const int b = blockIdx.y;
  if (act && !act[b]) return;
  load_twiddles(tw, twg);
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2], L0 = g.L[0], P0 = L0 + 1;
  const int mz = blockIdx.x / nchunk, my0 = (blockIdx.x % nchunk) * rows;
  const int nr = min(rows, N1 - my0);
  const C *Xb = X + b * xstride;
  C *Tb = T + b * g.Tst;
  const R s = scale ? scale[b] : (R)1;
  const long long Nh = g.Nh;
  Team tm(g.L[0]);
  // Green tensor ingredients for the adjoint form (G applied before the
  // Toeplitz product; G is real symmetric for real k and k_b^2) and the wave
  // vector of the H-field form
  R kb2 = 0, kz = 0;
  if (PRE) {
    kb2 = (R)inst[b].kb2;
    kz = (R)(inst[b].kinc[2] + (mz - g.n[2]) * g.K[2]);
  }
  for (int c = 0; c < 3; ++c) {
    for (int e = threadIdx.x; e < nr * P0; e += blockDim.x) S[e] = czero<C>();
    __syncthreads();
    for (int e = threadIdx.x; e < nr * N0; e += blockDim.x) {
      const int row = e / N0, mx = e - row * N0;
      const long long h = ((long long)mz * N1 + my0 + row) * N0 + mx;
      C v;
      if (PRE == 0) {
        v = cscale(Xb[c * Nh + h], s);
      } else {
        const R kx = (R)(inst[b].kinc[0] + (mx - g.n[0]) * g.K[0]);
        const R ky = (R)(inst[b].kinc[1] + (my0 + row - g.n[1]) * g.K[1]);
        const C v0 = cscale(Xb[h], s), v1 = cscale(Xb[Nh + h], s), v2 = cscale(Xb[2 * Nh + h], s);
        if (PRE == 1) {
          const C kv = mk(kx * v0.x + ky * v1.x + kz * v2.x, kx * v0.y + ky * v1.y + kz * v2.y);
          const R kc = c == 0 ? kx : (c == 1 ? ky : kz);
          const C vc = c == 0 ? v0 : (c == 1 ? v1 : v2);
          const R id = iden[b * g.ist + h];
          v = mk(id * (kb2 * vc.x - kc * kv.x), id * (kb2 * vc.y - kc * kv.y));
        } else {
          // (k x v)_c
          if (c == 0) v = csub(cscale(v2, ky), cscale(v1, kz));
          else if (c == 1) v = csub(cscale(v0, kz), cscale(v2, kx));
          else v = csub(cscale(v1, kx), cscale(v0, ky));
        }
      }
      S[row * P0 + wrap(mx, g.n[0], L0)] = v;
    }
    __syncthreads();
    for (int row = tm.id; row < nr; row += tm.count) team_fft<+1>(S + row * P0, g.L[0], tm.lane, tm.ts, tm.mask, tw);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * L0; e += blockDim.x) {
      const int rx = e / nr, row = e - rx * nr;
      Tb[(((long long)rx * 3 + c) * N2 + mz) * N1 + my0 + row] = S[row * P0 + rx];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- pass 2
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_yz(Geo g, typename Cx<R>::T *__restrict__ T, const R *__restrict__ D,
                     const int *__restrict__ act, const typename Cx<R>::T *__restrict__ twg) {
  using C = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C *tw = reinterpret_cast<C *>(sm_raw);
  const int N1 = g.N[1], N2 = g.N[2], L1 = g.L[1], L2 = g.L[2], P1 = L1 + 1, P2 = L2 + 1;
  C *A = tw + TWN;
  C *buf = A + N2 * P1;
  const int rx = blockIdx.x, c = blockIdx.y, b = blockIdx.z;
  if (act && !act[b]) return;
  load_twiddles(tw, twg);
  C *Tb = T + b * g.Tst + ((long long)rx * 3 + c) * N2 * N1;
  for (int e = threadIdx.x; e < N2 * P1; e += blockDim.x) A[e] = czero<C>();
  __syncthreads();
  for (int e = threadIdx.x; e < N2 * N1; e += blockDim.x) {
    const int mz = e / N1, my = e - mz * N1;
    A[mz * P1 + wrap(my, g.n[1], L1)] = Tb[e];
  }
  __syncthreads();
  Team ty(g.L[1]);
  for (int row = ty.id; row < N2; row += ty.count) team_fft<+1>(A + row * P1, g.L[1], ty.lane, ty.ts, ty.mask, tw);
  __syncthreads();
  Team tz(g.L[2]);
  const R *Dx = D + (long long)rx * L1 * L2;
  for (int ry = tz.id; ry < L1; ry += tz.count) {
    C *bf = buf + tz.id * P2;   // this team's column buffer
    for (int i = tz.lane; i < L2; i += tz.ts) bf[i] = czero<C>();
    __syncwarp(tz.mask);
    for (int mz = tz.lane; mz < N2; mz += tz.ts) bf[wrap(mz, g.n[2], L2)] = A[mz * P1 + ry];
    __syncwarp(tz.mask);
    team_fft<+1>(bf, g.L[2], tz.lane, tz.ts, tz.mask, tw);
    const R *Dc = Dx + (long long)ry * L2;
    for (int i = tz.lane; i < L2; i += tz.ts) bf[i] = cscale(bf[i], Dc[i]);
    __syncwarp(tz.mask);
    team_fft<-1>(bf, g.L[2], tz.lane, tz.ts, tz.mask, tw);
    for (int mz = tz.lane; mz < N2; mz += tz.ts) A[mz * P1 + ry] = bf[wrap(mz, g.n[2], L2)];
    __syncwarp(tz.mask);
  }
  __syncthreads();
  for (int row = ty.id; row < N2; row += ty.count) team_fft<-1>(A + row * P1, g.L[1], ty.lane, ty.ts, ty.mask, tw);
  __syncthreads();
  for (int e = threadIdx.x; e < N2 * N1; e += blockDim.x) {
    const int mz = e / N1, my = e - mz * N1;
    Tb[e] = A[mz * P1 + wrap(my, g.n[1], L1)];
  }
}

// ---------------------------------------------------------------- pass 3
// MODE 0: Y = X - G u          (forward operator)
// MODE 1: Y = b - (X - G u)    (residual of Eq. 4; b = a at m = 0)
// MODE 2: Y = X - u            (adjoint operator: G was applied in pass 1)
// MODE 3: Y = b - (X - u)      (residual of the adjoint system)
// HF = 1 (modes 0, 1): Eq. 5, G u replaced by k_m x u / (k_m^2 - k_b^2)
template <typename R, int MODE, int HF>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_inv_x(Geo g, const typename Cx<R>::T *__restrict__ T, const typename Cx<R>::T *__restrict__ X,
                        long long xstride, typename Cx<R>::T *__restrict__ Y, long long ystride,
                        const int *__restrict__ act, const Inst *__restrict__ inst, const R *__restrict__ iden,
                        const typename Cx<R>::T *__restrict__ twg, int rows, int nchunk, double *partial,
                        unsigned *counter, double *norm_out, const int *__restrict__ jdev, long long jstride,
                        const R *__restrict__ scale) {
  using C = typename Cx<R>::T;
  if (jdev) {
    X += (long long)(*jdev) * jstride;
    Y += (long long)(*jdev) * jstride;
  }
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ double red[32];
  C *tw = reinterpret_cast<C *>(sm_raw);
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2], L0 = g.L[0], P0 = L0 + 1;
  C *S = tw + TWN;
  R *kxs = reinterpret_cast<R *>(S + 3 * rows * P0);
  R *kys = kxs + N0;
  const int b = blockIdx.y;
  if (act && !act[b]) return;
  load_twiddles(tw, twg);
  const int mz = blockIdx.x / nchunk, my0 = (blockIdx.x % nchunk) * rows;
  const int nr = min(rows, N1 - my0);
  const C *Tb = T + b * g.Tst;
  const long long Nh = g.Nh;
  for (int c = 0; c < 3; ++c)
    for (int e = threadIdx.x; e < nr * L0; e += blockDim.x) {
      const int rx = e / nr, row = e - rx * nr;
      S[(c * rows + row) * P0 + rx] = Tb[(((long long)rx * 3 + c) * N2 + mz) * N1 + my0 + row];
    }
  if (!(MODE & 2)) {
    for (int i = threadIdx.x; i < N0; i += blockDim.x) kxs[i] = (R)(inst[b].kinc[0] + (i - g.n[0]) * g.K[0]);
    for (int i = threadIdx.x; i < nr; i += blockDim.x) kys[i] = (R)(inst[b].kinc[1] + (my0 + i - g.n[1]) * g.K[1]);
  }
  __syncthreads();
  Team tm(g.L[0]);
  for (int q = tm.id; q < 3 * rows; q += tm.count)
    if (q % rows < nr) team_fft<-1>(S + q * P0, g.L[0], tm.lane, tm.ts, tm.mask, tw);
  __syncthreads();
  const R kz = (R)(inst[b].kinc[2] + (mz - g.n[2]) * g.K[2]);
  const R kb2 = (R)inst[b].kb2;
  const long long h0 = ((long long)g.n[2] * N1 + g.n[1]) * N0 + g.n[0];
  const C *Xb = X + b * xstride;
  C *Yb = Y + b * ystride;
  double acc = 0;
  for (int e = threadIdx.x; e < nr * N0; e += blockDim.x) {
    const int row = e / N0, mx = e - row * N0;
    const long long h = ((long long)mz * N1 + my0 + row) * N0 + mx;
    const int px = wrap(mx, g.n[0], L0);
    C u0 = S[(0 * rows + row) * P0 + px], u1 = S[(1 * rows + row) * P0 + px], u2 = S[(2 * rows + row) * P0 + px];
    if (HF) {
      const R kx = kxs[mx], ky = kys[row], id = iden[b * g.ist + h];
      const C w0 = csub(cscale(u2, ky), cscale(u1, kz)), w1 = csub(cscale(u0, kz), cscale(u2, kx)),
              w2 = csub(cscale(u1, kx), cscale(u0, ky));
      u0 = cscale(w0, id);
      u1 = cscale(w1, id);
      u2 = cscale(w2, id);
    } else if (!(MODE & 2)) {
      const R kx = kxs[mx], ky = kys[row], id = iden[b * g.ist + h];
      const C ku = mk(kx * u0.x + ky * u1.x + kz * u2.x, kx * u0.y + ky * u1.y + kz * u2.y);
      u0 = mk(id * (kb2 * u0.x - kx * ku.x), id * (kb2 * u0.y - kx * ku.y));
      u1 = mk(id * (kb2 * u1.x - ky * ku.x), id * (kb2 * u1.y - ky * ku.y));
      u2 = mk(id * (kb2 * u2.x - kz * ku.x), id * (kb2 * u2.y - kz * ku.y));
    }
    // the identity term takes the input as pass 1 did (scaled by 1 / ||v_j||:
    // the stored Krylov vector is unnormalised)
    const R sx = scale ? scale[b] : (R)1;
    C y0 = csub(cscale(Xb[h], sx), u0), y1 = csub(cscale(Xb[Nh + h], sx), u1), y2 = csub(cscale(Xb[2 * Nh + h], sx), u2);
    if (MODE & 1) {
      C b0 = czero<C>(), b1 = czero<C>(), b2 = czero<C>();
      if (h == h0) {
        b0 = mk((R)inst[b].a[0], (R)inst[b].a[1]);
        b1 = mk((R)inst[b].a[2], (R)inst[b].a[3]);
        b2 = mk((R)inst[b].a[4], (R)inst[b].a[5]);
      }
      y0 = csub(b0, y0);
      y1 = csub(b1, y1);
      y2 = csub(b2, y2);
    }
    if (norm_out)
      acc += (double)y0.x * y0.x + (double)y0.y * y0.y + (double)y1.x * y1.x + (double)y1.y * y1.y +
             (double)y2.x * y2.x + (double)y2.y * y2.y;
    Yb[h] = y0;
    Yb[Nh + h] = y1;
    Yb[2 * Nh + h] = y2;
  }
  if (norm_out) last_block_sum(acc, red, partial, counter, norm_out, b, gridDim.x, blockIdx.x);
}

// ------------------------------------------------ 1/(k_m^2 - k_b^2) tables
__global__ void k_iden(Geo g, const Inst *__restrict__ inst, int B, double *id64, float *id32, dfl *iddf) {
  const long long tot = (long long)B * g.Nh;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / g.Nh);
    long long h = t - (long long)b * g.Nh;
    const long long e = (long long)b * g.ist + h;
    const int mx = (int)(h % g.N[0]);
    h /= g.N[0];
    const int my = (int)(h % g.N[1]);
    const int mz = (int)(h / g.N[1]);
    const double kx = inst[b].kinc[0] + (mx - g.n[0]) * g.K[0];
    const double ky = inst[b].kinc[1] + (my - g.n[1]) * g.K[1];
    const double kz = inst[b].kinc[2] + (mz - g.n[2]) * g.K[2];
    const double den = kx * kx + ky * ky + kz * kz - inst[b].kb2;  // FP64: cancellation near k_b
    const double v = 1.0 / den;
    id64[e] = v;
    id32[e] = (float)v;
    if (iddf) iddf[e] = dfl(v);
  }
}

__global__ void k_d2df(const double *__restrict__ in, dfl *__restrict__ out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = dfl(in[e]);
}

// ------------------------------------------------ precision conversions
template <typename Ci, typename Co>
__global__ void k_convert(const Ci *__restrict__ in, Co *__restrict__ out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    Ci v = in[e];
    out[e] = mk((decltype(out[0].x))v.x, (decltype(out[0].x))v.y);
  }
}

// ------------------------------------------------ launchers
static int pick_rows(int N1, int L0, size_t csize, int reps, size_t budget) {
  const int ts = L0 >= 8 ? L0 / 8 : 1;
  int rows = N1;
  while (rows > 1 && ((size_t)reps * rows * (L0 + 1) * csize > budget || rows * ts > 256)) rows = (rows + 1) / 2;
  return rows;
}

static int round_warp(int t) { return ((t + 31) / 32) * 32; }

template <typename R> size_t pass2_smem(const Geo &g) {
  using C = typename Cx<R>::T;
  const int tsz = g.L[2] >= 8 ? g.L[2] / 8 : 1;
  const int nteams = 256 / tsz;
  return sizeof(C) * (TWN + (size_t)g.N[2] * (g.L[1] + 1) + (size_t)nteams * (g.L[2] + 1));
}

template <typename R>
cudaError_t launch_matvec(const MatvecArgs<R> &a, cudaStream_t st, Profiler *prof) {
  using C = typename Cx<R>::T;
  const Geo &g = a.g;
  const size_t cs = sizeof(C);
  // pass 1
  {
    const int rows = pick_rows(g.N[1], g.L[0], cs, 1, 40 * 1024);
    const int nchunk = (g.N[1] + rows - 1) / rows;
    const int ts = g.L[0] >= 8 ? g.L[0] / 8 : 1;
    const int threads = max(64, round_warp(rows * ts));
    const size_t smem = cs * (TWN + (size_t)rows * (g.L[0] + 1));
    dim3 grid(g.N[2] * nchunk, a.B);
    if (prof) prof->begin(KIND_FWD_X, st);
#define GSM_P1(PRE)                                                                                       \
  cudaFuncSetAttribute(k_fwd_x<R, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);          \
  k_fwd_x<R, PRE><<<grid, threads, smem, st>>>(g, a.X, a.xstride, a.T, a.scale, a.act, a.inst, \
                                               a.iden, a.tw, rows, nchunk, a.jdev, a.jstride)
    if (a.mode & 2) { GSM_P1(1); }
    else if (a.form) { GSM_P1(2); }
    else { GSM_P1(0); }
#undef GSM_P1
    if (prof) prof->end(KIND_FWD_X, st, (double)a.B * (cs * (double)(g.U + g.Tsz)));
  }
  // pass 2
  {
    const size_t smem = pass2_smem<R>(g);
    cudaFuncSetAttribute(k_yz<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(g.L[0], 3, a.B);
    if (prof) prof->begin(KIND_YZ, st);
    k_yz<R><<<grid, 256, smem, st>>>(g, a.T, a.D, a.act, a.tw);
    if (prof)
      prof->end(KIND_YZ, st,
                (double)a.B * 2.0 * cs * (double)g.Tsz + sizeof(R) * (double)g.L[0] * g.L[1] * g.L[2]);
  }
  // pass 3
  {
    const int rows = pick_rows(g.N[1], g.L[0], cs, 3, 40 * 1024);
    const int nchunk = (g.N[1] + rows - 1) / rows;
    const int ts = g.L[0] >= 8 ? g.L[0] / 8 : 1;
    const int threads = max(64, round_warp(std::min(256, 3 * rows * ts)));
    const size_t smem = cs * (TWN + 3 * (size_t)rows * (g.L[0] + 1)) + sizeof(R) * (g.N[0] + rows) + 16;
    dim3 grid(g.N[2] * nchunk, a.B);
    if (prof) prof->begin(KIND_INV_X, st);
#define GSM_P3(M, HF)                                                                                           \
  cudaFuncSetAttribute(k_inv_x<R, M, HF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);            \
  k_inv_x<R, M, HF><<<grid, threads, smem, st>>>(g, a.T, a.X, a.xstride, a.Y, a.ystride, a.act, a.inst, a.iden, \
                                                 a.tw, rows, nchunk, a.partial, a.counter, a.norm_out, a.jdev,  \
                                                 a.jstride, a.scale)
    if (a.mode == 0) { if (a.form) { GSM_P3(0, 1); } else { GSM_P3(0, 0); } }
    else if (a.mode == 1) { if (a.form) { GSM_P3(1, 1); } else { GSM_P3(1, 0); } }
    else if (a.mode == 2) { GSM_P3(2, 0); }
    else { GSM_P3(3, 0); }
#undef GSM_P3
    if (prof)
      prof->end(KIND_INV_X, st,
                (double)a.B * (cs * (double)(g.Tsz + 2 * g.U) + (!(a.mode & 2) ? sizeof(R) * (double)g.Nh : 0.0)));
  }
  return cudaGetLastError();
}

int matvec_blocks_pass3(const Geo &g, size_t csize) {
  const int rows = pick_rows(g.N[1], g.L[0], csize, 3, 40 * 1024);
  return g.N[2] * ((g.N[1] + rows - 1) / rows);
}

size_t matvec_max_smem(const Geo &g, size_t csize) {
  size_t p2 = csize == 8 ? pass2_smem<float>(g) : pass2_smem<double>(g);
  const int r1 = pick_rows(g.N[1], g.L[0], csize, 1, 40 * 1024);
  size_t p1 = csize * (TWN + (size_t)r1 * (g.L[0] + 1));
  return p2 > p1 ? p2 : p1;
}

cudaError_t launch_iden(const Geo &g, const Inst *inst, int B, double *id64, float *id32, cudaStream_t st,
                        dfl *iddf) {
  long long tot = (long long)B * g.Nh;
  int blocks = (int)std::min<long long>((tot + 255) / 256, 148 * 16);
  k_iden<<<blocks, 256, 0, st>>>(g, inst, B, id64, id32, iddf);
  return cudaGetLastError();
}

cudaError_t launch_d2df(const double *in, dfl *out, long long n, cudaStream_t st) {
  int blocks = (int)std::min<long long>((n + 255) / 256, 148 * 8);
  k_d2df<<<blocks, 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_convert_d2f(const double2 *in, float2 *out, long long n, cudaStream_t st) {
  int blocks = (int)std::min<long long>((n + 255) / 256, 148 * 16);
  k_convert<double2, float2><<<blocks, 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}
cudaError_t launch_convert_f2d(const float2 *in, double2 *out, long long n, cudaStream_t st) {
  int blocks = (int)std::min<long long>((n + 255) / 256, 148 * 16);
  k_convert<float2, double2><<<blocks, 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

template cudaError_t launch_matvec<float>(const MatvecArgs<float> &, cudaStream_t, Profiler *);
template cudaError_t launch_matvec<double>(const MatvecArgs<double> &, cudaStream_t, Profiler *);

}  // namespace gsm
