// Complex64 fast path of the Eq. 4 operator for FFT sizes 32 and 64 per
// axis: the same three passes as matvec.cu, but every 1D transform is held
// by one thread in registers (fft_reg.cuh), so the only shared-memory
// traffic is the staging of rows and columns.  Forward transforms leave the
// spectrum in the permuted register order, the multiplier D is stored in
// that order (k_d_permute), and the inverse transforms return natural order.
//
//   pass 1  k_fwd_x_reg  : thread per x-row (c, m_z, m_y): N_x -> L_x
//   pass 2  k_yz_reg     : per r_x plane, thread per y-row (forward), thread
//                          per y-frequency column (z forward, x D, z inverse),
//                          thread per y-row (inverse)
//   pass 3  k_inv_x_reg  : thread per x-row: L_x -> N_x, then per harmonic
//                          the Green tensor, y = x - G u (or the residual)
#include "fft_reg.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace gsm {

// harmonic index (0..N-1) held at natural grid position k, or -1
__device__ __forceinline__ int harm_at(int k, int n, int L) {
  if (k <= n) return k + n;
  if (k >= L - n) return k - L + n;
  return -1;
}

constexpr int RT = 128;  // threads per block of the register kernels

template <int L0>
__global__ void __launch_bounds__(RT, 2) k_fwd_x_reg(Geo g, float2 *__restrict__ X, long long xstride,
                                                     float2 *__restrict__ T, const float *__restrict__ scale,
                                                     int write_back, const int *__restrict__ act,
                                                     const float2 *__restrict__ twg, int planes) {
  __shared__ float2 tw[TWN];
  extern __shared__ __align__(16) float2 S[];   // [planes * N1][N0 + 1]
  const int b = blockIdx.y;
  if (act && !act[b]) return;
  for (int i = threadIdx.x; i < TWN; i += blockDim.x) tw[i] = twg[i];
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2], P = N0 + 1;
  const long long Nh = g.Nh;
  const int p0 = blockIdx.x * planes;
  const int np = min(planes, 3 * N2 - p0);
  float2 *Xb = X + b * xstride;
  float2 *Tb = T + b * g.Tsz;
  const float s = scale ? scale[b] : 1.f;
  // planes (c, m_z) are consecutive N1 x N0 blocks of the field
  for (int e = threadIdx.x; e < np * N1 * N0; e += blockDim.x) {
    const int pl = e / (N1 * N0), r = e - pl * (N1 * N0);
    const int plane = p0 + pl;
    const long long idx = (long long)plane * N1 * N0 + r;   // c Nh + m_z N1 N0 + m_y N0 + m_x
    float2 v = Xb[idx];
    v.x *= s;
    v.y *= s;
    if (write_back) Xb[idx] = v;
    const int my = r / N0, mx = r - my * N0;
    S[(pl * N1 + my) * P + mx] = v;
  }
  __syncthreads();
  const int row = threadIdx.x;
  if (row >= np * N1) return;
  const int pl = row / N1, my = row - pl * N1;
  const int plane = p0 + pl, c = plane / N2, mz = plane - c * N2;
  float2 v[L0];
#pragma unroll
  for (int k = 0; k < L0; ++k) {
    const int h = harm_at(k, g.n[0], L0);
    v[k] = h >= 0 ? S[row * P + h] : make_float2(0.f, 0.f);
  }
  RegFFT<L0>::template forward<+1>(v, tw);
  (void)Nh;
#pragma unroll
  for (int i = 0; i < L0; ++i) {
    const int rx = RegFFT<L0>::freq(i);
    Tb[(((long long)rx * 3 + c) * N2 + mz) * N1 + my] = v[i];
  }
}

template <int LY, int LZ>
__global__ void __launch_bounds__(RT, 2) k_yz_reg(Geo g, float2 *__restrict__ T, const float *__restrict__ Dp,
                                                  const int *__restrict__ act, const float2 *__restrict__ twg) {
  constexpr int PPB = RT / LY;   // r_x planes per block
  __shared__ float2 tw[TWN];
  extern __shared__ __align__(16) float2 A[];   // [PPB][N2][LY + 1]
  const int b = blockIdx.z, c = blockIdx.y, rx0 = blockIdx.x * PPB;
  if (act && !act[b]) return;
  for (int i = threadIdx.x; i < TWN; i += blockDim.x) tw[i] = twg[i];
  const int N1 = g.N[1], N2 = g.N[2], PY = LY + 1;
  const int nq = min(PPB, g.L[0] - rx0);
  float2 *Tb = T + b * g.Tsz;
  for (int e = threadIdx.x; e < nq * N2 * N1; e += blockDim.x) {
    const int q = e / (N2 * N1), r = e - q * (N2 * N1);
    const int mz = r / N1, my = r - mz * N1;
    A[(q * N2 + mz) * PY + my] = Tb[((long long)(rx0 + q) * 3 + c) * N2 * N1 + r];
  }
  __syncthreads();
  // y forward: one thread per (plane, m_z) row
  for (int t = threadIdx.x; t < nq * N2; t += blockDim.x) {
    float2 *row = A + t * PY;
    float2 v[LY];
#pragma unroll
    for (int k = 0; k < LY; ++k) {
      const int h = harm_at(k, g.n[1], LY);
      v[k] = h >= 0 ? row[h] : make_float2(0.f, 0.f);
    }
    RegFFT<LY>::template forward<+1>(v, tw);
#pragma unroll
    for (int i = 0; i < LY; ++i) row[i] = v[i];
  }
  __syncthreads();
  // z forward, times D, z inverse: one thread per (plane, y-frequency column)
  {
    const int q = threadIdx.x / LY, col = threadIdx.x - q * LY;
    if (q < nq) {
      float2 *base = A + q * N2 * PY + col;
      float2 v[LZ];
#pragma unroll
      for (int k = 0; k < LZ; ++k) {
        const int h = harm_at(k, g.n[2], LZ);
        v[k] = h >= 0 ? base[h * PY] : make_float2(0.f, 0.f);
      }
      RegFFT<LZ>::template forward<+1>(v, tw);
      const float *Dq = Dp + (long long)(rx0 + q) * LZ * LY + col;
#pragma unroll
      for (int i = 0; i < LZ; ++i) {
        const float d = Dq[i * LY];
        v[i].x *= d;
        v[i].y *= d;
      }
      RegFFT<LZ>::template inverse<-1>(v, tw);
#pragma unroll
      for (int k = 0; k < LZ; ++k) {
        const int h = harm_at(k, g.n[2], LZ);
        if (h >= 0) base[h * PY] = v[k];
      }
    }
  }
  __syncthreads();
  // y inverse: one thread per row, back to natural order
  for (int t = threadIdx.x; t < nq * N2; t += blockDim.x) {
    float2 *row = A + t * PY;
    float2 v[LY];
#pragma unroll
    for (int i = 0; i < LY; ++i) v[i] = row[i];
    RegFFT<LY>::template inverse<-1>(v, tw);
#pragma unroll
    for (int k = 0; k < LY; ++k) {
      const int h = harm_at(k, g.n[1], LY);
      if (h >= 0) row[h] = v[k];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nq * N2 * N1; e += blockDim.x) {
    const int q = e / (N2 * N1), r = e - q * (N2 * N1);
    const int mz = r / N1, my = r - mz * N1;
    Tb[((long long)(rx0 + q) * 3 + c) * N2 * N1 + r] = A[(q * N2 + mz) * PY + my];
  }
}

// MODE 0: Y = X - G u; MODE 1: Y = b - (X - G u)
template <int L0, int MODE>
__global__ void __launch_bounds__(RT, 2) k_inv_x_reg(Geo g, const float2 *__restrict__ T,
                                                     const float2 *__restrict__ X, long long xstride,
                                                     float2 *__restrict__ Y, long long ystride,
                                                     const int *__restrict__ act, const Inst *__restrict__ inst,
                                                     const float *__restrict__ iden,
                                                     const float2 *__restrict__ twg, int rows, double *partial,
                                                     unsigned *counter, double *norm_out) {
  __shared__ float2 tw[TWN];
  __shared__ double red[32];
  extern __shared__ __align__(16) float2 S3[];   // [3][rows][N0 + 1], then kx[N0]
  const int b = blockIdx.y;
  if (act && !act[b]) return;
  for (int i = threadIdx.x; i < TWN; i += blockDim.x) tw[i] = twg[i];
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2], P = N0 + 1;
  float *kxs = reinterpret_cast<float *>(S3 + 3 * rows * P);
  const long long Nh = g.Nh;
  const long long r0 = (long long)blockIdx.x * rows;          // first (m_z, m_y) row
  const long long left = (long long)N1 * N2 - r0;
  const int nr = (int)(left < rows ? left : rows);
  for (int i = threadIdx.x; i < N0; i += blockDim.x) kxs[i] = (float)(inst[b].kinc[0] + (i - g.n[0]) * g.K[0]);
  __syncthreads();
  const float2 *Tb = T + b * g.Tsz;
  if (threadIdx.x < 3 * nr) {
    const int c = threadIdx.x / nr, row = threadIdx.x - c * nr;
    const long long rr = r0 + row;                            // = m_z N1 + m_y
    float2 v[L0];
#pragma unroll
    for (int i = 0; i < L0; ++i) {
      const int rx = RegFFT<L0>::freq(i);
      v[i] = Tb[((long long)rx * 3 + c) * N2 * N1 + rr];
    }
    RegFFT<L0>::template inverse<-1>(v, tw);
#pragma unroll
    for (int k = 0; k < L0; ++k) {
      const int h = harm_at(k, g.n[0], L0);
      if (h >= 0) S3[(c * rows + row) * P + h] = v[k];
    }
  }
  __syncthreads();
  const float kb2 = (float)inst[b].kb2;
  const long long h0 = ((long long)g.n[2] * N1 + g.n[1]) * N0 + g.n[0];
  const float2 *Xb = X + b * xstride;
  float2 *Yb = Y + b * ystride;
  double acc = 0;
  for (int e = threadIdx.x; e < nr * N0; e += blockDim.x) {
    const int row = e / N0, mx = e - row * N0;
    const long long rr = r0 + row;
    const int mz = (int)(rr / N1), my = (int)(rr - (long long)mz * N1);
    const long long h = rr * N0 + mx;
    float2 u0 = S3[(0 * rows + row) * P + mx], u1 = S3[(1 * rows + row) * P + mx], u2 = S3[(2 * rows + row) * P + mx];
    const float kx = kxs[mx];
    const float ky = (float)(inst[b].kinc[1] + (my - g.n[1]) * g.K[1]);
    const float kz = (float)(inst[b].kinc[2] + (mz - g.n[2]) * g.K[2]);
    const float id = iden[b * Nh + h];
    const float kux = kx * u0.x + ky * u1.x + kz * u2.x, kuy = kx * u0.y + ky * u1.y + kz * u2.y;
    float2 y0 = Xb[h], y1 = Xb[Nh + h], y2 = Xb[2 * Nh + h];
    y0.x -= id * (kb2 * u0.x - kx * kux);
    y0.y -= id * (kb2 * u0.y - kx * kuy);
    y1.x -= id * (kb2 * u1.x - ky * kux);
    y1.y -= id * (kb2 * u1.y - ky * kuy);
    y2.x -= id * (kb2 * u2.x - kz * kux);
    y2.y -= id * (kb2 * u2.y - kz * kuy);
    if (MODE == 1) {
      float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0;
      if (h == h0) {
        a0 = make_float2((float)inst[b].a[0], (float)inst[b].a[1]);
        a1 = make_float2((float)inst[b].a[2], (float)inst[b].a[3]);
        a2 = make_float2((float)inst[b].a[4], (float)inst[b].a[5]);
      }
      y0 = make_float2(a0.x - y0.x, a0.y - y0.y);
      y1 = make_float2(a1.x - y1.x, a1.y - y1.y);
      y2 = make_float2(a2.x - y2.x, a2.y - y2.y);
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

// Dp[r_x][i][c] = D[r_x][freq_y(c)][freq_z(i)]: the multiplier in the
// register order of the z and y transforms.
template <int LY, int LZ>
__global__ void k_d_permute(const float *__restrict__ D, int L0, float *Dp) {
  const long long tot = (long long)L0 * LY * LZ;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % LY);
    const long long t = e / LY;
    const int i = (int)(t % LZ);
    const int rx = (int)(t / LZ);
    Dp[e] = D[((long long)rx * LY + RegFFT<LY>::freq(c)) * LZ + RegFFT<LZ>::freq(i)];
  }
}

bool reg_path_ok(const Geo &g) {
  auto ok = [](int L) { return L == 32 || L == 64; };
  return ok(g.L[0]) && ok(g.L[1]) && ok(g.L[2]);
}

cudaError_t launch_d_permute(const Geo &g, const float *D, float *Dp, cudaStream_t st) {
  const long long tot = (long long)g.L[0] * g.L[1] * g.L[2];
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 148 * 16);
#define GSM_DP(LY, LZ) k_d_permute<LY, LZ><<<blocks, 256, 0, st>>>(D, g.L[0], Dp)
  if (g.L[1] == 64 && g.L[2] == 64) GSM_DP(64, 64);
  else if (g.L[1] == 64) GSM_DP(64, 32);
  else if (g.L[2] == 64) GSM_DP(32, 64);
  else GSM_DP(32, 32);
#undef GSM_DP
  return cudaGetLastError();
}

static int rwarp(int t) { return ((t + 31) / 32) * 32; }

cudaError_t launch_matvec_reg(const MatvecArgs<float> &a, const float *Dp, cudaStream_t st, Profiler *prof) {
  const Geo &g = a.g;
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  // pass 1
  {
    const int planes = std::max(1, RT / N1);
    const int threads = std::max(32, rwarp(std::min(RT, planes * N1)));
    const size_t smem = sizeof(float2) * (size_t)planes * N1 * (N0 + 1);
    dim3 grid((3 * N2 + planes - 1) / planes, a.B);
    if (prof) prof->begin(KIND_FWD_X, st);
    if (g.L[0] == 64) {
      cudaFuncSetAttribute(k_fwd_x_reg<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_fwd_x_reg<64><<<grid, threads, smem, st>>>(g, a.X, a.xstride, a.T, a.scale, a.write_back, a.act, a.tw, planes);
    } else {
      cudaFuncSetAttribute(k_fwd_x_reg<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_fwd_x_reg<32><<<grid, threads, smem, st>>>(g, a.X, a.xstride, a.T, a.scale, a.write_back, a.act, a.tw, planes);
    }
    if (prof) prof->end(KIND_FWD_X, st, (double)a.B * 8.0 * (double)(g.U + g.Tsz));
  }
  // pass 2
  {
    const int PPB = RT / g.L[1];
    const size_t smem = sizeof(float2) * (size_t)PPB * N2 * (g.L[1] + 1);
    dim3 grid((g.L[0] + PPB - 1) / PPB, 3, a.B);
    if (prof) prof->begin(KIND_YZ, st);
#define GSM_YZ(LY, LZ)                                                                                      \
  cudaFuncSetAttribute(k_yz_reg<LY, LZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);           \
  k_yz_reg<LY, LZ><<<grid, RT, smem, st>>>(g, a.T, Dp, a.act, a.tw)
    if (g.L[1] == 64 && g.L[2] == 64) { GSM_YZ(64, 64); }
    else if (g.L[1] == 64) { GSM_YZ(64, 32); }
    else if (g.L[2] == 64) { GSM_YZ(32, 64); }
    else { GSM_YZ(32, 32); }
#undef GSM_YZ
    if (prof) prof->end(KIND_YZ, st, (double)a.B * 16.0 * (double)g.Tsz + 4.0 * (double)g.L[0] * g.L[1] * g.L[2]);
  }
  // pass 3
  {
    const int rows = std::max(1, std::min(RT / 3, N1));
    const int threads = std::max(64, rwarp(3 * rows));
    const size_t smem = sizeof(float2) * 3 * (size_t)rows * (N0 + 1) + sizeof(float) * N0 + 16;
    dim3 grid((int)(((long long)N1 * N2 + rows - 1) / rows), a.B);
    if (prof) prof->begin(KIND_INV_X, st);
#define GSM_P3(L0, M)                                                                                           \
  cudaFuncSetAttribute(k_inv_x_reg<L0, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);            \
  k_inv_x_reg<L0, M><<<grid, threads, smem, st>>>(g, a.T, a.X, a.xstride, a.Y, a.ystride, a.act, a.inst, a.iden, \
                                                  a.tw, rows, a.partial, a.counter, a.norm_out)
    if (g.L[0] == 64) {
      if (a.mode == 1) { GSM_P3(64, 1); } else { GSM_P3(64, 0); }
    } else {
      if (a.mode == 1) { GSM_P3(32, 1); } else { GSM_P3(32, 0); }
    }
#undef GSM_P3
    if (prof) prof->end(KIND_INV_X, st, (double)a.B * (8.0 * (double)(g.Tsz + 2 * g.U) + 4.0 * (double)g.Nh));
  }
  return cudaGetLastError();
}

int matvec_reg_blocks_pass3(const Geo &g) {
  const int rows = std::max(1, std::min(RT / 3, g.N[1]));
  return (int)(((long long)g.N[1] * g.N[2] + rows - 1) / rows);
}

}  // namespace gsm
