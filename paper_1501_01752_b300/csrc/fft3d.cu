// Full (unpruned) FP64 FFTs along one axis of [L_z][L_y][L_x] arrays, used
// off the hot path: building the convolution multiplier D(r) from the
// Toeplitz generator once per structure, and the correlation and voxel
// chain of the adjoint gradient.
#include "fft.cuh"
#include "kernels.h"

namespace gsm {

template <int S>
__global__ void __launch_bounds__(256) k_fft_axis(double2 *data, int Lx, int Ly, int Lz, int axis, int Ln, long long bstride, int nl,
                           const double2 *__restrict__ twg) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  double2 *tw = reinterpret_cast<double2 *>(sm_raw);
  double2 *Sm = tw + TWN;
  load_twiddles(tw, twg);
  const int L = Ln, P = L + 1;
  const long long nlines = axis == 0 ? (long long)Ly * Lz : (axis == 1 ? (long long)Lz * Lx : (long long)Ly * Lx);
  const long long stride = axis == 0 ? 1 : (axis == 1 ? Lx : (long long)Lx * Ly);
  double2 *d = data + blockIdx.y * bstride;
  const long long l0 = (long long)blockIdx.x * nl;
  const long long left = nlines - l0;
  const int cnt = (int)(left < nl ? left : nl);
  auto base = [&](long long line) -> long long {
    if (axis == 0) return line * Lx;
    if (axis == 1) return (line / Lx) * (long long)Lx * Ly + line % Lx;
    return line;
  };
  for (int e = threadIdx.x; e < cnt * L; e += blockDim.x) {
    int l, i;
    if (axis == 0) { l = e / L; i = e - l * L; }
    else { i = e / cnt; l = e - i * cnt; }
    Sm[l * P + i] = d[base(l0 + l) + i * stride];
  }
  __syncthreads();
  Team tm(L);
  for (int l = tm.id; l < cnt; l += tm.count) team_fft<S>(Sm + l * P, L, tm.lane, tm.ts, tm.mask, tw);
  __syncthreads();
  for (int e = threadIdx.x; e < cnt * L; e += blockDim.x) {
    int l, i;
    if (axis == 0) { l = e / L; i = e - l * L; }
    else { i = e / cnt; l = e - i * cnt; }
    d[base(l0 + l) + i * stride] = Sm[l * P + i];
  }
}

cudaError_t launch_fft_axis(double2 *data, int Lx, int Ly, int Lz, int axis, int sign, int batch,
                            long long batch_stride, const double2 *tw, cudaStream_t st) {
  const int L = axis == 0 ? Lx : (axis == 1 ? Ly : Lz);
  if (L == 1) return cudaSuccess;
  const long long nlines = axis == 0 ? (long long)Ly * Lz : (axis == 1 ? (long long)Lz * Lx : (long long)Ly * Lx);
  int nl = std::max(1, 4096 / L);
  const int ts = L >= 8 ? L / 8 : 1;
  const int threads = std::min(256, std::max(64, ((nl * ts + 31) / 32) * 32));
  nl = std::min(nl, threads / ts);
  const size_t smem = sizeof(double2) * (TWN + (size_t)nl * (L + 1));
  dim3 grid((unsigned)((nlines + nl - 1) / nl), batch);
  if (sign > 0) {
    cudaFuncSetAttribute(k_fft_axis<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_fft_axis<1><<<grid, threads, smem, st>>>(data, Lx, Ly, Lz, axis, L, batch_stride, nl, tw);
  } else {
    cudaFuncSetAttribute(k_fft_axis<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_fft_axis<-1><<<grid, threads, smem, st>>>(data, Lx, Ly, Lz, axis, L, batch_stride, nl, tw);
  }
  return cudaGetLastError();
}

// D(r) from the transformed generator: real part, scaled by 1/(L_x L_y L_z),
// transposed from [z][y][x] to the [x][y][z] order the yz pass reads.
__global__ void k_d_finalize(const double2 *__restrict__ Dc, Geo g, double scale, double *D64, float *D32) {
  const long long tot = (long long)g.L[0] * g.L[1] * g.L[2];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int rz = (int)(e % g.L[2]);
    const long long t = e / g.L[2];
    const int ry = (int)(t % g.L[1]);
    const int rx = (int)(t / g.L[1]);
    const double v = Dc[((long long)rz * g.L[1] + ry) * g.L[0] + rx].x * scale;
    D64[e] = v;
    D32[e] = (float)v;
  }
}

cudaError_t launch_d_finalize(const double2 *Dc, const Geo &g, double scale, double *D64, float *D32,
                              cudaStream_t st) {
  const long long tot = (long long)g.L[0] * g.L[1] * g.L[2];
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 148 * 16);
  k_d_finalize<<<blocks, 256, 0, st>>>(Dc, g, scale, D64, D32);
  return cudaGetLastError();
}

}  // namespace gsm
