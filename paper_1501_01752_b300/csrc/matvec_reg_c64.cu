// Lane-team product (matvec_reg.cuh) instantiated for complex64, with the
// helpers shared by every precision.
#include "matvec_reg.cuh"

namespace gsm {

GSM_EXTERN_REG_PASSES(float)

// Dp[r_x / 2][r_y][r_z] = (D[r_x][r_y][r_z], D[r_x + 1][r_y][r_z])
__global__ void k_pair_d(const float *__restrict__ D, float2 *__restrict__ Dp, long long plane, long long npairs) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npairs * plane;
       i += (long long)gridDim.x * blockDim.x) {
    const long long xp = i / plane, e = i - xp * plane;
    Dp[i] = make_float2(D[(2 * xp) * plane + e], D[(2 * xp + 1) * plane + e]);
  }
}

cudaError_t launch_pair_d(const float *D, float2 *Dp, const Geo &g, cudaStream_t st) {
  const long long plane = (long long)g.L[1] * g.L[2], npairs = g.L[0] / 2;
  k_pair_d<<<148 * 4, 256, 0, st>>>(D, Dp, plane, npairs);
  return cudaGetLastError();
}

bool packed_yz_ok(const Geo &g) { return g.L[1] == 64 && g.L[2] == 64 && g.L[0] % 2 == 0; }

bool reg_path_ok(const Geo &g) {
  auto ok = [](int L) { return L == 32 || L == 64; };
  if (g.L[0] == 128 && g.L[1] == 128 && g.L[2] == 128) return true;   // 16-lane teams, cubic grids only
  return ok(g.L[0]) && ok(g.L[1]) && ok(g.L[2]);
}

int matvec_reg_blocks_pass3(const Geo &g) {
  if (!reg_path_ok(g)) return 1;
  // the smallest block the autotuner may pick, with the fewest items per team
  // (16-byte values): the most blocks any precision launches
  const int rows = p3_rows<double>(g, 128);
  return (int)(((long long)g.N[1] * g.N[2] + rows - 1) / rows);
}

template cudaError_t launch_matvec_reg<float>(const MatvecArgs<float> &, cudaStream_t, Profiler *, const int *);
template cudaError_t launch_reg_pass<float>(int, int, const MatvecArgs<float> &, cudaStream_t);

}  // namespace gsm
