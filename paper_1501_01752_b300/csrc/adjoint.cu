// Gradient of a real objective with respect to voxel permittivities through
// the Eq. 4 solve (the paper has no adjoint; this is the calculus of Eq. 4).
//
// With A = I - G T(Delta), A E = b and A^H lambda = g (g the objective's
// gradient with respect to E at m = 0), dL = Re sum_d C_d dDelta_d with
//   C_d = sum_{m - m' = d} sum_c conj(mu_{c m}) E_{c m'},   mu = G lambda
// (G is real symmetric for real k and k_b^2).  On the L grid,
//   C_d = L^-3 sum_r conj(F_mu(r)) . F_E(r) exp(2 pi i d.r / L),
// F(r) = sum_m f_m exp(2 pi i m.r / L), exact for |d| <= 2n because L >= 4n+1.
// A voxel grid gives Delta_d = (sum_v eps_v phi_v(d) - eps_b delta_d0)/eps_b,
//   phi_v(d) = prod_a M_a^-1 exp(-2 pi i d_a (v_a + 1/2) / M_a) sinc(pi d_a / M_a),
// so dL/d eps_v = Re( M^-3 eps_b^-1 sum_d C_d w(d) exp(-2 pi i d.v / M) ),
//   w(d) = prod_a sinc(pi d_a / M_a) exp(-i pi d_a / M_a):
// one more FFT on the voxel grid after folding d onto it modulo M.
#include "kernels.h"

namespace gsm {

__device__ __forceinline__ long long grid_pos(const Geo &g, int mx, int my, int mz) {
  const int rx = wrap(mx, g.n[0], g.L[0]), ry = wrap(my, g.n[1], g.L[1]), rz = wrap(mz, g.n[2], g.L[2]);
  return ((long long)rz * g.L[1] + ry) * g.L[0] + rx;
}

// grid[0..2] = G lambda, grid[3..5] = E on the L^3 grid (zero elsewhere)
__global__ void k_adj_scatter(Geo g, const double2 *__restrict__ lam, const double2 *__restrict__ E,
                              const Inst *__restrict__ inst, const double *__restrict__ iden, double2 *grid) {
  const long long LL = (long long)g.L[0] * g.L[1] * g.L[2];
  for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h < g.Nh; h += (long long)gridDim.x * blockDim.x) {
    const int mx = (int)(h % g.N[0]);
    const int my = (int)((h / g.N[0]) % g.N[1]);
    const int mz = (int)(h / ((long long)g.N[0] * g.N[1]));
    const double kx = inst->kinc[0] + (mx - g.n[0]) * g.K[0];
    const double ky = inst->kinc[1] + (my - g.n[1]) * g.K[1];
    const double kz = inst->kinc[2] + (mz - g.n[2]) * g.K[2];
    const double2 l0 = lam[h], l1 = lam[g.Nh + h], l2 = lam[2 * g.Nh + h];
    const double2 kl = mk(kx * l0.x + ky * l1.x + kz * l2.x, kx * l0.y + ky * l1.y + kz * l2.y);
    const double id = iden[h], kb2 = inst->kb2;
    const long long r = grid_pos(g, mx, my, mz);
    grid[r] = mk(id * (kb2 * l0.x - kx * kl.x), id * (kb2 * l0.y - kx * kl.y));
    grid[LL + r] = mk(id * (kb2 * l1.x - ky * kl.x), id * (kb2 * l1.y - ky * kl.y));
    grid[2 * LL + r] = mk(id * (kb2 * l2.x - kz * kl.x), id * (kb2 * l2.y - kz * kl.y));
    grid[3 * LL + r] = E[h];
    grid[4 * LL + r] = E[g.Nh + h];
    grid[5 * LL + r] = E[2 * g.Nh + h];
  }
}

__global__ void k_adj_accum(const double2 *__restrict__ grid, long long LL, double2 *P) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < LL; r += (long long)gridDim.x * blockDim.x) {
    double2 s = P[r];
    for (int c = 0; c < 3; ++c) s = cadd(s, cmulc(grid[c * LL + r], grid[(3 + c) * LL + r]));
    P[r] = s;
  }
}

__device__ __forceinline__ double sincd(double u) { return u == 0.0 ? 1.0 : sin(u) / u; }

// Q[t] = sum_{d = t mod M, |d_a| <= 2 n_a} (P(d)/L^3) w(d)
__global__ void k_adj_fold(const double2 *__restrict__ P, Geo g, int M0, int M1, int M2, double2 *Q) {
  const long long MM = (long long)M0 * M1 * M2;
  const double invLL = 1.0 / ((double)g.L[0] * g.L[1] * g.L[2]);
  const int D0 = 2 * g.n[0], D1 = 2 * g.n[1], D2 = 2 * g.n[2];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < MM; t += (long long)gridDim.x * blockDim.x) {
    const int tx = (int)(t % M0), ty = (int)((t / M0) % M1), tz = (int)(t / ((long long)M0 * M1));
    double2 s = mk(0.0, 0.0);
    for (int dz = tz - ((tz + D2) / M2) * M2; dz <= D2; dz += M2) {
      const double wz = sincd(M_PI * dz / M2);
      for (int dy = ty - ((ty + D1) / M1) * M1; dy <= D1; dy += M1) {
        const double wy = sincd(M_PI * dy / M1);
        for (int dx = tx - ((tx + D0) / M0) * M0; dx <= D0; dx += M0) {
          const double wx = sincd(M_PI * dx / M0);
          const double ph = -M_PI * ((double)dx / M0 + (double)dy / M1 + (double)dz / M2);
          double sn, cs;
          sincos(ph, &sn, &cs);
          const double w = wx * wy * wz;
          const long long r = ((long long)((dz + g.L[2]) % g.L[2]) * g.L[1] + (dy + g.L[1]) % g.L[1]) * g.L[0] +
                              (dx + g.L[0]) % g.L[0];
          const double2 c = P[r];
          s.x += w * invLL * (c.x * cs - c.y * sn);
          s.y += w * invLL * (c.x * sn + c.y * cs);
        }
      }
    }
    Q[t] = s;
  }
}

__global__ void k_adj_real(const double2 *__restrict__ Q, long long n, double scale, double *out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = Q[t].x * scale;
}

static int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 148 * 16); }

cudaError_t launch_adj_scatter(const Geo &g, const double2 *lam, const double2 *E, const Inst *inst, const double *iden,
                               double2 *grid, cudaStream_t st) {
  k_adj_scatter<<<blocks_for(g.Nh), 256, 0, st>>>(g, lam, E, inst, iden, grid);
  return cudaGetLastError();
}
cudaError_t launch_adj_accum(const double2 *grid, long long LL, double2 *P, cudaStream_t st) {
  k_adj_accum<<<blocks_for(LL), 256, 0, st>>>(grid, LL, P);
  return cudaGetLastError();
}
cudaError_t launch_adj_fold(const double2 *P, const Geo &g, const int M[3], double2 *Q, cudaStream_t st) {
  k_adj_fold<<<blocks_for((long long)M[0] * M[1] * M[2]), 256, 0, st>>>(P, g, M[0], M[1], M[2], Q);
  return cudaGetLastError();
}
cudaError_t launch_adj_real(const double2 *Q, long long n, double scale, double *out, cudaStream_t st) {
  k_adj_real<<<blocks_for(n), 256, 0, st>>>(Q, n, scale, out);
  return cudaGetLastError();
}

}  // namespace gsm
