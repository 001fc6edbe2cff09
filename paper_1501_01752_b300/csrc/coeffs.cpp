// Analytic Fourier coefficients of the unit-cell permittivity (host, FP64).
//
// The paper never samples eps(r): it combines exact Fourier images of simple
// shapes ("Calculation details", first paragraph).  With
// eps(r) = sum_m eps_m exp(i K_m . r) and eps_m = V^-1 \int_cell eps e^{-i K_m.r}:
//   ball of radius R:      f * 3 (sin x - x cos x) / x^3,   x = |K_m| R
//   box of sides s:        f * prod_a sin(K_a m_a s_a / 2) / (K_a m_a s_a / 2)
//   ellipsoid (a, b, c):   the ball image at x = |(K_x m_x a, K_y m_y b, K_z m_z c)|
// (f = shape volume / cell volume) times exp(-i K_m . c) for a shape centred
// at c, and (eps_shape - eps_host) as weight.  A voxel grid is integrated
// exactly voxel by voxel; its coefficient factorises per axis into
// M^-1 exp(-2 pi i d (v + 1/2) / M) sinc(pi d / M).
#include <cmath>
#include <complex>
#include <vector>

#include "../../include/gsm.h"

namespace gsm {

using cd = std::complex<double>;

static double ball(double x) {
  if (std::fabs(x) < 1e-2) {
    const double x2 = x * x;
    return 1.0 - x2 / 10.0 + x2 * x2 / 280.0;
  }
  return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}

static double sinc(double u) { return u == 0.0 ? 1.0 : std::sin(u) / u; }

// out[(dz + D2) * (2 D1 + 1) (2 D0 + 1) + (dy + D1) * (2 D0 + 1) + dx + D0]
void shapes_coefficients(cd eps_host, const gsm_shape *shapes, int n, const double period[3], const int D[3],
                         std::vector<cd> &out) {
  const int W0 = 2 * D[0] + 1, W1 = 2 * D[1] + 1, W2 = 2 * D[2] + 1;
  out.assign((size_t)W0 * W1 * W2, cd(0.0, 0.0));
  const double V = period[0] * period[1] * period[2];
  const double K[3] = {2 * M_PI / period[0], 2 * M_PI / period[1], 2 * M_PI / period[2]};
  out[((size_t)D[2] * W1 + D[1]) * W0 + D[0]] += eps_host;
  for (int s = 0; s < n; ++s) {
    const gsm_shape &sh = shapes[s];
    const cd w = cd(sh.eps[0], sh.eps[1]) - eps_host;
    double f = 0;
    if (sh.kind == GSM_SPHERE) f = 4.0 * M_PI * sh.size[0] * sh.size[0] * sh.size[0] / (3.0 * V);
    else if (sh.kind == GSM_BOX) f = sh.size[0] * sh.size[1] * sh.size[2] / V;
    else f = 4.0 * M_PI * sh.size[0] * sh.size[1] * sh.size[2] / (3.0 * V);
    for (int dz = -D[2]; dz <= D[2]; ++dz) {
      const double gz = dz * K[2];
      for (int dy = -D[1]; dy <= D[1]; ++dy) {
        const double gy = dy * K[1];
        for (int dx = -D[0]; dx <= D[0]; ++dx) {
          const double gx = dx * K[0];
          double img;
          if (sh.kind == GSM_SPHERE) img = ball(std::sqrt(gx * gx + gy * gy + gz * gz) * sh.size[0]);
          else if (sh.kind == GSM_BOX)
            img = sinc(0.5 * gx * sh.size[0]) * sinc(0.5 * gy * sh.size[1]) * sinc(0.5 * gz * sh.size[2]);
          else {
            const double ax = gx * sh.size[0], ay = gy * sh.size[1], az = gz * sh.size[2];
            img = ball(std::sqrt(ax * ax + ay * ay + az * az));
          }
          const double ph = -(gx * sh.center[0] + gy * sh.center[1] + gz * sh.center[2]);
          out[((size_t)(dz + D[2]) * W1 + dy + D[1]) * W0 + dx + D[0]] += w * f * img * cd(std::cos(ph), std::sin(ph));
        }
      }
    }
  }
}

// voxels[(vz * M1 + vy) * M0 + vx], real; same output layout as above
void voxel_coefficients(const double *vox, const int M[3], const int D[3], std::vector<cd> &out) {
  const int W0 = 2 * D[0] + 1, W1 = 2 * D[1] + 1, W2 = 2 * D[2] + 1;
  auto factor = [](int Dm, int Mm) {
    std::vector<cd> f((size_t)(2 * Dm + 1) * Mm);
    for (int d = -Dm; d <= Dm; ++d)
      for (int v = 0; v < Mm; ++v) {
        const double ph = -2.0 * M_PI * d * (v + 0.5) / Mm;
        f[(size_t)(d + Dm) * Mm + v] = cd(std::cos(ph), std::sin(ph)) * sinc(M_PI * d / Mm) / (double)Mm;
      }
    return f;
  };
  const std::vector<cd> fx = factor(D[0], M[0]), fy = factor(D[1], M[1]), fz = factor(D[2], M[2]);
  // contract x: t1[vz][vy][dx]
  std::vector<cd> t1((size_t)M[2] * M[1] * W0);
  for (int vz = 0; vz < M[2]; ++vz)
    for (int vy = 0; vy < M[1]; ++vy) {
      const double *row = vox + ((size_t)vz * M[1] + vy) * M[0];
      for (int dx = 0; dx < W0; ++dx) {
        cd s = 0;
        const cd *f = &fx[(size_t)dx * M[0]];
        for (int vx = 0; vx < M[0]; ++vx) s += row[vx] * f[vx];
        t1[((size_t)vz * M[1] + vy) * W0 + dx] = s;
      }
    }
  // contract y: t2[vz][dy][dx]
  std::vector<cd> t2((size_t)M[2] * W1 * W0, cd(0, 0));
  for (int vz = 0; vz < M[2]; ++vz)
    for (int dy = 0; dy < W1; ++dy) {
      cd *o = &t2[((size_t)vz * W1 + dy) * W0];
      for (int vy = 0; vy < M[1]; ++vy) {
        const cd f = fy[(size_t)dy * M[1] + vy];
        const cd *in = &t1[((size_t)vz * M[1] + vy) * W0];
        for (int dx = 0; dx < W0; ++dx) o[dx] += f * in[dx];
      }
    }
  // contract z
  out.assign((size_t)W2 * W1 * W0, cd(0, 0));
  for (int dz = 0; dz < W2; ++dz)
    for (int vz = 0; vz < M[2]; ++vz) {
      const cd f = fz[(size_t)dz * M[2] + vz];
      const cd *in = &t2[(size_t)vz * W1 * W0];
      cd *o = &out[(size_t)dz * W1 * W0];
      for (size_t i = 0; i < (size_t)W1 * W0; ++i) o[i] += f * in[i];
    }
}

}  // namespace gsm
