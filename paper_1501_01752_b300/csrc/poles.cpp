// Pole fit of the "Modes in 3D crystals" section (host, FP64):
// Eq. 7 monic pole polynomial, Eq. 8 divided-difference annihilation of
// P(kappa) xi(kappa), Eq. 9 linear system for p_k, QR eigenvalues of the
// companion matrix, Eq. 10 residues.  Readings of the garbled passages:
//  * Eq. 9 is used with xi_i multiplying (the divided difference of P xi),
//    not dividing as printed;
//  * every window of N_d + 1 consecutive points of the equidistant grid
//    gives one row; the M - N_d rows are solved in the least-squares sense;
//  * Eq. 10's product runs over the N_p poles; (P xi)(eta_k) is the Lagrange
//    interpolant over the window whose centre is nearest Re eta_k;
//  * kappa is mapped to t = (kappa - c) / h, c, h the grid centre and
//    half-width, before the divided differences are formed.
// The pole sensitivity d eta / d xi_i linearises the Eq. 6 model around the
// poles that matter in the window (double-pole terms) plus a Chebyshev
// regular part of degree N_d - 2.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace gsm {

using cd = std::complex<double>;

// Least squares min ||A x - b|| for a complex m x n (m >= n) matrix,
// row-major, by Householder QR.  Returns false if rank deficient.
static bool lstsq(std::vector<cd> A, std::vector<cd> b, int m, int n, std::vector<cd> &x) {
  for (int k = 0; k < n; ++k) {
    double norm = 0;
    for (int i = k; i < m; ++i) norm += std::norm(A[i * n + k]);
    norm = std::sqrt(norm);
    if (norm == 0.0) return false;
    const cd akk = A[k * n + k];
    const cd alpha = -(std::abs(akk) > 0 ? akk / std::abs(akk) : cd(1, 0)) * norm;
    std::vector<cd> v(m, 0.0);
    v[k] = akk - alpha;
    for (int i = k + 1; i < m; ++i) v[i] = A[i * n + k];
    double vn = 0;
    for (int i = k; i < m; ++i) vn += std::norm(v[i]);
    if (vn == 0.0) continue;
    for (int j = k; j < n; ++j) {
      cd s = 0;
      for (int i = k; i < m; ++i) s += std::conj(v[i]) * A[i * n + j];
      s = 2.0 * s / vn;
      for (int i = k; i < m; ++i) A[i * n + j] -= s * v[i];
    }
    cd s = 0;
    for (int i = k; i < m; ++i) s += std::conj(v[i]) * b[i];
    s = 2.0 * s / vn;
    for (int i = k; i < m; ++i) b[i] -= s * v[i];
  }
  x.assign(n, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    cd s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
    if (std::abs(A[i * n + i]) == 0.0) return false;
    x[i] = s / A[i * n + i];
  }
  return true;
}

// Eigenvalues of a complex upper Hessenberg matrix (row-major n x n) by the
// single-shift QR algorithm with Wilkinson shifts and deflation.
static bool hessenberg_eig(std::vector<cd> H, int n, std::vector<cd> &ev) {
  ev.assign(n, 0.0);
  int hi = n - 1, iter = 0;
  auto at = [&](int i, int j) -> cd & { return H[i * n + j]; };
  while (hi >= 0) {
    if (hi == 0) { ev[0] = at(0, 0); break; }
    int l = hi;
    while (l > 0) {
      const double sc = std::abs(at(l - 1, l - 1)) + std::abs(at(l, l));
      if (std::abs(at(l, l - 1)) <= 1e-15 * (sc > 0 ? sc : 1.0)) break;
      --l;
    }
    if (l == hi) {
      ev[hi] = at(hi, hi);
      --hi;
      iter = 0;
      continue;
    }
    if (++iter > 200) return false;
    // Wilkinson shift from the trailing 2x2 of the active block
    const cd a = at(hi - 1, hi - 1), bq = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
    const cd tr = 0.5 * (a + d);
    const cd disc = std::sqrt(0.25 * (a - d) * (a - d) + bq * c);
    cd mu = (std::abs(tr + disc - d) < std::abs(tr - disc - d)) ? tr + disc : tr - disc;
    if (iter % 11 == 10) mu = d + std::abs(at(hi, hi - 1));  // exceptional shift
    cd x = at(l, l) - mu, y = at(l + 1, l);
    for (int k = l; k < hi; ++k) {
      const double r = std::sqrt(std::norm(x) + std::norm(y));
      double cs;
      cd sn;
      if (r == 0.0) { cs = 1.0; sn = 0.0; }
      else if (std::abs(x) == 0.0) { cs = 0.0; sn = 1.0; }
      else { cs = std::abs(x) / r; sn = (x / std::abs(x)) * std::conj(y) / r; }
      // rows k, k+1 from the left: G = [c s; -conj(s) c]
      for (int j = std::max(l, k - 1); j <= hi; ++j) {
        const cd p = at(k, j), q = at(k + 1, j);
        at(k, j) = cs * p + sn * q;
        at(k + 1, j) = -std::conj(sn) * p + cs * q;
      }
      // columns k, k+1 from the right: G^H = [c -s; conj(s) c]
      for (int i = l; i <= std::min(hi, k + 2); ++i) {
        const cd p = at(i, k), q = at(i, k + 1);
        at(i, k) = cs * p + std::conj(sn) * q;
        at(i, k + 1) = -sn * p + cs * q;
      }
      if (k < hi - 1) { x = at(k + 1, k); y = at(k + 2, k); }
    }
  }
  return true;
}

static std::vector<double> dd_weights(const double *t, int n) {
  std::vector<double> c(n);
  for (int i = 0; i < n; ++i) {
    double p = 1.0;
    for (int j = 0; j < n; ++j)
      if (j != i) p *= (t[i] - t[j]);
    c[i] = 1.0 / p;
  }
  return c;
}

struct Normal { double c, h; };

static Normal normalise(const double *kappa, int M, std::vector<double> &t) {
  double lo = kappa[0], hi = kappa[0];
  for (int i = 1; i < M; ++i) { lo = std::min(lo, kappa[i]); hi = std::max(hi, kappa[i]); }
  Normal nm{0.5 * (hi + lo), 0.5 * (hi - lo)};
  t.resize(M);
  for (int i = 0; i < M; ++i) t[i] = (kappa[i] - nm.c) / nm.h;
  return nm;
}

// Returns 0 on success, 1 on bad arguments, 2 on numerical failure.
int fit_poles(int M, const double *kappa, const cd *xi, int Np, int Nd, cd *eta, cd *zeta) {
  if (Np < 1 || Nd <= Np || M < Nd + Np) return 1;
  std::vector<double> t;
  const Normal nm = normalise(kappa, M, t);
  if (!(nm.h > 0)) return 1;
  const int S = M - Nd;
  std::vector<cd> A((size_t)S * Np), rhs(S);
  for (int w = 0; w < S; ++w) {
    const std::vector<double> c = dd_weights(&t[w], Nd + 1);
    for (int k = 0; k <= Np; ++k) {
      cd s = 0;
      for (int i = 0; i <= Nd; ++i) s += std::pow(t[w + i], k) * xi[w + i] * c[i];
      if (k < Np) A[(size_t)w * Np + k] = s;
      else rhs[w] = -s;
    }
  }
  std::vector<cd> p;
  if (!lstsq(A, rhs, S, Np, p)) return 2;
  // companion matrix of t^Np + sum p_k t^k (upper Hessenberg)
  std::vector<cd> C((size_t)Np * Np, 0.0);
  for (int i = 1; i < Np; ++i) C[(size_t)i * Np + i - 1] = 1.0;
  for (int i = 0; i < Np; ++i) C[(size_t)i * Np + Np - 1] = -p[i];
  std::vector<cd> tau;
  if (!hessenberg_eig(C, Np, tau)) return 2;
  for (int k = 0; k < Np; ++k) {
    int best = 0;
    double bd = 1e300;
    for (int w = 0; w < S; ++w) {
      const double dist = std::fabs(t[w + Nd / 2] - tau[k].real());
      if (dist < bd) { bd = dist; best = w; }
    }
    const double *tw = &t[best];
    cd pxi = 0;
    for (int i = 0; i <= Nd; ++i) {
      cd P = 1.0, Li = 1.0;
      for (int j = 0; j < Np; ++j) P *= (tw[i] - tau[j]);
      for (int j = 0; j <= Nd; ++j)
        if (j != i) Li *= (tau[k] - tw[j]) / (tw[i] - tw[j]);
      pxi += P * xi[best + i] * Li;
    }
    cd dP = 1.0;
    for (int j = 0; j < Np; ++j)
      if (j != k) dP *= (tau[k] - tau[j]);
    eta[k] = nm.c + nm.h * tau[k];
    zeta[k] = nm.h * pxi / dP;
  }
  return 0;
}

int select_pole(int Np, const cd *eta, const cd *zeta, double lo, double hi) {
  int best = -1;
  for (int j = 0; j < Np; ++j)
    if (eta[j].real() >= lo && eta[j].real() <= hi && (best < 0 || std::abs(zeta[j]) > std::abs(zeta[best]))) best = j;
  return best;
}

// w[i] = d eta_index / d xi_i (holomorphic; d/d Im xi_i = i w[i]).
int pole_sensitivity(int M, const double *kappa, const cd *eta, const cd *zeta, int Np, int Nd, int index, cd *w) {
  std::vector<double> t;
  const Normal nm = normalise(kappa, M, t);
  std::vector<cd> tau(Np), zt(Np);
  double zmax = 0;
  for (int j = 0; j < Np; ++j) {
    tau[j] = (eta[j] - nm.c) / nm.h;
    zt[j] = zeta[j] / nm.h;
    zmax = std::max(zmax, std::abs(zt[j]));
  }
  std::vector<int> cand;
  for (int j = 0; j < Np; ++j)
    if (j != index && std::abs(zt[j]) > 1e-8 * zmax && std::fabs(tau[j].real()) <= 1.5) cand.push_back(j);
  std::sort(cand.begin(), cand.end(),
            [&](int a, int b) { return std::abs(tau[a] - tau[index]) < std::abs(tau[b] - tau[index]); });
  std::vector<int> expl{index};
  const int extra = std::max(0, (M - Nd) / 2 - 1);
  for (int q = 0; q < (int)cand.size() && q < extra; ++q) expl.push_back(cand[q]);
  const int ncol = 2 * (int)expl.size() + (Nd - 1);
  std::vector<cd> J((size_t)M * ncol);
  for (int i = 0; i < M; ++i) {
    int c = 0;
    for (int j : expl) {
      const cd d = t[i] - tau[j];
      J[(size_t)i * ncol + c++] = 1.0 / d;
      J[(size_t)i * ncol + c++] = zt[j] / (d * d);
    }
    const double th = std::acos(std::max(-1.0, std::min(1.0, t[i])));
    for (int l = 0; l < Nd - 1; ++l) J[(size_t)i * ncol + c++] = std::cos(l * th);
  }
  // row 1 of pinv(J): w_i = conj((J u)_i), u = (J^H J)^-1 e_1
  std::vector<cd> G((size_t)ncol * ncol, 0.0), u(ncol, 0.0);
  for (int a = 0; a < ncol; ++a)
    for (int b = 0; b < ncol; ++b) {
      cd s = 0;
      for (int i = 0; i < M; ++i) s += std::conj(J[(size_t)i * ncol + a]) * J[(size_t)i * ncol + b];
      G[(size_t)a * ncol + b] = s;
    }
  std::vector<cd> e1(ncol, 0.0);
  e1[1] = 1.0;
  if (!lstsq(G, e1, ncol, ncol, u)) return 2;
  for (int i = 0; i < M; ++i) {
    cd s = 0;
    for (int c = 0; c < ncol; ++c) s += J[(size_t)i * ncol + c] * u[c];
    w[i] = std::conj(s) * nm.h;
  }
  return 0;
}

}  // namespace gsm
