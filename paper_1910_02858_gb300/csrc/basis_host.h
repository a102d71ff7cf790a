// Host construction of the 1-D DGSEM operators (Sec. 3.1): Legendre-Gauss and
// Gauss-Lobatto nodes/weights, the differentiation matrix D_rs = l_s'(xi_r),
// Lagrange interpolation matrices, l(+-1), and the weak-form operators
// Dhat_ij = -(w_j/w_i) D_ji, lhat = l/w (the operators after Eq. semiDiscrete;
// Dhat in the orientation for which a constant flux has zero divergence).
#pragma once
#include <cmath>
#include <vector>

namespace flexi {
namespace host {

// P_N(x) and P_N'(x) by the Bonnet recurrence
inline void legendre(int N, double x, double& p, double& dp) {
  if (N == 0) { p = 1.0; dp = 0.0; return; }
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  for (int k = 2; k <= N; ++k) {
    const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    const double d2 = d0 + (2.0 * k - 1.0) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  p = p1; dp = d1;
}

// N+1 Gauss nodes (roots of P_{N+1}) and weights, ascending
inline void gauss(int N, std::vector<double>& x, std::vector<double>& w) {
  const int n = N + 1;
  x.assign(n, 0.0); w.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    double xi = -std::cos(M_PI * (2.0 * j + 1.0) / (2.0 * n));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, xi, p, dp);
      const double dx = p / dp;
      xi -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double p, dp;
    legendre(n, xi, p, dp);
    x[j] = xi;
    w[j] = 2.0 / ((1.0 - xi * xi) * dp * dp);
  }
}

// N+1 Gauss-Lobatto nodes (+-1 and the roots of P_N') and weights, ascending
inline void lobatto(int N, std::vector<double>& x, std::vector<double>& w) {
  x.assign(N + 1, 0.0); w.assign(N + 1, 0.0);
  x[0] = -1.0; x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double xi = -std::cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(N, xi, p, dp);
      const double ddp = (2.0 * xi * dp - N * (N + 1.0) * p) / (1.0 - xi * xi);
      const double dx = dp / ddp;
      xi -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    x[j] = xi;
  }
  for (int j = 0; j <= N; ++j) {
    double p, dp;
    legendre(N, x[j], p, dp);
    w[j] = 2.0 / (N * (N + 1.0) * p * p);
  }
}

inline std::vector<double> bary_weights(const std::vector<double>& x) {
  const int n = (int)x.size();
  std::vector<double> b(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) b[j] /= (x[j] - x[k]);
  return b;
}

// D[r*n+s] = l_s'(x_r), barycentric form with negative-sum diagonal
inline std::vector<double> diff_matrix(const std::vector<double>& x) {
  const int n = (int)x.size();
  const std::vector<double> b = bary_weights(x);
  std::vector<double> D(n * n, 0.0);
  for (int r = 0; r < n; ++r) {
    double s = 0.0;
    for (int c = 0; c < n; ++c)
      if (c != r) {
        D[r * n + c] = (b[c] / b[r]) / (x[r] - x[c]);
        s += D[r * n + c];
      }
    D[r * n + r] = -s;
  }
  return D;
}

// V[r*nfrom + j] = l_j(xto[r]) on the nodes xfrom (product form)
inline std::vector<double> interp_matrix(const std::vector<double>& xfrom, const std::vector<double>& xto) {
  const int nf = (int)xfrom.size(), nt = (int)xto.size();
  std::vector<double> V(nt * nf, 1.0);
  for (int r = 0; r < nt; ++r)
    for (int j = 0; j < nf; ++j)
      for (int k = 0; k < nf; ++k)
        if (k != j) V[r * nf + j] *= (xto[r] - xfrom[k]) / (xfrom[j] - xfrom[k]);
  return V;
}

}  // namespace host
}  // namespace flexi
