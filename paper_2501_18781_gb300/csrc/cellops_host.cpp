// 1D tables of the Q2/Q1 elements at the 3-point Gauss rule, from closed forms.
#include <cmath>

#include "cellops.cuh"

namespace mf {

Tables make_tables() {
  Tables t{};
  const double r = std::sqrt(15.0) / 10.0;
  const double g[3] = {0.5 - r, 0.5, 0.5 + r};
  const double w[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  for (int q = 0; q < 3; ++q) {
    const double x = g[q];
    // quadratic Lagrange basis on nodes 0, 1/2, 1 and its derivative
    const double l[3] = {2.0 * (x - 0.5) * (x - 1.0), -4.0 * x * (x - 1.0), 2.0 * x * (x - 0.5)};
    const double dl[3] = {4.0 * x - 3.0, 4.0 - 8.0 * x, 4.0 * x - 1.0};
    for (int a = 0; a < 3; ++a) {
      t.S[3 * q + a] = l[a];
      t.Sp[3 * q + a] = dl[a];
      t.SS[3 * q + a] = l[a] * l[a];
      t.SSp[3 * q + a] = l[a] * dl[a];
      t.SpSp[3 * q + a] = dl[a] * dl[a];
    }
    // derivative of the Lagrange polynomials through the Gauss points, at g_q
    for (int p = 0; p < 3; ++p) {
      double d = 0.0;
      for (int m = 0; m < 3; ++m) {
        if (m == p) continue;
        double term = 1.0 / (g[p] - g[m]);
        for (int b = 0; b < 3; ++b)
          if (b != p && b != m) term *= (x - g[b]) / (g[p] - g[b]);
        d += term;
      }
      t.D[3 * q + p] = d;
    }
    t.W[q] = w[q];
    t.G[q] = g[q];
    t.P[2 * q] = 1.0 - x;
    t.P[2 * q + 1] = x;
    t.PP[2 * q] = (1.0 - x) * (1.0 - x);
    t.PP[2 * q + 1] = x * x;
    t.PpPp[2 * q] = 1.0;
    t.PpPp[2 * q + 1] = 1.0;
  }
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) {
        const int q = a + 3 * b + 9 * c;
        t.W3[q] = w[a] * w[b] * w[c];
        for (int n = 0; n < 8; ++n)
          t.PW[8 * q + n] = t.P[2 * a + (n & 1)] * t.P[2 * b + ((n >> 1) & 1)] * t.P[2 * c + (n >> 2)];
        for (int n = 0; n < 8; ++n) t.PWW[8 * q + n] = t.W3[q] * t.PW[8 * q + n];
      }
  return t;
}

}  // namespace mf
