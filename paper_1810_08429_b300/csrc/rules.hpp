// Quadrature rules handed to the kernels by value.
//
//  * the 7-point degree-5 triangle rule (centroid plus two symmetric orbits
//    of three points; coordinates and weights involve sqrt(15)) used for
//    every regular integral over a triangle,
//  * Gauss-Legendre on [-1, 1] with m points for the faces of the box omega
//    (the quadrature of Eq. (2)),
//  * Gauss-Legendre on [0, 1] with q points for the Sauter-Schwab rules.
//
// Gauss-Legendre nodes are the roots of P_q found by Newton's method on the
// three-term recurrence, weights 2 / ((1 - x^2) P_q'(x)^2).
#pragma once

#include <cmath>

#include "gca.h"

namespace gca {

struct Rules {
  double bary[7][3];
  double w7[7];
  double box_t[GCA_MAX_BOX_M];
  double box_w[GCA_MAX_BOX_M];
  double ss_t[GCA_MAX_SAUTER_Q];
  double ss_w[GCA_MAX_SAUTER_Q];
  int m;
  int q;
};

inline void gauss_legendre(int q, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < q; ++i) {
    // i-th root from the top, refined by Newton's method
    double z = std::cos(pi * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int l = 2; l <= q; ++l) {
        double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
        p0 = p1;
        p1 = p2;
      }
      double pq = (q == 1) ? z : p1;
      double pq1 = (q == 1) ? 1.0 : p0;
      dp = q * (z * pq - pq1) / (z * z - 1.0);
      double dz = pq / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int l = 2; l <= q; ++l) {
        double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
        p0 = p1;
        p1 = p2;
      }
      double pq = (q == 1) ? z : p1;
      double pq1 = (q == 1) ? 1.0 : p0;
      dp = q * (z * pq - pq1) / (z * z - 1.0);
    }
    // ascending order
    x[q - 1 - i] = z;
    w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

inline Rules make_rules(int m, int q) {
  Rules r{};
  const double s15 = std::sqrt(15.0);
  const double a1 = (6.0 - s15) / 21.0, b1 = 1.0 - 2.0 * a1;
  const double a2 = (6.0 + s15) / 21.0, b2 = 1.0 - 2.0 * a2;
  const double third = 1.0 / 3.0;
  const double pts[7][3] = {{third, third, third}, {b1, a1, a1}, {a1, b1, a1}, {a1, a1, b1},
                            {b2, a2, a2},          {a2, b2, a2}, {a2, a2, b2}};
  const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
  const double wts[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
  for (int i = 0; i < 7; ++i) {
    for (int j = 0; j < 3; ++j) r.bary[i][j] = pts[i][j];
    r.w7[i] = wts[i];
  }
  r.m = m;
  r.q = q;
  gauss_legendre(m, r.box_t, r.box_w);
  double t[GCA_MAX_SAUTER_Q], w[GCA_MAX_SAUTER_Q];
  gauss_legendre(q, t, w);
  for (int i = 0; i < q; ++i) {
    r.ss_t[i] = 0.5 * (t[i] + 1.0);
    r.ss_w[i] = 0.5 * w[i];
  }
  return r;
}

}  // namespace gca
