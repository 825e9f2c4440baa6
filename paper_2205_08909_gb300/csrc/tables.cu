// Host-side 1D tables of the Q_p basis (Sec. 2, Eq. 2): Gauss-Lobatto nodes
// (nodes of the Lagrange basis), the (p+1)-point Gauss rule (quadrature of
// Eq. 5), basis values and derivatives at the Gauss points, the Gauss
// collocation derivative and the 1D reference mass and stiffness matrices.
// All in FP64, computed by Newton's method on the Legendre recurrence.
#include <cmath>

#include "mfcg_internal.h"

namespace mfcg {

namespace {

// Legendre P_n and P_n' at x in [-1,1] by the three-term recurrence
void legendre(int n, double x, double& P, double& dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    P = 1.0;
    dP = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  dP = n * (x * p1 - p0) / (x * x - 1.0);
}

}  // namespace

// n Gauss points and weights on [0,1]
void gauss_rule_01(int n, double* x01, double* w01) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double x = std::cos(pi * (i + 0.75) / (n + 0.5));
    double P, dP;
    for (int it = 0; it < 100; ++it) {
      legendre(n, x, P, dP);
      const double dx = P / dP;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    legendre(n, x, P, dP);
    const double w = 2.0 / ((1.0 - x * x) * dP * dP);
    // ascending order on [0,1]
    x01[n - 1 - i] = 0.5 * (x + 1.0);
    w01[n - 1 - i] = 0.5 * w;
  }
}

// p+1 Gauss-Lobatto points on [0,1]: ends and the roots of P_p'
void gauss_lobatto_01(int p, double* x01) {
  const double pi = 3.14159265358979323846;
  x01[0] = 0.0;
  x01[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double x = -std::cos(pi * i / p);  // Chebyshev-Lobatto start, ascending
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, x, P, dP);
      // (1-x^2) P'' = 2x P' - p(p+1) P  (Legendre equation)
      const double d2P = (2.0 * x * dP - p * (p + 1.0) * P) / (1.0 - x * x);
      const double dx = dP / d2P;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    x01[i] = 0.5 * (x + 1.0);
  }
}

// value and derivative of the Lagrange polynomial j on nodes[0..m) at x
void lagrange_eval(const double* nodes, int m, int j, double x, double& val, double& der) {
  val = 1.0;
  der = 0.0;
  for (int k = 0; k < m; ++k) {
    if (k == j) continue;
    const double f = 1.0 / (nodes[j] - nodes[k]);
    der = der * (x - nodes[k]) * f + val * f;
    val *= (x - nodes[k]) * f;
  }
}

// Fills the 1D matrices of OperatorCoeffs for degree p and cell sizes h.
void build_coeffs(int p, const double h[3], double amplitude, int coef, OperatorCoeffs& c) {
  const int n1 = p + 1;
  double nodes[kMaxDegree + 1], g[kMaxDegree + 1], w[kMaxDegree + 1];
  gauss_lobatto_01(p, nodes);
  gauss_rule_01(n1, g, w);
  double S[(kMaxDegree + 1) * (kMaxDegree + 1)], D[(kMaxDegree + 1) * (kMaxDegree + 1)];
  for (int q = 0; q < n1; ++q)
    for (int a = 0; a < n1; ++a) lagrange_eval(nodes, n1, a, g[q], S[q * n1 + a], D[q * n1 + a]);
  // Gauss collocation derivative: Dc[q][q'] = L^G_{q'}'(g_q)
  double Dc[(kMaxDegree + 1) * (kMaxDegree + 1)];
  for (int q = 0; q < n1; ++q)
    for (int r = 0; r < n1; ++r) {
      double v, d;
      lagrange_eval(g, n1, r, g[q], v, d);
      Dc[q * n1 + r] = d;
    }
  // reference 1D matrices: M = S^T W S, K = D^T W D
  double M[(kMaxDegree + 1) * (kMaxDegree + 1)], K[(kMaxDegree + 1) * (kMaxDegree + 1)];
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n1; ++j) {
      double m = 0.0, k = 0.0;
      for (int q = 0; q < n1; ++q) {
        m += w[q] * S[q * n1 + i] * S[q * n1 + j];
        k += w[q] * D[q * n1 + i] * D[q * n1 + j];
      }
      M[i * n1 + j] = m;
      K[i * n1 + j] = k;
    }
  // affine box cell: x-stiffness scaled by h_y h_z / h_x, etc.; mass unscaled
  const double scale[3] = {h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2]};
  for (int i = 0; i < n1 * n1; ++i) {
    c.mat[MAT_M][i] = M[i];
    for (int d = 0; d < 3; ++d) c.mat[MAT_K0 + d][i] = scale[d] * K[i];
    c.mat[MAT_S][i] = S[i];
    c.mat[MAT_DC][i] = Dc[i];
    c.mat[MAT_MV][i] = h[0] * h[1] * h[2] * M[i];
    c.T2[0][i] = S[i] * S[i];
    c.T2[1][i] = D[i] * S[i];
    c.T2[2][i] = D[i] * D[i];
  }
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n1; ++j) {
      c.mat[MAT_ST][i * n1 + j] = S[j * n1 + i];
      c.mat[MAT_DCT][i * n1 + j] = Dc[j * n1 + i];
    }
  // even-odd halves of every matrix (layouts in OperatorCoeffs); float
  // pairs: hi = nearest float, lo = nearest float of the remainder
  const int hh = n1 / 2, ne = n1 - hh;
  for (int m = 0; m < NMAT; ++m) {
    const double* A = c.mat[m];
    const bool anti = m == MAT_DC || m == MAT_DCT;
    if (!anti) {
      double* E = c.eo[m];
      double* O = c.eo[m] + ne * ne;
      for (int i = 0; i < ne; ++i)
        for (int j = 0; j < ne; ++j) {
          double v;
          if (j < hh)
            v = i < hh ? 0.5 * (A[i * n1 + j] + A[i * n1 + (n1 - 1 - j)]) : A[i * n1 + j];
          else
            v = A[i * n1 + j];  // middle column (odd n)
          E[i * ne + j] = v;
        }
      for (int i = 0; i < hh; ++i)
        for (int j = 0; j < hh; ++j) O[i * hh + j] = 0.5 * (A[i * n1 + j] - A[i * n1 + (n1 - 1 - j)]);
    } else {
      double* E = c.eo[m];            // hh x ne, multiplies e
      double* O = c.eo[m] + hh * ne;  // ne x hh, multiplies o
      for (int i = 0; i < hh; ++i)
        for (int j = 0; j < ne; ++j)
          E[i * ne + j] = j < hh ? 0.5 * (A[i * n1 + j] + A[i * n1 + (n1 - 1 - j)]) : A[i * n1 + j];
      for (int i = 0; i < ne; ++i)
        for (int j = 0; j < hh; ++j)
          O[i * hh + j] = i < hh ? 0.5 * (A[i * n1 + j] - A[i * n1 + (n1 - 1 - j)]) : A[i * n1 + j];
    }
    for (int i = 0; i < ne * ne + hh * hh; ++i) {
      const float hi = (float)c.eo[m][i];
      c.eoh[m][i] = hi;
      c.eol[m][i] = (float)(c.eo[m][i] - (double)hi);
    }
  }
  const double support[3] = {0.0, 0.5, 1.0};
  for (int q = 0; q < n1; ++q) {
    c.w[q] = w[q];
    c.g[q] = g[q];
    for (int a = 0; a < 3; ++a) lagrange_eval(support, 3, a, g[q], c.q2v[q][a], c.q2d[q][a]);
  }
  for (int d = 0; d < 3; ++d) c.h[d] = h[d];
  c.amplitude = amplitude;
  c.coef = coef;
}

}  // namespace mfcg
