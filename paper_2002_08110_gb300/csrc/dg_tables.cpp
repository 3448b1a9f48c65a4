// Host-side 1D tables of the collocated elements, in FP64.
//
// Gauss-Legendre points (Sec. 2.5 of arXiv 2002.08110) by Newton's method on
// the three-term recurrence of the Legendre polynomials, weights
// w = 2 / ((1 - x^2) P_n'(x)^2); Gauss-Lobatto points: the endpoints and the
// roots of P_{n-1}' (Newton's method, second derivative from Legendre's
// equation), weights 2 / (n (n-1) P_{n-1}(x)^2).  Lagrange derivatives by the
// barycentric formula D[p][i] = (lambda_i / lambda_p) / (x_p - x_i) (p != i),
// with the diagonal making each row sum to zero (derivative of a constant).
#include <cmath>
#include <cstring>

#include "dg_internal.h"

namespace dg {

static void legendre_eval(int n, double z, double* pn, double* dpn) {
  double p0 = 1.0, p1 = z;
  if (n == 0) { *pn = 1.0; *dpn = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  // P_n'(z) = n (z P_n - P_{n-1}) / (z^2 - 1)
  *dpn = n * (z * p1 - p0) / (z * z - 1.0);
}

bool gauss_legendre(int n, double* x, double* w) {
  if (n < 1 || n > kMaxN) return false;
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double pn = 0.0, dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      legendre_eval(n, z, &pn, &dp);
      const double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre_eval(n, z, &pn, &dp);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  return true;
}

bool gauss_lobatto(int n, double* x, double* w) {
  if (n < 2 || n > kMaxN) return false;
  const double pi = 3.14159265358979323846;
  const int m = n - 1;
  x[0] = -1.0;
  x[m] = 1.0;
  for (int i = 1; i < m; ++i) {
    // interior nodes: roots of P_m', started from the Chebyshev-Lobatto points
    double z = -std::cos(pi * i / m);
    for (int it = 0; it < 100; ++it) {
      double pn = 0.0, dp = 0.0;
      legendre_eval(m, z, &pn, &dp);
      const double d2 = (2.0 * z * dp - m * (m + 1.0) * pn) / (1.0 - z * z);
      const double dz = dp / d2;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  for (int i = 0; i < n; ++i) {
    double pn = 1.0, dp = 0.0;
    if (i == 0 || i == m) {
      pn = (i == 0 && (m % 2 == 1)) ? -1.0 : 1.0;   // P_m(-1) = (-1)^m, P_m(1) = 1
    } else {
      legendre_eval(m, x[i], &pn, &dp);
    }
    w[i] = 2.0 / (n * (n - 1.0) * pn * pn);
  }
  return true;
}

bool basis_points(int basis, int n, double* dof_nodes, double* qpoints, double* qweights) {
  double gx[kMaxN], gw[kMaxN], lx[kMaxN], lw[kMaxN];
  if (!gauss_legendre(n, gx, gw)) return false;
  if (basis != DG_BASIS_GL && !gauss_lobatto(n, lx, lw)) return false;
  for (int i = 0; i < n; ++i) {
    const bool lob_q = basis == DG_BASIS_GLL;        // quadrature at the Lobatto points
    const bool lob_n = basis != DG_BASIS_GL;         // DoFs at the Lobatto points
    if (dof_nodes) dof_nodes[i] = lob_n ? lx[i] : gx[i];
    if (qpoints) qpoints[i] = lob_q ? lx[i] : gx[i];
    if (qweights) qweights[i] = lob_q ? lw[i] : gw[i];
  }
  return true;
}

// Lagrange polynomial i through nodes z (n points) at x.
static double lagrange(const double* z, int n, int i, double x) {
  double v = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != i) v *= (x - z[m]) / (z[i] - z[m]);
  return v;
}

void build_tables(int n, int basis, HostTables* t) {
  std::memset(t, 0, sizeof(*t));
  t->n = n;
  t->basis = basis;
  // the operator is collocated at the quadrature points (Gauss-Legendre for
  // bases 0 and 2, Gauss-Lobatto for basis 1); basis 2 keeps its DoFs at the
  // Lobatto nodes and changes basis around the Gauss-Legendre operator
  basis_points(basis, n, t->dofz, t->zeta, t->w);
  for (int q = 0; q < n; ++q)
    for (int i = 0; i < n; ++i) t->V[q][i] = lagrange(t->dofz, n, i, t->zeta[q]);
  {
    // Vinv by Gauss-Jordan elimination with partial pivoting (n <= 6)
    double a[kMaxN][2 * kMaxN];
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < 2 * n; ++c) a[r][c] = c < n ? t->V[r][c] : (c - n == r ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
      int piv = c;
      for (int r = c + 1; r < n; ++r)
        if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
      if (piv != c)
        for (int k = 0; k < 2 * n; ++k) std::swap(a[c][k], a[piv][k]);
      const double inv = 1.0 / a[c][c];
      for (int k = 0; k < 2 * n; ++k) a[c][k] *= inv;
      for (int r = 0; r < n; ++r) {
        if (r == c) continue;
        const double f = a[r][c];
        for (int k = 0; k < 2 * n; ++k) a[r][k] -= f * a[c][k];
      }
    }
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) t->Vinv[r][c] = a[r][n + c];
  }
  const double* x = t->zeta;
  double lam[kMaxN];
  for (int i = 0; i < n; ++i) {
    double prod = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != i) prod *= (x[i] - x[m]);
    lam[i] = 1.0 / prod;
  }
  for (int p = 0; p < n; ++p) {
    double diag = 0.0;
    for (int i = 0; i < n; ++i) {
      if (i == p) continue;
      t->D[p][i] = (lam[i] / lam[p]) / (x[p] - x[i]);
      diag -= t->D[p][i];
    }
    t->D[p][p] = diag;
  }
  for (int i = 0; i < n; ++i) {
    double a = 1.0, b = 1.0;
    for (int m = 0; m < n; ++m) {
      if (m == i) continue;
      a *= (1.0 - x[m]) / (x[i] - x[m]);
      b *= (-1.0 - x[m]) / (x[i] - x[m]);
    }
    t->lp[i] = a;
    t->lm[i] = b;
  }
  // Iq[q][i] = int_{-1}^{zeta_q} phi_i: the n-point Gauss rule mapped onto
  // [-1, zeta_q] is exact for the degree n - 1 integrand.
  for (int q = 0; q < n; ++q) {
    const double half = 0.5 * (x[q] + 1.0);
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int r = 0; r < n; ++r) {
        const double xi = -1.0 + half * (x[r] + 1.0);
        double phi = 1.0;
        for (int m = 0; m < n; ++m)
          if (m != i) phi *= (xi - x[m]) / (x[i] - x[m]);
        s += t->w[r] * phi;
      }
      t->Iq[q][i] = half * s;
    }
  }
  Tab1D<double>& d = t->t64;
  for (int q = 0; q < n; ++q) {
    d.lp[q] = t->lp[q];
    d.lm[q] = t->lm[q];
    d.w[q] = t->w[q];
    d.winv[q] = 1.0 / t->w[q];
    d.Lp[q] = t->lp[q] / t->w[q];
    d.Lm[q] = t->lm[q] / t->w[q];
  }
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < n; ++p) {
      const double dt = t->D[p][q] * t->w[p] / t->w[q];
      d.Dt[q * n + p] = dt;
      d.Gp[q * n + p] = dt - d.Lp[q] * t->lp[p];
      d.Gn[q * n + p] = dt + d.Lm[q] * t->lm[p];
    }
  Tab1D<float>& f = t->t32;
  for (int i = 0; i < kMaxN * kMaxN; ++i) {
    f.Dt[i] = static_cast<float>(d.Dt[i]);
    f.Gp[i] = static_cast<float>(d.Gp[i]);
    f.Gn[i] = static_cast<float>(d.Gn[i]);
  }
  for (int i = 0; i < kMaxN; ++i) {
    f.Lp[i] = static_cast<float>(d.Lp[i]);
    f.Lm[i] = static_cast<float>(d.Lm[i]);
    f.lp[i] = static_cast<float>(d.lp[i]);
    f.lm[i] = static_cast<float>(d.lm[i]);
    f.w[i] = static_cast<float>(d.w[i]);
    f.winv[i] = static_cast<float>(d.winv[i]);
  }
}

}  // namespace dg
