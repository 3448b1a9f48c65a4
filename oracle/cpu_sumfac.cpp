// Sum-factorised FP64 CPU evaluation of the DG advection operator (oracle;
// test infrastructure only -- the product path never links or calls this).
//
// This is the CPU implementation kind the paper itself measures: matrix-free
// evaluation cell by cell (Algorithm 1, element-centric loop over the cell
// pairs), each cell's weak form (Sec. 1.3, Eq. into:adv:ref, with the
// phase-space Jacobian J = diag(J_x, J_v) of Sec. 3) evaluated by 1D sweeps
// along every direction (sum factorisation, Sec. 2.4 and Algorithm 2), the
// upwind flux on the 2d faces with the neighbour's trace across periodic
// boundaries, and the inverse of the diagonal mass matrix of the
// Gauss-Legendre collocation (Algorithm 2 step 4), or of the Gauss-Lobatto
// collocation (nodes and quadrature at the Lobatto points).  FP64
// throughout, OpenMP over cells.  It shares no code with the CUDA library:
// its 1D tables come from its own Newton iterations on the Legendre
// polynomials, and it keeps
// the cell and face terms apart as the weak form states them.
//
// Per direction j and line of n nodes (all other node digits fixed), with
// c the contravariant speed (J^{-1} a)_j -- constant along the line, since
// a_x depends on v only and a_v on x only -- and W_perp |J| the transverse
// weights times the Jacobian determinant:
//   cell term:  b_q += W_perp |J| sum_p phi_q'(zeta_p) w_p c u_p
//   face +1:    b_q -= W_perp |J| phi_q(+1) c u*(+1)
//   face -1:    b_q += W_perp |J| phi_q(-1) c u*(-1)
// u*(s) is the trace from the side the flow leaves: this cell's line if
// s c > 0, else the neighbour's line across that face.  Finally
// K_q = b_q / (W_q |J|).
//
// C entry points (ctypes, oracle/sumfac.py):
//   sf_create(...) -> plan, sf_destroy(plan), sf_apply(plan, src, dst),
//   sf_apply_abs(plan, src, dst) (the term scale),
//   sf_rk_stage(plan, w_in, w_out, u, a_dt, b_dt, last, cell_lo, cell_hi),
//   sf_threads().
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int kMaxD = 6;
constexpr int kMaxN = 6;

// n-point Gauss-Legendre rule by Newton's method on P_n (three-term
// recurrence for P_n and its derivative), the textbook construction.
void gauss_legendre(int n, double* x, double* w) {
  if (n == 1) {
    x[0] = 0.0;
    w[0] = 2.0;
    return;
  }
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));   // initial guess near root i
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int m = 2; m <= n; ++m) {
        const double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // P_n' at the converged root for the weight 2 / ((1 - z^2) P_n'(z)^2)
    double p0 = 1.0, p1 = z;
    for (int m = 2; m <= n; ++m) {
      const double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;                      // ascending order
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// n-point Gauss-Lobatto rule (n >= 2): the end points and the N - 1 interior
// roots of P_N' (N = n - 1), by Newton's method on P_N' with P_N'' from
// Legendre's equation (1 - z^2) P'' - 2 z P' + N (N + 1) P = 0, started from
// the Chebyshev-Lobatto points; weights 2 / (N (N + 1) P_N(z)^2).
void gauss_lobatto(int n, double* x, double* w) {
  const int N = n - 1;
  const double pi = 3.14159265358979323846;
  auto legendre = [N](double z, double& pN, double& pNm1) {
    double p0 = 1.0, p1 = z;
    for (int m = 2; m <= N; ++m) {
      const double p2 = ((2.0 * m - 1.0) * z * p1 - (m - 1.0) * p0) / m;
      p0 = p1;
      p1 = p2;
    }
    pN = p1;
    pNm1 = p0;
  };
  for (int i = 0; i < n; ++i) {
    double z = -std::cos(pi * i / N);
    if (i > 0 && i < N) {
      for (int it = 0; it < 100; ++it) {
        double pN, pNm1;
        legendre(z, pN, pNm1);
        const double d1 = N * (z * pN - pNm1) / (z * z - 1.0);                 // P_N'
        const double d2 = (2.0 * z * d1 - N * (N + 1.0) * pN) / (1.0 - z * z);   // P_N''
        const double dz = d1 / d2;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
    }
    double pN, pNm1;
    legendre(z, pN, pNm1);
    x[i] = z;
    w[i] = 2.0 / (N * (N + 1.0) * pN * pN);
  }
}

// Lagrange basis through the nodes z: value of phi_i at t.
double lagrange(const double* z, int n, int i, double t) {
  double v = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != i) v *= (t - z[m]) / (z[i] - z[m]);
  return v;
}
// derivative of phi_i at t (product rule)
double lagrange_d(const double* z, int n, int i, double t) {
  double s = 0.0;
  for (int r = 0; r < n; ++r) {
    if (r == i) continue;
    double term = 1.0 / (z[i] - z[r]);
    for (int m = 0; m < n; ++m)
      if (m != i && m != r) term *= (t - z[m]) / (z[i] - z[m]);
    s += term;
  }
  return s;
}

}  // namespace

extern "C" {

// Problem description (mirrors the library's geometry conventions: lattice
// box in x mapped by x = S y, velocity box in v, all periodic; cell index
// c_x + N_x c_v, node index lexicographic with the first direction fastest).
typedef struct {
  int dx, dv, k;
  int cells[6];
  double lo[6], hi[6];
  double S[9];              // row-major dx x dx; all zero = identity
  int field_kind;           // 0 constant a; 1 a = (v_1..v_dx, E(x))
  double a[6];
  const double* e_nodes;    // kind 1: [ncx][n^dx][dv], E at the x nodes (NULL: E = 0)
  int basis;                // 0: Gauss-Legendre collocation; 1: Gauss-Lobatto
                            // collocation (nodes and quadrature at the GLL points, k >= 1)
} sf_problem;

struct sf_plan {
  int dx, dv, d, n, npc, nqx, nqv;
  int cells[kMaxD];
  long long cstride[kMaxD], ncells, ncx, ncv;
  double detJ;
  double zeta[kMaxN], w[kMaxN];
  double Dw[kMaxN][kMaxN];   // Dw[q][p] = phi_q'(zeta_p) w_p (cell term of direction j)
  double lp[kMaxN], lm[kMaxN];
  std::vector<double> cx;    // [ncv][nqv][dx]: x speeds at the v nodes
  std::vector<double> cv;    // [ncx][nqx][dv]: v speeds at the x nodes
};

int sf_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

sf_plan* sf_create(const sf_problem* pb) {
  if (!pb || pb->dx < 1 || pb->dv < 1 || pb->dx + pb->dv > kMaxD || pb->k < 0 ||
      pb->k + 1 > kMaxN || pb->basis < 0 || pb->basis > 1 || (pb->basis == 1 && pb->k < 1))
    return nullptr;
  sf_plan* p = new sf_plan();
  p->dx = pb->dx;
  p->dv = pb->dv;
  p->d = pb->dx + pb->dv;
  p->n = pb->k + 1;
  const int n = p->n, d = p->d, dx = p->dx, dv = p->dv;
  p->npc = 1;
  for (int j = 0; j < d; ++j) p->npc *= n;
  p->nqx = 1;
  for (int j = 0; j < dx; ++j) p->nqx *= n;
  p->nqv = p->npc / p->nqx;
  long long st = 1;
  for (int j = 0; j < d; ++j) {
    p->cells[j] = pb->cells[j];
    p->cstride[j] = st;
    st *= pb->cells[j];
  }
  p->ncells = st;
  p->ncx = 1;
  for (int j = 0; j < dx; ++j) p->ncx *= pb->cells[j];
  p->ncv = p->ncells / p->ncx;
  if (pb->basis == 1) gauss_lobatto(n, p->zeta, p->w);
  else gauss_legendre(n, p->zeta, p->w);
  for (int q = 0; q < n; ++q)
    for (int pp = 0; pp < n; ++pp) p->Dw[q][pp] = lagrange_d(p->zeta, n, q, p->zeta[pp]) * p->w[pp];
  for (int i = 0; i < n; ++i) {
    p->lp[i] = lagrange(p->zeta, n, i, 1.0);
    p->lm[i] = lagrange(p->zeta, n, i, -1.0);
  }
  // Jacobian J = diag(S diag(h_x / 2), diag(h_v / 2)); S^{-1} for the x speeds
  double h[kMaxD];
  for (int j = 0; j < d; ++j) h[j] = (pb->hi[j] - pb->lo[j]) / pb->cells[j];
  double S[3][3] = {{0}}, Si[3][3] = {{0}};
  bool zero = true;
  for (int i = 0; i < dx * dx; ++i) zero = zero && pb->S[i] == 0.0;
  for (int i = 0; i < dx; ++i)
    for (int m = 0; m < dx; ++m) S[i][m] = zero ? (i == m ? 1.0 : 0.0) : pb->S[i * dx + m];
  double detS;
  if (dx == 1) {
    detS = S[0][0];
    Si[0][0] = 1.0 / detS;
  } else if (dx == 2) {
    detS = S[0][0] * S[1][1] - S[0][1] * S[1][0];
    Si[0][0] = S[1][1] / detS;
    Si[0][1] = -S[0][1] / detS;
    Si[1][0] = -S[1][0] / detS;
    Si[1][1] = S[0][0] / detS;
  } else {
    // inverse by cofactors
    detS = S[0][0] * (S[1][1] * S[2][2] - S[1][2] * S[2][1]) -
           S[0][1] * (S[1][0] * S[2][2] - S[1][2] * S[2][0]) +
           S[0][2] * (S[1][0] * S[2][1] - S[1][1] * S[2][0]);
    for (int i = 0; i < 3; ++i)
      for (int m = 0; m < 3; ++m) {
        const int r0 = (m + 1) % 3, r1 = (m + 2) % 3, c0 = (i + 1) % 3, c1 = (i + 2) % 3;
        Si[i][m] = (S[r0][c0] * S[r1][c1] - S[r0][c1] * S[r1][c0]) / detS;
      }
  }
  p->detJ = std::fabs(detS);
  for (int j = 0; j < d; ++j) p->detJ *= h[j] / 2.0;
  // x speeds (2 / h_x) S^{-1} a_x at every v node of every v cell
  p->cx.assign(static_cast<size_t>(p->ncv) * p->nqv * dx, 0.0);
  for (long long cv = 0; cv < p->ncv; ++cv)
    for (int qv = 0; qv < p->nqv; ++qv) {
      double ax[3] = {0, 0, 0};
      if (pb->field_kind == 0) {
        for (int i = 0; i < dx; ++i) ax[i] = pb->a[i];
      } else {
        long long c = cv;
        int q = qv;
        for (int i = 0; i < dx; ++i) {       // a_x = (v_1, .., v_dx)
          const int jv = dx + i;
          const long long ci = c % pb->cells[jv];
          const int qi = q % n;
          ax[i] = pb->lo[jv] + h[jv] * (ci + (p->zeta[qi] + 1.0) / 2.0);
          c /= pb->cells[jv];
          q /= n;
        }
      }
      for (int i = 0; i < dx; ++i) {
        double s = 0.0;
        for (int m = 0; m < dx; ++m) s += Si[i][m] * ax[m];
        p->cx[(static_cast<size_t>(cv) * p->nqv + qv) * dx + i] = 2.0 / h[i] * s;
      }
    }
  // v speeds (2 / h_v) a_v at every x node of every x cell
  p->cv.assign(static_cast<size_t>(p->ncx) * p->nqx * dv, 0.0);
  for (long long cx = 0; cx < p->ncx; ++cx)
    for (int qx = 0; qx < p->nqx; ++qx)
      for (int i = 0; i < dv; ++i) {
        double a = 0.0;
        if (pb->field_kind == 0) a = pb->a[dx + i];
        else if (pb->e_nodes) a = pb->e_nodes[(static_cast<size_t>(cx) * p->nqx + qx) * dv + i];
        p->cv[(static_cast<size_t>(cx) * p->nqx + qx) * dv + i] = 2.0 / h[dx + i] * a;
      }
  return p;
}

void sf_destroy(sf_plan* p) { delete p; }

}  // extern "C"

namespace {

// K = M^{-1} A(src) on one cell (b: scratch of n^d doubles; K written to out).
// ABS: the same sums with the absolute value of every factor and term (the
// term scale M^{-1} |A| |src| that bounds the rounding error of an
// evaluation in reduced precision); the upwind choice stays with the sign of
// the speed.
template <bool ABS>
void cell_operator(const sf_plan* p, const double* src, long long cell, double* b, double* out) {
  auto f = [](double x) { return ABS ? std::fabs(x) : x; };
  const int n = p->n, d = p->d, dx = p->dx, npc = p->npc;
  const double* u = src + cell * npc;
  for (int q = 0; q < npc; ++q) b[q] = 0.0;
  long long cc[kMaxD];
  for (int j = 0; j < d; ++j) cc[j] = (cell / p->cstride[j]) % p->cells[j];
  const long long cx = cell % p->ncx, cv = cell / p->ncx;
  int nst[kMaxD + 1];
  nst[0] = 1;
  for (int j = 0; j < d; ++j) nst[j + 1] = nst[j] * n;
  for (int j = 0; j < d; ++j) {
    // neighbours across the faces -1 and +1 (periodic wrap)
    const long long st = p->cstride[j];
    const long long nbm = cc[j] == 0 ? cell + (p->cells[j] - 1) * st : cell - st;
    const long long nbp = cc[j] == p->cells[j] - 1 ? cell - (p->cells[j] - 1) * st : cell + st;
    const double* um = src + nbm * npc;
    const double* up = src + nbp * npc;
    const int s = nst[j];
    const int nlo = nst[j], nhi = npc / nst[j + 1];
    for (int hi = 0; hi < nhi; ++hi)
      for (int lo = 0; lo < nlo; ++lo) {
        const int base = lo + hi * nst[j + 1];
        // contravariant speed of the line and its transverse weights
        double c;
        if (j < dx) c = p->cx[(static_cast<size_t>(cv) * p->nqv + base / p->nqx) * dx + j];
        else c = p->cv[(static_cast<size_t>(cx) * p->nqx + base % p->nqx) * p->dv + (j - dx)];
        const double ca = f(c);
        double wperp = p->detJ;
        {
          int q = base;
          for (int m = 0; m < d; ++m) {
            if (m != j) wperp *= p->w[q % n];
            q /= n;
          }
        }
        // cell term
        for (int q = 0; q < n; ++q) {
          double acc = 0.0;
          for (int pp = 0; pp < n; ++pp) acc += f(p->Dw[q][pp]) * ca * f(u[base + pp * s]);
          b[base + q * s] += wperp * acc;
        }
        // upwind traces on the two faces
        double tp = 0.0, tm = 0.0;
        if (c > 0) {
          for (int pp = 0; pp < n; ++pp) {
            tp += f(p->lp[pp]) * f(u[base + pp * s]);     // own trace leaves through +1
            tm += f(p->lp[pp]) * f(um[base + pp * s]);    // the lower neighbour's +1 trace enters
          }
        } else {
          for (int pp = 0; pp < n; ++pp) {
            tp += f(p->lm[pp]) * f(up[base + pp * s]);    // the upper neighbour's -1 trace enters
            tm += f(p->lm[pp]) * f(u[base + pp * s]);     // own trace leaves through -1
          }
        }
        const double fp = ca * tp, fm = ca * tm;
        for (int q = 0; q < n; ++q)
          b[base + q * s] += ABS ? wperp * (f(p->lp[q]) * fp + f(p->lm[q]) * fm)
                                 : wperp * (-p->lp[q] * fp + p->lm[q] * fm);
      }
  }
  // inverse of the diagonal mass matrix W_q |J|
  for (int q = 0; q < npc; ++q) {
    double wq = p->detJ;
    int r = q;
    for (int m = 0; m < d; ++m) {
      wq *= p->w[r % n];
      r /= n;
    }
    out[q] = b[q] / wq;
  }
}

}  // namespace

extern "C" {

// dst = M^{-1} A(src) for every cell (src and dst must not overlap).
int sf_apply(const sf_plan* p, const double* src, double* dst) {
  if (!p || !src || !dst) return 1;
#pragma omp parallel
  {
    std::vector<double> b(p->npc);
#pragma omp for schedule(static)
    for (long long e = 0; e < p->ncells; ++e) cell_operator<false>(p, src, e, b.data(), dst + e * p->npc);
  }
  return 0;
}

// dst = M^{-1} |A| |src|, the term scale of every value (see cell_operator).
int sf_apply_abs(const sf_plan* p, const double* src, double* dst) {
  if (!p || !src || !dst) return 1;
#pragma omp parallel
  {
    std::vector<double> b(p->npc);
#pragma omp for schedule(static)
    for (long long e = 0; e < p->ncells; ++e) cell_operator<true>(p, src, e, b.data(), dst + e * p->npc);
  }
  return 0;
}

// One fused LSRK(5,4) stage on the cells [cell_lo, cell_hi): K = L(w_in);
// w_out = u + a_dt K (or the new u if last != 0); u += b_dt K.  (A cell
// range lets a caller time a bounded part of a large mesh; neighbours
// outside the range are read from w_in as usual.)
int sf_rk_stage(const sf_plan* p, const double* w_in, double* w_out, double* u, double a_dt,
                double b_dt, int last, long long cell_lo, long long cell_hi) {
  if (!p || !w_in || !w_out || !u || cell_lo < 0 || cell_hi > p->ncells || cell_lo > cell_hi)
    return 1;
#pragma omp parallel
  {
    std::vector<double> b(p->npc), K(p->npc);
#pragma omp for schedule(static)
    for (long long e = cell_lo; e < cell_hi; ++e) {
      cell_operator<false>(p, w_in, e, b.data(), K.data());
      double* ue = u + e * p->npc;
      double* we = w_out + e * p->npc;
      for (int q = 0; q < p->npc; ++q) {
        const double un = ue[q] + b_dt * K[q];
        we[q] = last ? un : ue[q] + a_dt * K[q];
        ue[q] = un;
      }
    }
  }
  return 0;
}

}  // extern "C"
