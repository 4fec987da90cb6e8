/*
 * Oracle (test infrastructure only): reference-element tables and Butcher
 * tableaux.  Plain FP64; see oracle.h for the rules this file follows.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

/* Legendre polynomial P_n on [-1,1] and its derivative, by the three-term
 * recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = n * (x * p1 - p0) / (x * x - 1.0);
}

/* Solution points of Sec. 2 eq. (soln.points): the N+1 Gauss-Legendre nodes,
 * i.e. the roots of P_{N+1}, found by Newton's method and mapped from [-1,1]
 * to [0,1].  Weights w_p = 2 / ((1 - x^2) P'(x)^2), halved for [0,1] so that
 * sum_p w_p = 1; the rule is exact to degree 2N+1. */
static void gauss_legendre01(int N, double* xi, double* w) {
  const int m = N + 1;
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < m; ++i) {
    double x = -cos(pi * (i + 0.75) / (m + 0.5)); /* ascending initial guess */
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(m, x, &P, &dP);
      double dx = P / dP;
      x -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    double P, dP;
    legendre(m, x, &P, &dP);
    xi[i] = 0.5 * (1.0 + x);
    w[i] = 0.5 * 2.0 / ((1.0 - x * x) * dP * dP);
  }
}

/* Lagrange polynomial l_q(x) of Sec. 2 eq. (defn.lagrange). */
static double lagrange(int N, const double* xi, int q, double x) {
  double r = 1.0;
  for (int p = 0; p <= N; ++p)
    if (p != q) r *= (x - xi[p]) / (xi[q] - xi[p]);
  return r;
}

/* Derivative l_j'(x) by the product rule:
 * sum_{m != j} 1/(xi_j - xi_m) prod_{k != j, m} (x - xi_k)/(xi_j - xi_k). */
static double lagrange_deriv(int N, const double* xi, int j, double x) {
  double s = 0.0;
  for (int m = 0; m <= N; ++m) {
    if (m == j) continue;
    double t = 1.0 / (xi[j] - xi[m]);
    for (int k = 0; k <= N; ++k)
      if (k != j && k != m) t *= (x - xi[k]) / (xi[j] - xi[k]);
    s += t;
  }
  return s;
}

/* P_n and P_n' anywhere on [-1,1], endpoints included, by the recurrences
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and P'_{k+1} = P'_{k-1} + (2k+1) P_k. */
static void legendre_all(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    double d2 = d0 + (2.0 * k + 1.0) * p1;
    p0 = p1; p1 = p2;
    d0 = d1; d1 = d2;
  }
  *P = p1;
  *dP = d1;
}

/* Gauss-Lobatto-Legendre solution points (Sec. 5.1, with the g2 correction):
 * x = -1, 1 and the N-1 roots of P_N' (Newton's method with P_N'' from
 * Legendre's equation (1 - x^2) P'' = 2 x P' - N (N+1) P), mapped to [0,1];
 * weights 2 / (N (N+1) P_N(x)^2), halved for [0,1]; exact to degree 2N-1. */
static void gauss_lobatto01(int N, double* xi, double* w) {
  const double pi = 3.14159265358979323846;
  double x[OR_MAXN + 1];
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double z = -cos(pi * i / N);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_all(N, z, &P, &dP);
      double d2P = (2.0 * z * dP - N * (N + 1.0) * P) / (1.0 - z * z);
      double dz = dP / d2P;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    x[i] = z;
  }
  for (int i = 0; i <= N; ++i) {
    double P, dP;
    legendre_all(N, x[i], &P, &dP);
    xi[i] = 0.5 * (1.0 + x[i]);
    w[i] = 0.5 * 2.0 / (N * (N + 1.0) * P * P);
  }
}

/* Derivative on [-1,1] of the left correction function g (g(-1) = 1,
 * g(1) = 0) of the FR update (Sec. 2), with the right Radau polynomials
 * R_k = (-1)^k (P_k - P_{k-1}) / 2:
 *   Radau (OR_POINTS_GL): g = R_{N+1};
 *   g2 (OR_POINTS_GLL):   g = ((N+1) R_N + N R_{N+1}) / (2N+1). */
static double radau_deriv(int k, double x) {
  double P, dP, Pm, dPm;
  legendre_all(k, x, &P, &dP);
  legendre_all(k - 1, x, &Pm, &dPm);
  return ((k % 2) ? -0.5 : 0.5) * (dP - dPm);
}

static double corr_deriv(int N, int points, double x) {
  if (points == OR_POINTS_GLL)
    return ((N + 1.0) * radau_deriv(N, x) + N * radau_deriv(N + 1, x)) / (2.0 * N + 1.0);
  return radau_deriv(N + 1, x);
}

void or_tables_pts(int N, int points, double* xi, double* w, double* l0, double* l1, double* D,
                   double* gL, double* gR) {
  or_tables(N, xi, w, l0, l1, D);
  if (points == OR_POINTS_GLL) {
    gauss_lobatto01(N, xi, w);
    for (int p = 0; p <= N; ++p) {
      l0[p] = lagrange(N, xi, p, 0.0);
      l1[p] = lagrange(N, xi, p, 1.0);
    }
    for (int i = 0; i <= N; ++i)
      for (int j = 0; j <= N; ++j) D[i * (N + 1) + j] = lagrange_deriv(N, xi, j, xi[i]);
  }
  /* on [0,1]: g_L'(xi) = 2 g'(2 xi - 1); g_R(xi) = g_L(1 - xi) and the nodes are
   * symmetric (xi_{N-p} = 1 - xi_p), so g_R'(xi_p) = -g_L'(xi_{N-p}) */
  for (int p = 0; p <= N; ++p) gL[p] = 2.0 * corr_deriv(N, points, 2.0 * xi[p] - 1.0);
  for (int p = 0; p <= N; ++p) gR[p] = -gL[N - p];
}

void or_tables(int N, double* xi, double* w, double* l0, double* l1, double* D) {
  gauss_legendre01(N, xi, w);
  for (int p = 0; p <= N; ++p) {
    l0[p] = lagrange(N, xi, p, 0.0);
    l1[p] = lagrange(N, xi, p, 1.0);
  }
  /* Sec. 2 eq. (diff.matrix): D_ij = l_j'(xi_i) */
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N; ++j) D[i * (N + 1) + j] = lagrange_deriv(N, xi, j, xi[i]);
}

/* Butcher tableaux (Sec. 2 eq. (butcher)), A row-major [6][6].
 * Degree N uses an RK method of order N+1 (Sec. 3):
 *   N=1 cRK22 eq. (crk22), N=2 cRK33 eq. (crk33), N=3 cRK44 eq. (crk44).
 * The paper prints no order-5 scheme for N=4; the reading taken is Butcher's
 * six-stage fifth-order method, c = (0, 1/4, 1/4, 1/2, 3/4, 1). */
int or_tableau(int N, double* A, double* b, double* c) {
  memset(A, 0, sizeof(double) * 36);
  memset(b, 0, sizeof(double) * 6);
  memset(c, 0, sizeof(double) * 6);
#define AA(i, j) A[(i) * 6 + (j)]
  int s = 0;
  switch (N) {
    case 1: /* u2 = u - dt/2 Dloc f(u); F = f(u2) */
      s = 2;
      AA(1, 0) = 0.5;
      b[0] = 0.0; b[1] = 1.0;
      break;
    case 2: /* u2 = u - dt/3 .. f(u); u3 = u - 2dt/3 .. f(u2); F = f(u)/4 + 3 f(u3)/4 */
      s = 3;
      AA(1, 0) = 1.0 / 3.0;
      AA(2, 1) = 2.0 / 3.0;
      b[0] = 0.25; b[1] = 0.0; b[2] = 0.75;
      break;
    case 3: /* classical RK4 */
      s = 4;
      AA(1, 0) = 0.5;
      AA(2, 1) = 0.5;
      AA(3, 2) = 1.0;
      b[0] = 1.0 / 6.0; b[1] = 1.0 / 3.0; b[2] = 1.0 / 3.0; b[3] = 1.0 / 6.0;
      break;
    case 4:
      s = 6;
      AA(1, 0) = 0.25;
      AA(2, 0) = 0.125; AA(2, 1) = 0.125;
      AA(3, 0) = 0.0; AA(3, 1) = -0.5; AA(3, 2) = 1.0;
      AA(4, 0) = 3.0 / 16.0; AA(4, 1) = 0.0; AA(4, 2) = 0.0; AA(4, 3) = 9.0 / 16.0;
      AA(5, 0) = -3.0 / 7.0; AA(5, 1) = 2.0 / 7.0; AA(5, 2) = 12.0 / 7.0;
      AA(5, 3) = -12.0 / 7.0; AA(5, 4) = 8.0 / 7.0;
      b[0] = 7.0 / 90.0; b[1] = 0.0; b[2] = 32.0 / 90.0; b[3] = 12.0 / 90.0;
      b[4] = 32.0 / 90.0; b[5] = 7.0 / 90.0;
      break;
    default:
      return 0;
  }
  for (int i = 0; i < s; ++i) {
    double r = 0.0;
    for (int j = 0; j < s; ++j) r += AA(i, j);
    c[i] = r; /* c_i = sum_j a_ij */
  }
#undef AA
  return s;
}
