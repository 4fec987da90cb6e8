/*
 * Oracle (test infrastructure only): physical fluxes, wave speeds,
 * admissibility constraints and source terms.  Plain FP64.
 */
#include <math.h>
#include "oracle.h"

int or_nvars(const or_desc* d) {
  switch (d->equation) {
    case OR_EQ_LINADV: return 1;
    case OR_EQ_EULER: return d->dim == 1 ? 3 : 4;
    case OR_EQ_TENMOMENT: return 6;
    case OR_EQ_BURGERS: return 1;
    case OR_EQ_VARADV: return 1;
  }
  return 0;
}

int or_nodes(const or_desc* d) {
  int n = d->degree + 1;
  return d->dim == 1 ? n : n * n;
}

/* Euler pressure from the equation of state, Sec. 5.2 eq. (state) in 1D and
 * Sec. 5.3 eq. (2dstate) in 2D: p = (gamma - 1) (E - rho |v|^2 / 2). */
static double euler_pressure(const or_desc* d, const double* u) {
  if (d->dim == 1) return (d->gamma - 1.0) * (u[2] - 0.5 * u[1] * u[1] / u[0]);
  return (d->gamma - 1.0) * (u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0]);
}

/* Ten-moment pressure tensor from E = P/2 + rho v (x) v / 2 (Sec. 5.4):
 * p_ij = 2 E_ij - rho v_i v_j. */
static void tm_pressure(const double* u, double* p11, double* p12, double* p22) {
  double rho = u[0], v1 = u[1] / rho, v2 = u[2] / rho;
  *p11 = 2.0 * u[3] - rho * v1 * v1;
  *p12 = 2.0 * u[4] - rho * v1 * v2;
  *p22 = 2.0 * u[5] - rho * v2 * v2;
}

/* a(x) of the variable advection equation, by Horner's rule. */
static double varadv_a(const or_desc* d, double x) {
  return ((d->adv_poly[3] * x + d->adv_poly[2]) * x + d->adv_poly[1]) * x + d->adv_poly[0];
}

void or_flux_x(const or_desc* d, const double* u, double x, int dir, double* f) {
  if (d->equation == OR_EQ_VARADV) { /* Sec. 5.1: f(x, u) = a(x) u */
    f[0] = varadv_a(d, x) * u[0];
    return;
  }
  or_flux(d, u, dir, f);
}

double or_wave_speed_x(const or_desc* d, const double* u, double x, int dir) {
  if (d->equation == OR_EQ_VARADV) return fabs(varadv_a(d, x));
  return or_wave_speed(d, u, dir);
}

void or_flux(const or_desc* d, const double* u, int dir, double* f) {
  if (d->equation == OR_EQ_LINADV) {
    f[0] = d->adv[dir] * u[0];
    return;
  }
  if (d->equation == OR_EQ_BURGERS) { /* Sec. 5.1: f(u) = u^2/2 */
    f[0] = 0.5 * u[0] * u[0];
    return;
  }
  if (d->equation == OR_EQ_EULER) {
    if (d->dim == 1) { /* Sec. 5.2 eq. (1deuler) */
      double rho = u[0], v1 = u[1] / rho, p = euler_pressure(d, u);
      f[0] = rho * v1;
      f[1] = p + rho * v1 * v1;
      f[2] = (u[2] + p) * v1;
      return;
    }
    /* Sec. 5.3 eq. (2deuler) */
    double rho = u[0], v1 = u[1] / rho, v2 = u[2] / rho, E = u[3];
    double p = euler_pressure(d, u);
    if (dir == 0) {
      f[0] = rho * v1;
      f[1] = p + rho * v1 * v1;
      f[2] = rho * v1 * v2;
      f[3] = (E + p) * v1;
    } else {
      f[0] = rho * v2;
      f[1] = rho * v1 * v2;
      f[2] = p + rho * v2 * v2;
      f[3] = (E + p) * v2;
    }
    return;
  }
  /* ten-moment, Sec. 5.4 eq. (tmp) */
  double rho = u[0], v1 = u[1] / rho, v2 = u[2] / rho;
  double E11 = u[3], E12 = u[4], E22 = u[5];
  double p11, p12, p22;
  tm_pressure(u, &p11, &p12, &p22);
  if (dir == 0) {
    f[0] = rho * v1;
    f[1] = p11 + rho * v1 * v1;
    f[2] = p12 + rho * v1 * v2;
    f[3] = (E11 + p11) * v1;
    f[4] = E12 * v1 + 0.5 * (p11 * v2 + p12 * v1);
    f[5] = E22 * v1 + p12 * v2;
  } else {
    f[0] = rho * v2;
    f[1] = p12 + rho * v1 * v2;
    f[2] = p22 + rho * v2 * v2;
    f[3] = E11 * v2 + p12 * v1;
    f[4] = E12 * v2 + 0.5 * (p12 * v2 + p22 * v1);
    f[5] = (E22 + p22) * v2;
  }
}

/* Spectral radius sigma of the flux Jacobian in direction dir.
 * Linear advection: |a|.  Burgers: |u|.  Euler: |v| + c, c = sqrt(gamma p / rho)
 * (Sec. 5.2 eq. (spectral.radius.1d), Sec. 5.3).  Ten-moment (not given in
 * the paper; reading): |v_dir| + sqrt(3 p_dirdir / rho), the largest
 * eigenvalue magnitude of the x-Jacobian v1 +- sqrt(3 p11/rho).
 * The square root is taken of max(., 0). */
double or_wave_speed(const or_desc* d, const double* u, int dir) {
  if (d->equation == OR_EQ_LINADV) return fabs(d->adv[dir]);
  if (d->equation == OR_EQ_BURGERS) return fabs(u[0]); /* f'(u) = u */
  double rho = u[0];
  if (d->equation == OR_EQ_EULER) {
    double v = u[1 + dir] / rho;
    double c2 = d->gamma * euler_pressure(d, u) / rho;
    return fabs(v) + sqrt(fmax(c2, 0.0));
  }
  double p11, p12, p22;
  tm_pressure(u, &p11, &p12, &p22);
  double v = u[1 + dir] / rho;
  double pdd = dir == 0 ? p11 : p22;
  return fabs(v) + sqrt(fmax(3.0 * pdd / rho, 0.0));
}

/* Admissibility constraints P_k of Sec. 2 eq. (uad.form), each concave once the
 * earlier ones are positive.  Euler: rho, p.  Ten-moment: rho and the smallest
 * eigenvalue of the pressure tensor (x^T P x > 0 for all x != 0 exactly when
 * lambda_min(P) > 0; lambda_min is concave in u for rho > 0). */
int or_num_constraints(const or_desc* d) {
  return (d->equation == OR_EQ_LINADV || d->equation == OR_EQ_BURGERS || d->equation == OR_EQ_VARADV) ? 0 : 2;
}

double or_constraint(const or_desc* d, const double* u, int k) {
  if (k == 0) return u[0];
  if (d->equation == OR_EQ_EULER) return euler_pressure(d, u);
  double p11, p12, p22;
  tm_pressure(u, &p11, &p12, &p22);
  double h = 0.5 * (p11 - p22);
  return 0.5 * (p11 + p22) - sqrt(h * h + p12 * p12);
}

/* Source terms.  Euler with gravity (Sec. 5.5): s = (0, rho g, g . (rho v)),
 * the momentum source rho g and the work of gravity on the gas in the energy
 * (reading: the printed energy component names the velocity across gravity;
 * the work of a force rho g is rho v . g).  Ten-moment source of Sec. 5.4
 * eq. (tenmom.source), s = s^x + s^y with W = amp exp(-k |x - c|^2) (in 1D
 * only the x part, W = amp exp(-k (x-cx)^2)). */
void or_source(const or_desc* d, const double* u, double x, double y, double* s) {
  int M = or_nvars(d);
  for (int v = 0; v < M; ++v) s[v] = 0.0;
  if (d->source == OR_SRC_GRAVITY && d->equation == OR_EQ_EULER) {
    double gx = d->gravity[0], gy = d->dim == 2 ? d->gravity[1] : 0.0;
    s[1] = u[0] * gx;
    if (d->dim == 2) {
      s[2] = u[0] * gy;
      s[3] = u[1] * gx + u[2] * gy;
    } else {
      s[2] = u[1] * gx;
    }
    return;
  }
  if (d->source != OR_SRC_TENMOMENT || d->equation != OR_EQ_TENMOMENT) return;
  double rx = x - d->src_cx, ry = (d->dim == 2) ? (y - d->src_cy) : 0.0;
  double W = d->src_amp * exp(-d->src_k * (rx * rx + ry * ry));
  double dWx = -2.0 * d->src_k * rx * W;
  double dWy = (d->dim == 2) ? -2.0 * d->src_k * ry * W : 0.0;
  double rho = u[0], v1 = u[1] / rho, v2 = u[2] / rho;
  /* s^x */
  s[1] += -0.5 * rho * dWx;
  s[3] += -0.5 * rho * v1 * dWx;
  s[4] += -0.25 * rho * v2 * dWx;
  /* s^y */
  s[2] += -0.5 * rho * dWy;
  s[4] += -0.25 * rho * v1 * dWy;
  s[5] += -0.5 * rho * v2 * dWy;
}
