/*
 * Oracle (test infrastructure only): one cRKFR time step with the blending
 * limiter, the flux limiter and the scaling limiter.  Plain FP64, straight
 * loops in the paper's order; see oracle.h for the rules this file follows.
 *
 * Face sides of an element: 0 = left x-face (xi = 0), 1 = right x-face
 * (xi = 1), 2 = bottom y-face (eta = 0), 3 = top y-face (eta = 1).  A face node
 * j runs along the face: j = q on x-faces, j = p on y-faces.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define NMAX (OR_MAXN + 1)
#define NPMAX (NMAX * NMAX)

typedef struct {
  const or_desc* d;
  int dim, N, n, nq, np, M, s, K, nx, ny, ne;
  double dx, dy;
  double xi[NMAX], w[NMAX], l0[NMAX], l1[NMAX], D[NMAX * NMAX];
  double gL[NMAX], gR[NMAX]; /* correction derivatives g_L'(xi_p), g_R'(xi_p) */
  double A[36], b[6], c[6];
  double xsub[NMAX + 1]; /* subface positions x_{p-1/2}, p = 0..N+1, in units of dx (eq. subcell.defn) */
} ctx;

static void ctx_init(ctx* c, const or_desc* d) {
  memset(c, 0, sizeof(*c));
  c->d = d;
  c->dim = d->dim;
  c->N = d->degree;
  c->n = d->degree + 1;
  c->nq = d->dim == 2 ? c->n : 1;
  c->np = c->n * c->nq;
  c->M = or_nvars(d);
  c->K = or_num_constraints(d);
  c->nx = d->nx;
  c->ny = d->dim == 2 ? d->ny : 1;
  c->ne = c->nx * c->ny;
  c->dx = (d->x1 - d->x0) / d->nx;
  c->dy = d->dim == 2 ? (d->y1 - d->y0) / d->ny : 1.0;
  or_tables_pts(c->N, d->points, c->xi, c->w, c->l0, c->l1, c->D, c->gL, c->gR);
  c->s = or_tableau(c->N, c->A, c->b, c->c);
  /* Sec. 4 eq. (subcell.defn): x_{p+1/2} - x_{p-1/2} = w_p dx, x_{-1/2} = 0 */
  c->xsub[0] = 0.0;
  for (int p = 0; p <= c->N; ++p) c->xsub[p + 1] = c->xsub[p] + c->w[p];
}

static int node(const ctx* c, int p, int q) { return p + c->n * q; }

/* quadrature weight of node k for element means: w_p (1D) or w_p w_q (2D) */
static double node_weight(const ctx* c, int k) {
  int p = k % c->n, q = k / c->n;
  return c->dim == 2 ? c->w[p] * c->w[q] : c->w[p];
}

/* neighbour of element e across face side f; -1 at an outflow or wall boundary */
static int neighbour(const ctx* c, int e, int f) {
  int ix = e % c->nx, iy = e / c->nx;
  if (f == 0) { if (ix > 0) return e - 1; return c->d->bc_x == OR_BC_PERIODIC ? e + c->nx - 1 : -1; }
  if (f == 1) { if (ix < c->nx - 1) return e + 1; return c->d->bc_x == OR_BC_PERIODIC ? e - c->nx + 1 : -1; }
  if (f == 2) { if (iy > 0) return e - c->nx; return c->d->bc_y == OR_BC_PERIODIC ? e + c->nx * (c->ny - 1) : -1; }
  if (iy < c->ny - 1) return e + c->nx;
  return c->d->bc_y == OR_BC_PERIODIC ? e - c->nx * (c->ny - 1) : -1;
}

/* gather element e of the SoA state into ue[k][v] */
static void gather(const ctx* c, const double* u, int e, double* ue) {
  for (int k = 0; k < c->np; ++k)
    for (int v = 0; v < c->M; ++v) ue[k * c->M + v] = u[((size_t)v * c->ne + e) * c->np + k];
}

static void scatter(const ctx* c, double* u, int e, const double* ue) {
  for (int k = 0; k < c->np; ++k)
    for (int v = 0; v < c->M; ++v) u[((size_t)v * c->ne + e) * c->np + k] = ue[k * c->M + v];
}

static int admissible(const ctx* c, const double* u) {
  for (int k = 0; k < c->K; ++k)
    if (!(or_constraint(c->d, u, k) > 0.0)) return 0;
  return 1;
}

/* HLLC flux of the Euler equations (the upwind flux Sec. 3.3 names for
 * boundaries that mix inflow and outflow), normal direction dir, from states
 * UL, UR and fluxes FL, FR given separately (the time averages at a boundary
 * face; f(U) for the low-order flux).  Wave speeds S_L = min(v_L - c_L,
 * v_R - c_R), S_R = max(v_L + c_L, v_R + c_R); contact speed
 *   S* = (p_R - p_L + rho_L v_L (S_L - v_L) - rho_R v_R (S_R - v_R))
 *        / (rho_L (S_L - v_L) - rho_R (S_R - v_R));
 * star states U*_K = rho_K (S_K - v_K)/(S_K - S*) (1, S* in the normal
 * momentum, the tangential velocity, E_K/rho_K + (S* - v_K)(S* + p_K/(rho_K (S_K - v_K))));
 * F = F_L, F_L + S_L (U*_L - U_L), F_R + S_R (U*_R - U_R) or F_R by the signs
 * of S_L, S*, S_R (the classical three-wave solver of gas dynamics). */
static void hllc(const ctx* c, int dir, const double* UL, const double* UR, const double* FL,
                 const double* FR, double* out) {
  const int M = c->M, mn = 1 + dir, E = M - 1;
  const double g = c->d->gamma;
  double rl = UL[0], rr = UR[0], vl = UL[mn] / rl, vr = UR[mn] / rr;
  double pl = or_constraint(c->d, UL, 1), pr = or_constraint(c->d, UR, 1);
  double cl = sqrt(fmax(g * pl / rl, 0.0)), cr = sqrt(fmax(g * pr / rr, 0.0));
  double sl = fmin(vl - cl, vr - cr), sr = fmax(vl + cl, vr + cr);
  if (sl >= 0.0) { for (int v = 0; v < M; ++v) out[v] = FL[v]; return; }
  if (sr <= 0.0) { for (int v = 0; v < M; ++v) out[v] = FR[v]; return; }
  double ss = (pr - pl + rl * vl * (sl - vl) - rr * vr * (sr - vr)) / (rl * (sl - vl) - rr * (sr - vr));
  const double* U = ss >= 0.0 ? UL : UR;
  const double* F = ss >= 0.0 ? FL : FR;
  double r = ss >= 0.0 ? rl : rr, vn = ss >= 0.0 ? vl : vr, p = ss >= 0.0 ? pl : pr, sk = ss >= 0.0 ? sl : sr;
  double fac = r * (sk - vn) / (sk - ss), us[OR_MAXM];
  for (int v = 0; v < M; ++v) us[v] = fac * U[v] / r; /* tangential momentum: rho* v_t */
  us[0] = fac;
  us[mn] = fac * ss;
  us[E] = fac * (U[E] / r + (ss - vn) * (ss + p / (r * (sk - vn))));
  for (int v = 0; v < M; ++v) out[v] = F[v] + sk * (us[v] - U[v]);
}

/* Rusanov flux of Sec. 2 eq. (num.flux.fr) with eq. (rusanov.wave.speed), at
 * position x along the face normal (used by variable advection only). */
static void rusanov(const ctx* c, const double* uL, const double* uR, int dir, double x, double* out) {
  double fL[OR_MAXM], fR[OR_MAXM];
  or_flux_x(c->d, uL, x, dir, fL);
  or_flux_x(c->d, uR, x, dir, fR);
  double lam = fmax(or_wave_speed_x(c->d, uL, x, dir), or_wave_speed_x(c->d, uR, x, dir));
  for (int v = 0; v < c->M; ++v) out[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * lam * (uR[v] - uL[v]);
}

/* ------------------------------------------------------------------------ */
/* Local cRK procedure (Sec. 3 eqs. (crkfr1), (disc.avg.flux), (time.avg.sol);
 * App. B eqs. (crkfr.source), (crk33.source) for the source) and the EA face
 * fluxes of Sec. 3.1.2 eq. (evaluate).
 *   u^(i) = u^n - dt sum_{j<i} a_ij [ Dloc f(u^(j)) - s(u^(j)) ]
 *   F = sum_i b_i f(u^(i)), G likewise in y, U = sum_i b_i u^(i), S = sum_i b_i s(u^(i))
 *   EA: F^{+-} = sum_i b_i f(u^(i)(face))
 * ea is [4][NMAX][M] (face side, face node, variable); stg (may be NULL)
 * receives the stage traces u^(i)(face), [s][4][NMAX][M], for D-CSX. */
static void local_crk_ea(const ctx* c, const double* ue, double dt, int ix, int iy, double* F,
                         double* G, double* U, double* S, double* ea, double* stg) {
  const int M = c->M, n = c->n, nq = c->nq, np = c->np;
  static double ui[OR_MAXS][NPMAX][OR_MAXM];
  static double L[OR_MAXS][NPMAX][OR_MAXM];
  double f[NPMAX][OR_MAXM], g[NPMAX][OR_MAXM], src[NPMAX][OR_MAXM];
  for (int k = 0; k < np; ++k)
    for (int v = 0; v < M; ++v) F[k * M + v] = G[k * M + v] = U[k * M + v] = S[k * M + v] = 0.0;
  if (ea)
    for (int t = 0; t < 4 * NMAX * OR_MAXM; ++t) ea[t] = 0.0;

  for (int i = 0; i < c->s; ++i) {
    /* stage value */
    for (int k = 0; k < np; ++k)
      for (int v = 0; v < M; ++v) {
        double acc = ue[k * M + v];
        for (int j = 0; j < i; ++j) acc -= dt * c->A[i * 6 + j] * L[j][k][v];
        ui[i][k][v] = acc;
      }
    /* fluxes and source at the solution points */
    for (int k = 0; k < np; ++k) {
      int p = k % n, q = k / n;
      double x = c->d->x0 + (ix + c->xi[p]) * c->dx;
      double y = c->dim == 2 ? c->d->y0 + (iy + c->xi[q]) * c->dy : 0.0;
      or_flux_x(c->d, ui[i][k], x, 0, f[k]);
      if (c->dim == 2) or_flux(c->d, ui[i][k], 1, g[k]);
      or_source(c->d, ui[i][k], x, y, src[k]);
    }
    /* Dloc f = (1/dx) D f along x-lines (+ (1/dy) D g along y-lines), Sec. 3 */
    for (int k = 0; k < np; ++k) {
      int p = k % n, q = k / n;
      for (int v = 0; v < M; ++v) {
        double dfx = 0.0, dgy = 0.0;
        for (int r = 0; r < n; ++r) dfx += c->D[p * n + r] * f[node(c, r, q)][v];
        if (c->dim == 2)
          for (int r = 0; r < n; ++r) dgy += c->D[q * n + r] * g[node(c, p, r)][v];
        L[i][k][v] = dfx / c->dx + (c->dim == 2 ? dgy / c->dy : 0.0) - src[k][v];
      }
    }
    /* time averages */
    for (int k = 0; k < np; ++k)
      for (int v = 0; v < M; ++v) {
        F[k * M + v] += c->b[i] * f[k][v];
        if (c->dim == 2) G[k * M + v] += c->b[i] * g[k][v];
        U[k * M + v] += c->b[i] * ui[i][k][v];
        S[k * M + v] += c->b[i] * src[k][v];
      }
    if (!ea) continue;
    /* EA: evaluate the flux at the extrapolated stage traces */
    for (int q = 0; q < nq; ++q) {
      double uL[OR_MAXM], uR[OR_MAXM], fL[OR_MAXM], fR[OR_MAXM];
      for (int v = 0; v < M; ++v) {
        uL[v] = uR[v] = 0.0;
        for (int p = 0; p < n; ++p) {
          uL[v] += c->l0[p] * ui[i][node(c, p, q)][v];
          uR[v] += c->l1[p] * ui[i][node(c, p, q)][v];
        }
      }
      or_flux_x(c->d, uL, c->d->x0 + ix * c->dx, 0, fL);
      or_flux_x(c->d, uR, c->d->x0 + (ix + 1) * c->dx, 0, fR);
      for (int v = 0; v < M; ++v) {
        ea[(0 * NMAX + q) * OR_MAXM + v] += c->b[i] * fL[v];
        ea[(1 * NMAX + q) * OR_MAXM + v] += c->b[i] * fR[v];
        if (stg) {
          stg[((i * 4 + 0) * NMAX + q) * OR_MAXM + v] = uL[v];
          stg[((i * 4 + 1) * NMAX + q) * OR_MAXM + v] = uR[v];
        }
      }
    }
    if (c->dim == 2)
      for (int p = 0; p < n; ++p) {
        double uB[OR_MAXM], uT[OR_MAXM], gB[OR_MAXM], gT[OR_MAXM];
        for (int v = 0; v < M; ++v) {
          uB[v] = uT[v] = 0.0;
          for (int q = 0; q < n; ++q) {
            uB[v] += c->l0[q] * ui[i][node(c, p, q)][v];
            uT[v] += c->l1[q] * ui[i][node(c, p, q)][v];
          }
        }
        or_flux(c->d, uB, 1, gB);
        or_flux(c->d, uT, 1, gT);
        for (int v = 0; v < M; ++v) {
          ea[(2 * NMAX + p) * OR_MAXM + v] += c->b[i] * gB[v];
          ea[(3 * NMAX + p) * OR_MAXM + v] += c->b[i] * gT[v];
          if (stg) {
            stg[((i * 4 + 2) * NMAX + p) * OR_MAXM + v] = uB[v];
            stg[((i * 4 + 3) * NMAX + p) * OR_MAXM + v] = uT[v];
          }
        }
      }
  }
}

void or_local_crk(const or_desc* d, const double* ue, double dt, int ix, int iy, double* F,
                  double* G, double* U, double* S) {
  ctx c;
  ctx_init(&c, d);
  local_crk_ea(&c, ue, dt, ix, iy, F, G, U, S, NULL, NULL);
}

/* trace of nodal data X[k][v] on face side f at face node j (Sec. 2 eq. (soln.poly)
 * evaluated at xi = 0 or 1 along one line) */
static void trace(const ctx* c, const double* X, int f, int j, double* out) {
  for (int v = 0; v < c->M; ++v) {
    double acc = 0.0;
    for (int r = 0; r < c->n; ++r) {
      int k = f < 2 ? node(c, r, j) : node(c, j, r);
      double l = (f == 0 || f == 2) ? c->l0[r] : c->l1[r];
      acc += l * X[k * c->M + v];
    }
    out[v] = acc;
  }
}

/* ------------------------------------------------------------------------ */
/* Smoothness indicator (Sec. 4, cited from Hennemann et al. 2021; constants are
 * the reading of that paper):
 *   eps = u (scalar), rho p (Euler), rho (p11 + p22)/2 (ten-moment);
 *   Legendre modes m_j = (2j+1) sum_p w_p eps_p L_j(2 xi_p - 1) (tensor modes in 2D);
 *   E = max(top-mode energy / total, next-to-top energy / energy up to N-1)
 *   (the second ratio only for N >= 2);
 *   T = 0.5 10^(-1.8 (N+1)^0.25), s = ln((1 - 1e-4)/1e-4),
 *   alpha = 1 / (1 + exp(-s (E - T) / T)), alpha < 1e-3 -> 0, alpha > 1 - 1e-3 -> 1. */
static double legendre01(int j, double xi) {
  double x = 2.0 * xi - 1.0, p0 = 1.0, p1 = x;
  if (j == 0) return 1.0;
  for (int k = 1; k < j; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

static double indicator_variable(const or_desc* d, const double* u) {
  if (d->equation == OR_EQ_LINADV || d->equation == OR_EQ_BURGERS || d->equation == OR_EQ_VARADV) return u[0];
  if (d->equation == OR_EQ_EULER) return u[0] * or_constraint(d, u, 1);
  double rho = u[0], v1 = u[1] / rho, v2 = u[2] / rho;
  double p11 = 2.0 * u[3] - rho * v1 * v1, p22 = 2.0 * u[5] - rho * v2 * v2;
  return rho * 0.5 * (p11 + p22);
}

/* Legendre modes of the indicator variable of one element, m[i + n j] for the
 * x-mode i and the y-mode j (j = 0 in 1D): the indicator's own modes, which
 * both the indicator and the learned alpha's inputs are built from. */
static void indicator_modes(const ctx* c, const or_desc* d, const double* ue, double* m) {
  const int n = c->n;
  double eps[NPMAX];
  for (int k = 0; k < c->np; ++k) eps[k] = indicator_variable(d, ue + k * c->M);
  for (int k = 0; k < c->np; ++k) {
    int i = k % n, j = k / n;
    double acc = 0.0;
    if (c->dim == 1) {
      for (int p = 0; p < n; ++p) acc += c->w[p] * eps[p] * legendre01(i, c->xi[p]);
      m[k] = (2.0 * i + 1.0) * acc;
    } else {
      for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
          acc += c->w[p] * c->w[q] * eps[node(c, p, q)] * legendre01(i, c->xi[p]) * legendre01(j, c->xi[q]);
      m[k] = (2.0 * i + 1.0) * (2.0 * j + 1.0) * acc;
    }
  }
}

void or_modal_energies(const or_desc* d, const double* ue, double* e) {
  ctx c;
  ctx_init(&c, d);
  double m[NPMAX], tot = 0.0;
  indicator_modes(&c, d, ue, m);
  for (int k = 0; k < c.np; ++k) tot += m[k] * m[k];
  for (int k = 0; k < c.np; ++k) e[k] = tot > 0.0 ? m[k] * m[k] / tot : 0.0;
}

double or_indicator(const or_desc* d, const double* ue) {
  ctx c;
  ctx_init(&c, d);
  const int n = c.n, N = c.N;
  double m[NPMAX];
  indicator_modes(&c, d, ue, m);
  double E;
  if (c.dim == 1) {
    double tot = 0.0, tot1 = 0.0;
    for (int j = 0; j <= N; ++j) tot += m[j] * m[j];
    for (int j = 0; j <= N - 1; ++j) tot1 += m[j] * m[j];
    double r1 = tot > 0.0 ? m[N] * m[N] / tot : 0.0;
    double r2 = (N >= 2 && tot1 > 0.0) ? m[N - 1] * m[N - 1] / tot1 : 0.0;
    E = fmax(r1, r2);
  } else {
    double tot = 0.0, top = 0.0, low = 0.0, top1 = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double e2 = m[i + n * j] * m[i + n * j];
        int mx = i > j ? i : j;
        tot += e2;
        if (mx == N) top += e2;
        if (mx <= N - 1) low += e2;
        if (mx == N - 1) top1 += e2;
      }
    double r1 = tot > 0.0 ? top / tot : 0.0;
    double r2 = (N >= 2 && low > 0.0) ? top1 / low : 0.0;
    E = fmax(r1, r2);
  }
  double T = 0.5 * pow(10.0, -1.8 * pow(N + 1.0, 0.25));
  double s = log((1.0 - 1e-4) / 1e-4);
  double alpha = 1.0 / (1.0 + exp(-s / T * (E - T)));
  if (alpha < 1e-3) alpha = 0.0;
  if (alpha > 1.0 - 1e-3) alpha = 1.0;
  return fmin(alpha, 1.0);
}

/* ------------------------------------------------------------------------ */
/* MUSCL-Hancock on the subcells (Sec. 4.2; the scheme on non-centred subcells is
 * cited from another paper, reading):
 *   slope s_p = minmod(beta D-/h-, Dc/hc, beta D+/h+), beta = 2 - alpha_e, per
 *   conserved variable, with the neighbour element's node across a face;
 *   face states u_p^{-+} = u_p + s_p (x_{p-+1/2} - x_p);
 *   Hancock: u^{*} = u^{face} - dt/2 [ (f(u^{x+}) - f(u^{x-}))/(w_p dx)
 *                                     + (g(u^{y+}) - g(u^{y-}))/(w_q dy) ];
 *   if any face state or evolved state is inadmissible the slopes are zeroed.
 * First order (Sec. 4.1) is the same with all slopes zero.
 * ustar is [Np][4][M] for one element (x-, x+, y-, y+). */
static double minmod3(double a, double b, double c) {
  if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
  if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
  return 0.0;
}

/* Solid wall (Sec. 3.3 eq. (reflect.time.avg), Euler): the ghost state is the
 * interior state with the velocity normal to the face (direction dir)
 * reversed; the ghost normal flux is the interior one with every component
 * but the normal momentum reversed. */
/* Boundary type of side s (0 x-, 1 x+, 2 y-, 3 y+). */
static int side_bc(const ctx* c, int s) {
  if (c->d->bc_side[s] != 0) return c->d->bc_side[s];
  return s < 2 ? c->d->bc_x : c->d->bc_y;
}

/* Given ghost state g of side s at time t: bc_state, or for a scalar equation
 * with bc_time_terms > 0 the Chebyshev series sum_k a_k T_k(tau) (Clenshaw's
 * recurrence), tau = 2 (t - t0)/(t1 - t0) - 1 clamped to [-1, 1]. */
static void ghost_at(const ctx* c, int s, double t, double* g) {
  const or_desc* d = c->d;
  if (d->bc_time_terms <= 0 || c->M != 1) {
    for (int v = 0; v < c->M; ++v) g[v] = d->bc_state[s][v];
    return;
  }
  double tau = 2.0 * (t - d->bc_time_span[0]) / (d->bc_time_span[1] - d->bc_time_span[0]) - 1.0;
  tau = fmin(1.0, fmax(-1.0, tau));
  double b1 = 0.0, b2 = 0.0;
  for (int k = d->bc_time_terms - 1; k >= 1; --k) {
    double b0 = 2.0 * tau * b1 - b2 + d->bc_time_coef[s][k];
    b2 = b1;
    b1 = b0;
  }
  g[0] = tau * b1 - b2 + d->bc_time_coef[s][0];
}

/* Ghost node of the MUSCL-Hancock reconstruction beyond side s, from the own
 * boundary node ub: the node itself (outflow), its reflection (wall), or the
 * given state at t^n (Dirichlet, inflow). */
static void ghost_node(const ctx* c, int s, const double* ub, double* out) {
  int bc = side_bc(c, s);
  if (bc == OR_BC_WALL) { for (int v = 0; v < c->M; ++v) out[v] = (v == 1 + s / 2) ? -ub[v] : ub[v]; }
  else if (bc == OR_BC_DIRICHLET || bc == OR_BC_INFLOW) ghost_at(c, s, c->d->time, out);
  else { for (int v = 0; v < c->M; ++v) out[v] = ub[v]; }
}

/* Time-dependent ghost values of a Dirichlet / inflow side (Sec. 3.3):
 * g at the stage times t^n + c_i dt, U^- = sum_i b_i g_i and F^- =
 * sum_i b_i f(x, g_i); for a time-independent g they are g and f(g). */
static void ghost_averages(const ctx* c, int s, double dt, double x, int dir, double gst[][OR_MAXM],
                           double* Ug, double* Fg) {
  const int M = c->M;
  if (c->d->bc_time_terms <= 0 || M != 1) {
    for (int i = 0; i < c->s; ++i)
      for (int v = 0; v < M; ++v) gst[i][v] = c->d->bc_state[s][v];
    for (int v = 0; v < M; ++v) Ug[v] = c->d->bc_state[s][v];
    or_flux_x(c->d, c->d->bc_state[s], x, dir, Fg);
    return;
  }
  for (int v = 0; v < M; ++v) Ug[v] = Fg[v] = 0.0;
  for (int i = 0; i < c->s; ++i) {
    double f[OR_MAXM];
    ghost_at(c, s, c->d->time + c->c[i] * dt, gst[i]);
    or_flux_x(c->d, gst[i], x, dir, f);
    for (int v = 0; v < M; ++v) {
      Ug[v] += c->b[i] * gst[i][v];
      Fg[v] += c->b[i] * f[v];
    }
  }
}

static void reflect_state(const ctx* c, const double* u, int dir, double* out) {
  for (int v = 0; v < c->M; ++v) out[v] = (v == 1 + dir) ? -u[v] : u[v];
}

static void reflect_flux(const ctx* c, const double* f, int dir, double* out) {
  for (int v = 0; v < c->M; ++v) out[v] = (v == 1 + dir) ? f[v] : -f[v];
}

static void line_slope(const ctx* c, const double* u_line /* [N+3][M], index p+1 */,
                       const double* X /* [N+3] positions */, int p, double beta, double* slope) {
  for (int v = 0; v < c->M; ++v) {
    double um = u_line[(p) * c->M + v], u0 = u_line[(p + 1) * c->M + v],
           up = u_line[(p + 2) * c->M + v];
    double hm = X[p + 1] - X[p], hp = X[p + 2] - X[p + 1], hc = X[p + 2] - X[p];
    slope[v] = minmod3(beta * (u0 - um) / hm, (up - um) / hc, beta * (up - u0) / hp);
  }
}

static void muscl_hancock_element(const ctx* c, const double* u, int e, double alpha, double dt,
                                  int use_mh, double* ustar) {
  const int M = c->M, n = c->n, N = c->N;
  const double xe = c->d->x0 + (e % c->nx) * c->dx; /* left face of the element */
  double ue[NPMAX * OR_MAXM];
  gather(c, u, e, ue);
  double sx[NPMAX][OR_MAXM], sy[NPMAX][OR_MAXM];
  memset(sx, 0, sizeof(sx));
  memset(sy, 0, sizeof(sy));
  if (use_mh) {
    double beta = 2.0 - alpha;
    double X[NMAX + 2];
    X[0] = c->xi[N] - 1.0;
    for (int p = 0; p <= N; ++p) X[p + 1] = c->xi[p];
    X[N + 2] = 1.0 + c->xi[0];
    double line[(NMAX + 2) * OR_MAXM];
    double nb[NPMAX * OR_MAXM];
    /* x-lines */
    int eL = neighbour(c, e, 0), eR = neighbour(c, e, 1);
    for (int q = 0; q < c->nq; ++q) {
      for (int p = 0; p <= N; ++p)
        for (int v = 0; v < M; ++v) line[(p + 1) * M + v] = ue[node(c, p, q) * M + v];
      /* across a boundary: the ghost node of that side */
      if (eL >= 0) { gather(c, u, eL, nb); for (int v = 0; v < M; ++v) line[v] = nb[node(c, N, q) * M + v]; }
      else ghost_node(c, 0, ue + node(c, 0, q) * M, line);
      if (eR >= 0) { gather(c, u, eR, nb); for (int v = 0; v < M; ++v) line[(N + 2) * M + v] = nb[node(c, 0, q) * M + v]; }
      else ghost_node(c, 1, ue + node(c, N, q) * M, line + (N + 2) * M);
      for (int p = 0; p <= N; ++p) line_slope(c, line, X, p, beta, sx[node(c, p, q)]);
    }
    if (c->dim == 2) {
      int eB = neighbour(c, e, 2), eT = neighbour(c, e, 3);
      for (int p = 0; p <= N; ++p) {
        for (int q = 0; q <= N; ++q)
          for (int v = 0; v < M; ++v) line[(q + 1) * M + v] = ue[node(c, p, q) * M + v];
        if (eB >= 0) { gather(c, u, eB, nb); for (int v = 0; v < M; ++v) line[v] = nb[node(c, p, N) * M + v]; }
        else ghost_node(c, 2, ue + node(c, p, 0) * M, line);
        if (eT >= 0) { gather(c, u, eT, nb); for (int v = 0; v < M; ++v) line[(N + 2) * M + v] = nb[node(c, p, 0) * M + v]; }
        else ghost_node(c, 3, ue + node(c, p, N) * M, line + (N + 2) * M);
        for (int q = 0; q <= N; ++q) line_slope(c, line, X, q, beta, sy[node(c, p, q)]);
      }
    }
  }
  for (int k = 0; k < c->np; ++k) {
    int p = k % n, q = k / n;
    const double* uk = ue + k * M;
    double st[4][OR_MAXM];
    for (int pass = 0; pass < 2; ++pass) {
      /* pass 0 with the limited slopes, pass 1 with zero slopes (fallback) */
      double ax = pass == 0 ? 1.0 : 0.0;
      double face[4][OR_MAXM];
      for (int v = 0; v < M; ++v) {
        face[0][v] = uk[v] + ax * sx[k][v] * (c->xsub[p] - c->xi[p]);
        face[1][v] = uk[v] + ax * sx[k][v] * (c->xsub[p + 1] - c->xi[p]);
        face[2][v] = uk[v] + ax * sy[k][v] * (c->xsub[q] - c->xi[q]);
        face[3][v] = uk[v] + ax * sy[k][v] * (c->xsub[q + 1] - c->xi[q]);
      }
      double fm[OR_MAXM], fp[OR_MAXM], gm[OR_MAXM], gp[OR_MAXM], delta[OR_MAXM];
      or_flux_x(c->d, face[0], xe + c->xsub[p] * c->dx, 0, fm);
      or_flux_x(c->d, face[1], xe + c->xsub[p + 1] * c->dx, 0, fp);
      if (c->dim == 2) {
        or_flux(c->d, face[2], 1, gm);
        or_flux(c->d, face[3], 1, gp);
      }
      for (int v = 0; v < M; ++v) {
        delta[v] = 0.5 * dt * (fp[v] - fm[v]) / (c->w[p] * c->dx);
        if (c->dim == 2) delta[v] += 0.5 * dt * (gp[v] - gm[v]) / (c->w[q] * c->dy);
      }
      int nface = c->dim == 2 ? 4 : 2;
      int ok = 1;
      for (int f = 0; f < nface; ++f) {
        for (int v = 0; v < M; ++v) st[f][v] = face[f][v] - delta[v];
        if (!admissible(c, face[f]) || !admissible(c, st[f])) ok = 0;
      }
      if (ok || pass == 1) break;
    }
    for (int f = 0; f < 4; ++f)
      for (int v = 0; v < M; ++v) ustar[(k * 4 + f) * M + v] = (c->dim == 2 || f < 2) ? st[f][v] : 0.0;
  }
}

/* ------------------------------------------------------------------------ */
/* Zhang-Shu scaling limiter (cited in Sec. 3.2; reading): with the element mean
 * u_bar admissible, eps_k = min(1e-12, P_k(u_bar));
 *   density:  rho_p <- rho_bar + theta1 (rho_p - rho_bar),
 *             theta1 = (rho_bar - eps1)/(rho_bar - min rho) if min rho < eps1;
 *   next constraint: for each checked point with P_2 < eps2, t solves
 *             P_2(u_bar + t (u - u_bar)) = eps2 by 50 bisection steps (taking the
 *             admissible end); theta2 = min t; u_p <- u_bar + theta2 (u_p - u_bar).
 * Checked points: the solution points (Definition 1) and, with OR_LIM_TRACES,
 * the traces on the element faces. */
static int check_points(const ctx* c, const double* ue, double* pts /* [*][M] */) {
  int npts = 0;
  for (int k = 0; k < c->np; ++k, ++npts)
    for (int v = 0; v < c->M; ++v) pts[npts * c->M + v] = ue[k * c->M + v];
  if (c->d->limiter & OR_LIM_TRACES) {
    int nside = c->dim == 2 ? 4 : 2;
    for (int f = 0; f < nside; ++f) {
      int nj = f < 2 ? c->nq : c->n;
      for (int j = 0; j < nj; ++j, ++npts) trace(c, ue, f, j, pts + npts * c->M);
    }
  }
  return npts;
}

int or_scaling_limiter(const or_desc* d, double* ue) {
  ctx c;
  ctx_init(&c, d);
  const int M = c.M;
  if (c.K == 0) return 0;
  double ubar[OR_MAXM] = {0};
  for (int k = 0; k < c.np; ++k)
    for (int v = 0; v < M; ++v) ubar[v] += node_weight(&c, k) * ue[k * M + v];
  double rho_bar = ubar[0];
  if (!(rho_bar > 0.0) || !(or_constraint(d, ubar, 1) > 0.0)) return 1;
  double pts[(NPMAX + 4 * NMAX) * OR_MAXM];
  /* density */
  double eps1 = fmin(1e-12, rho_bar);
  int npts = check_points(&c, ue, pts);
  double rmin = pts[0];
  for (int t = 1; t < npts; ++t) rmin = fmin(rmin, pts[t * M]);
  if (rmin < eps1) {
    double th = (rho_bar - eps1) / (rho_bar - rmin);
    for (int k = 0; k < c.np; ++k) ue[k * M] = rho_bar + th * (ue[k * M] - rho_bar);
  }
  /* second constraint */
  double eps2 = fmin(1e-12, or_constraint(d, ubar, 1));
  npts = check_points(&c, ue, pts);
  double th2 = 1.0;
  for (int t = 0; t < npts; ++t) {
    const double* up = pts + t * M;
    if (or_constraint(d, up, 1) >= eps2) continue;
    double lo = 0.0, hi = 1.0, tmp[OR_MAXM];
    for (int it = 0; it < 50; ++it) {
      double mid = 0.5 * (lo + hi);
      for (int v = 0; v < M; ++v) tmp[v] = ubar[v] + mid * (up[v] - ubar[v]);
      if (or_constraint(d, tmp, 1) >= eps2) lo = mid; else hi = mid;
    }
    th2 = fmin(th2, lo);
  }
  if (th2 < 1.0)
    for (int k = 0; k < c.np; ++k)
      for (int v = 0; v < M; ++v) ue[k * M + v] = ubar[v] + th2 * (ue[k * M + v] - ubar[v]);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Time step, Sec. 5 eq. (time.step.2d) from the element means. */
double or_max_rate(const or_desc* d, const double* u) {
  ctx c;
  ctx_init(&c, d);
  double ue[NPMAX * OR_MAXM], rmax = 0.0;
  for (int e = 0; e < c.ne; ++e) {
    gather(&c, u, e, ue);
    double ubar[OR_MAXM] = {0};
    for (int k = 0; k < c.np; ++k)
      for (int v = 0; v < c.M; ++v) ubar[v] += node_weight(&c, k) * ue[k * c.M + v];
    double r;
    if (c.dim == 2) {
      r = or_wave_speed(d, ubar, 0) / c.dx + or_wave_speed(d, ubar, 1) / c.dy;
    } else {
      /* sigma of the mean at the element's faces and solution points (they
       * differ only for variable advection; reading) */
      double xe = d->x0 + (e % c.nx) * c.dx, s = fmax(or_wave_speed_x(d, ubar, xe, 0),
                                                       or_wave_speed_x(d, ubar, xe + c.dx, 0));
      for (int p = 0; p < c.n; ++p) s = fmax(s, or_wave_speed_x(d, ubar, xe + c.xi[p] * c.dx, 0));
      r = s / c.dx;
    }
    rmax = fmax(rmax, r);
  }
  return rmax;
}

double or_dt(const or_desc* d, const double* u) {
  return d->cfl_safety * d->cfl / or_max_rate(d, u);
}

/* ------------------------------------------------------------------------ */
typedef struct {
  double *F, *G, *S;      /* [ne][np][M] */
  double *ea, *Ut, *unt, *Fd; /* [ne][4][NMAX][M] */
  double *ustar;          /* [ne][np][4][M] */
  double *fsx, *fsy;      /* [ne][NMAX][NMAX+1][M]: line, subface p-1/2 (p=0..N+1), var */
  double *alpha;          /* [ne] */
  double *fnum;           /* [ne][4][NMAX][M] numerical flux on each face side */
  double *theta;          /* [ne][4][NMAX] */
  double *stg;            /* [ne][s][4][NMAX][M] stage traces (D-CSX) */
} work_t;

#define W4(arr, e, f, j, v) arr[((((size_t)(e)) * 4 + (f)) * NMAX + (j)) * OR_MAXM + (v)]
#define WST(arr, e, i, f, j, v) arr[(((((size_t)(e)) * OR_MAXS + (i)) * 4 + (f)) * NMAX + (j)) * OR_MAXM + (v)]
#define WS(arr, e, l, j, v) arr[((((size_t)(e)) * NMAX + (l)) * (NMAX + 1) + (j)) * OR_MAXM + (v)]

/* Central part F^{+-} of eq. (numflux.general) on face side f of element e at
 * face node j: EA, eq. (evaluate) (the stage fluxes at the face, averaged), or
 * AE, eq. (extrapolate) (the trace of the time-averaged flux). */
static const double* central_part(const ctx* c, const work_t* W, int e, int f, int j) {
  return c->d->central == OR_CENTRAL_AE ? &W4(W->Fd, e, f, j, 0) : &W4(W->ea, e, f, j, 0);
}

/* High-order numerical flux eq. (numflux.general), F = (F^- + F^+)/2 - D, from
 * the face data of the left (L) and right (R) sides: central parts Fc, u^n
 * traces un, time-averaged solution traces U and stage traces st.
 *   D2,    eq. (D2):   D = lambda/2 (U^+ - U^-),
 *   D1,    eq. (D1):   D = lambda/2 (u^+ - u^-),
 *          lambda = max(sigma(u^-), sigma(u^+)) from the u^n traces (eq. (rusanov.wave.speed));
 *   D-CSX, eq. (dcsx): D = sum_i b_i lambda_i/2 (u^(i)+ - u^(i)-), lambda_i from the stage traces. */
static void high_order_flux(const ctx* c, int dir, double x, const double* FcL, const double* FcR,
                            const double* unL, const double* unR, const double* UL, const double* UR,
                            double stL[][OR_MAXM], double stR[][OR_MAXM], double* FHO) {
  const int M = c->M;
  if (c->d->dissipation == OR_DISS_DCSX) {
    double Dv[OR_MAXM] = {0};
    for (int i = 0; i < c->s; ++i) {
      if (c->b[i] == 0.0) continue;
      double lam = fmax(or_wave_speed_x(c->d, stL[i], x, dir), or_wave_speed_x(c->d, stR[i], x, dir));
      for (int v = 0; v < M; ++v) Dv[v] += c->b[i] * 0.5 * lam * (stR[i][v] - stL[i][v]);
    }
    for (int v = 0; v < M; ++v) FHO[v] = 0.5 * (FcL[v] + FcR[v]) - Dv[v];
    return;
  }
  double lam = fmax(or_wave_speed_x(c->d, unL, x, dir), or_wave_speed_x(c->d, unR, x, dir));
  const double* jL = c->d->dissipation == OR_DISS_D1 ? unL : UL;
  const double* jR = c->d->dissipation == OR_DISS_D1 ? unR : UR;
  for (int v = 0; v < M; ++v) FHO[v] = 0.5 * (FcL[v] + FcR[v]) - 0.5 * lam * (jR[v] - jL[v]);
}

/* Numerical flux on one face node between elements eL (left/bottom) and eR
 * (right/top) in direction dir; either may be -1 at an outflow or wall boundary.
 *   high order: Sec. 3.1 eq. (numflux.general) with D2 (eq. (D2)) and EA (eq. (evaluate)),
 *               lambda from the u^n traces (eq. (rusanov.wave.speed));
 *   outflow boundary: F = the interior trace flux (Sec. 3.3);
 *   wall boundary: the same D2 flux with the ghost values of eq.
 *     (reflect.time.avg) (u^n trace, time-averaged flux and solution reflected)
 *     and, for the low-order flux, the reflected evolved boundary state;
 *   Dirichlet boundary (the inflow/outflow ghost values of Sec. 3.3 for a
 *     time-independent g): u^- = U^- = g, F^- = f(g), stage traces g, then the
 *     scheme's own flux (the paper takes an HLLC flux there; reading) and,
 *     for the low-order flux, Rusanov between the evolved boundary state and g;
 *   fully inflow boundary: F = F^- = f(g) (Sec. 3.3), high and low order;
 *   low order: the subcell flux at the element face (eqs. (fo.at.face), (mh.at.face));
 *   blend: eq. (Fblend) with alpha_{e+1/2} = (alpha_L + alpha_R)/2 (reading);
 *   flux limiter (Sec. 4.3, Theorem 1; the algorithm is cited, reading):
 *     candidates u~_L = u_{L,N} - dt/(kappa w_N dx) (F - f^L_{N-1/2}),
 *                u~_R = u_{R,0} - dt/(kappa w_0 dx) (f^R_{1/2} - F),
 *     kappa = 1 (1D) or 1/2 (2D); per constraint k: eps_k = 0.1 min P_k(u~(f_LO));
 *     F_theta = theta F + (1 - theta) f_LO is shrunk towards f_LO until
 *     P_k(u~) >= eps_k on both sides, using concavity of P_k. */
static void face_flux(const ctx* c, const double* u, const work_t* W, int dir, int eL, int eR, int j,
                      double dt, double* Fout, double* theta_out) {
  const int M = c->M, N = c->N;
  const int fL = dir == 0 ? 1 : 3, fR = dir == 0 ? 0 : 2;
  const int kL = dir == 0 ? node(c, N, j) : node(c, j, N);
  const int kR = dir == 0 ? node(c, 0, j) : node(c, j, 0);
  const int hL = dir == 0 ? 1 : 3, hR = dir == 0 ? 0 : 2; /* ustar slots x+ / x- (y+ / y-) */
  double FHO[OR_MAXM], fLO[OR_MAXM], alpha_f;
  const int S = c->s;
  /* boundary side of this face when one neighbour is missing */
  const int side = eR >= 0 ? (dir == 0 ? 0 : 2) : (dir == 0 ? 1 : 3);
  const int bc = (eL >= 0 && eR >= 0) ? OR_BC_PERIODIC : side_bc(c, side);
  /* position of the face along x (variable advection) */
  const double xf = dir == 1 ? 0.0
                    : c->d->x0 + (eR >= 0 ? (eR % c->nx) : (eL % c->nx) + 1) * c->dx;
  if (eL >= 0 && eR >= 0) {
    double stL[OR_MAXS][OR_MAXM], stR[OR_MAXS][OR_MAXM];
    for (int i = 0; i < S; ++i)
      for (int v = 0; v < M; ++v) {
        stL[i][v] = WST(W->stg, eL, i, fL, j, v);
        stR[i][v] = WST(W->stg, eR, i, fR, j, v);
      }
    high_order_flux(c, dir, xf, central_part(c, W, eL, fL, j), central_part(c, W, eR, fR, j),
                    &W4(W->unt, eL, fL, j, 0), &W4(W->unt, eR, fR, j, 0), &W4(W->Ut, eL, fL, j, 0),
                    &W4(W->Ut, eR, fR, j, 0), stL, stR, FHO);
    rusanov(c, &W->ustar[(((size_t)eL * c->np + kL) * 4 + hL) * M],
            &W->ustar[(((size_t)eR * c->np + kR) * 4 + hR) * M], dir, xf, fLO);
    alpha_f = 0.5 * (W->alpha[eL] + W->alpha[eR]);
  } else if (bc == OR_BC_WALL || bc == OR_BC_DIRICHLET) {
    /* the interior side (ei, face side fi) and its ghost: reflected (wall) or
     * the given state g with F^- = f(g) (Dirichlet) */
    const int ei = eR >= 0 ? eR : eL, fi = eR >= 0 ? fR : fL;
    const int ki = eR >= 0 ? kR : kL, hi = eR >= 0 ? hR : hL;
    double ug[OR_MAXM], Fg[OR_MAXM], Ug[OR_MAXM], usg[OR_MAXM];
    double sti[OR_MAXS][OR_MAXM], stg[OR_MAXS][OR_MAXM];
    const double* Fi = central_part(c, W, ei, fi, j);
    const double* usi = &W->ustar[(((size_t)ei * c->np + ki) * 4 + hi) * M];
    for (int i = 0; i < S; ++i)
      for (int v = 0; v < M; ++v) sti[i][v] = WST(W->stg, ei, i, fi, j, v);
    if (bc == OR_BC_WALL) {
      reflect_state(c, &W4(W->unt, ei, fi, j, 0), dir, ug);
      reflect_flux(c, Fi, dir, Fg);
      reflect_state(c, &W4(W->Ut, ei, fi, j, 0), dir, Ug);
      for (int i = 0; i < S; ++i) reflect_state(c, sti[i], dir, stg[i]);
      reflect_state(c, usi, dir, usg);
    } else {
      ghost_at(c, side, c->d->time, ug);
      for (int v = 0; v < M; ++v) usg[v] = ug[v];
      ghost_averages(c, side, dt, xf, dir, stg, Ug, Fg);
    }
    /* (left, right) = (ghost, interior) at a left/bottom wall, (interior, ghost) at a right/top wall */
    if (bc == OR_BC_DIRICHLET && c->d->bc_flux == 1) {
      /* HLLC on the time-averaged ghost values (high order) and on the evolved
       * boundary state against g (low order) */
      double fi_lo[OR_MAXM], fg_lo[OR_MAXM];
      const double* Ui = &W4(W->Ut, ei, fi, j, 0);
      or_flux(c->d, usi, dir, fi_lo);
      or_flux(c->d, usg, dir, fg_lo);
      if (eR >= 0) { hllc(c, dir, Ug, Ui, Fg, Fi, FHO); hllc(c, dir, usg, usi, fg_lo, fi_lo, fLO); }
      else { hllc(c, dir, Ui, Ug, Fi, Fg, FHO); hllc(c, dir, usi, usg, fi_lo, fg_lo, fLO); }
      alpha_f = W->alpha[ei];
    } else {
    if (eR >= 0)
      high_order_flux(c, dir, xf, Fg, Fi, ug, &W4(W->unt, ei, fi, j, 0), Ug, &W4(W->Ut, ei, fi, j, 0),
                      stg, sti, FHO);
    else
      high_order_flux(c, dir, xf, Fi, Fg, &W4(W->unt, ei, fi, j, 0), ug, &W4(W->Ut, ei, fi, j, 0), Ug,
                      sti, stg, FHO);
    if (eR >= 0) rusanov(c, usg, usi, dir, xf, fLO);
    else rusanov(c, usi, usg, dir, xf, fLO);
    alpha_f = W->alpha[ei];
    }
  } else if (bc == OR_BC_INFLOW) {
    /* fully inflow (Sec. 3.3): F = F^- (f(g) for a time-independent g) for both fluxes */
    double gst[OR_MAXS][OR_MAXM], Ug[OR_MAXM];
    ghost_averages(c, side, dt, xf, dir, gst, Ug, FHO);
    for (int v = 0; v < M; ++v) fLO[v] = FHO[v];
    alpha_f = W->alpha[eR >= 0 ? eR : eL];
  } else if (eR >= 0) {
    const double* Fc = central_part(c, W, eR, fR, j);
    for (int v = 0; v < M; ++v) FHO[v] = Fc[v];
    or_flux_x(c->d, &W->ustar[(((size_t)eR * c->np + kR) * 4 + hR) * M], xf, dir, fLO);
    alpha_f = W->alpha[eR];
  } else {
    const double* Fc = central_part(c, W, eL, fL, j);
    for (int v = 0; v < M; ++v) FHO[v] = Fc[v];
    or_flux_x(c->d, &W->ustar[(((size_t)eL * c->np + kL) * 4 + hL) * M], xf, dir, fLO);
    alpha_f = W->alpha[eL];
  }
  double F[OR_MAXM];
  int blend = (c->d->limiter & OR_LIM_BLEND) || c->d->alpha_mode == OR_ALPHA_FIXED;
  for (int v = 0; v < M; ++v) F[v] = blend ? (1.0 - alpha_f) * FHO[v] + alpha_f * fLO[v] : FHO[v];
  double theta = 1.0;
  if ((c->d->limiter & OR_LIM_FLUX) && c->K > 0) {
    double kappa = c->dim == 2 ? 0.5 : 1.0;
    double h = dir == 0 ? c->dx : c->dy;
    double cL = dt / (kappa * c->w[N] * h), cR = dt / (kappa * c->w[0] * h);
    double baseL[OR_MAXM], baseR[OR_MAXM], adjL[OR_MAXM], adjR[OR_MAXM];
    if (eL >= 0)
      for (int v = 0; v < M; ++v) {
        baseL[v] = u[((size_t)v * c->ne + eL) * c->np + kL];
        adjL[v] = WS((dir == 0 ? W->fsx : W->fsy), eL, j, N, v); /* f_{N-1/2} */
      }
    if (eR >= 0)
      for (int v = 0; v < M; ++v) {
        baseR[v] = u[((size_t)v * c->ne + eR) * c->np + kR];
        adjR[v] = WS((dir == 0 ? W->fsx : W->fsy), eR, j, 1, v); /* f_{1/2} */
      }
    for (int k = 0; k < c->K; ++k) {
      double cand[OR_MAXM], PlowL = 0.0, PlowR = 0.0, eps = INFINITY;
      if (eL >= 0) {
        for (int v = 0; v < M; ++v) cand[v] = baseL[v] - cL * (fLO[v] - adjL[v]);
        PlowL = or_constraint(c->d, cand, k);
        eps = fmin(eps, PlowL);
      }
      if (eR >= 0) {
        for (int v = 0; v < M; ++v) cand[v] = baseR[v] - cR * (adjR[v] - fLO[v]);
        PlowR = or_constraint(c->d, cand, k);
        eps = fmin(eps, PlowR);
      }
      eps *= 0.1;
      if (!(eps > 0.0)) { theta = 0.0; break; } /* the low-order update itself is not admissible */
      double Ft[OR_MAXM], tk = 1.0;
      for (int v = 0; v < M; ++v) Ft[v] = theta * F[v] + (1.0 - theta) * fLO[v];
      if (eL >= 0) {
        for (int v = 0; v < M; ++v) cand[v] = baseL[v] - cL * (Ft[v] - adjL[v]);
        double P = or_constraint(c->d, cand, k);
        if (P < eps) tk = fmin(tk, (PlowL - eps) / (PlowL - P));
      }
      if (eR >= 0) {
        for (int v = 0; v < M; ++v) cand[v] = baseR[v] - cR * (adjR[v] - Ft[v]);
        double P = or_constraint(c->d, cand, k);
        if (P < eps) tk = fmin(tk, (PlowR - eps) / (PlowR - P));
      }
      theta *= tk;
    }
  }
  for (int v = 0; v < M; ++v) Fout[v] = theta * F[v] + (1.0 - theta) * fLO[v];
  *theta_out = theta;
}

int or_step(const or_desc* d, const double* u_in, double dt, double* u_out, or_diag* diag) {
  ctx c;
  ctx_init(&c, d);
  const int M = c.M, n = c.n, N = c.N, np = c.np, ne = c.ne;
  int status = 0, bad = -1;
  work_t W;
  size_t nodal = (size_t)ne * np * M;
  W.F = calloc(nodal, sizeof(double));
  W.G = calloc(nodal, sizeof(double));
  W.S = calloc(nodal, sizeof(double));
  size_t facesz = (size_t)ne * 4 * NMAX * OR_MAXM;
  W.ea = calloc(facesz, sizeof(double));
  W.Ut = calloc(facesz, sizeof(double));
  W.unt = calloc(facesz, sizeof(double));
  W.Fd = calloc(facesz, sizeof(double));
  W.fnum = calloc(facesz, sizeof(double));
  W.theta = calloc((size_t)ne * 4 * NMAX, sizeof(double));
  W.ustar = calloc((size_t)ne * np * 4 * M, sizeof(double));
  size_t subsz = (size_t)ne * NMAX * (NMAX + 1) * OR_MAXM;
  W.fsx = calloc(subsz, sizeof(double));
  W.fsy = calloc(subsz, sizeof(double));
  W.alpha = calloc(ne, sizeof(double));
  W.stg = calloc((size_t)ne * OR_MAXS * 4 * NMAX * OR_MAXM, sizeof(double));
  double* alpha_raw = calloc(ne, sizeof(double));
  double ue[NPMAX * OR_MAXM], U[NPMAX * OR_MAXM], ea[4 * NMAX * OR_MAXM];
  const int nside = c.dim == 2 ? 4 : 2;

  /* 1. blending coefficient alpha_e from u^n (Sec. 4 eq. (blended.scheme)),
   *    smoothed as alpha_e <- max(alpha_e, max_neighbour alpha / 2) (reading) */
  for (int e = 0; e < ne; ++e) {
    if (d->alpha_mode == OR_ALPHA_FIXED) alpha_raw[e] = d->alpha_fixed;
    else if (!(d->limiter & OR_LIM_BLEND)) alpha_raw[e] = 0.0;
    else if (d->alpha_mode == OR_ALPHA_GIVEN) alpha_raw[e] = d->alpha_given[e];
    else { gather(&c, u_in, e, ue); alpha_raw[e] = or_indicator(d, ue); }
  }
  for (int e = 0; e < ne; ++e) {
    double a = alpha_raw[e];
    if (d->alpha_mode != OR_ALPHA_FIXED)
      for (int f = 0; f < nside; ++f) {
        int nb = neighbour(&c, e, f);
        if (nb >= 0) a = fmax(a, 0.5 * alpha_raw[nb]);
      }
    W.alpha[e] = a;
  }

  /* 2. local cRK, time averages and face traces of every element */
  for (int e = 0; e < ne; ++e) {
    int ix = e % c.nx, iy = e / c.nx;
    gather(&c, u_in, e, ue);
    local_crk_ea(&c, ue, dt, ix, iy, W.F + (size_t)e * np * M, W.G + (size_t)e * np * M, U,
                 W.S + (size_t)e * np * M, ea, &WST(W.stg, e, 0, 0, 0, 0));
    for (int f = 0; f < nside; ++f) {
      int nj = f < 2 ? c.nq : n;
      for (int j = 0; j < nj; ++j) {
        double tU[OR_MAXM], tu[OR_MAXM], tF[OR_MAXM];
        trace(&c, U, f, j, tU);                                              /* U^{+-}, eq. (D2) */
        trace(&c, ue, f, j, tu);                                             /* u^{n,+-} */
        trace(&c, (f < 2 ? W.F : W.G) + (size_t)e * np * M, f, j, tF);       /* F^delta at the face */
        for (int v = 0; v < M; ++v) {
          W4(W.ea, e, f, j, v) = ea[(f * NMAX + j) * OR_MAXM + v];
          W4(W.Ut, e, f, j, v) = tU[v];
          W4(W.unt, e, f, j, v) = tu[v];
          W4(W.Fd, e, f, j, v) = tF[v];
        }
      }
    }
  }

  /* 3. low-order subcell scheme: evolved face states and interior subcell fluxes */
  for (int e = 0; e < ne; ++e) {
    muscl_hancock_element(&c, u_in, e, W.alpha[e], dt, (d->limiter & OR_LIM_MH) != 0,
                          W.ustar + (size_t)e * np * 4 * M);
    const double* us = W.ustar + (size_t)e * np * 4 * M;
    const double xe = d->x0 + (e % c.nx) * c.dx;
    for (int q = 0; q < c.nq; ++q)
      for (int p = 1; p <= N; ++p) /* subface p-1/2 between nodes p-1 and p */
        rusanov(&c, &us[(node(&c, p - 1, q) * 4 + 1) * M], &us[(node(&c, p, q) * 4 + 0) * M], 0,
                xe + c.xsub[p] * c.dx, &WS(W.fsx, e, q, p, 0));
    if (c.dim == 2)
      for (int p = 0; p <= N; ++p)
        for (int q = 1; q <= N; ++q)
          rusanov(&c, &us[(node(&c, p, q - 1) * 4 + 3) * M], &us[(node(&c, p, q) * 4 + 2) * M], 1,
                  0.0, &WS(W.fsy, e, p, q, 0));
  }

  /* 4. one numerical flux per face node; each face is visited from the element on
   *    its right/top, plus the right/top boundary faces under outflow */
  for (int e = 0; e < ne; ++e) {
    for (int dir = 0; dir < c.dim; ++dir) {
      int nj = dir == 0 ? c.nq : n;
      int fneg = dir == 0 ? 0 : 2, fpos = dir == 0 ? 1 : 3;
      int eL = neighbour(&c, e, fneg);
      for (int j = 0; j < nj; ++j) {
        double Fn[OR_MAXM], th;
        face_flux(&c, u_in, &W, dir, eL, e, j, dt, Fn, &th);
        for (int v = 0; v < M; ++v) {
          W4(W.fnum, e, fneg, j, v) = Fn[v];
          if (eL >= 0) W4(W.fnum, eL, fpos, j, v) = Fn[v];
        }
        W.theta[((size_t)e * 4 + fneg) * NMAX + j] = th;
        if (eL >= 0) W.theta[((size_t)eL * 4 + fpos) * NMAX + j] = th;
      }
      if (neighbour(&c, e, fpos) < 0)
        for (int j = 0; j < nj; ++j) {
          double Fn[OR_MAXM], th;
          face_flux(&c, u_in, &W, dir, e, -1, j, dt, Fn, &th);
          for (int v = 0; v < M; ++v) W4(W.fnum, e, fpos, j, v) = Fn[v];
          W.theta[((size_t)e * 4 + fpos) * NMAX + j] = th;
        }
    }
  }

  /* 5. blended update (Sec. 4 eq. (blended.scheme)):
   *   R^H = D F + (F_{e+1/2} - F^delta(1)) g_R' + (F_{e-1/2} - F^delta(0)) g_L'
   *         with g_R'(xi_p) = l_p(1)/w_p, g_L'(xi_p) = -l_p(0)/w_p (Sec. 2, eq. (crkfr.avg));
   *   R^L_p = (f_{p+1/2} - f_{p-1/2}) / w_p with the element-face values F_{e-+1/2}
   *         (eq. (low.order.update));
   *   u^{n+1} = u^n - dt/dx [(1-alpha) R^H + alpha R^L] (+ y part) + dt S (App. B). */
  int use_blend = (d->limiter & OR_LIM_BLEND) || d->alpha_mode == OR_ALPHA_FIXED;
  for (int e = 0; e < ne; ++e) {
    gather(&c, u_in, e, ue);
    const double* Fe = W.F + (size_t)e * np * M;
    const double* Ge = W.G + (size_t)e * np * M;
    const double* Se = W.S + (size_t)e * np * M;
    double a = use_blend ? W.alpha[e] : 0.0;
    double un[NPMAX * OR_MAXM];
    for (int k = 0; k < np; ++k) {
      int p = k % n, q = k / n;
      for (int v = 0; v < M; ++v) {
        double RHx = 0.0;
        for (int r = 0; r < n; ++r) RHx += c.D[p * n + r] * Fe[node(&c, r, q) * M + v];
        RHx += (W4(W.fnum, e, 1, q, v) - W4(W.Fd, e, 1, q, v)) * c.gR[p];
        RHx += (W4(W.fnum, e, 0, q, v) - W4(W.Fd, e, 0, q, v)) * c.gL[p];
        double fr = p == N ? W4(W.fnum, e, 1, q, v) : WS(W.fsx, e, q, p + 1, v);
        double fl = p == 0 ? W4(W.fnum, e, 0, q, v) : WS(W.fsx, e, q, p, v);
        double RLx = (fr - fl) / c.w[p];
        double val = ue[k * M + v] - dt / c.dx * ((1.0 - a) * RHx + a * RLx);
        if (c.dim == 2) {
          double RHy = 0.0;
          for (int r = 0; r < n; ++r) RHy += c.D[q * n + r] * Ge[node(&c, p, r) * M + v];
          RHy += (W4(W.fnum, e, 3, p, v) - W4(W.Fd, e, 3, p, v)) * c.gR[q];
          RHy += (W4(W.fnum, e, 2, p, v) - W4(W.Fd, e, 2, p, v)) * c.gL[q];
          double gt = q == N ? W4(W.fnum, e, 3, p, v) : WS(W.fsy, e, p, q + 1, v);
          double gb = q == 0 ? W4(W.fnum, e, 2, p, v) : WS(W.fsy, e, p, q, v);
          double RLy = (gt - gb) / c.w[q];
          val -= dt / c.dy * ((1.0 - a) * RHy + a * RLy);
        }
        val += dt * Se[k * M + v];
        un[k * M + v] = val;
      }
    }
    /* 6. positivity scaling limiter */
    if ((d->limiter & OR_LIM_SCALING) && c.K > 0) {
      if (or_scaling_limiter(d, un) != 0 && status == 0) { status = 1; bad = e; }
    }
    for (int t = 0; t < np * M; ++t)
      if (!isfinite(un[t]) && status == 0) { status = 2; bad = e; }
    /* status: the element mean must be admissible.  The checked points are
     * the scaling limiter's business; it makes them admissible in exact
     * arithmetic, but a face trace interpolated from nodal values many orders of
     * magnitude larger than it carries a rounding error larger than a tiny
     * pressure, so the sign of P_k there is not decidable in FP64 and is not
     * tested (wave speeds take sqrt(max(c^2, 0))). */
    if (c.K > 0 && status == 0) {
      double ubar[OR_MAXM] = {0};
      for (int k = 0; k < np; ++k)
        for (int v = 0; v < M; ++v) ubar[v] += node_weight(&c, k) * un[k * M + v];
      if (!admissible(&c, ubar)) { status = 1; bad = e; }
    }
    scatter(&c, u_out, e, un);
  }

  if (diag) {
    diag->status = status;
    diag->bad_element = bad;
    for (int e = 0; e < ne; ++e) {
      if (diag->alpha) diag->alpha[e] = W.alpha[e];
      if (diag->alpha_raw) diag->alpha_raw[e] = alpha_raw[e];
      for (int j = 0; j < c.nq; ++j) {
        for (int v = 0; v < M; ++v) {
          if (diag->fnum_x) diag->fnum_x[((size_t)v * ne + e) * c.nq + j] = W4(W.fnum, e, 0, j, v);
          if (diag->fnum_x_right) diag->fnum_x_right[((size_t)v * ne + e) * c.nq + j] = W4(W.fnum, e, 1, j, v);
        }
        if (diag->theta_x) diag->theta_x[(size_t)e * c.nq + j] = W.theta[((size_t)e * 4 + 0) * NMAX + j];
      }
      if (c.dim == 2)
        for (int j = 0; j < n; ++j) {
          for (int v = 0; v < M; ++v) {
            if (diag->fnum_y) diag->fnum_y[((size_t)v * ne + e) * n + j] = W4(W.fnum, e, 2, j, v);
            if (diag->fnum_y_top) diag->fnum_y_top[((size_t)v * ne + e) * n + j] = W4(W.fnum, e, 3, j, v);
          }
          if (diag->theta_y) diag->theta_y[(size_t)e * n + j] = W.theta[((size_t)e * 4 + 2) * NMAX + j];
        }
      if (diag->source_mean)
        for (int v = 0; v < M; ++v) {
          double acc = 0.0;
          for (int k = 0; k < np; ++k) acc += node_weight(&c, k) * W.S[((size_t)e * np + k) * M + v];
          diag->source_mean[(size_t)v * ne + e] = acc;
        }
    }
  }
  free(W.F); free(W.G); free(W.S); free(W.ea); free(W.Ut); free(W.unt); free(W.Fd);
  free(W.fnum); free(W.theta); free(W.ustar); free(W.fsx); free(W.fsy); free(W.alpha); free(W.stg);
  free(alpha_raw);
  return status;
}

/* Time loop: dt from eq. (time.step.2d) each step, the last step clipped to land
 * exactly on t_final. */
int or_run(const or_desc* d, double* u, int max_steps, double t_final, double* t_out,
           int* steps_out) {
  ctx c;
  ctx_init(&c, d);
  size_t nvals = (size_t)c.ne * c.np * c.M;
  double* tmp = malloc(nvals * sizeof(double));
  double t = 0.0;
  int steps = 0, status = 0;
  or_desc dl = *d; /* its time field follows t^n */
  while (steps < max_steps && t < t_final) {
    double dt = or_dt(d, u);
    double remaining = t_final - t;
    int last = dt >= remaining;
    if (last) dt = remaining;
    dl.time = t;
    status = or_step(&dl, u, dt, tmp, NULL);
    memcpy(u, tmp, nvals * sizeof(double));
    t = last ? t_final : t + dt;
    ++steps;
    if (status) break;
  }
  free(tmp);
  if (t_out) *t_out = t;
  if (steps_out) *steps_out = steps;
  return status;
}
