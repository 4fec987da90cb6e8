// Host side of libcrkfr.so: reference tables, the Fourier CFL analysis, the
// device workspace, CUDA-graph launches of whole steps and the C ABI of
// include/cr.h.
#include <climits>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/cr.h"
#include "cr_batch.cuh"
#include "cr_launch.cuh"

using namespace crk;

namespace {

// ---------------------------------------------------------------------------
// Reference element (Sec. 2): Gauss-Legendre nodes on [0,1] by Newton's method
// on P_{N+1} from Chebyshev starting points; Lagrange values and the
// differentiation matrix from barycentric weights.
void legendre_pd(int n, double x, double* P, double* dP) {
  double pm = 1.0, p = x;
  if (n == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    const double pn = ((2 * k - 1) * x * p - (k - 1) * pm) / k;
    pm = p;
    p = pn;
  }
  *P = p;
  *dP = n * (pm - x * p) / (1.0 - x * x);
}

struct HostTables {
  int N, points;
  double xi[kMaxNodes1], w[kMaxNodes1], l0[kMaxNodes1], l1[kMaxNodes1];
  double D[kMaxNodes1 * kMaxNodes1];
};

// Gauss-Lobatto-Legendre nodes on [0,1] (Sec. 5.1): the end points and the
// roots of P_N', by Newton's method with P_N'' from Legendre's equation
// (1 - x^2) P'' = 2x P' - N(N+1) P, from the Chebyshev-Lobatto points;
// weights 2 / (N (N+1) P_N(x)^2), halved for [0,1].
void gll_nodes(int N, HostTables* t) {
  for (int i = 0; i <= N; ++i) {
    double x = i == 0 ? -1.0 : (i == N ? 1.0 : -std::cos(M_PI * i / N));
    if (i > 0 && i < N) {
      for (int it = 0; it < 60; ++it) {
        double P, dP;
        legendre_pd(N, x, &P, &dP);
        const double d2P = (2.0 * x * dP - N * (N + 1.0) * P) / (1.0 - x * x);
        const double dx = dP / d2P;
        x -= dx;
        if (std::fabs(dx) <= 1e-16) break;
      }
    }
    double P, dP;
    legendre_pd(N, x, &P, &dP);  // P is exact at the end points too (dP is not used)
    t->xi[i] = 0.5 * (x + 1.0);
    t->w[i] = 1.0 / (N * (N + 1.0) * P * P);
  }
}

void build_tables(int N, int points, HostTables* t) {
  const int n = N + 1;
  t->N = N;
  t->points = points;
  if (points == CR_POINTS_GLL) gll_nodes(N, t);
  for (int i = 0; points != CR_POINTS_GLL && i < n; ++i) {
    double x = -std::cos(M_PI * (2.0 * i + 1.0) / (2.0 * n));
    for (int it = 0; it < 60; ++it) {
      double P, dP;
      legendre_pd(n, x, &P, &dP);
      const double dx = P / dP;
      x -= dx;
      if (std::fabs(dx) <= 1e-16) break;
    }
    double P, dP;
    legendre_pd(n, x, &P, &dP);
    t->xi[i] = 0.5 * (x + 1.0);
    t->w[i] = 1.0 / ((1.0 - x * x) * dP * dP);  // 2/((1-x^2)P'^2), halved for [0,1]
  }
  double lam[kMaxNodes1];
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) prod *= (t->xi[j] - t->xi[m]);
    lam[j] = 1.0 / prod;
  }
  for (int side = 0; side < 2; ++side) {
    const double x = side;
    double* l = side ? t->l1 : t->l0;
    int at = -1;  // a node on the face (Gauss-Lobatto): the trace is its value
    for (int m = 0; m < n; ++m)
      if (t->xi[m] == x) at = m;
    if (at >= 0) {
      for (int j = 0; j < n; ++j) l[j] = j == at ? 1.0 : 0.0;
      continue;
    }
    double den = 0.0;
    for (int m = 0; m < n; ++m) den += lam[m] / (x - t->xi[m]);
    for (int j = 0; j < n; ++j) l[j] = lam[j] / (x - t->xi[j]) / den;
  }
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      const double d = (lam[j] / lam[i]) / (t->xi[i] - t->xi[j]);
      t->D[i * n + j] = d;
      diag -= d;
    }
    t->D[i * n + i] = diag;
  }
}

double legendre01(int j, double xi) {
  double P, dP;
  legendre_pd(j, 2.0 * xi - 1.0, &P, &dP);
  return P;
}

template <typename real>
void fill_tab(const HostTables& h, Tab<real>* t) {
  memset(t, 0, sizeof(*t));
  const int N = h.N, n = N + 1;
  double X[kMaxNodes1 + 2];
  X[0] = h.xi[N] - 1.0;  // neighbour node across the left face
  for (int p = 0; p < n; ++p) X[p + 1] = h.xi[p];
  X[n + 1] = 1.0 + h.xi[0];
  double xs = 0.0;
  for (int p = 0; p < n; ++p) {
    t->xi[p] = real(h.xi[p]);
    t->w[p] = real(h.w[p]);
    t->invw[p] = real(1.0 / h.w[p]);
    t->l0[p] = real(h.l0[p]);
    t->l1[p] = real(h.l1[p]);
    // correction derivatives at the solution points: the Radau correction with
    // Gauss-Legendre points and g2 with Gauss-Lobatto points both satisfy
    // g_R'(xi_p) = l_p(1)/w_p and g_L'(xi_p) = -l_p(0)/w_p
    t->gR[p] = real(h.l1[p] / h.w[p]);
    t->gL[p] = real(-h.l0[p] / h.w[p]);
    // subcells of Sec. 4 eq. (subcell.defn): widths w_p
    t->xs[p] = real(xs);
    t->dm[p] = real(xs - h.xi[p]);
    t->dp[p] = real(xs + h.w[p] - h.xi[p]);
    xs += h.w[p];
    // (Gauss-Lobatto points meet their neighbour's across a face: zero spacing,
    // and no MUSCL-Hancock subcells there)
    auto inv = [](double h) { return h > 0.0 ? 1.0 / h : 0.0; };
    t->ihm[p] = real(inv(X[p + 1] - X[p]));
    t->ihp[p] = real(inv(X[p + 2] - X[p + 1]));
    t->ihc[p] = real(inv(X[p + 2] - X[p]));
  }
  t->xs[n] = real(xs);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      t->V[i * n + j] = real((2.0 * i + 1.0) * h.w[j] * legendre01(i, h.xi[j]));
    }
}

// ---------------------------------------------------------------------------
// CFL(N) of eq. (time.step.2d) by Fourier analysis of the linear D2 scheme
// (u_t + u_x = 0, periodic).  With exact linear time averages
// U = T u, T = sum_{m<=N} (-nu)^m/(m+1)! D^m, the upwind D2 flux and the FR
// update give the amplification matrix
//   G(k) = I - nu [ D T - g_L' l(0)^T T + exp(-ik) g_L' l(1)^T T ];
// CFL is the largest nu with spectral radius <= 1 + 1e-4 on 721 wave numbers
// (the tolerance passes over the weak ~5e-6 growth of the fifth-order average
// at N = 4 and stops at the genuine k = pi instability).  Eigenvalues: the
// characteristic polynomial by Faddeev-LeVerrier, roots by Durand-Kerner.
using cd = std::complex<double>;

double spectral_radius(const cd* G, int n) {
  cd Mk[25] = {}, GM[25], c[6];
  c[n] = 1.0;
  for (int k = 1; k <= n; ++k) {
    // Mk = G * M_{k-1} + c_{n-k+1} I
    cd T[25];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        cd acc = 0.0;
        for (int r = 0; r < n; ++r) acc += G[i * n + r] * Mk[r * n + j];
        T[i * n + j] = acc + (i == j ? c[n - k + 1] : cd(0.0));
      }
    for (int i = 0; i < n * n; ++i) Mk[i] = T[i];
    cd tr = 0.0;
    for (int i = 0; i < n; ++i)
      for (int r = 0; r < n; ++r) tr += G[i * n + r] * Mk[r * n + i];
    c[n - k] = -tr / double(k);
  }
  (void)GM;
  cd z[5];
  const cd seed(0.4, 0.9);
  z[0] = 1.0;
  for (int i = 1; i < n; ++i) z[i] = z[i - 1] * seed;
  for (int it = 0; it < 2000; ++it) {
    double change = 0.0;
    for (int i = 0; i < n; ++i) {
      cd pv = 1.0;
      for (int k = n - 1; k >= 0; --k) pv = pv * z[i] + c[k];
      cd den = 1.0;
      for (int j = 0; j < n; ++j)
        if (j != i) den *= (z[i] - z[j]);
      const cd dz = pv / den;
      z[i] -= dz;
      change = std::fmax(change, std::abs(dz));
    }
    if (change < 1e-15) break;
  }
  double r = 0.0;
  for (int i = 0; i < n; ++i) r = std::fmax(r, std::abs(z[i]));
  return r;
}

double max_growth(const HostTables& h, double nu, bool d1) {
  const int n = h.N + 1;
  double T[25] = {}, Dm[25] = {}, tmp[25];
  for (int i = 0; i < n; ++i) Dm[i * n + i] = 1.0;
  double fact = 1.0;
  for (int m = 0; m <= h.N; ++m) {
    fact *= (m + 1);
    const double cm = std::pow(-nu, m) / fact;
    for (int i = 0; i < n * n; ++i) T[i] += cm * Dm[i];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int r = 0; r < n; ++r) acc += Dm[i * n + r] * h.D[r * n + j];
        tmp[i * n + j] = acc;
      }
    memcpy(Dm, tmp, sizeof(tmp));
  }
  // the jump term uses V = T (D2) or V = I (D1): with g_R' = l(1)/w,
  //   A0 = D T + g_R' (l1^T V - l1^T T)/2 - g_L' (l0^T T + l0^T V)/2   (k independent)
  //   Ap = g_R' (l0^T T - l0^T V)/2 (times exp(ik)), A1 = g_L' (l1^T T + l1^T V)/2 (exp(-ik))
  double A0[25], A1[25], Ap[25];
  for (int i = 0; i < n; ++i) {
    const double gL = -h.l0[i] / h.w[i], gR = h.l1[i] / h.w[i];
    for (int j = 0; j < n; ++j) {
      double dt = 0.0, l0T = 0.0, l1T = 0.0;
      for (int r = 0; r < n; ++r) {
        dt += h.D[i * n + r] * T[r * n + j];
        l0T += h.l0[r] * T[r * n + j];
        l1T += h.l1[r] * T[r * n + j];
      }
      const double l0V = d1 ? h.l0[j] : l0T, l1V = d1 ? h.l1[j] : l1T;
      A0[i * n + j] = dt + 0.5 * gR * (l1V - l1T) - 0.5 * gL * (l0T + l0V);
      Ap[i * n + j] = 0.5 * gR * (l0T - l0V);
      A1[i * n + j] = 0.5 * gL * (l1T + l1V);
    }
  }
  double g = 0.0;
  const int nk = 721;
  for (int ik = 0; ik < nk; ++ik) {
    const double k = 2.0 * M_PI * ik / (nk - 1);
    const cd ph = std::exp(cd(0.0, -k)), pp = std::exp(cd(0.0, k));
    cd G[25];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        G[i * n + j] = (i == j ? 1.0 : 0.0) - nu * (A0[i * n + j] + ph * A1[i * n + j] + pp * Ap[i * n + j]);
    g = std::fmax(g, spectral_radius(G, n));
  }
  return g;
}

double cfl_compute(int N, bool d1 = false, int points = CR_POINTS_GL) {
  static double cache[2][2][kMaxN + 1] = {};
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  const int pt = points == CR_POINTS_GLL ? 1 : 0;
  if (cache[pt][d1][N] > 0.0) return cache[pt][d1][N];
  HostTables h;
  build_tables(N, points, &h);
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 40; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (max_growth(h, mid, d1) <= 1.0 + 1e-4) lo = mid;
    else hi = mid;
  }
  cache[pt][d1][N] = lo;
  return lo;
}

std::string g_init_error;

__global__ void k_reset_ctl(TimeCtl* c, double cfl_factor) {
  c->t = 0.0;
  c->t_final = 0.0;
  c->dt_fixed = 0.0;
  c->cfl_factor = cfl_factor;
  c->rate_last = 0.0;
  c->rate_acc = 0ull;
  c->blocks_done = 0u;
  c->status = 0;
  c->bad_elem = INT_MAX;
  c->steps = 0;
  c->dt_step = 0.0;
  c->dt_step_f = 0.0f;
  c->last_step = 0;
  c->out = nullptr;
  c->out_done = 0;
  for (int i = 0; i < kRateParts; ++i) *rate_part(c, i) = 0ull;
}

__global__ void k_set_out(TimeCtl* c, double* out) {
  c->out = out;
  if (out) c->out_done = 0;
}

__global__ void k_set_run(TimeCtl* c, double t_final, double dt_fixed) {
  c->t_final = t_final;
  c->dt_fixed = dt_fixed;
  plan_step(c);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t ctl, u, umean, umean_f, P, smean, slot, fx, fy, alpha_raw, alpha_raw_f, alpha, mlp, staging,
      total;
};

int nvars_of(const cr_mesh_desc* d) {
  if (d->equation == CR_EQ_LINADV || d->equation == CR_EQ_BURGERS || d->equation == CR_EQ_VARADV) return 1;
  if (d->equation == CR_EQ_EULER) return d->dim == 1 ? 3 : 4;
  return 6;
}

Layout layout_of(const cr_mesh_desc* d) {
  const int n = d->degree + 1, dim = d->dim;
  const int np = dim == 2 ? n * n : n, M = nvars_of(d);
  const size_t ny = dim == 2 ? d->ny : 1, nx = d->nx, ne = nx * ny;
  const size_t nfx = d->bc_x == CR_BC_PERIODIC ? nx : nx + 1;
  const size_t nfy = dim == 2 ? (d->bc_y == CR_BC_PERIODIC ? ny : ny + 1) : 0;
  const size_t rs = d->precision == CR_FP32_BULK ? sizeof(float) : sizeof(double);
  const size_t nside = dim == 2 ? 4 : 2, nfn = dim == 2 ? n : 1;
  const bool mixed = d->precision == CR_FP32_BULK;
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  L.ctl = take(kCtlBytes);
  L.u = take(M * ne * np * rs);
  L.umean = take(mixed ? M * ne * sizeof(double) : 0);
  L.umean_f = take(mixed ? M * ne * sizeof(float) : 0);
  L.P = take(M * ne * np * rs);
  L.smean = take(mixed ? M * ne * sizeof(double) : 0);
  // face-node slots: 4M+1 fields, plus the stage traces for D-CSX
  const int nstage = d->degree == 4 ? 6 : d->degree + 1;
  const size_t nslotf = 4 * M + 1 + (d->dissipation == CR_DISS_DCSX ? (size_t)nstage * M : 0);
  L.slot = take(nslotf * nside * ne * nfn * rs);
  L.fx = take(M * ny * nfx * nfn * rs);
  L.fy = take(dim == 2 ? M * nfy * nx * n * rs : 0);
  L.alpha_raw = take(ne * sizeof(double));
  L.alpha_raw_f = take(mixed ? ne * sizeof(float) : 0);
  L.alpha = take(ne * sizeof(double));
  L.mlp = take(16 + 2 * (size_t)(32 * np + 32 + 32 * 32 + 32 + 32 + 1));  // flag + BF16 weights
  L.staging = take(mixed ? M * ne * np * sizeof(double) : 0);
  L.total = off;
  return L;
}

const KernelSet* lookup(const cr_mesh_desc* d) {
  const int mixed = d->precision == CR_FP32_BULK;
  if (d->equation == CR_EQ_LINADV)
    return d->dim == 1 ? kernels_linadv1d(d->degree, mixed) : kernels_linadv2d(d->degree, mixed);
  if (d->equation == CR_EQ_EULER && d->source == CR_SRC_GRAVITY)
    return d->dim == 1 ? kernels_euler1d_grav(d->degree, mixed) : kernels_euler2d_grav(d->degree, mixed);
  if (d->equation == CR_EQ_EULER)
    return d->dim == 1 ? kernels_euler1d(d->degree, mixed) : kernels_euler2d(d->degree, mixed);
  if (d->equation == CR_EQ_BURGERS) return d->dim == 1 ? kernels_burgers1d(d->degree, mixed) : nullptr;
  if (d->equation == CR_EQ_VARADV) return d->dim == 1 ? kernels_varadv1d(d->degree, mixed) : nullptr;
  return d->dim == 1 ? kernels_tenmoment1d(d->degree, mixed)
                     : kernels_tenmoment2d(d->degree, mixed);
}

// Boundary type of side s (0 x-, 1 x+, 2 y-, 3 y+): the per-side override or
// the direction's type.
int side_bc(const cr_mesh_desc* d, int s) {
  if (d->bc_side[s] != 0) return d->bc_side[s];
  return s < 2 ? d->bc_x : d->bc_y;
}

// A Dirichlet / inflow ghost state must be finite and, for Euler and
// ten-moment, admissible (rho > 0 and p > 0, or a positive-definite pressure
// tensor).
const char* check_ghost_state(const cr_mesh_desc* d, const double* g) {
  const int M = nvars_of(d);
  for (int v = 0; v < M; ++v)
    if (!std::isfinite(g[v])) return "a boundary state is not finite";
  if (d->equation == CR_EQ_EULER) {
    const double kin = d->dim == 1 ? 0.5 * g[1] * g[1] : 0.5 * (g[1] * g[1] + g[2] * g[2]);
    if (!(g[0] > 0.0) || !((d->gamma - 1.0) * (g[M - 1] - kin / g[0]) > 0.0))
      return "a boundary state is not admissible (rho > 0, p > 0)";
  } else if (d->equation == CR_EQ_TENMOMENT) {
    const double p11 = 2.0 * g[3] - g[1] * g[1] / g[0], p22 = 2.0 * g[5] - g[2] * g[2] / g[0];
    const double p12 = 2.0 * g[4] - g[1] * g[2] / g[0];
    if (!(g[0] > 0.0) || !(p11 > 0.0) || !(p11 * p22 - p12 * p12 > 0.0))
      return "a boundary state is not admissible (rho > 0, positive-definite pressure tensor)";
  }
  return nullptr;
}

const char* check_desc(const cr_mesh_desc* d) {
  if (!d) return "descriptor is NULL";
  if (d->dim != 1 && d->dim != 2) return "dim must be 1 or 2";
  if (d->degree < 1 || d->degree > kMaxN) return "degree must be in 1..4";
  if (d->nx < 1 || (d->dim == 2 && d->ny < 1)) return "nx, ny must be >= 1";
  if ((double)d->nx * (d->dim == 2 ? d->ny : 1) > 2.0e8) return "too many elements";
  if (!(d->x1 > d->x0) || (d->dim == 2 && !(d->y1 > d->y0))) return "empty domain";
  if (d->bc_x < 0 || d->bc_x > 4 || (d->dim == 2 && (d->bc_y < 0 || d->bc_y > 4)))
    return "unknown boundary condition";
  for (int s = 0; s < (d->dim == 2 ? 4 : 2); ++s) {
    const int dirbc = s < 2 ? d->bc_x : d->bc_y;
    if (d->bc_side[s] < 0 || d->bc_side[s] > 4) return "unknown per-side boundary condition";
    if (d->bc_side[s] != 0 && dirbc == CR_BC_PERIODIC)
      return "a periodic direction takes no per-side boundary condition";
    const int bc = side_bc(d, s);
    if (bc == CR_BC_WALL && d->equation != CR_EQ_EULER)
      return "wall boundaries are defined for the Euler equations";
    if (bc == CR_BC_DIRICHLET || bc == CR_BC_INFLOW) {
      const char* why = check_ghost_state(d, d->bc_state[s]);
      if (why) return why;
    }
  }
  if (d->equation < 0 || d->equation > 4) return "unknown equation";
  if (d->equation == CR_EQ_BURGERS && d->dim != 1) return "Burgers' equation is 1D";
  if (d->equation == CR_EQ_VARADV && d->dim != 1) return "variable advection is 1D";
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(d->adv_poly[k])) return "adv_poly is not finite";
  if (d->bc_time_terms < 0 || d->bc_time_terms > 16) return "bc_time_terms must be in 0..16";
  if (d->bc_flux < 0 || d->bc_flux > 1) return "unknown boundary flux";
  if (d->bc_flux == 1 && d->equation != CR_EQ_EULER) return "the HLLC boundary flux is for the Euler equations";
  if (d->bc_flux == 1 && d->dissipation == CR_DISS_D1)
    return "the HLLC boundary flux takes the time-averaged solution traces, which D1 does not keep";
  if (d->bc_time_terms > 0) {
    if (nvars_of(d) != 1) return "time-dependent boundary states are for scalar equations";
    if (!std::isfinite(d->bc_time_span[0]) || !(d->bc_time_span[1] > d->bc_time_span[0]) ||
        !std::isfinite(d->bc_time_span[1]))
      return "bc_time_span must be a finite interval t0 < t1";
    for (int s = 0; s < 4; ++s)
      for (int k = 0; k < d->bc_time_terms; ++k)
        if (!std::isfinite(d->bc_time_coef[s][k])) return "a boundary-state coefficient is not finite";
  }
  if (d->dissipation < 0 || d->dissipation > 2) return "unknown dissipation model";
  if (d->central < 0 || d->central > 1) return "unknown central flux";
  if (d->points != CR_POINTS_GL && d->points != CR_POINTS_GLL) return "unknown solution points";
  if (d->points == CR_POINTS_GLL &&
      ((d->limiter & (CR_LIM_BLEND | CR_LIM_MH | CR_LIM_FLUX)) || d->alpha_mode == CR_ALPHA_FIXED))
    return "Gauss-Lobatto points take no blending or flux limiter: their low-order subcell "
           "update would outrun its CFL condition at the GLL time step";
  if (d->equation == CR_EQ_EULER && !(d->gamma > 1.0)) return "gamma must be > 1";
  if (d->precision != CR_FP64 && d->precision != CR_FP32_BULK) return "unknown precision";
  if (d->alpha_mode != CR_ALPHA_INDICATOR && d->alpha_mode != CR_ALPHA_FIXED &&
      d->alpha_mode != CR_ALPHA_MLP)
    return "unknown alpha mode";
  if (d->alpha_mode == CR_ALPHA_FIXED && !(d->alpha_fixed >= 0.0 && d->alpha_fixed <= 1.0))
    return "alpha_fixed must be in [0,1]";
  if (d->source < 0 || d->source > 2) return "unknown source";
  if (d->source == CR_SRC_TENMOMENT && d->equation != CR_EQ_TENMOMENT)
    return "source 1 needs the ten-moment equations";
  if (d->source == CR_SRC_GRAVITY &&
      (d->equation != CR_EQ_EULER || !std::isfinite(d->gravity[0]) || !std::isfinite(d->gravity[1])))
    return "source 2 (gravity) needs the Euler equations and a finite gravity vector";
  if (d->limiter < 0 || d->limiter > 31) return "unknown limiter bits";
  return nullptr;
}

}  // namespace

namespace crk {

// Per-side boundary types, ghost states and gravity of the kernels' Mesh.
void fill_mesh_extras(const cr_mesh_desc* d, Mesh* m) {
  const int M = nvars_of(d);
  for (int s = 0; s < 4; ++s) {
    m->bcs[s] = (d->dim == 2 || s < 2) ? side_bc(d, s) : CR_BC_PERIODIC;
    for (int v = 0; v < 6; ++v) m->bcg[s][v] = v < M ? d->bc_state[s][v] : 0.0;
  }
  m->grav[0] = d->source == CR_SRC_GRAVITY ? d->gravity[0] : 0.0;
  m->grav[1] = d->source == CR_SRC_GRAVITY && d->dim == 2 ? d->gravity[1] : 0.0;
  m->bcflux = d->bc_flux;
  m->bcnt = d->bc_time_terms;
  m->bct0 = d->bc_time_span[0];
  m->bct1 = d->bc_time_span[1];
  for (int s = 0; s < 4; ++s)
    for (int k = 0; k < 16; ++k) m->bcc[s][k] = k < d->bc_time_terms ? d->bc_time_coef[s][k] : 0.0;
}

}  // namespace crk

struct cr_ctx {
  cr_mesh_desc d;
  const KernelSet* ks = nullptr;
  KParams<double> pd;
  KParams<float> pf;
  const void* params = nullptr;
  Layout L;
  unsigned char* ws = nullptr;
  bool owns_ws = false;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  cudaGraphExec_t g1 = nullptr, g8 = nullptr;
  bool graphs_tried = false;
  TimeCtl* h_ctl = nullptr;  // pinned mirror
  TimeCtl* d_ctl = nullptr;
  double cfl = 0.0;
  std::string err;
};

namespace {

// NVTX range for the duration of a scope (visible to ncu --nvtx and other
// CUDA tools; a few nanoseconds when no tool listens).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

cr_status fail(cr_ctx* c, cr_status st, const std::string& msg) {
  if (c) c->err = msg;
  else g_init_error = msg;
  return st;
}

cr_status cuda_fail(cr_ctx* c, cudaError_t e, const char* where) {
  return fail(c, CR_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CR_CUDA(c, call)                                    \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return cuda_fail((c), _e, #call); \
  } while (0)

// Mesh, physics and table parameters of the kernels for a description
// (everything but the buffers).
template <typename real>
void fill_desc_params(const cr_mesh_desc& d, KParams<real>* P, const HostTables& h) {
  Mesh& m = P->m;
  memset(&m, 0, sizeof(m));
  m.nx = d.nx;
  m.ny = d.dim == 2 ? d.ny : 1;
  m.ne = m.nx * m.ny;
  m.nfx = d.bc_x == CR_BC_PERIODIC ? m.nx : m.nx + 1;
  m.nfy = d.dim == 2 ? (d.bc_y == CR_BC_PERIODIC ? m.ny : m.ny + 1) : 0;
  m.bcx = d.bc_x;
  m.bcy = d.dim == 2 ? d.bc_y : 0;
  m.x0 = d.x0;
  m.y0 = d.dim == 2 ? d.y0 : 0.0;
  m.dx = (d.x1 - d.x0) / d.nx;
  m.dy = d.dim == 2 ? (d.y1 - d.y0) / d.ny : 1.0;
  m.invdx = 1.0 / m.dx;
  m.invdy = d.dim == 2 ? 1.0 / m.dy : 0.0;
  m.limiter = d.limiter;
  m.dissipation = d.dissipation;
  m.central = d.central;
  m.alpha_mode = d.alpha_mode;
  m.alpha_fixed = d.alpha_fixed;
  m.gamma = d.gamma;
  m.ax = d.adv[0];
  m.ay = d.adv[1];
  m.source = d.source;
  m.src_amp = d.src_amp;
  m.src_k = d.src_k;
  m.src_cx = d.src_cx;
  m.src_cy = d.src_cy;
  fill_mesh_extras(&d, &m);
  // indicator constants (Hennemann et al. form): T(N) = 0.5 10^(-1.8 (N+1)^(1/4)),
  // s = ln((1 - 1e-4)/1e-4)
  m.T_ind = 0.5 * std::pow(10.0, -1.8 * std::pow(d.degree + 1.0, 0.25));
  m.s_ind = std::log((1.0 - 1e-4) / 1e-4);
  {
    // flux-limiter candidates: u~ = u -+ dt/(kappa w h) (F - f_adj), kappa = 1 (1D), 1/2 (2D)
    const double kappa = d.dim == 2 ? 0.5 : 1.0;
    m.cflim[0] = 1.0 / (kappa * h.w[0] * m.dx);
    m.cflim[1] = 1.0 / (kappa * h.w[d.degree] * m.dx);
    m.cflim[2] = 1.0 / (kappa * h.w[0] * m.dy);
    m.cflim[3] = 1.0 / (kappa * h.w[d.degree] * m.dy);
  }
  P->ph.gamma = real(d.gamma);
  P->ph.gm1 = real(d.gamma - 1.0);
  P->ph.ax = real(d.adv[0]);
  P->ph.ay = real(d.adv[1]);
  P->ph.a0 = real(d.adv_poly[0]);
  P->ph.a1 = real(d.adv_poly[1]);
  P->ph.a2 = real(d.adv_poly[2]);
  P->ph.a3 = real(d.adv_poly[3]);
  P->ph.invdx = real(m.invdx);
  P->ph.invdy = real(m.invdy);
  for (int i = 0; i < 4; ++i) {
    P->ph.cflim[i] = real(m.cflim[i]);
    P->phd.cflim[i] = m.cflim[i];
  }
  P->phd.invdx = m.invdx;
  P->phd.invdy = m.invdy;
  P->phd.gamma = d.gamma;
  P->phd.gm1 = d.gamma - 1.0;
  P->phd.ax = d.adv[0];
  P->phd.ay = d.adv[1];
  P->phd.a0 = d.adv_poly[0];
  P->phd.a1 = d.adv_poly[1];
  P->phd.a2 = d.adv_poly[2];
  P->phd.a3 = d.adv_poly[3];
  fill_tab(h, &P->tb);
  fill_tab(h, &P->td);
  fill_scaled(h.D, h.w, h.l0, h.l1, d.degree, m.invdx, m.invdy, &P->ds);
}

template <typename real>
void fill_params(cr_ctx* c, KParams<real>* P, const HostTables& h) {
  fill_desc_params(c->d, P, h);
  Bufs<real>& b = P->b;
  unsigned char* w = c->ws;
  b.ctl = reinterpret_cast<TimeCtl*>(w + c->L.ctl);
  b.u = reinterpret_cast<real*>(w + c->L.u);
  b.umean = reinterpret_cast<double*>(w + c->L.umean);
  b.umean_f = reinterpret_cast<float*>(w + c->L.umean_f);
  b.P = reinterpret_cast<real*>(w + c->L.P);
  b.smean = reinterpret_cast<double*>(w + c->L.smean);
  b.slot = reinterpret_cast<real*>(w + c->L.slot);
  b.fx = reinterpret_cast<real*>(w + c->L.fx);
  b.fy = reinterpret_cast<real*>(w + c->L.fy);
  b.alpha_raw = reinterpret_cast<double*>(w + c->L.alpha_raw);
  b.alpha_raw_f = sizeof(real) == 4 ? reinterpret_cast<float*>(w + c->L.alpha_raw_f) : nullptr;
  b.alpha = reinterpret_cast<double*>(w + c->L.alpha);
  b.mlp_flag = reinterpret_cast<const int*>(w + c->L.mlp);
  b.mlp_w = reinterpret_cast<const unsigned short*>(w + c->L.mlp + 16);
  b.feat = nullptr;
  b.u_src = nullptr;
}

cr_status read_ctl(cr_ctx* c) {
  CR_CUDA(c, cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(TimeCtl), cudaMemcpyDeviceToHost, c->stream));
  CR_CUDA(c, cudaStreamSynchronize(c->stream));
  return CR_OK;
}

cr_status build_graphs(cr_ctx* c) {
  c->graphs_tried = true;
  for (int which = 0; which < 2; ++which) {
    const int nsteps = which == 0 ? 1 : 8;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return CR_OK;  // launch directly instead
    }
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < nsteps && e == cudaSuccess; ++s) e = c->ks->step(c->params, c->stream);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return CR_OK;
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return CR_OK;
    }
    (which == 0 ? c->g1 : c->g8) = ex;
  }
  return CR_OK;
}

// Enqueue n steps (graphs of 8 and 1 steps; direct launches if capture failed).
// A step whose planned dt is 0 (run finished or failed) does no work.
cr_status launch_steps(cr_ctx* c, int n) {
  while (n > 0) {
    if (n >= 8 && c->g8) {
      CR_CUDA(c, cudaGraphLaunch(c->g8, c->stream));
      n -= 8;
    } else if (c->g1) {
      CR_CUDA(c, cudaGraphLaunch(c->g1, c->stream));
      n -= 1;
    } else {
      CR_CUDA(c, c->ks->step(c->params, c->stream));
      n -= 1;
    }
  }
  return CR_OK;
}

}  // namespace

namespace crk {

// The kernel parameters of a description as a context sets them, in FP64,
// without the buffers (cr_step_static points those at its own scratch).
void fill_static_params(const cr_mesh_desc* d, KParams<double>* P) {
  HostTables h;
  build_tables(d->degree, d->points, &h);
  fill_desc_params(*d, P, h);
}

// The message cr_last_error(NULL) returns, for the entry points without a
// context.
void record_global_error(const std::string& msg) { g_init_error = msg; }

}  // namespace crk

// ===========================================================================
extern "C" {

cr_status cr_cfl_number_for(int degree, int dissipation, double* cfl) {
  if (degree < 1 || degree > kMaxN || !cfl || dissipation < 0 || dissipation > 2) return CR_E_INVALID_ARG;
  *cfl = cfl_compute(degree, dissipation == CR_DISS_D1);
  return CR_OK;
}

cr_status cr_cfl_number(int degree, double* cfl) {
  if (degree < 1 || degree > kMaxN || !cfl) return CR_E_INVALID_ARG;
  *cfl = cfl_compute(degree);
  return CR_OK;
}

cr_status cr_cfl_number_points(int degree, int dissipation, int points, double* cfl) {
  if (degree < 1 || degree > kMaxN || !cfl || dissipation < 0 || dissipation > 2 ||
      (points != CR_POINTS_GL && points != CR_POINTS_GLL))
    return CR_E_INVALID_ARG;
  *cfl = cfl_compute(degree, dissipation == CR_DISS_D1, points);
  return CR_OK;
}

cr_status cr_reference_tables_points(int degree, int points, double* xi, double* w, double* D) {
  if (degree < 1 || degree > kMaxN || (points != CR_POINTS_GL && points != CR_POINTS_GLL))
    return CR_E_INVALID_ARG;
  HostTables h;
  build_tables(degree, points, &h);
  const int n = degree + 1;
  for (int i = 0; i < n; ++i) {
    if (xi) xi[i] = h.xi[i];
    if (w) w[i] = h.w[i];
  }
  if (D) memcpy(D, h.D, sizeof(double) * n * n);
  return CR_OK;
}

cr_status cr_reference_tables(int degree, double* xi, double* w, double* D) {
  if (degree < 1 || degree > kMaxN) return CR_E_INVALID_ARG;
  HostTables h;
  build_tables(degree, CR_POINTS_GL, &h);
  const int n = degree + 1;
  for (int i = 0; i < n; ++i) {
    if (xi) xi[i] = h.xi[i];
    if (w) w[i] = h.w[i];
  }
  if (D) memcpy(D, h.D, sizeof(double) * n * n);
  return CR_OK;
}

cr_status cr_workspace_bytes(const cr_mesh_desc* desc, size_t* bytes) {
  if (!bytes) return fail(nullptr, CR_E_INVALID_ARG, "bytes is NULL");
  if (const char* why = check_desc(desc)) return fail(nullptr, CR_E_INVALID_ARG, why);
  *bytes = layout_of(desc).total;
  return CR_OK;
}

cr_status cr_init_mesh(const cr_mesh_desc* desc, void* workspace, size_t workspace_bytes,
                       cr_ctx** out) {
  if (!out) return fail(nullptr, CR_E_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (const char* why = check_desc(desc)) return fail(nullptr, CR_E_INVALID_ARG, why);
  const KernelSet* ks = lookup(desc);
  if (!ks) return fail(nullptr, CR_E_UNSUPPORTED, "this equation/dimension/degree/precision is not built");
  cr_ctx* c = new (std::nothrow) cr_ctx();
  if (!c) return fail(nullptr, CR_E_NOMEM, "host allocation failed");
  c->d = *desc;
  c->ks = ks;
  c->L = layout_of(desc);
  auto bail = [&](cr_status st) {
    g_init_error = c->err;
    cr_destroy(c);
    return st;
  };
  if (workspace) {
    if (workspace_bytes < c->L.total || (reinterpret_cast<uintptr_t>(workspace) & 255u))
      return bail(fail(c, CR_E_INVALID_ARG, "workspace too small or not 256-byte aligned"));
    c->ws = static_cast<unsigned char*>(workspace);
  } else {
    cudaError_t e = cudaMalloc(&c->ws, c->L.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bail(fail(c, CR_E_NOMEM, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e)));
    }
    c->owns_ws = true;
  }
  if (desc->stream) {
    c->stream = static_cast<cudaStream_t>(desc->stream);
  } else {
    cudaError_t e = cudaStreamCreate(&c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaStreamCreate"));
    c->owns_stream = true;
  }
  cudaError_t e = cudaMallocHost(&c->h_ctl, sizeof(TimeCtl));
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMallocHost"));
  e = ks->configure();
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaFuncSetAttribute"));
  c->cfl = desc->cfl > 0.0 ? desc->cfl
                           : cfl_compute(desc->degree, desc->dissipation == CR_DISS_D1, desc->points);
  if (!(c->d.cfl_safety > 0.0)) c->d.cfl_safety = 0.98;
  HostTables h;
  build_tables(desc->degree, desc->points, &h);
  if (ks->mixed) {
    fill_params(c, &c->pf, h);
    c->params = &c->pf;
    c->d_ctl = c->pf.b.ctl;
  } else {
    fill_params(c, &c->pd, h);
    c->params = &c->pd;
    c->d_ctl = c->pd.b.ctl;
  }
  k_reset_ctl<<<1, 1, 0, c->stream>>>(c->d_ctl, c->d.cfl_safety * c->cfl);
  e = cudaGetLastError();
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "k_reset_ctl"));
  e = cudaMemsetAsync(c->ws + c->L.mlp, 0, 16, c->stream);  // no network loaded
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemsetAsync"));
  *out = c;
  return CR_OK;
}

void cr_destroy(cr_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->g1) cudaGraphExecDestroy(c->g1);
  if (c->g8) cudaGraphExecDestroy(c->g8);
  if (c->owns_ws && c->ws) cudaFree(c->ws);
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  if (c->owns_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

cr_status cr_set_state(cr_ctx* c, const double* u, int on_device) {
  Range range("cr_set_state");
  if (!c || !u) return fail(c, CR_E_INVALID_ARG, "NULL argument");
  const size_t nvals = (size_t)c->ks->nvars * c->d.nx * (c->d.dim == 2 ? c->d.ny : 1) * c->ks->nodes;
  // (non-finite and inadmissible values are found by the prologue kernel, on
  // the device, for host and device input alike)
  k_reset_ctl<<<1, 1, 0, c->stream>>>(c->d_ctl, c->d.cfl_safety * c->cfl);
  CR_CUDA(c, cudaGetLastError());
  const double* src = u;
  // FP64 input in pinned host memory: the prologue kernel reads it over the
  // host link itself and keeps the copy, so the transfer and the input check,
  // indicator and CFL rate overlap instead of running one after the other
  const double* pinned = nullptr;
  if (!on_device && !c->ks->mixed) {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, u) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer)
      pinned = static_cast<const double*>(pa.devicePointer);
    cudaGetLastError();
  }
  if (pinned) {
    KParams<double> P = c->pd;
    P.b.u_src = pinned;
    CR_CUDA(c, c->ks->prologue(&P, c->stream));
  } else {
    if (c->ks->mixed) {
      double* staging = reinterpret_cast<double*>(c->ws + c->L.staging);
      CR_CUDA(c, cudaMemcpyAsync(staging, u, nvals * sizeof(double), cudaMemcpyDefault, c->stream));
      src = staging;
    }
    CR_CUDA(c, c->ks->split(c->params, src, c->stream));
    CR_CUDA(c, c->ks->prologue(c->params, c->stream));
  }
  cr_status st = read_ctl(c);
  if (st != CR_OK) return st;
  if (c->h_ctl->status & kStInvalidInput)
    return fail(c, CR_E_INVALID_STATE,
                "inadmissible or non-finite input at element " + std::to_string(c->h_ctl->bad_elem));
  return CR_OK;
}

cr_status cr_get_state(cr_ctx* c, double* u, int on_device) {
  Range range("cr_get_state");
  if (!c || !u) return fail(c, CR_E_INVALID_ARG, "NULL argument");
  const size_t nvals = (size_t)c->ks->nvars * c->d.nx * (c->d.dim == 2 ? c->d.ny : 1) * c->ks->nodes;
  if (c->ks->mixed && !on_device) {
    double* staging = reinterpret_cast<double*>(c->ws + c->L.staging);
    CR_CUDA(c, c->ks->join(c->params, staging, c->stream));
    CR_CUDA(c, cudaMemcpyAsync(u, staging, nvals * sizeof(double), cudaMemcpyDefault, c->stream));
  } else {
    CR_CUDA(c, c->ks->join(c->params, u, c->stream));
  }
  if (!on_device) CR_CUDA(c, cudaStreamSynchronize(c->stream));
  return CR_OK;
}

cr_status cr_step_async(cr_ctx* c, int max_steps, double t_final, double dt_fixed) {
  Range range("cr_step_async");
  if (!c) return fail(c, CR_E_INVALID_ARG, "NULL context");
  if (max_steps < 0 || !(t_final == t_final)) return fail(c, CR_E_INVALID_ARG, "bad max_steps or t_final");
  if (!c->graphs_tried) {
    cr_status st = build_graphs(c);
    if (st != CR_OK) return st;
  }
  k_set_run<<<1, 1, 0, c->stream>>>(c->d_ctl, t_final, dt_fixed);
  CR_CUDA(c, cudaGetLastError());
  return launch_steps(c, max_steps);
}

cr_status cr_profile_steps(cr_ctx* c, int max_steps, double t_final, double dt_fixed,
                           double* kernel_ms) {
  if (!c || !kernel_ms || max_steps < 0) return fail(c, CR_E_INVALID_ARG, "bad argument");
  const int nk = c->ks->launches_per_step;
  cudaEvent_t ev[5];
  for (int i = 0; i <= nk; ++i) CR_CUDA(c, cudaEventCreate(&ev[i]));
  k_set_run<<<1, 1, 0, c->stream>>>(c->d_ctl, t_final, dt_fixed);
  CR_CUDA(c, cudaGetLastError());
  cr_status st = CR_OK;
  for (int s = 0; s < max_steps && st == CR_OK; ++s) {
    for (int i = 0; i < nk; ++i) {
      Range range(c->ks->names[i]);
      CR_CUDA(c, cudaEventRecord(ev[i], c->stream));
      CR_CUDA(c, c->ks->launch[i](c->params, c->stream));
    }
    CR_CUDA(c, cudaEventRecord(ev[nk], c->stream));
    CR_CUDA(c, cudaEventSynchronize(ev[nk]));
    for (int i = 0; i < nk; ++i) {
      float ms = 0.0f;
      CR_CUDA(c, cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
      kernel_ms[i] += ms;
    }
  }
  for (int i = 0; i <= nk; ++i) cudaEventDestroy(ev[i]);
  return st;
}

cr_status cr_sync(cr_ctx* c, double* t_out, int* steps_out) {
  if (!c) return fail(c, CR_E_INVALID_ARG, "NULL context");
  cr_status st = read_ctl(c);
  if (st != CR_OK) return st;
  if (t_out) *t_out = c->h_ctl->t;
  if (steps_out) *steps_out = c->h_ctl->steps;
  if (c->h_ctl->status & (kStInadmissible | kStNonFinite))
    return fail(c, CR_E_INADMISSIBLE,
                "inadmissible or non-finite state after a step, element " +
                    std::to_string(c->h_ctl->bad_elem));
  return CR_OK;
}

cr_status cr_step(cr_ctx* c, int max_steps, double t_final, double dt_fixed, double* t_out,
                  int* steps_out) {
  // Steps go out in chunks of 64, 128, ... 4096; between chunks the time
  // record is read back, and launching stops once the run has reached
  // t_final or failed, so a generous max_steps costs nothing extra.
  const int first = max_steps < 64 ? max_steps : 64;
  cr_status st = cr_step_async(c, first, t_final, dt_fixed);
  if (st != CR_OK) return st;
  int left = max_steps - first, chunk = 64;
  while (left > 0) {
    st = read_ctl(c);
    if (st != CR_OK) return st;
    if (c->h_ctl->status != 0 || !(c->h_ctl->dt_step > 0.0)) break;
    chunk = chunk < 4096 ? 2 * chunk : chunk;
    const int n = left < chunk ? left : chunk;
    st = launch_steps(c, n);
    if (st != CR_OK) return st;
    left -= n;
  }
  return cr_sync(c, t_out, steps_out);
}

cr_status cr_step_get(cr_ctx* c, int max_steps, double t_final, double dt_fixed, double* u,
                      double* t_out, int* steps_out) {
  Range range("cr_step_get");
  if (!c || !u) return fail(c, CR_E_INVALID_ARG, "NULL argument");
  cudaPointerAttributes attr;
  const bool pinned = cudaPointerGetAttributes(&attr, u) == cudaSuccess && attr.type == cudaMemoryTypeHost;
  cudaGetLastError();  // a pageable pointer may leave an error behind
  if (!pinned || max_steps <= 0) {
    cr_status st = cr_step(c, max_steps, t_final, dt_fixed, t_out, steps_out);
    return st != CR_OK ? st : cr_get_state(c, u, 0);
  }
  if (max_steps > 1) {
    cr_status st = cr_step(c, max_steps - 1, t_final, dt_fixed, nullptr, nullptr);
    if (st != CR_OK) return st;
  }
  // the last step writes the state into u while its update kernel runs
  k_set_out<<<1, 1, 0, c->stream>>>(c->d_ctl, u);
  CR_CUDA(c, cudaGetLastError());
  cr_status st = cr_step_async(c, 1, t_final, dt_fixed);
  k_set_out<<<1, 1, 0, c->stream>>>(c->d_ctl, nullptr);
  CR_CUDA(c, cudaGetLastError());
  if (st != CR_OK) return st;
  st = cr_sync(c, t_out, steps_out);
  if (st != CR_OK) return st;
  // the run ended before that step (t_final reached): copy the state
  return c->h_ctl->out_done ? CR_OK : cr_get_state(c, u, 0);
}

cr_status cr_get_alpha(cr_ctx* c, double* alpha, int on_device) {
  if (!c || !alpha) return fail(c, CR_E_INVALID_ARG, "NULL argument");
  const size_t ne = (size_t)c->d.nx * (c->d.dim == 2 ? c->d.ny : 1);
  CR_CUDA(c, cudaMemcpyAsync(alpha, c->ws + c->L.alpha, ne * sizeof(double), cudaMemcpyDefault,
                             c->stream));
  if (!on_device) CR_CUDA(c, cudaStreamSynchronize(c->stream));
  return CR_OK;
}

cr_status cr_mlp_load(cr_ctx* c, const float* params, int nparams) {
  if (!c || !params) return fail(c, CR_E_INVALID_ARG, "NULL argument");
  const int np = c->ks->nodes;
  const int want = 32 * np + 32 + 32 * 32 + 32 + 32 + 1;
  if (nparams != want)
    return fail(c, CR_E_INVALID_ARG, "expected " + std::to_string(want) + " network parameters");
  // Device layout: the weight matrices transposed (W1T[Np][32], W2T[32][32])
  // so that the 32 lanes of a warp read 32 consecutive entries.
  const int H = 32;
  std::vector<int> src(nparams);
  for (int i = 0; i < nparams; ++i) src[i] = i;
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < np; ++i) src[i * H + j] = j * np + i;
  const int o2 = H * np + H;
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < H; ++i) src[o2 + i * H + j] = o2 + j * H + i;
  std::vector<unsigned short> h(nparams);
  for (int i = 0; i < nparams; ++i) {  // FP32 -> BF16, round to nearest even
    uint32_t b;
    memcpy(&b, &params[src[i]], 4);
    if ((b & 0x7f800000u) == 0x7f800000u && (b & 0x007fffffu)) return fail(c, CR_E_INVALID_ARG, "NaN parameter");
    b += 0x7fffu + ((b >> 16) & 1u);
    h[i] = (unsigned short)(b >> 16);
  }
  const int one = 1;
  CR_CUDA(c, cudaMemcpyAsync(c->ws + c->L.mlp + 16, h.data(), h.size() * 2, cudaMemcpyHostToDevice, c->stream));
  CR_CUDA(c, cudaMemcpyAsync(c->ws + c->L.mlp, &one, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CR_CUDA(c, cudaStreamSynchronize(c->stream));
  return CR_OK;
}

cr_status cr_get_features(cr_ctx* c, float* features, double* alpha_raw, int on_device) {
  if (!c || (!features && !alpha_raw)) return fail(c, CR_E_INVALID_ARG, "NULL argument");
  const size_t ne = (size_t)c->d.nx * (c->d.dim == 2 ? c->d.ny : 1);
  const size_t nf = ne * c->ks->nodes;
  float* staging = reinterpret_cast<float*>(c->ws + c->L.P);  // P is free between steps
  cudaError_t e;
  if (c->ks->mixed) {
    KParams<float> P = c->pf;
    P.b.feat = staging;
    e = c->ks->prologue(&P, c->stream);
  } else {
    KParams<double> P = c->pd;
    P.b.feat = staging;
    e = c->ks->prologue(&P, c->stream);
  }
  CR_CUDA(c, e);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (features) CR_CUDA(c, cudaMemcpyAsync(features, staging, nf * sizeof(float), kind, c->stream));
  if (alpha_raw)
    CR_CUDA(c, cudaMemcpyAsync(alpha_raw, c->ws + c->L.alpha_raw, ne * sizeof(double), kind, c->stream));
  if (!on_device) CR_CUDA(c, cudaStreamSynchronize(c->stream));
  return CR_OK;
}

cr_status cr_get_means(cr_ctx* c, double* means, int on_device) {
  if (!c || !means) return fail(c, CR_E_INVALID_ARG, "NULL argument");
  const size_t ne = (size_t)c->d.nx * (c->d.dim == 2 ? c->d.ny : 1);
  if (on_device) {
    CR_CUDA(c, c->ks->means(c->params, means, c->stream));
    return CR_OK;
  }
  double* staging = reinterpret_cast<double*>(c->ws + c->L.P);  // P is free between steps
  if (c->ks->mixed) staging = reinterpret_cast<double*>(c->ws + c->L.staging);
  CR_CUDA(c, c->ks->means(c->params, staging, c->stream));
  CR_CUDA(c, cudaMemcpyAsync(means, staging, (size_t)c->ks->nvars * ne * sizeof(double),
                             cudaMemcpyDeviceToHost, c->stream));
  CR_CUDA(c, cudaStreamSynchronize(c->stream));
  return CR_OK;
}

cr_status cr_next_dt(cr_ctx* c, double* dt) {
  if (!c || !dt) return fail(c, CR_E_INVALID_ARG, "NULL argument");
  cr_status st = read_ctl(c);
  if (st != CR_OK) return st;
  *dt = c->h_ctl->cfl_factor / c->h_ctl->rate_last;
  return CR_OK;
}

cr_status cr_launches_per_step(cr_ctx* c, int* launches) {
  if (!c || !launches) return CR_E_INVALID_ARG;
  *launches = c->ks->launches_per_step;
  return CR_OK;
}

const char* cr_last_error(const cr_ctx* c) {
  return c ? c->err.c_str() : g_init_error.c_str();
}

}  // extern "C"

// ===========================================================================
// Batches: many contexts advanced together by the kernels of cr_batch.cu.
struct cr_batch {
  std::vector<cr_ctx*> ctx;
  bool fp32 = false;
  cudaStream_t stream = nullptr;
  int threads = 256, mode = CR_BATCH_FUSED, tiles = 1;
  unsigned long long spin_limit = 1ull << 26;  // polls of a fused-launch wait (>= 64 ns each): >= 4 s
  int phantom = 0;                             // test hook: completions that never come
  int fused_grid = 0;
  unsigned char* dmem = nullptr;     // parameters, degrees, block counts, tiles, queue, error flag
  size_t params_off = 0, deg_off = 0, nblk_off = 0, nface_off = 0, nupd_off = 0, tel_off = 0,
         tface_off = 0, tupd_off = 0, queue_off = 0, err_off = 0;
  size_t max_el = 0, max_face = 0;   // tile capacity (the smallest block size)
  BatchArgs<float> af{};
  BatchArgs<double> ad{};
  cudaGraphExec_t g1 = nullptr, g8 = nullptr;
  std::vector<cudaEvent_t> ev;       // one per context stream (ordering before a step)
  int* h_err = nullptr;              // pinned copy of the barrier error flag
  std::string err;
};

namespace {

cr_status bfail(cr_batch* b, cr_status st, const std::string& msg) {
  if (b) b->err = msg;
  else g_init_error = msg;
  return st;
}

#define CR_BCUDA(b, call)                                                                  \
  do {                                                                                     \
    cudaError_t _e = (call);                                                               \
    if (_e != cudaSuccess) return bfail((b), CR_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// Element and face-node tile counts of one problem for a block of `threads`.
void tile_counts(const cr_ctx* c, int threads, int* nel, int* nface) {
  const int n = c->d.degree + 1, np = n * n;
  const int epr = threads / np;
  const int nx = c->d.nx, ny = c->d.ny;
  const int ne = nx * ny;
  const int nfx = c->d.bc_x == CR_BC_PERIODIC ? nx : nx + 1;
  const int nfy = c->d.bc_y == CR_BC_PERIODIC ? ny : ny + 1;
  const long long fnodes = (long long)ny * nfx * n + (long long)nfy * nx * n;
  *nel = (ne + epr - 1) / epr;
  *nface = (int)((fnodes + threads - 1) / threads);
}

void destroy_graphs(cr_batch* b) {
  if (b->g1) cudaGraphExecDestroy(b->g1);
  if (b->g8) cudaGraphExecDestroy(b->g8);
  b->g1 = b->g8 = nullptr;
}

// Tiles, block counts and launch arguments for b->threads; graphs of 1 and 8
// steps in b->mode.
cr_status batch_build(cr_batch* b) {
  destroy_graphs(b);
  const int nprob = (int)b->ctx.size();
  // the update phase of FP32-bulk batches launched per phase runs in 128-thread
  // blocks, as the single-problem FP32-bulk update (barrier bound: smaller
  // blocks wait less); every other phase in blocks of b->threads
  const int upd_threads = (b->fp32 && b->mode == CR_BATCH_PHASES) ? kBatchThreadChoices[0] : b->threads;
  // element tiles grouped by degree (3, then 4): the element phases launch one
  // kernel per degree over its contiguous range
  std::vector<BatchTile> tel, tface, tupd;
  std::vector<int> nblk(nprob), nblkf(nprob), nblku(nprob);
  int el_first[2] = {0, 0}, el_count[2] = {0, 0}, upd_first[2] = {0, 0}, upd_count[2] = {0, 0};
  for (int g = 0; g < 2; ++g) {
    el_first[g] = (int)tel.size();
    upd_first[g] = (int)tupd.size();
    for (int i = 0; i < nprob; ++i) {
      if (b->ctx[i]->d.degree != 3 + g) continue;
      int nel, nface, nupd, unused;
      tile_counts(b->ctx[i], b->threads, &nel, &nface);
      tile_counts(b->ctx[i], upd_threads, &nupd, &unused);
      nblk[i] = nel;
      nblkf[i] = nface;
      nblku[i] = nupd;
      for (int k = 0; k < nupd; ++k) tupd.push_back({i, k});
      for (int k = 0; k < nel; ++k) tel.push_back({i, k});
      for (int k = 0; k < nface; ++k) tface.push_back({i, k});
    }
    el_count[g] = (int)tel.size() - el_first[g];
    upd_count[g] = (int)tupd.size() - upd_first[g];
  }
  if (tel.size() > b->max_el || tface.size() > b->max_face || tupd.size() > b->max_el)
    return bfail(b, CR_E_INVALID_ARG, "tile capacity exceeded");
  unsigned char* d = b->dmem;
  CR_BCUDA(b, cudaMemcpyAsync(d + b->nblk_off, nblk.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  CR_BCUDA(b, cudaMemcpyAsync(d + b->nface_off, nblkf.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  CR_BCUDA(b, cudaMemcpyAsync(d + b->nupd_off, nblku.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  CR_BCUDA(b, cudaMemcpyAsync(d + b->tupd_off, tupd.data(), tupd.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, b->stream));
  CR_BCUDA(b, cudaMemcpyAsync(d + b->tel_off, tel.data(), tel.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, b->stream));
  CR_BCUDA(b, cudaMemcpyAsync(d + b->tface_off, tface.data(), tface.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, b->stream));
  CR_BCUDA(b, cudaStreamSynchronize(b->stream));
  auto fill = [&](auto& A, auto* P) {
    A.P = P;
    A.deg = reinterpret_cast<const int*>(d + b->deg_off);
    A.nblk_el = reinterpret_cast<const int*>(d + b->nblk_off);
    A.nblk_face = reinterpret_cast<const int*>(d + b->nface_off);
    A.t_el = reinterpret_cast<const BatchTile*>(d + b->tel_off);
    A.n_el = (int)tel.size();
    A.t_face = reinterpret_cast<const BatchTile*>(d + b->tface_off);
    A.n_face = (int)tface.size();
    A.t_upd = reinterpret_cast<const BatchTile*>(d + b->tupd_off);
    A.n_upd = (int)tupd.size();
    A.nblk_upd = reinterpret_cast<const int*>(d + b->nupd_off);
    A.upd_threads = upd_threads;
    for (int g = 0; g < 2; ++g) {
      A.el_first[g] = el_first[g];
      A.el_count[g] = el_count[g];
      A.upd_first[g] = upd_first[g];
      A.upd_count[g] = upd_count[g];
    }
    A.nprob = nprob;
    A.tiles = b->tiles;
    A.queue = reinterpret_cast<unsigned*>(d + b->queue_off);
    A.err = reinterpret_cast<int*>(d + b->err_off);
    A.spin_limit = b->spin_limit;
    A.phantom = b->phantom;
  };
  fill(b->af, reinterpret_cast<const KParams<float>*>(d + b->params_off));
  fill(b->ad, reinterpret_cast<const KParams<double>*>(d + b->params_off));
  for (cr_ctx* c : b->ctx) {  // the tables depend only on the degree
    const int i = c->d.degree - 3;
    b->af.tb[i] = c->pf.tb;
    b->af.td[i] = c->pf.td;
    b->ad.tb[i] = c->pd.tb;
    b->ad.td[i] = c->pd.td;
  }
  CR_BCUDA(b, batch_configure(b->threads, b->fp32));
  if (b->mode == CR_BATCH_FUSED) {
    int maxb = 0;
    CR_BCUDA(b, batch_fused_max_blocks(b->threads, b->fp32, &maxb));
    if (maxb < 1) return bfail(b, CR_E_CUDA, "the fused batch kernel does not fit on an SM");
    const int most = b->af.n_el > b->af.n_face ? b->af.n_el : b->af.n_face;
    const int per_claim = b->tiles * kFusedClaim;
    const int want = (most + per_claim - 1) / per_claim;
    b->fused_grid = want < maxb ? want : maxb;
  }
  // graphs of 1 and 8 steps (direct launches if capture is refused)
  for (int which = 0; which < 2; ++which) {
    const int nsteps = which == 0 ? 1 : 8;
    b->af.nsteps = b->ad.nsteps = nsteps;
    const void* args = b->fp32 ? static_cast<const void*>(&b->af) : static_cast<const void*>(&b->ad);
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    cudaError_t e = cudaSuccess;
    if (b->mode == CR_BATCH_FUSED) {
      e = batch_launch_fused(b->threads, b->fused_grid, args, b->fp32, b->stream);
    } else {
      for (int s = 0; s < nsteps && e == cudaSuccess; ++s)
        for (int ph = 0; ph < 3 && e == cudaSuccess; ++ph)
          e = batch_launch_phase(b->threads, ph, args, b->fp32, b->stream);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess && e2 == cudaSuccess && g) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || e2 != cudaSuccess || !ex) {
      cudaGetLastError();
      destroy_graphs(b);
      break;
    }
    (which == 0 ? b->g1 : b->g8) = ex;
  }
  return CR_OK;
}

cr_status batch_launch_steps(cr_batch* b, int nsteps) {
  const void* args = b->fp32 ? static_cast<const void*>(&b->af) : static_cast<const void*>(&b->ad);
  while (nsteps > 0) {
    const int k = nsteps >= 8 ? 8 : 1;
    cudaGraphExec_t g = k == 8 ? b->g8 : b->g1;
    if (g) {
      CR_BCUDA(b, cudaGraphLaunch(g, b->stream));
    } else {
      b->af.nsteps = b->ad.nsteps = k;
      if (b->mode == CR_BATCH_FUSED) {
        CR_BCUDA(b, batch_launch_fused(b->threads, b->fused_grid, args, b->fp32, b->stream));
      } else {
        for (int s = 0; s < k; ++s)
          for (int ph = 0; ph < 3; ++ph) CR_BCUDA(b, batch_launch_phase(b->threads, ph, args, b->fp32, b->stream));
      }
    }
    nsteps -= k;
  }
  return CR_OK;
}

}  // namespace

extern "C" {

cr_status cr_batch_init(cr_ctx* const* ctxs, int n, cr_batch** out) {
  if (!ctxs || n < 1 || !out) return bfail(nullptr, CR_E_INVALID_ARG, "cr_batch_init: bad arguments");
  *out = nullptr;
  cr_batch* b = new (std::nothrow) cr_batch();
  if (!b) return bfail(nullptr, CR_E_NOMEM, "cr_batch_init: out of host memory");
  auto bail = [&](cr_status st) {
    if (st != CR_OK) g_init_error = b->err;
    cr_batch_destroy(b);
    return st;
  };
  for (int i = 0; i < n; ++i) {
    cr_ctx* c = ctxs[i];
    if (!c) return bail(bfail(b, CR_E_INVALID_ARG, "cr_batch_init: NULL context"));
    const cr_mesh_desc& d = c->d;
    if (d.dim != 2 || d.equation != CR_EQ_EULER || (d.degree != 3 && d.degree != 4) ||
        d.points != CR_POINTS_GL || d.source != CR_SRC_NONE)
      return bail(bfail(b, CR_E_UNSUPPORTED,
                        "cr_batch_init: batches hold 2D Euler problems of degree 3 or 4 on Gauss-Legendre points, without a source"));
    if (i > 0 && d.precision != ctxs[0]->d.precision)
      return bail(bfail(b, CR_E_INVALID_ARG, "cr_batch_init: mixed precisions"));
    b->ctx.push_back(c);
  }
  b->fp32 = ctxs[0]->d.precision == CR_FP32_BULK;
  b->stream = ctxs[0]->stream;
  // capacity for the smallest block size
  size_t mel = 0, mface = 0;
  for (cr_ctx* c : b->ctx) {
    int nel, nface;
    tile_counts(c, kBatchThreadChoices[0], &nel, &nface);
    mel += nel;
    mface += nface;
  }
  b->max_el = mel;
  b->max_face = mface;
  const size_t psz = b->fp32 ? sizeof(KParams<float>) : sizeof(KParams<double>);
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += align256(bytes); return o; };
  b->params_off = take(psz * n);
  b->deg_off = take(sizeof(int) * n);
  b->nblk_off = take(sizeof(int) * n);
  b->nface_off = take(sizeof(int) * n);
  b->nupd_off = take(sizeof(int) * n);
  b->tel_off = take(sizeof(BatchTile) * mel);
  b->tface_off = take(sizeof(BatchTile) * mface);
  b->tupd_off = take(sizeof(BatchTile) * mel);
  b->queue_off = take(sizeof(unsigned) * (1 + 3 * (size_t)n));
  b->err_off = take(16);
  cudaError_t e = cudaMalloc(&b->dmem, off);
  if (e != cudaSuccess) return bail(bfail(b, CR_E_NOMEM, "cr_batch_init: cudaMalloc failed"));
  e = cudaMallocHost(&b->h_err, sizeof(int));
  if (e != cudaSuccess) return bail(bfail(b, CR_E_NOMEM, "cr_batch_init: cudaMallocHost failed"));
  std::vector<unsigned char> hp(psz * n);
  std::vector<int> deg(n);
  for (int i = 0; i < n; ++i) {
    memcpy(hp.data() + psz * i, b->fp32 ? static_cast<const void*>(&b->ctx[i]->pf)
                                        : static_cast<const void*>(&b->ctx[i]->pd), psz);
    deg[i] = b->ctx[i]->d.degree;
  }
  for (cr_ctx* c : b->ctx)  // the contexts' queued work (cr_set_state) comes first
    if (c->stream != b->stream && cudaStreamSynchronize(c->stream) != cudaSuccess)
      return bail(bfail(b, CR_E_CUDA, "cr_batch_init: a context stream failed"));
  e = cudaMemcpyAsync(b->dmem + b->params_off, hp.data(), hp.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->dmem + b->deg_off, deg.data(), n * sizeof(int), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->dmem + b->err_off, 0, 16, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bail(bfail(b, CR_E_CUDA, std::string("cr_batch_init: ") + cudaGetErrorString(e)));
  for (cr_ctx* c : b->ctx) {
    if (c->stream == b->stream) continue;
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      return bail(bfail(b, CR_E_CUDA, "cr_batch_init: cudaEventCreate failed"));
    b->ev.push_back(ev);
  }
  cr_status st = batch_build(b);
  if (st != CR_OK) return bail(st);
  *out = b;
  return CR_OK;
}

void cr_batch_destroy(cr_batch* b) {
  if (!b) return;
  destroy_graphs(b);
  for (cudaEvent_t ev : b->ev) cudaEventDestroy(ev);
  if (b->dmem) cudaFree(b->dmem);
  if (b->h_err) cudaFreeHost(b->h_err);
  delete b;
}

cr_status cr_batch_config(cr_batch* b, int threads, int mode, int tiles) {
  if (!b) return bfail(nullptr, CR_E_INVALID_ARG, "NULL batch");
  if ((threads != kBatchThreadChoices[0] && threads != kBatchThreadChoices[1]) ||
      (mode != CR_BATCH_PHASES && mode != CR_BATCH_FUSED) ||
      (tiles != kBatchTileChoices[0] && tiles != kBatchTileChoices[1] && tiles != kBatchTileChoices[2]))
    return bfail(b, CR_E_INVALID_ARG,
                 "cr_batch_config: threads must be 128 or 256, mode PHASES or FUSED, tiles 1, 2 or 4");
  b->threads = threads;
  b->mode = mode;
  b->tiles = tiles;
  return batch_build(b);
}

cr_status cr_batch_step_async(cr_batch* b, int nsteps, double t_final) {
  Range range("cr_batch_step_async");
  if (!b) return bfail(nullptr, CR_E_INVALID_ARG, "NULL batch");
  if (nsteps < 0 || !(t_final == t_final)) return bfail(b, CR_E_INVALID_ARG, "bad nsteps or t_final");
  size_t k = 0;
  for (cr_ctx* c : b->ctx) {  // work queued on the contexts' own streams comes first
    if (c->stream == b->stream) continue;
    CR_BCUDA(b, cudaEventRecord(b->ev[k], c->stream));
    CR_BCUDA(b, cudaStreamWaitEvent(b->stream, b->ev[k], 0));
    ++k;
  }
  const void* P = b->dmem + b->params_off;
  CR_BCUDA(b, batch_set_run(P, (int)b->ctx.size(), t_final, b->fp32, b->stream));
  return batch_launch_steps(b, nsteps);
}

cr_status cr_batch_sync(cr_batch* b) {
  if (!b) return bfail(nullptr, CR_E_INVALID_ARG, "NULL batch");
  CR_BCUDA(b, cudaMemcpyAsync(b->h_err, b->dmem + b->err_off, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  CR_BCUDA(b, cudaStreamSynchronize(b->stream));
  if (*b->h_err) {  // clear the flag so that the batch can run again
    CR_BCUDA(b, cudaMemsetAsync(b->dmem + b->err_off, 0, 16, b->stream));
    CR_BCUDA(b, cudaStreamSynchronize(b->stream));
    return bfail(b, CR_E_TIMEOUT, "cr_batch_sync: a wait of the fused kernel gave up");
  }
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    cr_ctx* c = b->ctx[i];
    cr_status st = read_ctl(c);
    if (st != CR_OK) return bfail(b, st, "cr_batch_sync: problem " + std::to_string(i) + ": " + c->err);
    if (c->h_ctl->status & (kStInadmissible | kStNonFinite))
      return bfail(b, CR_E_INADMISSIBLE, "problem " + std::to_string(i) +
                                             ": inadmissible or non-finite state after a step, element " +
                                             std::to_string(c->h_ctl->bad_elem));
  }
  return CR_OK;
}

cr_status cr_batch_step(cr_batch* b, int nsteps, double t_final) {
  cr_status st = cr_batch_step_async(b, nsteps, t_final);
  if (st != CR_OK) return st;
  return cr_batch_sync(b);
}

cr_status cr_batch_autotune(cr_batch* b, int trial_steps, int* threads_out, int* mode_out,
                            int* tiles_out, double* ms_per_step) {
  if (!b || trial_steps < 1) return bfail(b, CR_E_INVALID_ARG, "cr_batch_autotune: bad arguments");
  // candidates, per thread count: PHASES, then FUSED with tiles 1, 2, 4 (the
  // order of ms_per_step)
  constexpr int NC = CR_BATCH_CANDIDATES;
  int cand_t[NC], cand_m[NC], cand_k[NC];
  for (int i = 0; i < NC; ++i) {
    cand_t[i] = kBatchThreadChoices[i / 4];
    cand_m[i] = i % 4 == 0 ? CR_BATCH_PHASES : CR_BATCH_FUSED;
    cand_k[i] = i % 4 == 0 ? 1 : kBatchTileChoices[i % 4 - 1];
  }
  double best_ms[NC];
  for (int i = 0; i < NC; ++i) best_ms[i] = 1e300;
  cudaEvent_t e0, e1;
  CR_BCUDA(b, cudaEventCreate(&e0));
  CR_BCUDA(b, cudaEventCreate(&e1));
  const void* P = b->dmem + b->params_off;
  cr_status st = CR_OK;
  // Pass 0 warms every candidate up (graph upload, first launch); passes
  // 1..trial_steps time one step of each candidate in turn, so the state the
  // problems reach as they advance is shared fairly between the candidates;
  // each candidate keeps its fastest step.
  for (int r = 0; r <= trial_steps && st == CR_OK; ++r) {
    for (int i = 0; i < NC && st == CR_OK; ++i) {
      b->threads = cand_t[i];
      b->mode = cand_m[i];
      b->tiles = cand_k[i];
      st = batch_build(b);
      if (st != CR_OK) break;
      if (batch_set_run(P, (int)b->ctx.size(), 1e300, b->fp32, b->stream) != cudaSuccess) {
        st = bfail(b, CR_E_CUDA, "cr_batch_autotune: launch failed");
        break;
      }
      cudaEventRecord(e0, b->stream);
      st = batch_launch_steps(b, 1);
      cudaEventRecord(e1, b->stream);
      if (st == CR_OK) st = cr_batch_sync(b);
      float ms = 0.0f;
      if (st == CR_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        st = bfail(b, CR_E_CUDA, "cr_batch_autotune: event timing");
      if (st == CR_OK && r > 0 && ms < best_ms[i]) best_ms[i] = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != CR_OK) return st;
  int bi = 0;
  for (int i = 1; i < NC; ++i)
    if (best_ms[i] < best_ms[bi]) bi = i;
  if (ms_per_step)
    for (int i = 0; i < NC; ++i) ms_per_step[i] = best_ms[i];
  b->threads = cand_t[bi];
  b->mode = cand_m[bi];
  b->tiles = cand_k[bi];
  st = batch_build(b);
  if (threads_out) *threads_out = cand_t[bi];
  if (mode_out) *mode_out = cand_m[bi];
  if (tiles_out) *tiles_out = cand_k[bi];
  return st;
}

cr_status cr_batch_barrier_test(cr_batch* b, unsigned long long polls, int phantom) {
  if (!b || phantom < 0) return bfail(b, CR_E_INVALID_ARG, "cr_batch_barrier_test: bad arguments");
  b->spin_limit = polls ? polls : (1ull << 26);
  b->phantom = phantom;
  return batch_build(b);
}

const char* cr_batch_last_error(const cr_batch* b) { return b ? b->err.c_str() : g_init_error.c_str(); }

}  // extern "C"
