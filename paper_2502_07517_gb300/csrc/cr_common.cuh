// Shared device-side definitions of the cRKFR library: the time-control
// record, the per-degree tables, launch parameters, the Butcher tableaux and
// the equation functors.  Everything here is compiled for sm_103a only.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace crk {

constexpr int kMaxN = 4;
constexpr int kMaxNodes1 = kMaxN + 1;

// Status bits kept in TimeCtl::status.
enum : int { kStInadmissible = 1, kStNonFinite = 2, kStInvalidInput = 4 };

// Time control of one context, resident in device memory.  The step size of
// the next step is planned once (plan_step) by whoever changed its inputs: the
// one-warp kernel that ends a step (k_finish_step, k_batch_finish), the last
// block of the prologue or of the persistent batched kernel's update phase, or
// the run-setup kernel; the step kernels only read dt_step, so a whole run can
// be enqueued without host round trips.
struct TimeCtl {
  double t;                 // current time
  double t_final;           // the run stops here; the last step is clipped to it
  double dt_fixed;          // > 0: use this dt instead of the CFL rule
  double cfl_factor;        // C_s * CFL(N), eq. (time.step.2d)
  double rate_last;         // max_e sigma_x(mean)/dx + sigma_y(mean)/dy of the current state
  unsigned long long rate_acc;  // running max (bit pattern of a non-negative double)
  unsigned int blocks_done; // last-block counter (prologue, persistent batched update phase)
  int status;               // kSt* bits, sticky until cr_set_state
  int bad_elem;             // smallest element index that set a status bit
  int steps;                // steps taken since cr_set_state
  double dt_step;           // dt of the next step (0: nothing to do)
  float dt_step_f;          // the same in FP32
  int last_step;            // 1 when that step lands on t_final
  double* out;              // when set (cr_step_get), the single-problem update kernel also
                            // writes the new FP64 state here (page-locked host memory)
  int out_done;             // set by the step that wrote out
};

// The running maximum of the CFL rate in a single-problem step is spread over
// kRateParts counters, one per 256-byte line after the TimeCtl block of a
// context (its device allocation is kCtlBytes): the update blocks fold their
// rate into counter (block % kRateParts) without waiting, and k_finish_step
// takes the maximum of the counters.  One counter for all blocks serialised
// their reductions at one L2 slice.
constexpr int kRateParts = 32;
constexpr size_t kRateLine = 256;
constexpr size_t kCtlBytes = kRateLine * (1 + kRateParts);
static_assert(sizeof(TimeCtl) <= kRateLine, "TimeCtl fits its line");
__host__ __device__ inline unsigned long long* rate_part(TimeCtl* c, int i) {
  return reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(c) + kRateLine * (1 + i));
}

// Plan the next step from the current time, rate and run limits (one thread).
__device__ __forceinline__ void plan_step(TimeCtl* c) {
  double dt = 0.0;
  int last = 0;
  const double rem = c->t_final - c->t;
  if (c->status == 0 && rem > 0.0) {
    const double dtc = c->dt_fixed > 0.0 ? c->dt_fixed : c->cfl_factor / c->rate_last;
    if (dtc >= rem) {
      dt = rem;
      last = 1;
    } else {
      dt = dtc;
    }
  }
  c->dt_step = dt;
  c->dt_step_f = float(dt);
  c->last_step = last;
}

// Reference-element tables for degree N in the arithmetic type of the kernel
// (filled on the host from FP64 values).
template <typename real>
struct Tab {
  real xi[kMaxNodes1], w[kMaxNodes1], invw[kMaxNodes1];
  real l0[kMaxNodes1], l1[kMaxNodes1];     // l_p(0), l_p(1)
  real gR[kMaxNodes1], gL[kMaxNodes1];     // g_R'(xi_p) = l_p(1)/w_p, g_L'(xi_p) = -l_p(0)/w_p
  real dm[kMaxNodes1], dp[kMaxNodes1];     // subcell faces relative to the node: x_{p-+1/2} - xi_p
  real xs[kMaxNodes1 + 1];                 // subcell faces x_{p-1/2} (cumulative weights)
  real ihm[kMaxNodes1], ihp[kMaxNodes1], ihc[kMaxNodes1];  // inverse node spacings incl. halo nodes
  real V[kMaxNodes1 * kMaxNodes1];         // V[j*n+p] = (2j+1) w_p L_j(2 xi_p - 1) (Legendre modes)
};

// Mesh, physics and limiter switches (one struct per launch, by value).
struct Mesh {
  int nx, ny, ne, nfx, nfy;  // elements and faces per direction (nf = n or n+1)
  int bcx, bcy;              // 0 periodic, else not periodic (the side types are in bcs)
  double x0, y0, dx, dy, invdx, invdy;
  int limiter;               // CR_LIM_* bits
  int alpha_mode;            // 0 indicator, 1 fixed, 2 learned (network, indicator fallback)
  double alpha_fixed;
  double gamma, ax, ay;
  int source;
  double src_amp, src_k, src_cx, src_cy;
  double T_ind, s_ind;       // indicator threshold T(N) and sharpness s
  double cflim[4];           // 1/(kappa w h) of the flux-limiter candidates on face sides
                             // 0..3 (x-left: w_0 dx, x-right: w_N dx, y-bottom, y-top)
  int dissipation;           // 0 D2, 1 D1, 2 D-CSX (Sec. 3.1)
  int central;               // 0 EA, 1 AE (Sec. 3.1.2)
  int bcs[4];                // boundary type of sides x-, x+, y-, y+ (CR_BC_* codes)
  double bcg[4][6];          // ghost state g of Dirichlet / inflow sides
  double grav[2];            // gravity (g_x, g_y), source 2
  int bcflux;                // flux at Dirichlet sides: 0 the scheme's own, 1 HLLC (Euler)
  int bcnt;                  // > 0: Dirichlet / inflow ghost states are Chebyshev series in t
  double bct0, bct1;         // their time interval
  double bcc[4][16];         // their coefficients per side (scalar equations)
};

enum : int { kBcPeriodic = 0, kBcOutflow = 1, kBcWall = 2, kBcDirichlet = 3, kBcInflow = 4 };

enum : int { kLimBlend = 1, kLimMH = 2, kLimFlux = 4, kLimScaling = 8, kLimTraces = 16 };

// Device buffers of one context (all inside the workspace).
template <typename real>
struct Bufs {
  real* u;           // state [M][Ne][Np] (FP32_BULK: fluctuation about the mean)
  double* umean;     // FP32_BULK: element means [M][Ne] (FP64)
  float* umean_f;    // FP32_BULK: the same means rounded to FP32 (read by the FP32 kernels)
  real* P;           // partial update [M][Ne][Np] (everything but the element-face fluxes)
  double* smean;     // FP32_BULK: sum_k W_k S_k per element [M][Ne] (FP64)
  real* slot;        // per element face-node data [4M+1][nside][Ne][nfn]
  real* fx;          // x-face numerical flux [M][ny][nfx][nq]
  real* fy;          // y-face numerical flux [M][nfy][nx][n]
  double* alpha_raw; // indicator alpha of the current state [Ne]
  float* alpha_raw_f; // FP32_BULK: the same in FP32, what the FP32 element kernel reads [Ne]
  double* alpha;     // smoothed alpha used by the last step [Ne]
  TimeCtl* ctl;
  const int* mlp_flag;              // != 0 once network weights are loaded
  const unsigned short* mlp_w;      // BF16 network weights (learned alpha)
  float* feat;                      // when not null, the prologue writes network inputs [Ne][Np]
  const double* u_src;              // when not null (FP64), the prologue reads the state from
                                    // here (pinned host memory) and stores it into u
};

// Physical constants in the arithmetic type of the kernel (no FP64 work leaks
// into FP32 arithmetic through double constants).
template <typename real>
struct Phys {
  real gamma, gm1, ax, ay;
  real invdx, invdy;  // 1/dx, 1/dy of the mesh
  real a0, a1, a2, a3;  // a(x) = a0 + a1 x + a2 x^2 + a3 x^3 of variable advection
  real cflim[4];        // Mesh::cflim in the kernel's type (no FP64 conversion in the kernels)
};

// Differentiation matrix D[i*n+j] = l_j'(xi_i) (Sec. 2 eq. (diff.matrix)) and
// FR volume matrix Dt = D - g_R' l(1)^T - g_L' l(0)^T (the trace terms of eq.
// (crkfr.avg) folded in), scaled by the inverse element widths so that a stage
// residual (and the FR volume part) over both directions is one FMA chain:
// Dx = D / dx, Dy = D / dy, Dtx = Dt / dx, Dty = Dt / dy.  Per problem (a
// batch shares Tab between problems of different widths).
template <typename real>
struct DiffScaled {
  real Dx[kMaxNodes1 * kMaxNodes1], Dy[kMaxNodes1 * kMaxNodes1];
  real Dtx[kMaxNodes1 * kMaxNodes1], Dty[kMaxNodes1 * kMaxNodes1];
};

template <typename real>
struct KParams {
  Mesh m;
  Phys<real> ph;        // constants in the bulk type
  Phys<double> phd;     // FP64 constants (limiters, means)
  DiffScaled<real> ds;  // scaled differentiation matrices in the bulk type
  Bufs<real> b;
  // The tables last: they depend only on the degree, so the batched kernels take
  // them as kernel parameters and copy only the part before tb per problem.
  Tab<real> tb;         // tables in the bulk type
  Tab<double> td;       // FP64 tables (limiters, means)
};

// Host: fill ds from D and Dt of degree N (FP64, row-major n x n; each
// product rounded once), with w, l(0), l(1) of the nodes giving Dt.
template <typename real>
inline void fill_scaled(const double* D, const double* w, const double* l0, const double* l1, int N,
                        double invdx, double invdy, DiffScaled<real>* ds) {
  const int n = N + 1;
  for (int i = 0; i < kMaxNodes1 * kMaxNodes1; ++i)
    ds->Dx[i] = ds->Dy[i] = ds->Dtx[i] = ds->Dty[i] = real(0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double d = D[i * n + j];
      const double dt = d - (l1[i] / w[i]) * l1[j] + (l0[i] / w[i]) * l0[j];
      ds->Dx[i * n + j] = real(d * invdx);
      ds->Dy[i * n + j] = real(d * invdy);
      ds->Dtx[i * n + j] = real(dt * invdx);
      ds->Dty[i * n + j] = real(dt * invdy);
    }
}

// ---------------------------------------------------------------------------
// Butcher tableaux (Sec. 2 eq. (butcher)); degree N uses order N+1 (Sec. 3).
// N=1 cRK22 eq. (crk22), N=2 cRK33 eq. (crk33), N=3 cRK44 eq. (crk44).  The
// paper prints no fifth-order scheme for N=4; the six-stage fifth-order method
// of Butcher with c = (0, 1/4, 1/4, 1/2, 3/4, 1) is used.
template <int N> struct Tableau;
// c_i = sum_j a_ij (summed in j order)
template <int N>
__host__ __device__ constexpr double tableau_c(int i) {
  double r = 0.0;
  for (int j = 0; j < Tableau<N>::S; ++j) r += Tableau<N>::a(i, j);
  return r;
}
template <> struct Tableau<1> {
  static constexpr int S = 2;
  __host__ __device__ static constexpr double a(int i, int j) { return (i == 1 && j == 0) ? 0.5 : 0.0; }
  __host__ __device__ static constexpr double b(int i) { return i == 1 ? 1.0 : 0.0; }
};
template <> struct Tableau<2> {
  static constexpr int S = 3;
  __host__ __device__ static constexpr double a(int i, int j) {
    return (i == 1 && j == 0) ? 1.0 / 3.0 : (i == 2 && j == 1) ? 2.0 / 3.0 : 0.0;
  }
  __host__ __device__ static constexpr double b(int i) { return i == 0 ? 0.25 : i == 2 ? 0.75 : 0.0; }
};
template <> struct Tableau<3> {
  static constexpr int S = 4;
  __host__ __device__ static constexpr double a(int i, int j) {
    return (j == i - 1) ? (i == 3 ? 1.0 : 0.5) : 0.0;
  }
  __host__ __device__ static constexpr double b(int i) {
    return (i == 0 || i == 3) ? 1.0 / 6.0 : 1.0 / 3.0;
  }
};
template <> struct Tableau<4> {
  static constexpr int S = 6;
  __host__ __device__ static constexpr double a(int i, int j) {
    return i == 1 ? (j == 0 ? 0.25 : 0.0)
         : i == 2 ? (j < 2 ? 0.125 : 0.0)
         : i == 3 ? (j == 1 ? -0.5 : j == 2 ? 1.0 : 0.0)
         : i == 4 ? (j == 0 ? 3.0 / 16.0 : j == 3 ? 9.0 / 16.0 : 0.0)
         : i == 5 ? (j == 0 ? -3.0 / 7.0 : j == 1 ? 2.0 / 7.0 : j == 2 ? 12.0 / 7.0
                   : j == 3 ? -12.0 / 7.0 : j == 4 ? 8.0 / 7.0 : 0.0)
         : 0.0;
  }
  __host__ __device__ static constexpr double b(int i) {
    return i == 0 ? 7.0 / 90.0 : i == 2 ? 32.0 / 90.0 : i == 3 ? 12.0 / 90.0
         : i == 4 ? 32.0 / 90.0 : i == 5 ? 7.0 / 90.0 : 0.0;
  }
};

// ---------------------------------------------------------------------------
// Equation functors.  dir = 0 (x) or 1 (y); calls with a literal dir fold.
//   flux(u, dir, f)            physical flux in direction dir
//   flux_xy(u, f, g)           both directions, one reciprocal of rho
//   flux_speed(u, dir, f, s)   flux and spectral radius, one reciprocal
//   speed(u, dir)              spectral radius sigma of the flux Jacobian
//   constraint(u, k)           admissibility constraint P_k (Sec. 2 eq. (uad.form))
//   admissible_fast(u)         all P_k > 0, tested without division (multiplied by rho > 0)
//   indicator_var(u)           variable the smoothness indicator looks at
// x > 0, with the FP64 test on the integer pipe (the FP64 pipe is the scarce
// unit): as a signed 64-bit integer a double is positive exactly when its sign
// bit is clear and it is not +0; NaN patterns (above +inf) are excluded, as the
// floating-point comparison excludes them.
__device__ __forceinline__ bool gt0(float x) { return x > 0.0f; }
__device__ __forceinline__ bool gt0(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0ll && b <= 0x7ff0000000000000ll;
}
template <typename real>
__device__ __forceinline__ real sqrt_pos(real x) { return sqrt(gt0(x) ? x : real(0)); }

struct EqLinAdv {  // u_t + a . grad u = 0, Sec. 5.1.1
  static constexpr int M = 1, K = 0;
  template <typename real>
  __device__ static void flux(const real* u, int dir, real* f, const Phys<real>& ph) {
    f[0] = (dir == 0 ? ph.ax : ph.ay) * u[0];
  }
  template <typename real>
  __device__ static void flux_xy(const real* u, real* f, real* g, const Phys<real>& ph) {
    f[0] = ph.ax * u[0];
    g[0] = ph.ay * u[0];
  }
  template <typename real>
  __device__ static real speed(const real*, int dir, const Phys<real>& ph) {
    return fabs(dir == 0 ? ph.ax : ph.ay);
  }
  template <typename real>
  __device__ static void flux_speed(const real* u, int dir, real* f, real* s, const Phys<real>& ph) {
    flux(u, dir, f, ph);
    *s = speed(u, dir, ph);
  }
  template <typename real>
  __device__ static real constraint(const real*, int, const Phys<real>&) { return real(1); }
  template <typename real>
  __device__ static bool admissible_fast(const real*, const Phys<real>&) { return true; }
  template <typename real>
  __device__ static real indicator_var(const real* u, const Phys<real>&) { return u[0]; }
};

// Variable advection, Sec. 5.1: f(x, u) = a(x) u with a cubic a(x) (1D).
// The flux depends on the position: the kernels call it through flux_at /
// speed_at with the coordinate of the point; the position-free forms below
// (a at x = 0) exist only so that the shared templates compile.
struct EqVarAdv {
  static constexpr int M = 1, K = 0;
  template <typename real>
  __device__ static real coef(real x, const Phys<real>& ph) {
    return ((ph.a3 * x + ph.a2) * x + ph.a1) * x + ph.a0;
  }
  template <typename real>
  __device__ static void flux(const real* u, int, real* f, const Phys<real>& ph) { f[0] = ph.a0 * u[0]; }
  template <typename real>
  __device__ static void flux_xy(const real* u, real* f, real* g, const Phys<real>& ph) {
    f[0] = ph.a0 * u[0];
    g[0] = real(0);
  }
  template <typename real>
  __device__ static real speed(const real*, int, const Phys<real>& ph) { return fabs(ph.a0); }
  template <typename real>
  __device__ static void flux_speed(const real* u, int dir, real* f, real* s, const Phys<real>& ph) {
    flux(u, dir, f, ph);
    *s = speed(u, dir, ph);
  }
  template <typename real>
  __device__ static real constraint(const real*, int, const Phys<real>&) { return real(1); }
  template <typename real>
  __device__ static bool admissible_fast(const real*, const Phys<real>&) { return true; }
  template <typename real>
  __device__ static real indicator_var(const real* u, const Phys<real>&) { return u[0]; }
};

template <class EQ> struct IsVarAdv { static constexpr bool value = false; };
template <> struct IsVarAdv<EqVarAdv> { static constexpr bool value = true; };

// Flux, wave speed and both at position x along the face normal: variable
// advection evaluates a(x); every other equation ignores x.
template <class EQ, typename real>
__device__ __forceinline__ void flux_at(const real* u, int dir, real* f, const Phys<real>& ph, real x) {
  if constexpr (IsVarAdv<EQ>::value) f[0] = EqVarAdv::coef(x, ph) * u[0];
  else EQ::flux(u, dir, f, ph);
}
template <class EQ, typename real>
__device__ __forceinline__ real speed_at(const real* u, int dir, const Phys<real>& ph, real x) {
  if constexpr (IsVarAdv<EQ>::value) return fabs(EqVarAdv::coef(x, ph));
  else return EQ::speed(u, dir, ph);
}
template <class EQ, typename real>
__device__ __forceinline__ void flux_speed_at(const real* u, int dir, real* f, real* s,
                                              const Phys<real>& ph, real x) {
  if constexpr (IsVarAdv<EQ>::value) {
    const real a = EqVarAdv::coef(x, ph);
    f[0] = a * u[0];
    *s = fabs(a);
  } else {
    EQ::flux_speed(u, dir, f, s, ph);
  }
}

// Given ghost state of side s at time t (Dirichlet / inflow): the constant
// bcg, or for a scalar equation with bcnt > 0 the Chebyshev series
// sum_k bcc[s][k] T_k(tau), tau = 2 (t - t0)/(t1 - t0) - 1 clamped to [-1, 1],
// by Clenshaw's recurrence.
template <int M, typename real>
__device__ __forceinline__ void ghost_at(const Mesh& m, int s, double t, real* g) {
  if (M != 1 || m.bcnt <= 0) {
#pragma unroll
    for (int v = 0; v < M; ++v) g[v] = real(m.bcg[s][v]);
    return;
  }
  double tau = 2.0 * (t - m.bct0) / (m.bct1 - m.bct0) - 1.0;
  tau = fmin(1.0, fmax(-1.0, tau));
  double b1 = 0.0, b2 = 0.0;
  for (int k = m.bcnt - 1; k >= 1; --k) {
    const double b0 = 2.0 * tau * b1 - b2 + m.bcc[s][k];
    b2 = b1;
    b1 = b0;
  }
  g[0] = real(tau * b1 - b2 + m.bcc[s][0]);
}

struct EqBurgers {  // u_t + (u^2/2)_x = 0, Sec. 5.1 (1D); sigma = |u|
  static constexpr int M = 1, K = 0;
  template <typename real>
  __device__ static void flux(const real* u, int, real* f, const Phys<real>&) {
    f[0] = real(0.5) * u[0] * u[0];
  }
  template <typename real>
  __device__ static void flux_xy(const real* u, real* f, real* g, const Phys<real>&) {
    f[0] = real(0.5) * u[0] * u[0];
    g[0] = real(0);
  }
  template <typename real>
  __device__ static real speed(const real* u, int, const Phys<real>&) { return fabs(u[0]); }
  template <typename real>
  __device__ static void flux_speed(const real* u, int dir, real* f, real* s, const Phys<real>& ph) {
    flux(u, dir, f, ph);
    *s = speed(u, dir, ph);
  }
  template <typename real>
  __device__ static real constraint(const real*, int, const Phys<real>&) { return real(1); }
  template <typename real>
  __device__ static bool admissible_fast(const real*, const Phys<real>&) { return true; }
  template <typename real>
  __device__ static real indicator_var(const real* u, const Phys<real>&) { return u[0]; }
};

// Euler, Sec. 5.2 eq. (1deuler) (DIM 1, u = rho, rho v, E) and Sec. 5.3
// eq. (2deuler) (DIM 2, u = rho, rho v1, rho v2, E); p from eqs. (state), (2dstate);
// sigma = |v_dir| + c, c = sqrt(gamma p / rho) (eq. (spectral.radius.1d)).
template <int DIM>
struct EqEuler {
  static constexpr int M = DIM == 1 ? 3 : 4, K = 2;
  static constexpr int E = DIM == 1 ? 2 : 3;
  template <typename real>
  __device__ static real kinetic_rho(const real* u) {  // rho |v|^2 / 2 * rho = |m|^2 / 2
    return DIM == 1 ? real(0.5) * u[1] * u[1] : real(0.5) * (u[1] * u[1] + u[2] * u[2]);
  }
  template <typename real>
  __device__ static real pressure(const real* u, const Phys<real>& ph) {
    return ph.gm1 * (u[E] - kinetic_rho(u) / u[0]);
  }
  template <typename real>
  __device__ static void flux_r(const real* u, int dir, real rinv, real* f, real* p_out,
                                const Phys<real>& ph) {
    if (DIM == 1) {
      const real v = u[1] * rinv;
      const real p = ph.gm1 * (u[2] - real(0.5) * u[1] * v);
      f[0] = u[1];
      f[1] = u[1] * v + p;
      f[2] = (u[2] + p) * v;
      *p_out = p;
      return;
    }
    const real v1 = u[1] * rinv, v2 = u[2] * rinv;
    const real p = ph.gm1 * (u[3] - real(0.5) * (u[1] * v1 + u[2] * v2));
    const real vn = dir == 0 ? v1 : v2;
    f[0] = u[1 + dir];
    f[1] = u[1] * vn + (dir == 0 ? p : real(0));
    f[2] = u[2] * vn + (dir == 1 ? p : real(0));
    f[3] = (u[3] + p) * vn;
    *p_out = p;
  }
  template <typename real>
  __device__ static void flux(const real* u, int dir, real* f, const Phys<real>& ph) {
    real p;
    flux_r(u, dir, real(1) / u[0], f, &p, ph);
  }
  template <typename real>
  __device__ static void flux_xy(const real* u, real* f, real* g, const Phys<real>& ph) {
    const real rinv = real(1) / u[0];
    if (DIM == 1) {
      real p;
      flux_r(u, 0, rinv, f, &p, ph);
      return;
    }
    const real v1 = u[1] * rinv, v2 = u[2] * rinv;
    const real p = ph.gm1 * (u[3] - real(0.5) * (u[1] * v1 + u[2] * v2));
    const real Ep = u[3] + p;
    f[0] = u[1];
    f[1] = u[1] * v1 + p;
    f[2] = u[2] * v1;
    f[3] = Ep * v1;
    g[0] = u[2];
    g[1] = u[1] * v2;
    g[2] = u[2] * v2 + p;
    g[3] = Ep * v2;
  }
  template <typename real>
  __device__ static void flux_speed(const real* u, int dir, real* f, real* s, const Phys<real>& ph) {
    const real rinv = real(1) / u[0];
    real p;
    flux_r(u, dir, rinv, f, &p, ph);
    *s = fabs(u[1 + dir] * rinv) + sqrt_pos(ph.gamma * p * rinv);
  }
  template <typename real>
  __device__ static real speed(const real* u, int dir, const Phys<real>& ph) {
    const real rinv = real(1) / u[0];
    const real p = ph.gm1 * (u[E] - kinetic_rho(u) * rinv);
    return fabs(u[1 + dir] * rinv) + sqrt_pos(ph.gamma * p * rinv);
  }
  template <typename real>
  __device__ static real constraint(const real* u, int k, const Phys<real>& ph) {
    return k == 0 ? u[0] : pressure(u, ph);
  }
  template <typename real>
  __device__ static bool admissible_fast(const real* u, const Phys<real>&) {
    return gt0(u[0]) && gt0(u[E] * u[0] - kinetic_rho(u));
  }
  template <typename real>
  __device__ static real indicator_var(const real* u, const Phys<real>& ph) {
    return u[0] * pressure(u, ph);
  }
};

// Ten-moment equations, Sec. 5.4 eq. (tmp); u = (rho, rho v1, rho v2, E11, E12, E22),
// P = 2E - rho v (x) v.  Admissibility: rho > 0 and lambda_min(P) > 0; wave speed
// |v_dir| + sqrt(3 p_dirdir / rho).
struct EqTenMoment {
  static constexpr int M = 6, K = 2;
  template <typename real>
  __device__ static void flux_r(const real* u, int dir, real rinv, real* f, const Phys<real>&) {
    const real v1 = u[1] * rinv, v2 = u[2] * rinv;
    const real p11 = real(2) * u[3] - u[1] * v1;
    const real p12 = real(2) * u[4] - u[1] * v2;
    const real p22 = real(2) * u[5] - u[2] * v2;
    if (dir == 0) {
      f[0] = u[1];
      f[1] = p11 + u[1] * v1;
      f[2] = p12 + u[1] * v2;
      f[3] = (u[3] + p11) * v1;
      f[4] = u[4] * v1 + real(0.5) * (p11 * v2 + p12 * v1);
      f[5] = u[5] * v1 + p12 * v2;
    } else {
      f[0] = u[2];
      f[1] = p12 + u[1] * v2;
      f[2] = p22 + u[2] * v2;
      f[3] = u[3] * v2 + p12 * v1;
      f[4] = u[4] * v2 + real(0.5) * (p12 * v2 + p22 * v1);
      f[5] = (u[5] + p22) * v2;
    }
  }
  template <typename real>
  __device__ static void flux(const real* u, int dir, real* f, const Phys<real>& ph) {
    flux_r(u, dir, real(1) / u[0], f, ph);
  }
  template <typename real>
  __device__ static void flux_xy(const real* u, real* f, real* g, const Phys<real>& ph) {
    const real rinv = real(1) / u[0];
    flux_r(u, 0, rinv, f, ph);
    flux_r(u, 1, rinv, g, ph);
  }
  template <typename real>
  __device__ static real speed_r(const real* u, int dir, real rinv) {
    const real v = u[1 + dir] * rinv;
    const real pdd = real(2) * u[3 + 2 * dir] - u[1 + dir] * v;
    return fabs(v) + sqrt_pos(real(3) * pdd * rinv);
  }
  template <typename real>
  __device__ static void flux_speed(const real* u, int dir, real* f, real* s, const Phys<real>& ph) {
    const real rinv = real(1) / u[0];
    flux_r(u, dir, rinv, f, ph);
    *s = speed_r(u, dir, rinv);
  }
  template <typename real>
  __device__ static real speed(const real* u, int dir, const Phys<real>&) {
    return speed_r(u, dir, real(1) / u[0]);
  }
  template <typename real>
  __device__ static real constraint(const real* u, int k, const Phys<real>&) {
    if (k == 0) return u[0];
    const real rinv = real(1) / u[0];
    const real p11 = real(2) * u[3] - u[1] * u[1] * rinv;
    const real p12 = real(2) * u[4] - u[1] * u[2] * rinv;
    const real p22 = real(2) * u[5] - u[2] * u[2] * rinv;
    const real h = real(0.5) * (p11 - p22);
    return real(0.5) * (p11 + p22) - sqrt(h * h + p12 * p12);
  }
  template <typename real>
  __device__ static bool admissible_fast(const real* u, const Phys<real>&) {
    // rho P = 2 rho E - m m^T positive definite
    const real a11 = real(2) * u[0] * u[3] - u[1] * u[1];
    const real a22 = real(2) * u[0] * u[5] - u[2] * u[2];
    const real a12 = real(2) * u[0] * u[4] - u[1] * u[2];
    return gt0(u[0]) && gt0(a11) && gt0(a11 * a22 - a12 * a12);
  }
  template <typename real>
  __device__ static real indicator_var(const real* u, const Phys<real>&) {
    const real rinv = real(1) / u[0];
    const real p11 = real(2) * u[3] - u[1] * u[1] * rinv;
    const real p22 = real(2) * u[5] - u[2] * u[2] * rinv;
    return u[0] * real(0.5) * (p11 + p22);
  }
};

// Gradient of W = amp exp(-k |x - c|^2) for the ten-moment source (eq. (tenmom.source)),
// from the offsets rx = x - cx, ry = y - cy, in the kernel's arithmetic type.
template <int DIM, typename real>
__device__ __forceinline__ void source_grad(const Mesh& m, real rx, real ry, real* dWx, real* dWy) {
  const real kk = real(m.src_k);
  const real W = real(m.src_amp) * exp(-kk * (rx * rx + ry * ry));
  *dWx = real(-2) * kk * rx * W;
  *dWy = DIM == 2 ? real(-2) * kk * ry * W : real(0);
}

// Euler with the gravity source of Sec. 5.5: the same equations as a type of
// its own, so that kernels for problems without a source carry no source code
// (a runtime switch cost the FP32 element kernel 4%).
template <int DIM> struct EqEulerG : EqEuler<DIM> {};

template <class EQ> struct IsEuler { static constexpr bool value = false; };
template <int DIM> struct IsEuler<EqEuler<DIM>> { static constexpr bool value = true; };
template <int DIM> struct IsEuler<EqEulerG<DIM>> { static constexpr bool value = true; };
template <class EQ> struct HasGravity { static constexpr bool value = false; };
template <int DIM> struct HasGravity<EqEulerG<DIM>> { static constexpr bool value = true; };

// Source at one point.  Ten-moment: s = s^x + s^y of eq. (tenmom.source),
// linear in u for fixed grad W = (dWx, dWy).  Euler with gravity (Sec. 5.5):
// (dWx, dWy) holds g and s = (0, rho g, rho v . g) (the energy term is the
// work of the force rho g).
template <class EQ, typename real>
__device__ __forceinline__ void source_eval(const real* u, real dWx, real dWy, real* s) {
  if constexpr (IsEuler<EQ>::value) {
    s[0] = real(0);
    if constexpr (EQ::M == 3) {
      s[1] = u[0] * dWx;
      s[2] = u[1] * dWx;
    } else {
      s[1] = u[0] * dWx;
      s[2] = u[0] * dWy;
      s[3] = u[1] * dWx + u[2] * dWy;
    }
  } else if constexpr (EQ::M == 6) {
    s[0] = real(0);
    s[1] = real(-0.5) * u[0] * dWx;
    s[2] = real(-0.5) * u[0] * dWy;
    s[3] = real(-0.5) * u[1] * dWx;
    s[4] = real(-0.25) * (u[2] * dWx + u[1] * dWy);
    s[5] = real(-0.5) * u[2] * dWy;
  } else {
    for (int v = 0; v < EQ::M; ++v) s[v] = real(0);
  }
}

}  // namespace crk
