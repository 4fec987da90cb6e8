// cr_step_static: one FP64 cRKFR step that allocates no memory.
//
// Some callers cannot allocate device memory when they want to advance a
// state: a host application whose whole device memory is already handed to
// another allocator (a framework's memory pool) and that may not allocate
// around it, code that must not pay cudaMalloc/cudaFree's implicit device
// synchronisation in a time-critical loop, or software that forbids dynamic
// allocation once it has started.  For them this entry point keeps all of the
// step's scratch (partial update, face-node data, face fluxes, blending
// coefficients, time control) in one file-scope device array of
// kStaticScratchBytes bytes.  Every GPU that loads the library reserves that
// array until the process exits.  Inputs and outputs still come from the
// caller.  The step itself runs the same kernels as cr_step.
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/cr.h"
#include "cr_launch.cuh"

namespace crk {
// Per-side boundary types, ghost states and gravity of the kernels' Mesh
// (defined with the context code).
void fill_mesh_extras(const cr_mesh_desc* d, Mesh* m);
}  // namespace crk

using namespace crk;

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

// The shared scratch.  Device code may name it; host code must use the address
// from cudaGetSymbolAddress (the host-side name is only a stand-in).
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
unsigned char* g_static_ptr[kMaxDevices] = {};

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// The status code is the whole report; the message documents the cause here.
cr_status static_fail(cr_status st, const std::string&) { return st; }

__global__ void k_static_reset(TimeCtl* c, double dt) {
  c->t = 0.0;
  c->t_final = dt;
  c->dt_fixed = dt;
  c->cfl_factor = 0.0;
  c->rate_last = 0.0;
  c->rate_acc = 0ull;
  c->blocks_done = 0u;
  c->status = 0;
  c->bad_elem = INT_MAX;
  c->steps = 0;
  c->dt_step = 0.0;
  c->dt_step_f = 0.0f;
  c->last_step = 0;
}

// Reference tables of degree N from the public host routine, plus the derived
// per-kernel tables (same definitions as the context path); D receives the
// differentiation matrix (n x n).
void static_tables(int N, Tab<double>* t, double* D) {
  const int n = N + 1;
  double xi[kMaxNodes1], w[kMaxNodes1];
  cr_reference_tables(N, xi, w, D);
  double lam[kMaxNodes1], l0[kMaxNodes1], l1[kMaxNodes1];
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) prod *= xi[j] - xi[m];
    lam[j] = 1.0 / prod;
  }
  for (int side = 0; side < 2; ++side) {
    double den = 0.0;
    for (int m = 0; m < n; ++m) den += lam[m] / (side - xi[m]);
    for (int j = 0; j < n; ++j) (side ? l1 : l0)[j] = lam[j] / (side - xi[j]) / den;
  }
  memset(t, 0, sizeof(*t));
  double X[kMaxNodes1 + 2];
  X[0] = xi[N] - 1.0;
  for (int p = 0; p < n; ++p) X[p + 1] = xi[p];
  X[n + 1] = 1.0 + xi[0];
  double xs = 0.0;
  for (int p = 0; p < n; ++p) {
    t->xi[p] = xi[p];
    t->w[p] = w[p];
    t->invw[p] = 1.0 / w[p];
    t->l0[p] = l0[p];
    t->l1[p] = l1[p];
    t->gR[p] = l1[p] / w[p];
    t->gL[p] = -l0[p] / w[p];
    t->xs[p] = xs;
    t->dm[p] = xs - xi[p];
    t->dp[p] = xs + w[p] - xi[p];
    xs += w[p];
    t->ihm[p] = 1.0 / (X[p + 1] - X[p]);
    t->ihp[p] = 1.0 / (X[p + 2] - X[p + 1]);
    t->ihc[p] = 1.0 / (X[p + 2] - X[p]);
  }
  t->xs[n] = xs;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double pm = 1.0, pc = 2.0 * xi[j] - 1.0, x = pc;  // Legendre L_i(2 xi_j - 1)
      double Li = (i == 0) ? 1.0 : x;
      for (int k = 2; k <= i; ++k) {
        const double pn = ((2 * k - 1) * x * pc - (k - 1) * pm) / k;
        pm = pc;
        pc = pn;
        Li = pc;
      }
      t->V[i * n + j] = (2.0 * i + 1.0) * w[j] * Li;
    }
}

}  // namespace

extern "C" cr_status cr_step_static(const cr_mesh_desc* d, const double* u_in, double* u_out,
                                    double dt) {
  if (!d || !u_in || !u_out || !(dt > 0.0))
    return static_fail(CR_E_INVALID_ARG, "cr_step_static: NULL pointer or dt <= 0");
  if (d->bc_time_terms > 0)
    return static_fail(CR_E_UNSUPPORTED, "cr_step_static: time-independent boundary states only");
  if (d->dissipation != CR_DISS_D2 || d->central != CR_CENTRAL_EA || d->points != CR_POINTS_GL)
    return static_fail(CR_E_UNSUPPORTED,
                       "cr_step_static: D2 dissipation, EA flux and Gauss-Legendre points only");
  if (d->precision != CR_FP64)
    return static_fail(CR_E_UNSUPPORTED, "cr_step_static: FP64 precision only");
  size_t probe = 0;
  if (cr_workspace_bytes(d, &probe) != CR_OK)
    return static_fail(CR_E_INVALID_ARG, std::string("cr_step_static: ") + cr_last_error(nullptr));
  const KernelSet* ks = nullptr;
  {
    const int N = d->degree;
    if (d->equation == CR_EQ_LINADV) ks = d->dim == 1 ? kernels_linadv1d(N, 0) : kernels_linadv2d(N, 0);
    else if (d->equation == CR_EQ_EULER && d->source == CR_SRC_GRAVITY)
      ks = d->dim == 1 ? kernels_euler1d_grav(N, 0) : kernels_euler2d_grav(N, 0);
    else if (d->equation == CR_EQ_EULER) ks = d->dim == 1 ? kernels_euler1d(N, 0) : kernels_euler2d(N, 0);
    else if (d->equation == CR_EQ_BURGERS) ks = d->dim == 1 ? kernels_burgers1d(N, 0) : nullptr;
    else if (d->equation == CR_EQ_VARADV) ks = d->dim == 1 ? kernels_varadv1d(N, 0) : nullptr;
    else ks = d->dim == 1 ? kernels_tenmoment1d(N, 0) : kernels_tenmoment2d(N, 0);
  }
  if (!ks) return static_fail(CR_E_UNSUPPORTED, "cr_step_static: combination not built");

  // scratch layout inside the static array
  const int n = d->degree + 1, dim = d->dim, M = ks->nvars, np = ks->nodes;
  const size_t nx = d->nx, ny = dim == 2 ? d->ny : 1, ne = nx * ny;
  const size_t nfx = d->bc_x == CR_BC_PERIODIC ? nx : nx + 1;
  const size_t nfy = dim == 2 ? (d->bc_y == CR_BC_PERIODIC ? ny : ny + 1) : 0;
  const size_t nside = dim == 2 ? 4 : 2, nfn = dim == 2 ? n : 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += round256(bytes);
    return o;
  };
  const size_t o_ctl = take(sizeof(TimeCtl));
  const size_t o_P = take((size_t)M * ne * np * sizeof(double));
  const size_t o_slot = take((size_t)(4 * M + 1) * nside * ne * nfn * sizeof(double));
  const size_t o_fx = take((size_t)M * ny * nfx * nfn * sizeof(double));
  const size_t o_fy = take(dim == 2 ? (size_t)M * nfy * nx * n * sizeof(double) : 0);
  const size_t o_ar = take(ne * sizeof(double));
  const size_t o_al = take(ne * sizeof(double));
  if (off > kStaticScratchBytes)
    return static_fail(CR_E_TOO_LARGE,
                       "cr_step_static: mesh needs " + std::to_string(off) +
                           " bytes of scratch, the static limit is " +
                           std::to_string(kStaticScratchBytes));

  // once per device, with that device current: the device address of the array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return static_fail(CR_E_CUDA, "cr_step_static: no current CUDA device");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess || !ptr)
        return static_fail(CR_E_CUDA, std::string("cr_step_static: cudaGetSymbolAddress: ") +
                                          cudaGetErrorString(e));
      e = ks->configure();
      if (e != cudaSuccess)
        return static_fail(CR_E_CUDA, std::string("cr_step_static: ") + cudaGetErrorString(e));
      g_static_ptr[dev] = static_cast<unsigned char*>(ptr);
    } else if (ks->configure() != cudaSuccess) {
      return static_fail(CR_E_CUDA, "cr_step_static: kernel configuration failed");
    }
    base = g_static_ptr[dev];
  }

  KParams<double> P;
  memset(&P, 0, sizeof(P));
  Mesh& m = P.m;
  m.nx = (int)nx;
  m.ny = (int)ny;
  m.ne = (int)ne;
  m.nfx = (int)nfx;
  m.nfy = (int)nfy;
  m.bcx = d->bc_x;
  m.bcy = dim == 2 ? d->bc_y : 0;
  m.x0 = d->x0;
  m.y0 = dim == 2 ? d->y0 : 0.0;
  m.dx = (d->x1 - d->x0) / d->nx;
  m.dy = dim == 2 ? (d->y1 - d->y0) / d->ny : 1.0;
  m.invdx = 1.0 / m.dx;
  m.invdy = dim == 2 ? 1.0 / m.dy : 0.0;
  m.limiter = d->limiter;
  m.alpha_mode = d->alpha_mode;
  m.alpha_fixed = d->alpha_fixed;
  m.gamma = d->gamma;
  m.ax = d->adv[0];
  m.ay = d->adv[1];
  m.source = d->source;
  m.src_amp = d->src_amp;
  m.src_k = d->src_k;
  m.src_cx = d->src_cx;
  m.src_cy = d->src_cy;
  fill_mesh_extras(d, &m);
  m.T_ind = 0.5 * std::pow(10.0, -1.8 * std::pow(d->degree + 1.0, 0.25));
  m.s_ind = std::log((1.0 - 1e-4) / 1e-4);
  P.ph.gamma = d->gamma;
  P.ph.gm1 = d->gamma - 1.0;
  P.ph.ax = d->adv[0];
  P.ph.ay = d->adv[1];
  P.ph.a0 = d->adv_poly[0];
  P.ph.a1 = d->adv_poly[1];
  P.ph.a2 = d->adv_poly[2];
  P.ph.a3 = d->adv_poly[3];
  P.ph.invdx = m.invdx;
  P.ph.invdy = m.invdy;
  P.phd = P.ph;
  double Dref[kMaxNodes1 * kMaxNodes1];
  static_tables(d->degree, &P.tb, Dref);
  P.td = P.tb;
  fill_scaled(Dref, P.td.w, P.td.l0, P.td.l1, d->degree, m.invdx, m.invdy, &P.ds);
  {
    const double kappa = dim == 2 ? 0.5 : 1.0;
    m.cflim[0] = 1.0 / (kappa * P.td.w[0] * m.dx);
    m.cflim[1] = 1.0 / (kappa * P.td.w[d->degree] * m.dx);
    m.cflim[2] = 1.0 / (kappa * P.td.w[0] * m.dy);
    m.cflim[3] = 1.0 / (kappa * P.td.w[d->degree] * m.dy);
  }
  P.b.ctl = reinterpret_cast<TimeCtl*>(base + o_ctl);
  P.b.u = u_out;
  P.b.umean = nullptr;
  P.b.umean_f = nullptr;
  P.b.P = reinterpret_cast<double*>(base + o_P);
  P.b.smean = nullptr;
  P.b.slot = reinterpret_cast<double*>(base + o_slot);
  P.b.fx = reinterpret_cast<double*>(base + o_fx);
  P.b.fy = reinterpret_cast<double*>(base + o_fy);
  P.b.alpha_raw = reinterpret_cast<double*>(base + o_ar);
  P.b.alpha = reinterpret_cast<double*>(base + o_al);

  cudaStream_t s = static_cast<cudaStream_t>(d->stream);
  const size_t nbytes = (size_t)M * ne * np * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (u_out != u_in) e = cudaMemcpyAsync(u_out, u_in, nbytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) {
    k_static_reset<<<1, 1, 0, s>>>(P.b.ctl, dt);  // the array keeps the previous call's contents
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = ks->prologue(&P, s);
  if (e == cudaSuccess) e = ks->step(&P, s);
  int status = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&status, &P.b.ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess)
    return static_fail(CR_E_CUDA, std::string("cr_step_static: ") + cudaGetErrorString(e));
  if (status & kStInvalidInput)
    return static_fail(CR_E_INVALID_STATE, "cr_step_static: inadmissible or non-finite input");
  if (status) return static_fail(CR_E_INADMISSIBLE, "cr_step_static: inadmissible step");
  return CR_OK;
}
