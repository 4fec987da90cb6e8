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
// Defined with the context code: the kernel parameters of a description
// without the buffers (the same routine a context uses), and the message
// cr_last_error(NULL) returns.
void fill_static_params(const cr_mesh_desc* d, KParams<double>* P);
void record_global_error(const std::string& msg);
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

// The status code, with its message kept for cr_last_error(NULL).
cr_status static_fail(cr_status st, const std::string& msg) {
  record_global_error(msg);
  return st;
}

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
  c->out = nullptr;
  c->out_done = 0;
  for (int i = 0; i < kRateParts; ++i) *rate_part(c, i) = 0ull;
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
  const size_t o_ctl = take(kCtlBytes);
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
  fill_static_params(d, &P);
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
