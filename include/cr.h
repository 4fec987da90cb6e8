/*
 * cr.h - C ABI of libcrkfr.so, the GB300 (sm_103a) implementation of one time
 * step of compact Runge-Kutta Flux Reconstruction (cRKFR) with the subcell
 * blending limiter, the flux limiter for admissible means and the positivity
 * scaling limiter, after Babbar & Chen, "Compact Runge-Kutta Flux
 * Reconstruction for Hyperbolic Conservation Laws with admissibility
 * preservation", arXiv 2502.07517.
 *
 * Conventions shared by every entry point:
 *  - All calls return a cr_status; CR_OK is 0, errors are negative.  No call
 *    aborts the process.  cr_last_error(ctx) gives a one-line description of
 *    the last error on a context.
 *  - State arrays are FP64, structure-of-arrays u[v][e][k]: variable v,
 *    element e = ix + nx * iy, solution point k = p + (N+1) * q (p along x,
 *    q along y; in 1D k = p).  Solution points are the N+1 Gauss-Legendre
 *    nodes of [0,1] in each direction (Sec. 2, eq. (soln.points)).
 *  - A pointer argument with on_device != 0 is a CUDA device pointer that the
 *    caller owns and keeps valid until the stream work has finished; with
 *    on_device == 0 it is host memory.  The library never frees caller memory.
 *  - Work is ordered on the stream given in cr_mesh_desc.stream (NULL: the
 *    legacy default stream).  Calls that return results on the host
 *    synchronise that stream.
 *  - A context owns its device workspace: either the caller passes a device
 *    buffer of cr_workspace_bytes() bytes to cr_init_mesh, or passes NULL and
 *    the library allocates (and later frees) it with cudaMalloc.
 *  - Contexts are not thread-safe; use one context per host thread.
 */
#ifndef CRKFR_CR_H
#define CRKFR_CR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cr_ctx cr_ctx;

typedef enum {
  CR_OK = 0,
  CR_E_INVALID_ARG = -1,   /* a descriptor field, size or pointer is out of range */
  CR_E_INVALID_STATE = -2, /* cr_set_state: a solution point is inadmissible or not finite */
  CR_E_INADMISSIBLE = -3,  /* cr_step: an element mean left the admissible set,
                              or a value is not finite */
  CR_E_TIMEOUT = -4,       /* a bounded device wait gave up */
  CR_E_CUDA = -5,          /* a CUDA runtime call failed (message in cr_last_error) */
  CR_E_NOMEM = -6,         /* device or host allocation failed */
  CR_E_UNSUPPORTED = -7,   /* this combination (equation, dim, degree, precision) is not built */
  CR_E_TOO_LARGE = -8      /* cr_step_static: the mesh needs more scratch than its fixed array */
} cr_status;

/* CR_EQ_BURGERS: u_t + (u^2/2)_x = 0 (Sec. 5.1), 1D, FP64.  CR_EQ_VARADV:
 * u_t + (a(x) u)_x = 0 with a(x) = sum_k adv_poly[k] x^k (Sec. 5.1, variable
 * advection), 1D, FP64; the flux is evaluated at each point's position. */
enum { CR_EQ_LINADV = 0, CR_EQ_EULER = 1, CR_EQ_TENMOMENT = 2, CR_EQ_BURGERS = 3, CR_EQ_VARADV = 4 };
/* Boundary conditions of Sec. 3.3.  Outflow: the fully-outflow rule F = F^+.
 * Wall (Euler only): ghost values by reflecting the velocity normal to the
 * face, eq. (reflect.time.avg), then the D2 flux as at an interior face.
 * Dirichlet: the inflow/outflow ghost values for a time-independent boundary
 * state g (u^- = U^- = g, F^- = f(g)), then the scheme's own numerical flux
 * (the paper takes an HLLC flux there; Rusanov-type D2 here).  Inflow: the
 * fully-inflow rule F = F^- = f(g).  g is bc_state of the side. */
enum { CR_BC_PERIODIC = 0, CR_BC_OUTFLOW = 1, CR_BC_WALL = 2, CR_BC_DIRICHLET = 3, CR_BC_INFLOW = 4 };
/* Source terms (field source): none; the ten-moment potential of eq.
 * (tenmom.source) with W = src_amp exp(-src_k |x - (src_cx, src_cy)|^2);
 * Euler gravity of Sec. 5.5, s = (0, rho g, rho v . g) with g = gravity. */
enum { CR_SRC_NONE = 0, CR_SRC_TENMOMENT = 1, CR_SRC_GRAVITY = 2 };
/* Solution points and FR correction: Gauss-Legendre points with the Radau
 * correction (Sec. 2, the default), or Gauss-Lobatto-Legendre points with
 * the g2 correction (Sec. 5.1; there the evaluate and extrapolate central
 * fluxes coincide).  GLL takes no blending or flux limiter (the low-order
 * subcell update would outrun its CFL condition at the GLL time step), and
 * neither cr_step_static nor the batched entry points take it. */
enum { CR_POINTS_GL = 0, CR_POINTS_GLL = 1 };
/* Dissipative part D of the numerical flux eq. (numflux.general), Sec. 3.1:
 * D2 eq. (D2) (default: jump of the time-averaged solution traces), D1 eq.
 * (D1) (jump of the u^n traces; lower CFL numbers, computed for it), D-CSX
 * eq. (dcsx) (stage-trace jumps, one wave speed per stage; equal to D2 for
 * linear problems).  The wave speed of D2 and D1 comes from the u^n traces. */
enum { CR_DISS_D2 = 0, CR_DISS_D1 = 1, CR_DISS_DCSX = 2 };
/* Central part F^{+-}, Sec. 3.1.2: EA eq. (evaluate) (default: the stage
 * fluxes at the face, averaged), AE eq. (extrapolate) (the trace of the
 * time-averaged flux; equal to EA for linear problems). */
enum { CR_CENTRAL_EA = 0, CR_CENTRAL_AE = 1 };
enum {
  CR_LIM_BLEND = 1,   /* blend with the subcell scheme, Sec. 4 eq. (blended.scheme) */
  CR_LIM_MH = 2,      /* MUSCL-Hancock subcell fluxes (otherwise first order), Sec. 4.2 */
  CR_LIM_FLUX = 4,    /* flux limiter for admissibility in means, Sec. 4.3 */
  CR_LIM_SCALING = 8, /* Zhang-Shu positivity scaling after the update, Sec. 3.2 */
  CR_LIM_TRACES = 16  /* the scaling limiter also checks the element-face traces */
};
enum {
  CR_ALPHA_INDICATOR = 0, /* smoothness indicator of Sec. 4 (Hennemann form) */
  CR_ALPHA_FIXED = 1,     /* alpha_e = alpha_fixed everywhere (tests) */
  CR_ALPHA_MLP = 2        /* learned network on the indicator's modal energies (not in the
                             paper); the indicator is the fallback when no network is loaded
                             or its output is not finite */
};
enum { CR_FP64 = 0, CR_FP32_BULK = 1 };

typedef struct {
  int dim;               /* 1 or 2 */
  int nx, ny;            /* elements per direction, >= 1 (ny ignored in 1D) */
  double x0, x1, y0, y1; /* domain [x0,x1] x [y0,y1] */
  int bc_x, bc_y;        /* CR_BC_* of both sides of each direction (see bc_side) */
  int degree;            /* N, 1..4; the RK method has order N+1 (Sec. 3) */
  int equation;          /* CR_EQ_*: u_t + a.grad u = 0 (Sec. 5.1.1), Euler (Sec. 5.2,
                            5.3), ten-moment (Sec. 5.4), Burgers (Sec. 5.1, 1D) */
  double gamma;          /* Euler adiabatic constant */
  double adv[2];         /* linear advection velocity */
  int source;            /* CR_SRC_*: none, ten-moment potential, Euler gravity */
  double src_amp, src_k, src_cx, src_cy;
  int limiter;           /* CR_LIM_* bits */
  int alpha_mode;        /* CR_ALPHA_*: smoothness indicator, or alpha_e = alpha_fixed */
  double alpha_fixed;
  int precision;         /* CR_FP64, or CR_FP32_BULK: FP32 stage arithmetic with FP64
                            element means, FP64 flux-limiter and scaling-limiter theta */
  double cfl;            /* CFL(N) of eq. (time.step.2d); <= 0: Fourier analysis */
  double cfl_safety;     /* C_s of eq. (time.step.2d); <= 0: 0.98 */
  void* stream;          /* cudaStream_t or NULL */
  int dissipation;       /* CR_DISS_*; 0 (D2) when zero-initialised */
  int central;           /* CR_CENTRAL_*; 0 (EA) when zero-initialised */
  int bc_side[4];        /* per side x-, x+, y-, y+: 0 = as bc_x / bc_y, else a CR_BC_*
                            code other than periodic for that side alone (a periodic
                            direction takes no override) */
  double bc_state[4][6]; /* conservative ghost state g of each Dirichlet / inflow side
                            (first M entries; admissible for Euler and ten-moment) */
  double gravity[2];     /* (g_x, g_y) of CR_SRC_GRAVITY (Euler) */
  int points;            /* CR_POINTS_*; 0 (Gauss-Legendre, Radau) when zero-initialised */
  double adv_poly[4];    /* a(x) of CR_EQ_VARADV */
  int bc_time_terms;     /* 0..16; > 0 (scalar equations): the ghost states of Dirichlet and
                            inflow sides follow g(t) = sum_{k < terms} bc_time_coef[side][k]
                            T_k(tau), T_k the Chebyshev polynomials, tau = 2 (t - t0) / (t1 - t0)
                            - 1 clamped to [-1, 1], (t0, t1) = bc_time_span; the boundary
                            averages take g at the stage times (Sec. 3.3) */
  double bc_time_span[2];
  double bc_time_coef[4][16];
  int bc_flux;           /* flux at Dirichlet sides: 0 the scheme's own (Rusanov-type D2), 1 the
                            HLLC flux of Sec. 3.3 on the time-averaged ghost values (Euler; not
                            with D1) */
} cr_mesh_desc;

/* Device workspace needed by cr_init_mesh for this descriptor.
 * Errors: CR_E_INVALID_ARG for a bad descriptor or NULL bytes. */
cr_status cr_workspace_bytes(const cr_mesh_desc* desc, size_t* bytes);

/* Create a context for one mesh.  workspace: device buffer of at least
 * cr_workspace_bytes() bytes owned by the caller, aligned to 256 bytes, or
 * NULL to let the library allocate it.  The state is undefined until
 * cr_set_state.  Errors: CR_E_INVALID_ARG, CR_E_UNSUPPORTED, CR_E_NOMEM,
 * CR_E_CUDA; *out is NULL on error. */
cr_status cr_init_mesh(const cr_mesh_desc* desc, void* workspace, size_t workspace_bytes,
                       cr_ctx** out);

/* Release the context (and the workspace if the library allocated it). */
void cr_destroy(cr_ctx* ctx);

/* Copy the state u[M][Ne][Np] (FP64) in, reset time to 0, and compute the
 * first time step (eq. (time.step.2d)) and the indicator.  Synchronises.
 * on_device == 0: u is host memory (pageable or pinned); on_device == 1: a
 * device pointer.  In FP64, pinned host input is read by the kernel that
 * checks it (over the host link, the transfer overlapping the check, the
 * indicator and the CFL rate); other input is copied first.  The input is
 * checked on the device.  Errors: CR_E_INVALID_STATE when a solution point is
 * not finite or (for equations with an admissible set, Sec. 2 eq. (uad.form))
 * not admissible. */
cr_status cr_set_state(cr_ctx* ctx, const double* u, int on_device);

/* Copy the current state out as u[M][Ne][Np] (FP64); synchronises when
 * on_device == 0 (host memory as for cr_set_state).  In CR_FP32_BULK mode
 * values are mean + FP32 fluctuation. */
cr_status cr_get_state(cr_ctx* ctx, double* u, int on_device);

/* Advance up to max_steps cRKFR steps (Sec. 3 eq. (crkfr.avg), blended by
 * eq. (blended.scheme), with source eq. (crkfr.source)).  dt comes from eq.
 * (time.step.2d) on the current element means, or is dt_fixed when
 * dt_fixed > 0; the last step is shortened to land exactly on t_final.
 * Synchronises and returns the time reached and the number of steps taken
 * (either pointer may be NULL).  Steps are enqueued in growing chunks and
 * launching stops once t_final is reached, so max_steps may be generous.
 * Errors: CR_E_INADMISSIBLE (the step that failed is counted; the state is
 * the failed step's output). */
cr_status cr_step(cr_ctx* ctx, int max_steps, double t_final, double dt_fixed, double* t_out,
                  int* steps_out);

/* cr_step followed by cr_get_state(ctx, u, 0), for host memory u.  When u is
 * page-locked (pinned) host memory the update kernel of the last step writes
 * the new FP64 state into it while it runs, so the device->host transfer
 * overlaps that kernel instead of following the steps; otherwise, and when the
 * run reaches t_final before its last step, the state is copied after the
 * steps.  Synchronises.  Arguments and errors as cr_step; on an error the
 * contents of u are unspecified. */
cr_status cr_step_get(cr_ctx* ctx, int max_steps, double t_final, double dt_fixed, double* u,
                      double* t_out, int* steps_out);

/* As cr_step but only enqueues the work on the stream; cr_sync reports. */
cr_status cr_step_async(cr_ctx* ctx, int max_steps, double t_final, double dt_fixed);

/* Wait for the context's stream and report time, steps and the step status. */
cr_status cr_sync(cr_ctx* ctx, double* t_out, int* steps_out);

/* alpha_e (after neighbour smoothing) used by the most recent step, [Ne]
 * FP64.  Synchronises when on_device == 0. */
cr_status cr_get_alpha(cr_ctx* ctx, double* alpha, int on_device);

/* Learned blending coefficient (not in the paper: a small network replaces
 * the last step of the smoothness indicator, Sec. 4).  Inputs: the element's
 * normalised modal energies e_k = m_k^2 / sum m^2 of the indicator variable,
 * k = i + (N+1) j (Np of them), encoded x_k = log10(e_k + 1e-10)/10 + 1;
 * two hidden layers of 32 ReLU units and a sigmoid output, clipped like the
 * indicator (< 1e-3 -> 0, > 1 - 1e-3 -> 1) and then smoothed as usual.
 * Parameter vector (FP32): W1[32][Np], b1[32], W2[32][32], b2[32], w3[32], b3.
 * cr_mlp_param_count(Np) gives its length (-1 if Np is not 2,3,4,5,9,16,25). */
int cr_mlp_param_count(int nin);

/* Load network parameters into a context (stored as BF16, evaluated in FP32).
 * Used when desc.alpha_mode == CR_ALPHA_MLP.  Synchronises.
 * Errors: CR_E_INVALID_ARG (wrong count, NaN). */
cr_status cr_mlp_load(cr_ctx* ctx, const float* params, int nparams);

/* Network inputs x[Ne][Np] (FP32) of the current state and the raw alpha
 * [Ne] (before neighbour smoothing) under the context's alpha mode; either
 * pointer may be NULL.  Synchronises when on_device == 0. */
cr_status cr_get_features(cr_ctx* ctx, float* features, double* alpha_raw, int on_device);

/* Cross-entropy loss -mean(t log y + (1 - t) log(1 - y)) of the network on
 * samples X[n][nin] with targets t[n] in [0, 1] (the indicator's alpha taken
 * as a probability) and its gradient (same layout as the parameters), on the
 * GPU.  All pointers are device pointers; grad and loss are overwritten.
 * Per-block partial sums are added in a fixed order, so the result is the
 * same on every run.  Ordered on stream; takes a small stream-ordered scratch
 * allocation (cudaMallocAsync) for the partial sums. */
cr_status cr_mlp_grad(int nin, const float* params, const float* X, const float* t, int n,
                      float* grad, float* loss, void* stream);

/* Train the network in place (params: device pointer) with Adam (beta 0.9,
 * 0.999, eps 1e-8, learning rate lr) on minibatches of size batch from a
 * seeded shuffle of X[n][nin], t[n] (device), for the given number of epochs.
 * epoch_loss (host, may be NULL) receives the mean loss of the last epoch.
 * Deterministic: the same inputs and seed give the same parameters.
 * Allocates its own device scratch; synchronises stream. */
cr_status cr_mlp_train(int nin, float* params, const float* X, const float* t, int n, int batch,
                       int epochs, float lr, unsigned long long seed, float* epoch_loss,
                       void* stream);

/* Element means u_bar_e = sum_k W_k u_{e,k} (Sec. 3.2 eq. (upmean)), FP64
 * [M][Ne].  In CR_FP32_BULK mode these are the FP64 means the scheme updates
 * conservatively; totals sum_e u_bar_e dx dy are conserved to FP64 round-off
 * on periodic meshes without source.  Synchronises when on_device == 0. */
cr_status cr_get_means(cr_ctx* ctx, double* means, int on_device);

/* Time step the next cr_step would take without t_final clipping. Synchronises. */
cr_status cr_next_dt(cr_ctx* ctx, double* dt);

/* Number of kernel launches one step enqueues. */
cr_status cr_launches_per_step(cr_ctx* ctx, int* launches);

/* As cr_step_async, but launches every kernel of every step directly (no CUDA
 * graph) between CUDA events on the context's stream and adds each kernel's
 * device time in milliseconds to kernel_ms[i], i < cr_launches_per_step()
 * (in launch order: element-local kernel, face kernel, update kernel, and the
 * one-thread kernel that ends the step: time, rate, next step size).
 * Synchronises.  For measurement; the state advances exactly as in cr_step. */
cr_status cr_profile_steps(cr_ctx* ctx, int max_steps, double t_final, double dt_fixed,
                           double* kernel_ms);

/* CFL(N) of eq. (time.step.2d) from the library's Fourier analysis of the
 * D2 scheme for linear advection (host only, no device needed). */
cr_status cr_cfl_number(int degree, double* cfl);

/* CFL(N) for a dissipation model (CR_DISS_*): the same Fourier analysis of
 * the linear scheme with D1's dissipation for CR_DISS_D1; D2 and D-CSX share
 * one value.  Host only.  Errors: CR_E_INVALID_ARG. */
cr_status cr_cfl_number_for(int degree, int dissipation, double* cfl);

/* Reference-element tables the kernels use (host only): Gauss-Legendre nodes
 * xi[N+1] and weights w[N+1] on [0,1], and D[(N+1)*(N+1)], D_ij = l_j'(xi_i)
 * (Sec. 2 eq. (diff.matrix)).  Any pointer may be NULL. */
cr_status cr_reference_tables(int degree, double* xi, double* w, double* D);

/* CFL(N) for a dissipation model and a point set (CR_POINTS_*): the same
 * Fourier analysis with the tables of that point set.  Host only.
 * Errors: CR_E_INVALID_ARG. */
cr_status cr_cfl_number_points(int degree, int dissipation, int points, double* cfl);

/* cr_reference_tables for a point set (CR_POINTS_*): Gauss-Legendre, or
 * Gauss-Lobatto-Legendre nodes (end points included) with their weights.
 * Host only.  Errors: CR_E_INVALID_ARG. */
cr_status cr_reference_tables_points(int degree, int points, double* xi, double* w, double* D);

/* One FP64 step that allocates nothing (the paper has no counterpart; this is
 * a service for callers that may not allocate device memory, e.g. a host
 * whose device memory all belongs to another allocator, or code that must not
 * pay cudaMalloc's implicit synchronisation, or that forbids allocation once
 * running).  u_out = the state after one step of size dt from u_in, for the
 * mesh in desc; the limiters, indicator and source follow desc exactly as in
 * cr_step (desc->cfl is not used, desc->precision must be CR_FP64).
 * u_in and u_out are device pointers [M][Ne][Np] owned by the caller; they
 * may be equal.  The work is ordered on desc->stream and the call
 * synchronises that stream.
 * Scratch: one 16 MiB device array inside the library, reserved on every GPU
 * that loads it until the process exits; a mesh whose scratch does not fit
 * returns CR_E_TOO_LARGE (2D Euler N=4: up to about 4,000 elements).  The
 * first call on a device, with that device current, looks up the array's
 * device address and configures the kernels; make that first call before any
 * stream capture.  Every call reuses the same array (it is re-initialised at
 * the start of each call), so calls whose work overlaps on the GPU race.
 * Errors: CR_E_INVALID_ARG (bad desc, NULL pointer, dt <= 0),
 * CR_E_UNSUPPORTED, CR_E_TOO_LARGE, CR_E_INVALID_STATE (inadmissible input),
 * CR_E_INADMISSIBLE, CR_E_CUDA; cr_last_error(NULL) returns the failure's
 * message. */
cr_status cr_step_static(const cr_mesh_desc* desc, const double* u_in, double* u_out, double dt);

/* Last error message of ctx (or, when ctx is NULL, of the last failed call
 * without a context: cr_init_mesh, cr_workspace_bytes or cr_step_static). */
const char* cr_last_error(const cr_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Batches: many independent problems advanced together.  The paper treats one
 * problem at a time; a batch runs the same step (Sec. 3 eq. (crkfr.avg) with
 * the limiters of Sec. 4 and the time step of eq. (time.step.2d), each problem
 * with its own dt) for every problem of a set of contexts, in one launch per
 * phase or in one persistent launch, so many small meshes fill the GPU.  A
 * batched step computes exactly what cr_step computes on each context.
 * Supported: 2D Euler without a source on Gauss-Legendre points, degree 3 or 4
 * (mixed in one batch), all contexts in the same precision.  The contexts keep their state and remain usable with
 * cr_set_state / cr_get_state / cr_get_alpha / cr_mlp_load. */
typedef struct cr_batch cr_batch;
enum {
  CR_BATCH_PHASES = 0, /* three launches per step (local, face, update) over all problems */
  CR_BATCH_FUSED = 1   /* one cooperative persistent launch for all phases of up to 8 steps:
                          blocks claim work items (step, phase, tile) from one queue, and an
                          item waits (bounded) only for the work of its own problem it reads */
};
/* Number of configurations the autotuner tries. */
#define CR_BATCH_CANDIDATES 8

/* Group n contexts (pointers owned by the caller; they must outlive the
 * batch).  Allocates the batch's small device tables (parameters, tiles).
 * Default configuration: 256 threads per block, CR_BATCH_FUSED, 1 tile per
 * block.  Synchronises
 * the contexts' streams.  Errors: CR_E_INVALID_ARG, CR_E_UNSUPPORTED,
 * CR_E_NOMEM, CR_E_CUDA. */
cr_status cr_batch_init(cr_ctx* const* ctxs, int n, cr_batch** out);
void cr_batch_destroy(cr_batch* batch);

/* Threads per block (128 or 256: elements per block and tile = threads /
 * (N+1)^2), mode (CR_BATCH_PHASES or CR_BATCH_FUSED) and tiles (1, 2 or 4):
 * in FUSED a block takes 8 x tiles consecutive tiles from the queue per claim
 * (so a CTA works through 8 x tiles x threads / (N+1)^2 elements between
 * claims); PHASES runs one tile per block and ignores it.  Errors:
 * CR_E_INVALID_ARG for other values. */
cr_status cr_batch_config(cr_batch* batch, int threads, int mode, int tiles);

/* Autotuner: times one step of each (threads, mode, tiles) candidate in
 * turn, for trial_steps rounds after one warm-up round, on the batch's own
 * problems (CUDA events), and keeps the candidate with the fastest step.  The
 * problems advance by CR_BATCH_CANDIDATES * (trial_steps + 1) steps: tune
 * before setting the state of the real run.  ms_per_step (host, may be NULL)
 * receives CR_BATCH_CANDIDATES values, each candidate's fastest step, in the
 * order (128, PHASES), (128, FUSED, 1), (128, FUSED, 2), (128, FUSED, 4), then
 * the same four with 256 threads.  threads, mode and tiles (may be NULL)
 * receive the choice. */
cr_status cr_batch_autotune(cr_batch* batch, int trial_steps, int* threads, int* mode, int* tiles,
                            double* ms_per_step);

/* Advance every problem by up to nsteps steps (each stops at t_final, the
 * last step clipped to land on it).  Ordered after work already queued on the
 * contexts' streams; enqueued on the first context's stream.  Call
 * cr_batch_sync before using a context on its own again. */
cr_status cr_batch_step_async(cr_batch* batch, int nsteps, double t_final);
/* Wait for the batch; CR_E_TIMEOUT if a wait of the fused kernel gave up
 * (its blocks then returned early), CR_E_INADMISSIBLE naming the first
 * problem whose step produced an inadmissible state. */
cr_status cr_batch_sync(cr_batch* batch);
/* cr_batch_step_async followed by cr_batch_sync. */
cr_status cr_batch_step(cr_batch* batch, int nsteps, double t_final);
const char* cr_batch_last_error(const cr_batch* batch);

/* Fault injection for tests of the fused kernel's timeout path (no
 * counterpart in the paper).  Sets the budget of the fused kernel's waits to
 * `polls` polls of at least 64 ns each (0 restores the default, 2^26, at
 * least 4 s) and makes every wait require `phantom` further completed tiles
 * that never come.  With phantom > 0 the first wait runs out after its budget,
 * that block sets the batch's error flag and returns, and every other block
 * stops at its next claim or wait; no block traps or hangs.  The next
 * cr_batch_sync then returns CR_E_TIMEOUT and clears the flag; the problems'
 * states are undefined until they are set again.  No effect in
 * CR_BATCH_PHASES mode (no waits). */
cr_status cr_batch_barrier_test(cr_batch* batch, unsigned long long polls, int phantom);

#ifdef __cplusplus
}
#endif
#endif
