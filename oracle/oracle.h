/*
 * Plain FP64 CPU oracle for one time step of compact Runge-Kutta Flux
 * Reconstruction (cRKFR) with the subcell blending limiter, the flux limiter
 * and the positivity scaling limiter (Babbar & Chen, arXiv 2502.07517).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or constant generator with
 * the CUDA path, and it never reads anything the CUDA path produced.
 *
 * Every function follows one passage of the paper in the paper's order and
 * notation, with straightforward loops (per element, per stage, per node) and
 * no blocking, fusion or reordering.  Where the paper defers a detail to
 * another paper, the reading taken is stated beside the code.
 *
 * Pins (tests/test_oracle_pins.py, tests/test_oracle_mlp.py): closed forms,
 * exact solutions, invariants and brute force for every step of the scheme.
 * The smoothness indicator (or_indicator) follows a method the paper cites
 * without printing it (Sec. 4); its constants are readings of the cited
 * method.  It is pinned (tests/test_oracle_indicator.py) by elements made of
 * chosen Legendre modes, whose energy ratio is known in closed form and set to
 * the threshold and 5% either side of it, through the top ratio, the
 * next-to-top ratio or both, in 1D and 2D for N = 2, 3, 4; and by special
 * cases (constant and linear data give 0, a jump gives 1).  or_indicator and
 * or_modal_energies compute their modes with the same routine.
 *
 * Layout of a state vector: u[(v * Ne + e) * Np + k], variable v, element
 * e = ix + nx * iy, node k = p + (N + 1) * q (p along x, q along y).
 */
#ifndef CRKFR_ORACLE_H
#define CRKFR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAXN 4
#define OR_MAXS 6
#define OR_MAXM 6

/* Burgers: 1D only, f(u) = u^2/2 (Sec. 5.1, Burgers' equation).  Variable
 * advection: 1D only, f(x, u) = a(x) u with a(x) = sum_k adv_poly[k] x^k
 * (Sec. 5.1, variable advection equation). */
enum { OR_EQ_LINADV = 0, OR_EQ_EULER = 1, OR_EQ_TENMOMENT = 2, OR_EQ_BURGERS = 3, OR_EQ_VARADV = 4 };
/* Boundary conditions of Sec. 3.3: periodic; outflow (F = F^+, the fully
 * outflow rule); solid wall for the Euler equations (ghost values by
 * reflecting the normal velocity, eq. (reflect.time.avg)); a given ghost
 * state g (inflow/outflow: ghost values u^- = U^- = g, F^- = f(g), then the
 * scheme's own numerical flux); fully inflow (F = F^- = f(g)). */
enum { OR_BC_PERIODIC = 0, OR_BC_OUTFLOW = 1, OR_BC_WALL = 2, OR_BC_DIRICHLET = 3, OR_BC_INFLOW = 4 };
/* Source terms: ten-moment Gaussian potential (Sec. 5.4), Euler gravity (Sec. 5.5). */
enum { OR_SRC_NONE = 0, OR_SRC_TENMOMENT = 1, OR_SRC_GRAVITY = 2 };
enum {
  OR_LIM_BLEND = 1,    /* blend with the subcell scheme, Sec. 4 eq. (blended.scheme) */
  OR_LIM_MH = 2,       /* MUSCL-Hancock subcell fluxes (else first order), Sec. 4.2 */
  OR_LIM_FLUX = 4,     /* flux limiter for admissible means, Sec. 4.3 */
  OR_LIM_SCALING = 8,  /* Zhang-Shu positivity scaling, Sec. 3.2 */
  OR_LIM_TRACES = 16   /* scaling limiter also enforces admissibility at face traces */
};
enum { OR_ALPHA_INDICATOR = 0, OR_ALPHA_FIXED = 1, OR_ALPHA_GIVEN = 2 };
/* D2 eq. (D2) (time-averaged solution traces), D1 eq. (D1) (u^n traces),
 * D-CSX eq. (dcsx) (stage traces with a wave speed per stage) */
enum { OR_DISS_D2 = 0, OR_DISS_D1 = 1, OR_DISS_DCSX = 2 };
/* EA eq. (evaluate) (stage fluxes at the face), AE eq. (extrapolate) (trace of
 * the time-averaged flux) */
enum { OR_CENTRAL_EA = 0, OR_CENTRAL_AE = 1 };
/* Solution points and correction: Gauss-Legendre with Radau (Sec. 2, the
 * default), Gauss-Lobatto-Legendre with g2 (Sec. 5.1). */
enum { OR_POINTS_GL = 0, OR_POINTS_GLL = 1 };

typedef struct {
  int dim;                 /* 1 or 2 */
  int nx, ny;              /* elements per direction (ny = 1 in 1D) */
  double x0, x1, y0, y1;   /* domain */
  int bc_x, bc_y;          /* OR_BC_* */
  int degree;              /* N in 1..4 */
  int equation;            /* OR_EQ_* */
  double gamma;            /* Euler */
  double adv[2];           /* linear advection velocity */
  int source;              /* OR_SRC_* */
  double src_amp, src_k, src_cx, src_cy;
  int limiter;             /* OR_LIM_* bits */
  int alpha_mode;          /* OR_ALPHA_* */
  double alpha_fixed;      /* alpha_e when alpha_mode == OR_ALPHA_FIXED */
  double cfl;              /* CFL(N) of Sec. 5 eq. (time.step.2d) */
  double cfl_safety;       /* C_s */
  const double* alpha_given; /* [Ne] raw alpha_e (before smoothing) when alpha_mode == OR_ALPHA_GIVEN */
  int dissipation;         /* OR_DISS_*: dissipative part of eq. (numflux.general), Sec. 3.1.1 */
  int central;             /* OR_CENTRAL_*: central part F^{+-}, Sec. 3.1.2 */
  int bc_side[4];          /* per side (x-, x+, y-, y+): 0 = bc_x / bc_y, else OR_BC_* (not periodic) */
  double bc_state[4][OR_MAXM]; /* ghost state g of each side (conservative), OR_BC_DIRICHLET / OR_BC_INFLOW */
  double gravity[2];       /* acceleration (g_x, g_y) of OR_SRC_GRAVITY */
  int points;              /* OR_POINTS_*; GLL supports no MUSCL-Hancock subcells */
  double adv_poly[4];      /* a(x) of OR_EQ_VARADV */
  /* time-dependent ghost states of Dirichlet / inflow sides (scalar equations):
   * when bc_time_terms > 0, g(t) = sum_{k < terms} bc_time_coef[side][k] T_k(tau),
   * tau = 2 (t - t0) / (t1 - t0) - 1 clamped to [-1, 1], (t0, t1) = bc_time_span */
  int bc_time_terms;
  double bc_time_span[2];
  double bc_time_coef[4][16];
  double time;             /* t^n of or_step (or_run advances it in its own copy) */
  int bc_flux;             /* flux at Dirichlet sides: 0 the scheme's own, 1 HLLC (Euler) */
} or_desc;

/* Optional outputs of or_step; any pointer may be NULL. */
typedef struct {
  double* alpha;       /* [Ne] blending coefficient alpha_e after smoothing */
  double* alpha_raw;   /* [Ne] alpha_e straight from the indicator */
  double* fnum_x;      /* [M][Ne][nq] numerical flux on the LEFT x-face of each element */
  double* fnum_x_right;/* [M][Ne][nq] numerical flux on the RIGHT x-face of each element */
  double* fnum_y;      /* [M][Ne][n]  numerical flux on the BOTTOM y-face */
  double* fnum_y_top;  /* [M][Ne][n]  numerical flux on the TOP y-face */
  double* theta_x;     /* [Ne][nq] flux-limiter theta on the LEFT x-face */
  double* theta_y;     /* [Ne][n]  flux-limiter theta on the BOTTOM y-face */
  double* source_mean; /* [M][Ne] sum_k W_k S_k, the source part of the mean update */
  int status;          /* 0 ok, 1 inadmissible mean, 2 non-finite value */
  int bad_element;     /* first element that set status, -1 if none */
} or_diag;

int or_nvars(const or_desc* d);
int or_nodes(const or_desc* d);

/* Reference element tables of Sec. 2 on [0,1]: Gauss-Legendre nodes and
 * weights, l_p(0), l_p(1), and D_ij = l_j'(xi_i). */
void or_tables(int N, double* xi, double* w, double* l0, double* l1, double* D);
/* The tables of either point set, with the correction derivatives g_L', g_R'
 * at the solution points (Radau for Gauss-Legendre, g2 for Gauss-Lobatto). */
void or_tables_pts(int N, int points, double* xi, double* w, double* l0, double* l1, double* D,
                   double* gL, double* gR);
/* Butcher tableau used for degree N (cRK22/33/44, and the order-5 reading for N = 4). */
int or_tableau(int N, double* A /* [6][6] */, double* b, double* c);

/* Physics, exposed for the tests. dir 0 = x, 1 = y. */
void or_flux(const or_desc* d, const double* u, int dir, double* f);
/* The flux and wave speed at position x (variable advection depends on it;
 * the other equations ignore it). */
void or_flux_x(const or_desc* d, const double* u, double x, int dir, double* f);
double or_wave_speed_x(const or_desc* d, const double* u, double x, int dir);
double or_wave_speed(const or_desc* d, const double* u, int dir);
int or_num_constraints(const or_desc* d);
double or_constraint(const or_desc* d, const double* u, int k);
void or_source(const or_desc* d, const double* u, double x, double y, double* s);

/* Local cRK procedure of Sec. 3 for one element: time-averaged F, G, U, S at
 * the solution points, arrays [Np][M].  ue is [Np][M]. */
void or_local_crk(const or_desc* d, const double* ue, double dt, int ix, int iy,
                  double* F, double* G, double* U, double* S);

/* Smoothness indicator alpha of one element from its nodal values [Np][M]. */
double or_indicator(const or_desc* d, const double* ue);
/* Normalised modal energies e_k = m_k^2 / sum_j m_j^2 of the indicator variable
 * of one element (mode k = i + (N+1) j in 2D, k = i in 1D); all zero when the
 * sum is zero.  These are the inputs of the learned blending coefficient. */
void or_modal_energies(const or_desc* d, const double* ue, double* e);

/* max_e (sigma_x(mean_e)/dx + sigma_y(mean_e)/dy), Sec. 5 eq. (time.step.2d) */
double or_max_rate(const or_desc* d, const double* u);
double or_dt(const or_desc* d, const double* u);

/* One cRKFR step with the given dt. Returns diag->status (0 ok). */
int or_step(const or_desc* d, const double* u_in, double dt, double* u_out, or_diag* diag);

/* Steps with the CFL time step until t_final or max_steps; the last step is
 * clipped to land on t_final. u is updated in place. Returns the status. */
int or_run(const or_desc* d, double* u, int max_steps, double t_final, double* t_out,
           int* steps_out);

/* Zhang-Shu scaling limiter on one element, in place on ue [Np][M].
 * Returns 0 if the mean is admissible, 1 otherwise. */
int or_scaling_limiter(const or_desc* d, double* ue);

#ifdef __cplusplus
}
#endif
#endif
