"""FP64 CPU oracle for the cRKFR time step (Babbar & Chen, arXiv 2502.07517).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this package; the CUDA library never does, and
this package never imports the CUDA library.

The C sources (or_tables.c, or_physics.c, or_step.c) hold the scheme; this
module only marshals arguments.  The CFL number CFL(N) of Sec. 5 comes from
the Fourier analysis in ``oracle.cfl``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

EQ_LINADV, EQ_EULER, EQ_TENMOMENT, EQ_BURGERS, EQ_VARADV = 0, 1, 2, 3, 4
BC_PERIODIC, BC_OUTFLOW, BC_WALL, BC_DIRICHLET, BC_INFLOW = 0, 1, 2, 3, 4
SRC_NONE, SRC_TENMOMENT, SRC_GRAVITY = 0, 1, 2
LIM_BLEND, LIM_MH, LIM_FLUX, LIM_SCALING, LIM_TRACES = 1, 2, 4, 8, 16
LIM_ALL = LIM_BLEND | LIM_MH | LIM_FLUX | LIM_SCALING | LIM_TRACES
ALPHA_INDICATOR, ALPHA_FIXED, ALPHA_GIVEN = 0, 1, 2
DISS_D2, DISS_D1, DISS_DCSX = 0, 1, 2
CENTRAL_EA, CENTRAL_AE = 0, 1
POINTS_GL, POINTS_GLL = 0, 1


class Desc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
        ("degree", ctypes.c_int), ("equation", ctypes.c_int),
        ("gamma", ctypes.c_double), ("adv", ctypes.c_double * 2),
        ("source", ctypes.c_int),
        ("src_amp", ctypes.c_double), ("src_k", ctypes.c_double),
        ("src_cx", ctypes.c_double), ("src_cy", ctypes.c_double),
        ("limiter", ctypes.c_int), ("alpha_mode", ctypes.c_int),
        ("alpha_fixed", ctypes.c_double),
        ("cfl", ctypes.c_double), ("cfl_safety", ctypes.c_double),
        ("alpha_given", ctypes.POINTER(ctypes.c_double)),
        ("dissipation", ctypes.c_int), ("central", ctypes.c_int),
        ("bc_side", ctypes.c_int * 4), ("bc_state", (ctypes.c_double * 6) * 4),
        ("gravity", ctypes.c_double * 2), ("points", ctypes.c_int),
        ("adv_poly", ctypes.c_double * 4), ("bc_time_terms", ctypes.c_int),
        ("bc_time_span", ctypes.c_double * 2), ("bc_time_coef", (ctypes.c_double * 16) * 4),
        ("time", ctypes.c_double), ("bc_flux", ctypes.c_int),
    ]


class Diag(ctypes.Structure):
    _fields_ = [(name, ctypes.POINTER(ctypes.c_double)) for name in (
        "alpha", "alpha_raw", "fnum_x", "fnum_x_right", "fnum_y", "fnum_y_top",
        "theta_x", "theta_y", "source_mean")] + [
        ("status", ctypes.c_int), ("bad_element", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        D = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(Desc)
        _lib.or_tables.argtypes = [ctypes.c_int, D, D, D, D, D]
        _lib.or_tables_pts.argtypes = [ctypes.c_int, ctypes.c_int, D, D, D, D, D, D, D]
        _lib.or_tableau.argtypes = [ctypes.c_int, D, D, D]
        _lib.or_tableau.restype = ctypes.c_int
        _lib.or_nvars.argtypes = [P]
        _lib.or_nodes.argtypes = [P]
        _lib.or_flux.argtypes = [P, D, ctypes.c_int, D]
        _lib.or_wave_speed.argtypes = [P, D, ctypes.c_int]
        _lib.or_wave_speed.restype = ctypes.c_double
        _lib.or_flux_x.argtypes = [P, D, ctypes.c_double, ctypes.c_int, D]
        _lib.or_wave_speed_x.argtypes = [P, D, ctypes.c_double, ctypes.c_int]
        _lib.or_wave_speed_x.restype = ctypes.c_double
        _lib.or_num_constraints.argtypes = [P]
        _lib.or_constraint.argtypes = [P, D, ctypes.c_int]
        _lib.or_constraint.restype = ctypes.c_double
        _lib.or_source.argtypes = [P, D, ctypes.c_double, ctypes.c_double, D]
        _lib.or_local_crk.argtypes = [P, D, ctypes.c_double, ctypes.c_int, ctypes.c_int, D, D, D, D]
        _lib.or_indicator.argtypes = [P, D]
        _lib.or_indicator.restype = ctypes.c_double
        _lib.or_modal_energies.argtypes = [P, D, D]
        _lib.or_modal_energies.restype = None
        _lib.or_max_rate.argtypes = [P, D]
        _lib.or_max_rate.restype = ctypes.c_double
        _lib.or_dt.argtypes = [P, D]
        _lib.or_dt.restype = ctypes.c_double
        _lib.or_step.argtypes = [P, D, ctypes.c_double, D, ctypes.POINTER(Diag)]
        _lib.or_step.restype = ctypes.c_int
        _lib.or_run.argtypes = [P, D, ctypes.c_int, ctypes.c_double,
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
        _lib.or_run.restype = ctypes.c_int
        _lib.or_scaling_limiter.argtypes = [P, D]
        _lib.or_scaling_limiter.restype = ctypes.c_int
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_desc(dim=1, nx=16, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc_x=BC_PERIODIC,
              bc_y=BC_PERIODIC, degree=3, equation=EQ_LINADV, gamma=1.4, adv=(1.0, 0.0),
              source=0, src_amp=0.0, src_k=0.0, src_cx=0.5, src_cy=0.5, limiter=0,
              alpha_mode=ALPHA_INDICATOR, alpha_fixed=0.0, cfl=None, cfl_safety=0.98,
              alpha_given=None, dissipation=DISS_D2, central=CENTRAL_EA, bc_side=(0, 0, 0, 0),
              bc_state=None, gravity=(0.0, 0.0), points=POINTS_GL, adv_poly=(0.0, 0.0, 0.0, 0.0),
              bc_time=None, bc_flux=0):
    """Mesh/scheme description; cfl defaults to CFL(degree) from the Fourier analysis.
    alpha_given: per-element raw alpha array for alpha_mode ALPHA_GIVEN (kept alive on
    the returned object)."""
    if cfl is None:
        from .cfl import cfl_number
        cfl = cfl_number(degree, dissipation == DISS_D1, points=points)
    d = Desc()
    d.dim, d.nx, d.ny = dim, nx, (ny if dim == 2 else 1)
    d.x0, d.x1, d.y0, d.y1 = x0, x1, y0, y1
    d.bc_x, d.bc_y = bc_x, bc_y
    d.degree, d.equation, d.gamma = degree, equation, gamma
    d.adv[0], d.adv[1] = adv
    d.source, d.src_amp, d.src_k, d.src_cx, d.src_cy = source, src_amp, src_k, src_cx, src_cy
    d.limiter, d.alpha_mode, d.alpha_fixed = limiter, alpha_mode, alpha_fixed
    d.cfl, d.cfl_safety = cfl, cfl_safety
    d.dissipation, d.central = dissipation, central
    for s in range(4):
        d.bc_side[s] = bc_side[s]
        if bc_state is not None and bc_state[s] is not None:
            for v, x in enumerate(bc_state[s]):
                d.bc_state[s][v] = x
    d.gravity[0], d.gravity[1] = gravity
    d.points = points
    d.bc_flux = bc_flux
    for k in range(4):
        d.adv_poly[k] = adv_poly[k]
    if bc_time is not None:                  # (span, {side index: Chebyshev coefficients})
        span, coefs = bc_time
        d.bc_time_span[0], d.bc_time_span[1] = span
        d.bc_time_terms = max(len(c) for c in coefs.values())
        for s, c in coefs.items():
            for k, a in enumerate(c):
                d.bc_time_coef[s][k] = a
    if alpha_given is not None:
        arr = np.ascontiguousarray(alpha_given, dtype=np.float64)
        d._alpha_given_keep = arr
        d.alpha_given = _ptr(arr)
        d.alpha_mode = ALPHA_GIVEN
    return d


def nvars(d):
    return lib().or_nvars(ctypes.byref(d))


def nodes(d):
    return lib().or_nodes(ctypes.byref(d))


def nelem(d):
    return d.nx * (d.ny if d.dim == 2 else 1)


def state_shape(d):
    return (nvars(d), nelem(d), nodes(d))


def tables(N, points=POINTS_GL):
    """(xi, w, l0, l1, D) of the point set on [0,1]."""
    return tables_corr(N, points)[:5]


def tables_corr(N, points=POINTS_GL):
    """(xi, w, l0, l1, D, gL, gR): the tables with the correction derivatives
    g_L'(xi_p), g_R'(xi_p) (Radau for Gauss-Legendre, g2 for Gauss-Lobatto)."""
    n = N + 1
    xi, w, l0, l1, gL, gR = (np.zeros(n) for _ in range(6))
    D = np.zeros((n, n))
    lib().or_tables_pts(N, points, _ptr(xi), _ptr(w), _ptr(l0), _ptr(l1), _ptr(D), _ptr(gL), _ptr(gR))
    return xi, w, l0, l1, D, gL, gR


def tableau(N):
    A = np.zeros((6, 6))
    b = np.zeros(6)
    c = np.zeros(6)
    s = lib().or_tableau(N, _ptr(A), _ptr(b), _ptr(c))
    return A[:s, :s].copy(), b[:s].copy(), c[:s].copy()


def flux(d, u, direction):
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = np.zeros(nvars(d))
    lib().or_flux(ctypes.byref(d), _ptr(u), direction, _ptr(f))
    return f


def wave_speed(d, u, direction):
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().or_wave_speed(ctypes.byref(d), _ptr(u), direction)


def flux_x(d, u, x, direction):
    """Flux at position x (variable advection depends on it)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = np.zeros(nvars(d))
    lib().or_flux_x(ctypes.byref(d), _ptr(u), float(x), direction, _ptr(f))
    return f


def wave_speed_x(d, u, x, direction):
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().or_wave_speed_x(ctypes.byref(d), _ptr(u), float(x), direction)


def constraint(d, u, k):
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().or_constraint(ctypes.byref(d), _ptr(u), k)


def num_constraints(d):
    return lib().or_num_constraints(ctypes.byref(d))


def source(d, u, x, y):
    u = np.ascontiguousarray(u, dtype=np.float64)
    s = np.zeros(nvars(d))
    lib().or_source(ctypes.byref(d), _ptr(u), x, y, _ptr(s))
    return s


def local_crk(d, ue, dt, ix=0, iy=0):
    """Time-averaged F, G, U, S of one element; ue is [Np][M]."""
    ue = np.ascontiguousarray(ue, dtype=np.float64)
    F, G, U, S = (np.zeros_like(ue) for _ in range(4))
    lib().or_local_crk(ctypes.byref(d), _ptr(ue), dt, ix, iy, _ptr(F), _ptr(G), _ptr(U), _ptr(S))
    return F, G, U, S


def indicator(d, ue):
    ue = np.ascontiguousarray(ue, dtype=np.float64)
    return lib().or_indicator(ctypes.byref(d), _ptr(ue))


def modal_energies(d, ue):
    """Normalised modal energies of one element's indicator variable; ue [Np][M]."""
    ue = np.ascontiguousarray(ue, dtype=np.float64)
    e = np.zeros(nodes(d))
    lib().or_modal_energies(ctypes.byref(d), _ptr(ue), _ptr(e))
    return e


def max_rate(d, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().or_max_rate(ctypes.byref(d), _ptr(u))


def dt(d, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().or_dt(ctypes.byref(d), _ptr(u))


def step(d, u, dt_, want_diag=False, time=None):
    """One step from time t^n = time (default: d.time); returns (u_new, status)
    or (u_new, status, diag dict)."""
    if time is not None:
        d.time = time
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    M, ne, npn = state_shape(d)
    n = d.degree + 1
    nq = n if d.dim == 2 else 1
    diag = Diag()
    arrays = {}
    if want_diag:
        arrays = {
            "alpha": np.zeros(ne), "alpha_raw": np.zeros(ne),
            "fnum_x": np.zeros((M, ne, nq)), "fnum_x_right": np.zeros((M, ne, nq)),
            "fnum_y": np.zeros((M, ne, n)), "fnum_y_top": np.zeros((M, ne, n)),
            "theta_x": np.zeros((ne, nq)), "theta_y": np.zeros((ne, n)),
            "source_mean": np.zeros((M, ne)),
        }
        for k, a in arrays.items():
            setattr(diag, k, _ptr(a))
    st = lib().or_step(ctypes.byref(d), _ptr(u), float(dt_), _ptr(out), ctypes.byref(diag))
    if want_diag:
        arrays["bad_element"] = diag.bad_element
        return out, st, arrays
    return out, st


def run(d, u, max_steps, t_final):
    """CFL time stepping to t_final (last step clipped); returns (u, t, steps, status)."""
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    t = ctypes.c_double(0.0)
    n = ctypes.c_int(0)
    st = lib().or_run(ctypes.byref(d), _ptr(u), int(max_steps), float(t_final),
                      ctypes.byref(t), ctypes.byref(n))
    return u, t.value, n.value, st


def scaling_limiter(d, ue):
    ue = np.array(ue, dtype=np.float64, order="C", copy=True)
    st = lib().or_scaling_limiter(ctypes.byref(d), _ptr(ue))
    return ue, st


def node_coords(d):
    """Physical coordinates (x, y) of every solution point, arrays [Ne][Np]."""
    xi = tables(d.degree, d.points)[0]
    n = d.degree + 1
    ne = nelem(d)
    dx = (d.x1 - d.x0) / d.nx
    ix = np.arange(ne) % d.nx
    if d.dim == 1:
        x = d.x0 + (ix[:, None] + xi[None, :]) * dx
        return x, np.zeros_like(x)
    dy = (d.y1 - d.y0) / d.ny
    iy = np.arange(ne) // d.nx
    p = np.tile(np.arange(n), n)
    q = np.repeat(np.arange(n), n)
    x = d.x0 + (ix[:, None] + xi[p][None, :]) * dx
    y = d.y0 + (iy[:, None] + xi[q][None, :]) * dy
    return x, y


def element_means(d, u):
    """Element means sum_k W_k u_k, array [M][Ne]."""
    w = tables(d.degree, d.points)[1]
    n = d.degree + 1
    W = w if d.dim == 1 else np.array([w[k % n] * w[k // n] for k in range(n * n)])
    return np.einsum("vek,k->ve", u, W)
