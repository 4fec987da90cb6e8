"""Seeded synthetic initial states for the cRKFR workloads.

This module holds no part of the scheme: it only samples initial data at the
solution points (nodal interpolation) and describes each problem as a plain
dict.  Node positions come from numpy's Gauss-Legendre rule, so neither the
CUDA library nor the CPU checker is involved in making an input; both receive
the same arrays.

State layout: float64 array [M][Ne][Np], element e = ix + nx * iy, node
k = p + (N + 1) * q with p along x.

Problem dict keys: dim, nx, ny, x0, x1, y0, y1, bc_x, bc_y ("periodic",
"outflow" or "wall"), degree, equation ("linadv", "euler", "tenmoment",
"burgers"), gamma, adv,
source (None, dict amp, k, cx, cy for the ten-moment potential, or dict
gravity=(gx, gy) for Euler), limiter (set of "blend", "mh", "flux",
"scaling", "traces"), t_final, steps; optional bc_side (dict side -> bc name,
sides "x-", "x+", "y-", "y+", overriding bc_x / bc_y) and bc_state (dict side
-> conservative ghost state) for "dirichlet" and "inflow" sides; points
("gl", the default, or "gll" Gauss-Lobatto-Legendre).
"""
import math

import numpy as np

LIMITER_ALL = frozenset({"blend", "mh", "flux", "scaling", "traces"})


def gl_nodes01(N):
    x, w = np.polynomial.legendre.leggauss(N + 1)
    return 0.5 * (x + 1.0), 0.5 * w


def gll_nodes01(N):
    """Gauss-Lobatto-Legendre nodes and weights on [0,1] (numpy's Legendre
    class: the end points and the roots of P_N')."""
    PN = np.polynomial.legendre.Legendre.basis(N)
    inner = np.sort(PN.deriv().roots().real) if N > 1 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (N * (N + 1) * PN(x) ** 2)
    return 0.5 * (x + 1.0), 0.5 * w


def nodes01(prob):
    """Solution points and weights of the problem's point set ("gl" default, "gll")."""
    N = prob["degree"]
    return gll_nodes01(N) if prob.get("points", "gl") == "gll" else gl_nodes01(N)


def node_coords(prob):
    """(x, y) of every solution point, arrays [Ne][Np]."""
    N = prob["degree"]
    xi, _ = nodes01(prob)
    n = N + 1
    nx = prob["nx"]
    ny = prob["ny"] if prob["dim"] == 2 else 1
    dx = (prob["x1"] - prob["x0"]) / nx
    ix = np.arange(nx * ny) % nx
    if prob["dim"] == 1:
        x = prob["x0"] + (ix[:, None] + xi[None, :]) * dx
        return x, np.zeros_like(x)
    dy = (prob["y1"] - prob["y0"]) / ny
    iy = np.arange(nx * ny) // nx
    p = np.tile(np.arange(n), n)
    q = np.repeat(np.arange(n), n)
    x = prob["x0"] + (ix[:, None] + xi[p][None, :]) * dx
    y = prob["y0"] + (iy[:, None] + xi[q][None, :]) * dy
    return x, y


def element_centres(prob):
    nx = prob["nx"]
    ny = prob["ny"] if prob["dim"] == 2 else 1
    dx = (prob["x1"] - prob["x0"]) / nx
    ix = np.arange(nx * ny) % nx
    xc = prob["x0"] + (ix + 0.5) * dx
    if prob["dim"] == 1:
        return xc, np.zeros_like(xc)
    dy = (prob["y1"] - prob["y0"]) / ny
    iy = np.arange(nx * ny) // nx
    return xc, prob["y0"] + (iy + 0.5) * dy


def base_problem(**kw):
    prob = dict(dim=1, nx=16, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc_x="periodic",
                bc_y="periodic", degree=3, equation="linadv", gamma=1.4, adv=(1.0, 0.0),
                source=None, limiter=frozenset(), t_final=1.0, steps=None)
    prob.update(kw)
    if prob["dim"] == 1:
        prob["ny"] = 1
    return prob


def nvars(prob):
    return {"linadv": 1, "burgers": 1, "varadv": 1, "euler": 3 if prob["dim"] == 1 else 4,
            "tenmoment": 6}[prob["equation"]]


def euler_conservative(rho, v1, v2, p, gamma, dim):
    if dim == 1:
        return np.stack([rho, rho * v1, p / (gamma - 1.0) + 0.5 * rho * v1 * v1])
    E = p / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2)
    return np.stack([rho, rho * v1, rho * v2, E])


def tenmoment_conservative(rho, v1, v2, p11, p12, p22):
    return np.stack([rho, rho * v1, rho * v2, 0.5 * p11 + 0.5 * rho * v1 * v1,
                     0.5 * p12 + 0.5 * rho * v1 * v2, 0.5 * p22 + 0.5 * rho * v2 * v2])


# ---------------------------------------------------------------------------
def linadv_sine(nx=64, degree=3, t_final=1.0, a=1.0):
    """1D u_t + a u_x = 0 on [0,1] periodic, u0 = sin(2 pi x), no limiter."""
    prob = base_problem(dim=1, nx=nx, degree=degree, equation="linadv", adv=(a, 0.0),
                        t_final=t_final)
    x, _ = node_coords(prob)
    return prob, np.sin(2.0 * np.pi * x)[None, :, :].copy()


def burgers_sine(nx=64, degree=3, t_final=2.0, amp=0.2, points="gl"):
    """1D Burgers u_t + (u^2/2)_x = 0 on [0, 2 pi] periodic, u0 = amp sin(x)
    (Sec. 5.1): smooth until t = 1/amp = 5, no limiter; Gauss-Legendre or
    Gauss-Lobatto ("gll") solution points."""
    prob = base_problem(dim=1, nx=nx, degree=degree, equation="burgers", x0=0.0,
                        x1=2.0 * math.pi, t_final=t_final, points=points)
    prob["burgers_amp"] = amp
    x, _ = node_coords(prob)
    return prob, (amp * np.sin(x))[None, :, :].copy()


def varadv_exact(x, t):
    """Exact solution of u_t + (x^2 u)_x = 0 with u0 = cos(pi x / 2), by the
    characteristics x0 = x / (1 + t x): u = u0(x0) / (1 + t x)^2 (Sec. 5.1)."""
    s = 1.0 + t * x
    return np.cos(0.5 * math.pi * x / s) / (s * s)


def varadv_x2(nx=32, degree=3, t_final=1.0, terms=16):
    """Variable advection u_t + (a(x) u)_x = 0, a(x) = x^2, on [0.1, 1]
    (Sec. 5.1): u0 = cos(pi x / 2); inflow on the left with the exact solution
    as boundary data (a Chebyshev fit in t on [0, t_final] of u(0.1, t), numpy's
    chebinterpolate), outflow on the right; no limiter."""
    prob = base_problem(dim=1, nx=nx, degree=degree, equation="varadv", x0=0.1, x1=1.0,
                        bc_x="outflow", t_final=t_final, adv_poly=(0.0, 0.0, 1.0, 0.0))
    prob["bc_side"] = {"x-": "inflow"}
    tt = lambda tau: 0.5 * (tau + 1.0) * t_final
    coef = np.polynomial.chebyshev.chebinterpolate(lambda tau: varadv_exact(0.1, tt(tau)), terms - 1)
    prob["bc_time"] = {"span": (0.0, t_final), "coef": {"x-": [float(c) for c in coef]}}
    x, _ = node_coords(prob)
    return prob, np.cos(0.5 * math.pi * x)[None, :, :].copy()


def sedov1d(nx=201, degree=3, limiter=LIMITER_ALL, t_final=1e-3):
    """1D Sedov blast (Sec. 5.2): Euler (gamma 1.4) on [-1, 1] between solid
    walls, rho = 1, v = 0, total energy E = 3.2e6/dx in the centre element
    (|x| <= dx/2; nx odd) and 1e-12 elsewhere."""
    if nx % 2 == 0:
        raise ValueError("the 1D Sedov blast wants an odd element count")
    prob = base_problem(dim=1, nx=nx, degree=degree, equation="euler", x0=-1.0, x1=1.0,
                        bc_x="wall", limiter=frozenset(limiter), t_final=t_final)
    dx = 2.0 / nx
    x, _ = node_coords(prob)
    centre = (np.arange(nx) == nx // 2)[:, None]
    E = np.where(np.broadcast_to(centre, x.shape), 3.2e6 / dx, 1e-12)
    one = np.ones_like(x)
    return prob, np.stack([one, 0.0 * one, E])


def sedov2d_periodic(nx=64, degree=3, limiter=LIMITER_ALL, t_final=20.0):
    """2D periodic Sedov blast (Sec. 5.3): Euler (gamma 1.4) on [-1.5, 1.5]^2
    periodic, gas at rest, rho = rho0 + exp(-r^2/(2 s_rho^2))/(4 pi s_rho^2),
    p = p0 + (gamma - 1) exp(-r^2/(2 s_p^2))/(4 pi s_p^2), rho0 = 1, p0 = 1e-5,
    s_rho = 0.25, s_p = 0.15."""
    prob = base_problem(dim=2, nx=nx, ny=nx, degree=degree, equation="euler", x0=-1.5, x1=1.5,
                        y0=-1.5, y1=1.5, limiter=frozenset(limiter), t_final=t_final)
    g = prob["gamma"]
    x, y = node_coords(prob)
    r2 = x * x + y * y
    sr, sp = 0.25, 0.15
    rho = 1.0 + np.exp(-r2 / (2.0 * sr * sr)) / (4.0 * math.pi * sr * sr)
    p = 1e-5 + (g - 1.0) * np.exp(-r2 / (2.0 * sp * sp)) / (4.0 * math.pi * sp * sp)
    zero = np.zeros_like(x)
    return prob, euler_conservative(rho, zero, zero, p, g, 2)


def linadv_random(nx=8, ny=1, dim=1, degree=3, seed=0, adv=(1.0, 0.0), bc="periodic"):
    """Linear advection with seeded random nodal values (tests only)."""
    prob = base_problem(dim=dim, nx=nx, ny=ny, degree=degree, equation="linadv", adv=adv,
                        bc_x=bc, bc_y=bc)
    rng = np.random.default_rng(seed)
    ne = nx * (ny if dim == 2 else 1)
    npn = (degree + 1) ** dim
    return prob, rng.standard_normal((1, ne, npn))


def euler1d_riemann(nx=4000, degree=4, seed=0, limiter=LIMITER_ALL, t_final=0.2):
    """1D Euler (gamma 1.4) on [0,1] outflow; left/right states with
    rho log-uniform in [0.1, 10], v uniform in [-2, 2], p log-uniform in
    [0.01, 1000]; the jump sits on the element face nearest x = 0.5."""
    prob = base_problem(dim=1, nx=nx, degree=degree, equation="euler", bc_x="outflow",
                        limiter=frozenset(limiter), t_final=t_final)
    rng = np.random.default_rng(seed)
    rho = np.exp(rng.uniform(math.log(0.1), math.log(10.0), 2))
    vel = rng.uniform(-2.0, 2.0, 2)
    p = np.exp(rng.uniform(math.log(0.01), math.log(1000.0), 2))
    x, _ = node_coords(prob)
    xc, _ = element_centres(prob)
    right = (xc >= prob["x0"] + (nx // 2) * (prob["x1"] - prob["x0"]) / nx)[:, None]
    right = np.broadcast_to(right, x.shape)
    r = np.where(right, rho[1], rho[0])
    v = np.where(right, vel[1], vel[0])
    pp = np.where(right, p[1], p[0])
    prob["riemann"] = dict(rho=rho.tolist(), v=vel.tolist(), p=p.tolist())
    return prob, euler_conservative(r, v, None, pp, prob["gamma"], 1)


def isentropic_vortex(x, y, gamma=1.4, beta=5.0, u_inf=1.0, v_inf=1.0, xc=0.0, yc=0.0):
    """Sec. 5.3.1 vortex with free stream (u_inf, v_inf), rho_inf = p_inf = 1, p = rho^gamma."""
    r2 = (x - xc) ** 2 + (y - yc) ** 2
    rho = (1.0 - beta ** 2 * (gamma - 1.0) / (8.0 * gamma * math.pi ** 2) *
           np.exp(1.0 - r2)) ** (1.0 / (gamma - 1.0))
    v1 = u_inf - beta * (y - yc) / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    v2 = v_inf + beta * (x - xc) / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
    return rho, v1, v2, rho ** gamma


def euler2d_vortex(nx=512, ny=None, degree=4, seed=0, perturb=0.01, limiter=LIMITER_ALL,
                   steps=200):
    """2D Euler on [-5,5]^2 periodic: isentropic vortex (beta 5, free stream
    rho = 1, u = v = 1, p = 1) with the density multiplied by (1 + perturb Pi),
    Pi a seeded sum of 8 periodic sine modes scaled to max |Pi| = 1 on the nodes."""
    ny = nx if ny is None else ny
    prob = base_problem(dim=2, nx=nx, ny=ny, x0=-5.0, x1=5.0, y0=-5.0, y1=5.0, degree=degree,
                        equation="euler", limiter=frozenset(limiter), steps=steps, t_final=1e9)
    x, y = node_coords(prob)
    rho, v1, v2, p = isentropic_vortex(x, y, prob["gamma"])
    if perturb:
        rng = np.random.default_rng(seed)
        mk = rng.integers(1, 9, 8)
        nk = rng.integers(1, 9, 8)
        ak = rng.uniform(0.5, 1.0, 8)
        phi = rng.uniform(0.0, 2.0 * math.pi, 8)
        Pi = np.zeros_like(x)
        for k in range(8):
            Pi += ak[k] * np.sin(2.0 * math.pi * (mk[k] * x + nk[k] * y) / 10.0 + phi[k])
        Pi /= np.max(np.abs(Pi))
        rho = rho * (1.0 + perturb * Pi)
    return prob, euler_conservative(rho, v1, v2, p, prob["gamma"], 2)


def euler2d_vortex_riemann(nx=128, ny=None, degree=4, seed=0, limiter=LIMITER_ALL, steps=100):
    """2D Euler on [-5,5]^2 periodic: the isentropic vortex (as euler2d_vortex,
    unperturbed) with a seeded planar Riemann jump: a stripe of half the domain,
    normal to x or to y, bounded by element faces, where density and pressure
    are multiplied by (rho_R, p_R) and elsewhere by (rho_L, p_L); rho uniform
    in [0.5, 5], p uniform in [0.1, 10]."""
    ny = nx if ny is None else ny
    prob = base_problem(dim=2, nx=nx, ny=ny, x0=-5.0, x1=5.0, y0=-5.0, y1=5.0, degree=degree,
                        equation="euler", limiter=frozenset(limiter), steps=steps, t_final=1e9)
    rng = np.random.default_rng(seed)
    rho_s = rng.uniform(0.5, 5.0, 2)
    p_s = rng.uniform(0.1, 10.0, 2)
    along_x = bool(rng.integers(0, 2))
    n_dir = nx if along_x else ny
    lo = int(rng.integers(n_dir // 8, 3 * n_dir // 8 + 1))
    hi = lo + n_dir // 2
    x, y = node_coords(prob)
    rho, v1, v2, p = isentropic_vortex(x, y, prob["gamma"])
    e = np.arange(nx * ny)
    idx = (e % nx) if along_x else (e // nx)
    inside = ((idx >= lo) & (idx < hi))[:, None]
    rho = rho * np.where(inside, rho_s[1], rho_s[0])
    p = p * np.where(inside, p_s[1], p_s[0])
    prob["riemann2d"] = dict(rho=rho_s.tolist(), p=p_s.tolist(), along_x=along_x, lo=lo, hi=hi)
    return prob, euler_conservative(rho, v1, v2, p, prob["gamma"], 2)


def euler2d_ensemble(nprob=96, seed=0, nmin=32, nmax=512, limiter=LIMITER_ALL):
    """Independent 2D Euler problems for batched runs: side n uniform integer in
    [nmin, nmax] (n x n elements), degree uniform in {3, 4}, each with the
    vortex-plus-Riemann data of euler2d_vortex_riemann (its own seed).
    Returns a list of (problem, state)."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(nmin, nmax + 1, nprob)
    degs = rng.integers(3, 5, nprob)
    return [euler2d_vortex_riemann(nx=int(n), degree=int(N), seed=seed * 1000 + i, limiter=limiter)
            for i, (n, N) in enumerate(zip(sides, degs))]


def tenmoment2d_voronoi(nx=256, ny=None, degree=3, seed=0, ncells=16, limiter=LIMITER_ALL,
                        steps=200, source=True):
    """2D ten-moment on [0,1]^2 periodic with the Gaussian source
    W = 25 exp(-200 |x - (0.5, 0.5)|^2); each element takes the state of the
    seeded Voronoi cell (periodic distance) holding its centre: rho log-uniform
    in [0.1, 10], v uniform in [-1, 1]^2, P = R diag(l1, l2) R^T with l
    log-uniform in [0.01, 10] and R a random rotation."""
    ny = nx if ny is None else ny
    src = dict(amp=25.0, k=200.0, cx=0.5, cy=0.5) if source else None
    prob = base_problem(dim=2, nx=nx, ny=ny, degree=degree, equation="tenmoment",
                        limiter=frozenset(limiter), steps=steps, t_final=1e9, source=src)
    rng = np.random.default_rng(seed)
    sites = rng.uniform(0.0, 1.0, (ncells, 2))
    rho_c = np.exp(rng.uniform(math.log(0.1), math.log(10.0), ncells))
    v_c = rng.uniform(-1.0, 1.0, (ncells, 2))
    lam = np.exp(rng.uniform(math.log(0.01), math.log(10.0), (ncells, 2)))
    ang = rng.uniform(0.0, math.pi, ncells)
    c, s = np.cos(ang), np.sin(ang)
    p11 = c * c * lam[:, 0] + s * s * lam[:, 1]
    p22 = s * s * lam[:, 0] + c * c * lam[:, 1]
    p12 = c * s * (lam[:, 0] - lam[:, 1])
    xc, yc = element_centres(prob)
    dxs = np.abs(xc[:, None] - sites[None, :, 0])
    dys = np.abs(yc[:, None] - sites[None, :, 1])
    dxs = np.minimum(dxs, 1.0 - dxs)
    dys = np.minimum(dys, 1.0 - dys)
    cell = np.argmin(dxs ** 2 + dys ** 2, axis=1)
    npn = (degree + 1) ** 2
    rep = lambda a: np.repeat(a[cell][:, None], npn, axis=1)
    u = tenmoment_conservative(rep(rho_c), rep(v_c[:, 0]), rep(v_c[:, 1]), rep(p11), rep(p12),
                               rep(p22))
    return prob, u


def rayleigh_taylor(nx=64, ny=256, degree=3, limiter=LIMITER_ALL, t_final=2.5):
    """Rayleigh-Taylor instability (Sec. 5.5): Euler (gamma 5/3) with gravity
    g = (0, 1) (pointing to +y) on [0, 0.25] x [0, 1]; walls in x; given ghost
    states with the HLLC flux at the bottom (rho, v1, v2, p) = (2, 0, 0, 1) and
    top (1, 0, 0, 2.5);
    (rho, v1, v2, p) = (2, 0, -0.025 c cos(8 pi x), 2y + 1) for y <= 0.5 and
    (1, 0, -0.025 c cos(8 pi x), y + 1.5) above, c = sqrt(gamma p / rho)."""
    g = 5.0 / 3.0
    prob = base_problem(dim=2, nx=nx, ny=ny, degree=degree, equation="euler", gamma=g, x0=0.0,
                        x1=0.25, y0=0.0, y1=1.0, bc_x="wall", bc_y="dirichlet",
                        limiter=frozenset(limiter), t_final=t_final, source=dict(gravity=(0.0, 1.0)))
    bottom = euler_conservative(np.array(2.0), np.array(0.0), np.array(0.0), np.array(1.0), g, 2)
    top = euler_conservative(np.array(1.0), np.array(0.0), np.array(0.0), np.array(2.5), g, 2)
    prob["bc_state"] = {"y-": [float(x) for x in bottom], "y+": [float(x) for x in top]}
    prob["bc_flux"] = "hllc"
    x, y = node_coords(prob)
    _, yc = element_centres(prob)
    low = np.broadcast_to((yc <= 0.5)[:, None], x.shape)
    rho = np.where(low, 2.0, 1.0)
    p = np.where(low, 2.0 * y + 1.0, y + 1.5)
    c = np.sqrt(g * p / rho)
    v2 = -0.025 * c * np.cos(8.0 * math.pi * x)
    return prob, euler_conservative(rho, np.zeros_like(x), v2, p, g, 2)


def uniform_state(prob, prim):
    """Constant state everywhere (free-stream tests); prim is the primitive tuple."""
    x, y = node_coords(prob)
    one = np.ones_like(x)
    eq = prob["equation"]
    if eq == "linadv":
        return (prim[0] * one)[None].copy()
    if eq == "euler":
        if prob["dim"] == 1:
            rho, v1, p = prim
            return euler_conservative(rho * one, v1 * one, None, p * one, prob["gamma"], 1)
        rho, v1, v2, p = prim
        return euler_conservative(rho * one, v1 * one, v2 * one, p * one, prob["gamma"], 2)
    rho, v1, v2, p11, p12, p22 = prim
    return tenmoment_conservative(rho * one, v1 * one, v2 * one, p11 * one, p12 * one, p22 * one)
