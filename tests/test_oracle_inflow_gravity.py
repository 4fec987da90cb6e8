"""Pins of the oracle's given-state boundaries (Sec. 3.3: the inflow/outflow
ghost values u^- = U^- = g, F^- = f(g), and the fully-inflow rule F = f(g))
and of the Euler gravity source (Sec. 5.5), against what the mathematics
fixes:

* a uniform state equal to the ghost states stays uniform (free stream
  through every boundary kind, 1D and 2D, limiters on);
* the fully-inflow face flux is f(g) exactly;
* for linear advection the scheme's flux with a ghost state is the upwind
  flux, so given-state boundaries on both sides reproduce inflow + outflow
  to rounding;
* smooth data entering through an inflow boundary converge at order N + 1
  to the exact solution c + bump(x - t);
* gravity on a uniform state: the source ODE m' = rho g, E' = g . m has the
  quadratic solution m0 + rho g t, E0 + g.m0 t + rho |g|^2 t^2 / 2, which an
  RK method of order >= 2 reproduces exactly;
* the Rayleigh-Taylor data are mirror symmetric about x = 0.125 and the
  walls, ghost states and gravity keep them so to rounding.
"""
import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc


def _euler_uniform(dim, prim, nx=6, ny=5, N=3):
    prob = wl.base_problem(dim=dim, nx=nx, ny=ny, degree=N, equation="euler", limiter=wl.LIMITER_ALL)
    u = wl.uniform_state(prob, prim)
    return prob, u


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_free_stream_through_given_state_boundaries(N):
    prim = (1.3, 2.5, -0.4, 0.9)
    prob, u = _euler_uniform(2, prim, N=N)
    g = [float(x) for x in u[:, 0, 0]]
    for sides in ({"x-": "inflow", "x+": "outflow", "y-": "dirichlet", "y+": "dirichlet"},
                  {"x-": "dirichlet", "x+": "dirichlet", "y-": "wall", "y+": "dirichlet"}):
        pr = dict(prob, bc_x="outflow", bc_y="outflow", bc_side=sides,
                  bc_state={s: g for s in sides})
        if "wall" in sides.values():   # a wall keeps a uniform state only without normal velocity
            pr = dict(pr, bc_state={s: [g[0], g[1], 0.0, g[3] - 0.5 * g[2] ** 2 / g[0]] for s in sides})
            uu = wl.uniform_state(pr, (prim[0], prim[1], 0.0, prim[3]))
        else:
            uu = u
        d = oracle_desc(pr)
        out, t, n, st = oracle.run(d, uu, 5, 1e9)
        assert st == 0
        np.testing.assert_allclose(out, uu, rtol=0, atol=2e-14 * np.abs(uu).max())
    prob1, u1 = _euler_uniform(1, (0.7, -1.9, 2.2), nx=9, N=N)
    g1 = [float(x) for x in u1[:, 0, 0]]
    pr = dict(prob1, bc_x="dirichlet", bc_state={"x-": g1, "x+": g1})
    out, t, n, st = oracle.run(oracle_desc(pr), u1, 5, 1e9)
    assert st == 0
    np.testing.assert_allclose(out, u1, rtol=0, atol=2e-14 * np.abs(u1).max())


def test_fully_inflow_face_flux_is_f_of_g():
    prob, u = wl.euler1d_riemann(nx=12, degree=3, seed=2)
    g = [0.8, 0.8 * 3.0, 2.0 / 0.4 + 0.5 * 0.8 * 9.0]        # rho 0.8, v 3, p 2: supersonic inflow
    pr = dict(prob, bc_side={"x-": "inflow"}, bc_state={"x-": g})
    d = oracle_desc(pr)
    out, st, dg = oracle.step(d, u, 0.5 * oracle.dt(d, u), want_diag=True)
    assert st == 0
    rho, m, E = g
    p = 0.4 * (E - 0.5 * m * m / rho)
    f = np.array([m, m * m / rho + p, (E + p) * m / rho])
    np.testing.assert_allclose(dg["fnum_x"][:, 0, 0], f, rtol=1e-15, atol=0)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_linear_advection_ghost_state_is_upwind(N):
    prob, u = wl.linadv_random(nx=11, degree=N, seed=N, adv=(1.4, 0.0), bc="outflow")
    g = [0.37]
    upw = dict(prob, bc_side={"x-": "inflow"}, bc_state={"x-": g})
    dir_ = dict(prob, bc_x="dirichlet", bc_state={"x-": g, "x+": [-5.0]})
    d1, d2 = oracle_desc(upw), oracle_desc(dir_)
    dt = oracle.dt(d1, u)
    a, st1 = oracle.step(d1, u, dt)
    b, st2 = oracle.step(d2, u, dt)
    assert st1 == st2 == 0
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-14 * np.abs(a).max())


def _bump(x):
    return np.exp(-200.0 * (x - 0.5) ** 2)


@pytest.mark.parametrize("N", [2, 3])
def test_inflow_convergence(N):
    c, t_end = 0.3, 0.25
    errs = []
    for nx in (16, 32, 64):
        prob = wl.base_problem(dim=1, nx=nx, degree=N, equation="linadv", adv=(1.0, 0.0),
                               bc_x="outflow", bc_side={"x-": "inflow"}, bc_state={"x-": [c]})
        x, _ = wl.node_coords(prob)
        u0 = (c + _bump(x))[None]
        out, t, n, st = oracle.run(oracle_desc(prob), u0, 10 ** 6, t_end)
        assert st == 0 and t == t_end
        _, w = wl.gl_nodes01(N)
        errs.append(np.sqrt((((out[0] - c - _bump(x - t_end)) ** 2) * w / nx).sum()))
    order = np.log2(errs[1] / errs[2])
    assert order >= N + 1 - 0.3, (errs, order)


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("N", [1, 3, 4])
def test_gravity_on_a_uniform_state(dim, N):
    g = (0.7, -1.3) if dim == 2 else (-1.1, 0.0)
    prim = (1.6, 0.4, -0.2, 2.0) if dim == 2 else (1.6, 0.4, 2.0)
    prob = wl.base_problem(dim=dim, nx=5, ny=4, degree=N, equation="euler", source=dict(gravity=g))
    u = wl.uniform_state(prob, prim)
    d = oracle_desc(prob)
    dt = 0.8 * oracle.dt(d, u)
    out, st = oracle.step(d, u, dt)
    assert st == 0
    rho, m0, E0 = u[0, 0, 0], u[1:1 + dim, 0, 0], u[-1, 0, 0]
    gv = np.array(g[:dim])
    exp_m = m0 + rho * gv * dt
    exp_E = E0 + gv @ m0 * dt + 0.5 * rho * (gv @ gv) * dt * dt
    scale = np.abs(u).max()
    np.testing.assert_allclose(out[0], rho, rtol=0, atol=1e-15 * scale)
    for i in range(dim):
        np.testing.assert_allclose(out[1 + i], exp_m[i], rtol=0, atol=1e-14 * scale)
    np.testing.assert_allclose(out[-1], exp_E, rtol=0, atol=1e-14 * scale)


def test_rayleigh_taylor_keeps_mirror_symmetry():
    nx, ny, N = 8, 32, 3
    prob, u = wl.rayleigh_taylor(nx=nx, ny=ny, degree=N)
    d = oracle_desc(prob)
    out, t, n, st = oracle.run(d, u, 25, 1e9)
    assert st == 0 and n == 25
    n1 = N + 1
    G = out.reshape(4, ny, nx, n1, n1)             # [v][iy][ix][q][p]
    F = G[:, :, ::-1, :, ::-1]
    for v, sgn in enumerate((1, -1, 1, 1)):
        assert np.abs(G[v] - sgn * F[v]).max() <= 1e-13 * np.abs(G[v]).max()
    # gravity has accelerated the gas (heavy fluid pushed towards +y)
    m = oracle.element_means(d, out)
    assert m[0].min() > 0
