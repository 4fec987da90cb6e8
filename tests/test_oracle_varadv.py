"""Pins of the oracle on the variable advection equation u_t + (a(x) u)_x = 0
(Sec. 5.1, a(x) = x^2 on [0.1, 1]) with the exact solution as time-dependent
inflow data on the left and outflow on the right, against what the
mathematics and the paper fix:

* the exact solution by characteristics (u0(x/(1+tx))/(1+tx)^2) solves the
  equation (checked by finite differences) and the Chebyshev boundary data
  reproduce it;
* the EA (evaluate) flux converges at the optimal order N + 1 for N = 1..3;
  the AE (extrapolate) flux also reaches N + 1 (from 32 elements on) but with
  much larger errors for odd N (10x and 30x at 128 elements) and similar ones
  for N = 2, as the paper reports;
* conservation with boundaries: the change of the total over one step is
  dt times (inflow flux - outflow flux) of the step's own face fluxes;
* with a(x) constant the equation is linear advection: the step equals the
  linear advection step with the same velocity.
"""
import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc


def test_exact_solution_and_boundary_data():
    x = np.linspace(0.1, 1.0, 41)
    t, h = 0.6, 1e-5
    u = lambda x, t: wl.varadv_exact(x, t)
    ut = (u(x, t + h) - u(x, t - h)) / (2 * h)
    fx = ((x + h) ** 2 * u(x + h, t) - (x - h) ** 2 * u(x - h, t)) / (2 * h)
    assert np.abs(ut + fx).max() < 1e-8
    prob, _ = wl.varadv_x2(t_final=1.0)
    c = np.array(prob["bc_time"]["coef"]["x-"])
    tau = np.linspace(-1.0, 1.0, 201)
    assert np.abs(np.polynomial.chebyshev.chebval(tau, c) - u(0.1, 0.5 * (tau + 1.0))).max() < 1e-13


def test_flux_and_speed():
    d = oracle.make_desc(equation=oracle.EQ_VARADV, adv_poly=(0.3, -0.2, 1.0, 0.5), x0=0.1, x1=1.0)
    for x in (0.1, 0.55, 1.0):
        a = 0.3 - 0.2 * x + x * x + 0.5 * x ** 3
        assert oracle.wave_speed_x(d, [2.0], x, 0) == pytest.approx(abs(a), rel=1e-15)
        assert oracle.flux_x(d, [2.0], x, 0)[0] == pytest.approx(2.0 * a, rel=1e-15)


def _error(N, nx, central):
    prob, u = wl.varadv_x2(nx=nx, degree=N)
    g, t, n, st = oracle.run(oracle_desc(prob, central=central), u, 10 ** 6, 1.0)
    assert st == 0 and t == 1.0
    x, _ = wl.node_coords(prob)
    _, w = wl.nodes01(prob)
    return float(np.sqrt(((g[0] - wl.varadv_exact(x, 1.0)) ** 2 * w * 0.9 / nx).sum()))


@pytest.fixture(scope="module")
def study():
    return {(N, c): [_error(N, nx, cen) for nx in (32, 64, 128)]
            for N in (1, 2, 3) for c, cen in (("EA", oracle.CENTRAL_EA), ("AE", oracle.CENTRAL_AE))}


@pytest.mark.parametrize("N", [1, 2, 3])
def test_optimal_order(study, N):
    for c in ("EA", "AE"):
        e = study[N, c]
        assert np.log2(e[1] / e[2]) >= N + 1 - 0.3, (c, e)


def test_extrapolate_errors_larger_for_odd_degree(study):
    for N in (1, 3):
        assert study[N, "AE"][-1] >= 2.0 * study[N, "EA"][-1], (N, study[N, "AE"], study[N, "EA"])
    assert study[2, "AE"][-1] <= 2.0 * study[2, "EA"][-1]


def test_conservation_with_boundary_fluxes():
    prob, u = wl.varadv_x2(nx=12, degree=3)
    d = oracle_desc(prob)
    dt = oracle.dt(d, u)
    out, st, dg = oracle.step(d, u, dt, want_diag=True, time=0.3)
    assert st == 0
    m0, m1 = oracle.element_means(d, u)[0].sum(), oracle.element_means(d, out)[0].sum()
    dx = 0.9 / 12
    f_in, f_out = dg["fnum_x"][0, 0, 0], dg["fnum_x_right"][0, -1, 0]
    assert abs((m1 - m0) * dx - dt * (f_in - f_out)) <= 1e-15 * abs(m0 * dx)
    # the inflow flux is the b-weighted average of a(0.1) g(t) over the stage times
    A, b, c = oracle.tableau(3)
    g = np.array([wl.varadv_exact(0.1, 0.3 + ci * dt) for ci in c[:len(b)]])
    assert abs(f_in - 0.01 * (b @ g)) <= 1e-14


def test_constant_coefficient_is_linear_advection():
    prob, u = wl.linadv_random(nx=9, degree=3, seed=3, adv=(0.7, 0.0), bc="periodic")
    lin = oracle_desc(prob)
    var = oracle_desc(dict(prob, equation="varadv", adv_poly=(0.7, 0.0, 0.0, 0.0)))
    dt = oracle.dt(lin, u)
    a, _ = oracle.step(lin, u, dt)
    b, _ = oracle.step(var, u, dt)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-15 * np.abs(a).max())
