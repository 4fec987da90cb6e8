"""Pins of the oracle's HLLC flux at given-state boundaries (the upwind flux
that Sec. 3.3 names for boundaries mixing inflow and outflow), by the
properties that define the solver:

* consistency: a uniform state equal to the ghost states stays uniform, at
  rest and moving, 1D and 2D, with the limiters on;
* upwinding: when every wave leaves the ghost side (supersonic inflow) the
  flux is the ghost side's flux, so the step equals the fully-inflow rule;
* contact resolution: a fluid at rest next to a ghost state of another
  density at the same pressure feels no mass flux through the boundary
  (exact for HLLC), where the Rusanov-type flux diffuses mass across it.
"""
import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc


def _cons1(rho, v, p, g=1.4):
    return [rho, rho * v, p / (g - 1.0) + 0.5 * rho * v * v]


@pytest.mark.parametrize("N", [1, 3, 4])
@pytest.mark.parametrize("v", [0.0, 0.7, -2.9])
def test_free_stream(N, v):
    prob = wl.base_problem(dim=1, nx=9, degree=N, equation="euler", limiter=wl.LIMITER_ALL,
                           bc_x="dirichlet", bc_flux="hllc")
    u = wl.uniform_state(prob, (1.3, v, 0.8))
    g = [float(x) for x in u[:, 0, 0]]
    prob["bc_state"] = {"x-": g, "x+": g}
    out, t, n, st = oracle.run(oracle_desc(prob), u, 5, 1e9)
    assert st == 0
    np.testing.assert_allclose(out, u, rtol=0, atol=2e-14 * np.abs(u).max())
    prob2, u2 = wl.euler2d_vortex(nx=5, ny=4, degree=N, perturb=0.0)
    prob2 = dict(prob2, bc_x="dirichlet", bc_y="dirichlet", bc_flux="hllc", limiter=wl.LIMITER_ALL)
    u2 = wl.uniform_state(prob2, (0.9, v, 0.4, 1.7))
    g2 = [float(x) for x in u2[:, 0, 0]]
    prob2["bc_state"] = {s: g2 for s in ("x-", "x+", "y-", "y+")}
    out, t, n, st = oracle.run(oracle_desc(prob2), u2, 3, 1e9)
    assert st == 0
    np.testing.assert_allclose(out, u2, rtol=0, atol=2e-14 * np.abs(u2).max())


@pytest.mark.parametrize("N", [2, 3])
def test_supersonic_inflow_is_the_inflow_rule(N):
    prob, u = wl.euler1d_riemann(nx=15, degree=N, seed=4)
    x, _ = wl.node_coords(prob)
    one = np.ones_like(x)
    u = wl.euler_conservative(1.0 + 0.2 * np.sin(6 * x), 3.0 * one, None, 0.5 * one, 1.4, 1)
    g = _cons1(1.1, 3.2, 0.6)                      # Mach ~ 4.3 into the domain
    hllc = dict(prob, bc_x="outflow", bc_side={"x-": "dirichlet"}, bc_state={"x-": g}, bc_flux="hllc")
    infl = dict(prob, bc_x="outflow", bc_side={"x-": "inflow"}, bc_state={"x-": g})
    d1, d2 = oracle_desc(hllc), oracle_desc(infl)
    dt = oracle.dt(d1, u)
    a, s1 = oracle.step(d1, u, dt)
    b, s2 = oracle.step(d2, u, dt)
    assert s1 == s2 == 0
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14 * np.abs(b).max())


def test_contact_at_rest_passes_no_mass():
    prob = wl.base_problem(dim=1, nx=10, degree=3, equation="euler", limiter=wl.LIMITER_ALL,
                           bc_x="dirichlet")
    u = wl.uniform_state(prob, (1.0, 0.0, 1.0))
    g = _cons1(3.0, 0.0, 1.0)                      # denser gas, same pressure, at rest
    prob["bc_state"] = {"x-": g, "x+": g}
    mass0 = u[0].sum()
    out, st = oracle.step(oracle_desc(dict(prob, bc_flux="hllc")), u, 1e-3)
    assert st == 0
    np.testing.assert_allclose(out, u, rtol=0, atol=1e-15)     # the contact does not move
    out2, st = oracle.step(oracle_desc(prob), u, 1e-3)
    assert st == 0 and out2[0].sum() - mass0 > 1e-6           # Rusanov lets mass in
