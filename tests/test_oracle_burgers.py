"""Pins of the oracle on Burgers' equation f(u) = u^2/2 (Sec. 5.1), against
what the mathematics and the paper fix, not against the code:

* the exact solution of u0 = 0.2 sin(x) on [0, 2 pi] by characteristics,
  u = 0.2 sin(x - u t), smooth until t = 5: at t = 2 the EA central flux
  converges at the optimal order N + 1 for every degree, and the AE flux
  at about N + 1/2 with several times larger errors for odd N (the paper's
  finding for Radau correction and Gauss-Legendre points);
* D-CSX gives errors within a few percent of D2 (the paper calls the two
  virtually the same);
* conservation of the mean of u over the periodic domain, and a constant
  state kept to rounding;
* past the shock (t = 8) the blended scheme stays within the initial range
  (no Gibbs overshoot), while the unlimited scheme overshoots it.
"""
import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc

AMP = 0.2
LEVELS = (32, 64, 128)


def exact(x, t, a=AMP):
    """u = a sin(x - u t), by Newton's method from u0 (g' = 1 + a t cos > 0 for a t < 1)."""
    u = a * np.sin(x)
    for _ in range(100):
        g = u - a * np.sin(x - u * t)
        u = u - g / (1.0 + a * t * np.cos(x - u * t))
    return u


def test_exact_solution_helper():
    x = np.linspace(0.0, 2.0 * np.pi, 101)
    u = exact(x, 2.0)
    np.testing.assert_allclose(u, AMP * np.sin(x - 2.0 * u), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(exact(x, 0.0), AMP * np.sin(x))


def l2_error(N, nx, t=2.0, **over):
    prob, u = wl.burgers_sine(nx=nx, degree=N, t_final=t)
    g, tt, n, st = oracle.run(oracle_desc(prob, **over), u, 10 ** 6, t)
    assert st == 0 and tt == t
    x, _ = wl.node_coords(prob)
    _, w = wl.gl_nodes01(N)
    dx = 2.0 * np.pi / nx
    return float(np.sqrt(((g[0] - exact(x, t)) ** 2 * w * dx).sum()))


def orders(errs):
    return [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.fixture(scope="module")
def study():
    out = {}
    for N in (1, 2, 3, 4):
        for name, cen in (("EA", oracle.CENTRAL_EA), ("AE", oracle.CENTRAL_AE)):
            out[N, name] = [l2_error(N, nx, central=cen) for nx in LEVELS]
    return out


def test_flux_and_wave_speed():
    d = oracle.make_desc(equation=oracle.EQ_BURGERS)
    for u in (-1.7, 0.0, 0.3):
        assert oracle.flux(d, np.array([u]), 0)[0] == 0.5 * u * u
        assert oracle.wave_speed(d, np.array([u]), 0) == abs(u)
    assert oracle.num_constraints(d) == 0


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_evaluate_flux_optimal_order(study, N):
    e = study[N, "EA"]
    assert orders(e)[-1] >= N + 1 - 0.25, (e, orders(e))


@pytest.mark.parametrize("N", [1, 3])
def test_extrapolate_flux_suboptimal_for_odd_degree(study, N):
    ea, ae = study[N, "EA"], study[N, "AE"]
    assert N + 0.2 <= orders(ae)[-1] <= N + 0.75, orders(ae)
    assert ae[-1] >= 5.0 * ea[-1]


@pytest.mark.parametrize("N", [2, 4])
def test_extrapolate_flux_converges_for_even_degree(study, N):
    ae = study[N, "AE"]
    assert orders(ae)[-1] >= N + 1 - 0.25, orders(ae)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_dcsx_close_to_d2(N):
    for nx in (32, 64):
        d2 = l2_error(N, nx)
        dc = l2_error(N, nx, dissipation=oracle.DISS_DCSX)
        assert abs(dc - d2) <= 0.05 * d2, (nx, d2, dc)


def test_mean_conserved_and_constant_state_kept():
    prob, u = wl.burgers_sine(nx=40, degree=3)
    d = oracle_desc(prob, central=oracle.CENTRAL_AE)
    g, t, n, st = oracle.run(d, u, 10 ** 6, 3.0)
    assert st == 0 and n > 30
    m0, m1 = oracle.element_means(d, u)[0].sum(), oracle.element_means(d, g)[0].sum()
    assert abs(m1 - m0) <= 1e-15 * n * np.abs(u).max() * 40
    c = np.full_like(u, 0.37)
    g, t, n, st = oracle.run(oracle_desc(prob), c, 10 ** 6, 1.0)
    assert st == 0
    np.testing.assert_allclose(g, c, rtol=0, atol=1e-15)


def test_blending_past_the_shock_stays_in_range():
    prob, u = wl.burgers_sine(nx=64, degree=3)
    lim = oracle_desc(dict(prob, limiter=wl.LIMITER_ALL))
    g, t, n, st = oracle.run(lim, u, 10 ** 6, 8.0)
    assert st == 0 and t == 8.0
    assert np.abs(g).max() <= AMP
    g2, _, _, st = oracle.run(oracle_desc(prob), u, 10 ** 6, 8.0)
    assert st == 0 and np.abs(g2).max() >= AMP + 0.01
