"""Pins of the oracle with Gauss-Lobatto-Legendre solution points and the g2
correction (Sec. 5.1), against what the mathematics and the paper fix:

* the nodes and weights against numpy's Legendre class (end points and
  roots of P_N'; exact quadrature to degree 2N - 1, not 2N);
* the correction derivatives against g2 and the Radau polynomial built with
  numpy: g2' vanishes at every interior GLL node, so the FR correction
  reaches only the end nodes, with 1/w there; the Radau derivatives at the
  Gauss-Legendre nodes equal l(1)/w;
* the paper: with GLL points the evaluate (EA) and extrapolate (AE) central
  fluxes are the same scheme, also for nonlinear problems; Burgers converges
  at the optimal order for N = 2 but near N + 1/2 for odd N; linear
  advection converges at N + 1;
* the CFL number from the Fourier analysis is the stability limit of the
  computed GLL scheme (0.99 CFL bounded, 1.05 CFL blows up).
"""
import numpy as np
import pytest

import oracle
from oracle.cfl import cfl_number
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc
from tests.test_oracle_burgers import exact

Leg = np.polynomial.legendre.Legendre


def _radau(k):
    return ((-1) ** k / 2.0) * (Leg.basis(k) - Leg.basis(k - 1))


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_nodes_weights_and_quadrature(N):
    xi, w, l0, l1, D, gL, gR = oracle.tables_corr(N, oracle.POINTS_GLL)
    inner = np.sort(Leg.basis(N).deriv().roots().real) if N > 1 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    np.testing.assert_allclose(xi, 0.5 * (x + 1.0), rtol=0, atol=1e-15)
    for m in range(2 * N):
        assert abs(w @ xi ** m - 1.0 / (m + 1)) < 1e-14
    assert abs(w @ xi ** (2 * N) - 1.0 / (2 * N + 1)) > 1e-6
    np.testing.assert_array_equal(l0, np.eye(N + 1)[0])
    np.testing.assert_array_equal(l1, np.eye(N + 1)[N])
    for m in range(N + 1):
        np.testing.assert_allclose(D @ xi ** m, m * xi ** max(m - 1, 0) * (m > 0), atol=1e-12)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_correction_derivatives(N):
    xi, w, l0, l1, D, gL, gR = oracle.tables_corr(N, oracle.POINTS_GLL)
    g2 = ((N + 1) * _radau(N) + N * _radau(N + 1)) / (2 * N + 1)
    assert abs(g2(-1.0) - 1.0) < 1e-14 and abs(g2(1.0)) < 1e-14
    np.testing.assert_allclose(gL, 2.0 * g2.deriv()(2.0 * xi - 1.0), rtol=0, atol=1e-12)
    np.testing.assert_allclose(gR, -2.0 * g2.deriv()(1.0 - 2.0 * xi), rtol=0, atol=1e-12)
    expect_L = np.zeros(N + 1)
    expect_L[0] = -1.0 / w[0]
    np.testing.assert_allclose(gL, expect_L, rtol=0, atol=1e-12)
    np.testing.assert_allclose(gR, -expect_L[::-1], rtol=0, atol=1e-12)
    # Gauss-Legendre with the Radau correction
    xi, w, l0, l1, D, gL, gR = oracle.tables_corr(N, oracle.POINTS_GL)
    gdg = _radau(N + 1)
    np.testing.assert_allclose(gL, 2.0 * gdg.deriv()(2.0 * xi - 1.0), rtol=0, atol=1e-12)
    np.testing.assert_allclose(gR, l1 / w, rtol=0, atol=1e-12)
    np.testing.assert_allclose(gL, -l0 / w, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_evaluate_and_extrapolate_coincide(N):
    prob = wl.base_problem(dim=1, nx=13, degree=N, equation="burgers", points="gll")
    u = np.random.default_rng(N).standard_normal((1, 13, N + 1))
    d_ea = oracle_desc(prob)
    d_ae = oracle_desc(prob, central=oracle.CENTRAL_AE)
    dt = oracle.dt(d_ea, u)
    a, s1 = oracle.step(d_ea, u, dt)
    b, s2 = oracle.step(d_ae, u, dt)
    assert s1 == s2 == 0
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14 * np.abs(a).max())
    prob, u = wl.euler2d_vortex_riemann(nx=6, ny=5, degree=N, seed=N, limiter=())
    prob = dict(prob, points="gll")
    u = wl.euler_conservative(*_vortex_prims(prob), prob["gamma"], 2)
    d_ea, d_ae = oracle_desc(prob), oracle_desc(prob, central=oracle.CENTRAL_AE)
    dt = oracle.dt(d_ea, u)
    a, s1 = oracle.step(d_ea, u, dt)
    b, s2 = oracle.step(d_ae, u, dt)
    assert s1 == s2 == 0
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13 * np.abs(a).max())
    # while with Gauss-Legendre points they differ
    prob_gl = dict(prob, points="gl")
    if N > 1:
        u2 = wl.euler_conservative(*_vortex_prims(prob_gl), prob["gamma"], 2)
        d1, d2 = oracle_desc(prob_gl), oracle_desc(prob_gl, central=oracle.CENTRAL_AE)
        a2, _ = oracle.step(d1, u2, dt)
        b2, _ = oracle.step(d2, u2, dt)
        assert np.abs(a2 - b2).max() > 1e-9


def _vortex_prims(prob):
    x, y = wl.node_coords(prob)
    return wl.isentropic_vortex(x, y, prob["gamma"])


def _burgers_errors(N, central, levels):
    errs = []
    for nx in levels:
        prob, u = wl.burgers_sine(nx=nx, degree=N, points="gll")
        g, t, n, st = oracle.run(oracle_desc(prob, central=central), u, 10 ** 6, 2.0)
        assert st == 0 and t == 2.0
        x, _ = wl.node_coords(prob)
        _, w = wl.nodes01(prob)
        errs.append(np.sqrt(((g[0] - exact(x, 2.0)) ** 2 * w * 2 * np.pi / nx).sum()))
    return errs


def test_burgers_orders_with_gll():
    levels = (32, 64, 128)
    orders = {}
    for N in (1, 2, 3):
        e = _burgers_errors(N, oracle.CENTRAL_EA, levels)
        orders[N] = np.log2(e[1] / e[2])
    assert orders[2] >= 2.75, orders
    assert orders[1] <= 1.75 and orders[3] <= 3.75, orders


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_linear_advection_order(N):
    errs = []
    for nx in (8, 16, 32):
        prob = wl.base_problem(dim=1, nx=nx, degree=N, equation="linadv", points="gll")
        x, _ = wl.node_coords(prob)
        u = np.sin(2 * np.pi * x)[None]
        g, t, n, st = oracle.run(oracle_desc(prob), u, 10 ** 6, 1.0)
        assert st == 0
        _, w = wl.nodes01(prob)
        errs.append(np.sqrt(((g[0] - np.sin(2 * np.pi * (x - 1.0))) ** 2 * w / nx).sum()))
    assert np.log2(errs[1] / errs[2]) >= N + 1 - 0.3, errs


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_gll_cfl_is_the_stability_limit(N):
    cfl = cfl_number(N, points=oracle.POINTS_GLL)
    peaks = []
    for frac in (0.99, 1.05):
        prob, u = wl.linadv_random(nx=16, degree=N, seed=5)
        prob = dict(prob, points="gll")
        d = oracle_desc(prob, cfl=cfl * frac, cfl_safety=1.0)
        out, t, steps, st = oracle.run(d, u, 3000, 1e9)
        peaks.append(np.abs(out).max() / np.abs(u).max())
    assert peaks[0] < 1.05, peaks
    assert not np.isfinite(peaks[1]) or peaks[1] > 10.0, peaks   # overflowed, or grown


def test_subcell_scheme_outruns_its_cfl_with_gll():
    """Why the library takes GLL points without the blending and flux limiters
    (the paper uses them only for smooth, unlimited runs): the low-order
    subcell update of the smallest subcell (width w_0 dx) needs
    lambda dt / (w_0 dx) <= 1, but CFL(N) of the GLL scheme is larger than
    the Gauss-Legendre one while w_0 is smaller, so C_s CFL(N) / w_0 > 1 and
    the limited scheme loses admissible means within a few steps, where the
    same data on Gauss-Legendre points run on."""
    for N in (2, 3, 4):
        w0 = oracle.tables(N, oracle.POINTS_GLL)[1][0]
        assert 0.98 * cfl_number(N, points=oracle.POINTS_GLL) / w0 > 1.0
        w0gl = oracle.tables(N)[1][0]
        assert 0.98 * cfl_number(N) / w0gl < 1.0
    for pts, fails in (("gl", False), ("gll", True)):
        prob, _ = wl.euler1d_riemann(nx=40, degree=3, seed=2, limiter=("blend", "flux", "scaling", "traces"))
        prob = dict(prob, points=pts)
        x, _ = wl.node_coords(prob)
        xc, _ = wl.element_centres(prob)
        r = prob["riemann"]
        right = np.broadcast_to((xc >= 0.5)[:, None], x.shape)
        pick = lambda k: np.where(right, r[k][1], r[k][0])
        u = wl.euler_conservative(pick("rho"), pick("v"), None, pick("p"), 1.4, 1)
        g, t, n, st = oracle.run(oracle_desc(prob), u, 60, 1e9)
        assert (st != 0) == fails, (pts, n, st)
