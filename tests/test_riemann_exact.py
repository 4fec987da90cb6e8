"""Pins of the exact Riemann solver used to measure errors (tests/_riemann_exact.py):
Sod's problem against the star values printed in gas-dynamics textbooks, the
Rankine-Hugoniot conditions across the computed shock, and the isentropic
relations and Riemann invariant across the computed rarefaction."""
import math

import numpy as np

from tests import _riemann_exact as rx


def test_sod_star_state():
    ps, vs = rx.star((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(ps - 0.30313) < 1e-5 and abs(vs - 0.92745) < 1e-5
    r = rx.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), np.array([0.5, 1.5]))
    assert abs(r[0][0] - 0.42632) < 1e-5 and abs(r[0][1] - 0.26557) < 1e-5


def test_shock_satisfies_rankine_hugoniot():
    g = 1.4
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    s = np.linspace(-2, 2, 4001)
    W = rx.sample(L, R, s)
    # locate the right shock: last jump in rho
    i = np.argmax(np.abs(np.diff(W[0])) * (s[1:] > 1.0))
    a, b = W[:, i], W[:, i + 1]
    S = 0.5 * (s[i] + s[i + 1])
    U = lambda w: np.array([w[0], w[0] * w[1], w[2] / (g - 1) + 0.5 * w[0] * w[1] ** 2])
    F = lambda w: np.array([w[0] * w[1], w[0] * w[1] ** 2 + w[2], w[1] * (w[2] / (g - 1) + 0.5 * w[0] * w[1] ** 2 + w[2])])
    # exact shock speed from mass conservation, then momentum and energy must agree
    Sx = (F(a)[0] - F(b)[0]) / (U(a)[0] - U(b)[0])
    assert abs(Sx - S) < 2e-3
    np.testing.assert_allclose(F(a) - F(b), Sx * (U(a) - U(b)), rtol=1e-10, atol=1e-10)


def test_rarefaction_isentropic_and_invariant():
    g = 1.4
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    s = np.linspace(-1.18, -0.08, 200)   # inside the left fan
    rho, v, p = rx.sample(L, R, s)
    np.testing.assert_allclose(p / rho ** g, 1.0, rtol=1e-12)
    c = np.sqrt(g * p / rho)
    np.testing.assert_allclose(v + 2 * c / (g - 1), 2 * math.sqrt(g) / (g - 1), rtol=1e-12)
    np.testing.assert_allclose(v - c, s, rtol=1e-12, atol=1e-12)


def test_mirror_symmetry():
    L, R = (0.7, 0.3, 2.0), (2.5, -1.1, 40.0)
    s = np.linspace(-5, 5, 101)
    a = rx.sample(L, R, s)
    b = rx.sample((R[0], -R[1], R[2]), (L[0], -L[1], L[2]), -s)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-12)
    np.testing.assert_allclose(a[1], -b[1], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a[2], b[2], rtol=1e-12)
