"""Pins of the smoothness indicator between its limits (Sec. 4: the blending
coefficient comes from the indicator of Hennemann et al., which the paper cites
without printing it; the reading is stated in the oracle beside or_indicator).

The elements here hold an indicator variable that is a chosen combination of
Legendre polynomials, eps = sum_j c_j L_j(2 xi - 1) (tensor products in 2D).
Gauss-Legendre quadrature on N + 1 points integrates eps L_j exactly, so the
normalised modes the indicator computes are exactly the c_j, and its energy
ratio E is known in closed form from the c_j:

  1D  E = max(c_N^2 / sum_{j<=N} c_j^2,  c_{N-1}^2 / sum_{j<=N-1} c_j^2)
  2D  E = max(energy at max(i,j) = N / all energy,
              energy at max(i,j) = N-1 / energy at max(i,j) <= N-1)

The coefficients are chosen so that the firing ratio equals T(N) (1 + delta):
alpha is 1/2 at delta = 0 whatever the sharpness, and 1/(1 + exp(-s delta))
at delta = +-0.05, which fixes the threshold T(N) = 0.5 10^(-1.8 (N+1)^(1/4)),
the sharpness s = ln((1 - 1e-4)/1e-4), the (2j+1) normalisation, both ratios
and the 2D grouping: a wrong exponent in T, a dropped next-to-top ratio, a
grouping by i + j or along x only, or unnormalised modes each move alpha
far from the expected value in one of these cases."""
import math

import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc

# Hennemann et al. (2021), the indicator the paper cites in Sec. 4: threshold
# a 10^(-c (N+1)^(1/4)) with a = 0.5, c = 1.8, and alpha = 1e-4 at E = 0.
S_SHARP = math.log((1.0 - 1e-4) / 1e-4)
T_LITERAL = {2: 2.13814e-3, 3: 1.42359e-3, 4: 1.01705e-3}  # T(N) to 6 digits


def threshold(N):
    return 0.5 * 10.0 ** (-1.8 * (N + 1) ** 0.25)


def expected_alpha(delta):
    a = 1.0 / (1.0 + math.exp(-S_SHARP * delta))
    return 0.0 if a < 1e-3 else (1.0 if a > 1.0 - 1e-3 else a)


def test_threshold_values():
    for N, t in T_LITERAL.items():
        assert abs(threshold(N) - t) < 1e-8, N
    assert abs(S_SHARP - 9.21024) < 1e-5
    assert abs(expected_alpha(0.05) - 0.61314) < 1e-5


def _leg(j, x):
    return np.polynomial.legendre.legval(2.0 * x - 1.0, [0.0] * j + [1.0])


def eps_1d(c, N):
    xi, _ = wl.gl_nodes01(N)
    return sum(cj * _leg(j, xi) for j, cj in enumerate(c))


def eps_2d(c, N):
    """c: dict {(i, j): c_ij}, i the x-mode and j the y-mode; nodes k = p + n q."""
    xi, _ = wl.gl_nodes01(N)
    n = N + 1
    out = np.zeros(n * n)
    for (i, j), cij in c.items():
        out += cij * np.kron(_leg(j, xi), _leg(i, xi))  # [q][p] flattened = p + n q
    return out


def ratio_1d(c, N):
    e = np.asarray(c, float) ** 2
    r1 = e[N] / e[:N + 1].sum()
    r2 = e[N - 1] / e[:N].sum() if N >= 2 else 0.0
    return max(r1, r2)


def ratio_2d(c, N):
    top = sum(v * v for (i, j), v in c.items() if max(i, j) == N)
    nxt = sum(v * v for (i, j), v in c.items() if max(i, j) == N - 1)
    low = sum(v * v for (i, j), v in c.items() if max(i, j) <= N - 1)
    tot = sum(v * v for v in c.values())
    return max(top / tot, nxt / low)


def _solve(r, base):
    """x^2 with x^2 / (base + x^2) = r."""
    return r * base / (1.0 - r)


def cases_1d(N, delta):
    """Coefficients c_0..c_N for: the top ratio alone, the next-to-top ratio
    alone, both present with the next-to-top one firing, both present with the
    top one firing.  The fired ratio is T (1 + delta), the other T / 2."""
    T = threshold(N)
    r, half = T * (1.0 + delta), 0.5 * T
    fill = [1.0] + [0.15] * max(0, N - 2)  # c_0 .. c_{N-2}
    S = sum(v * v for v in fill)
    out = {}
    out["top"] = fill + [0.0, math.sqrt(_solve(r, S))]
    out["next"] = fill + [math.sqrt(_solve(r, S)), 0.0]
    b2 = _solve(r, S)
    out["both_next_fires"] = fill + [math.sqrt(b2), math.sqrt(_solve(half, S + b2))]
    b2 = _solve(half, S)
    out["both_top_fires"] = fill + [math.sqrt(b2), -math.sqrt(_solve(r, S + b2))]
    return out


def cases_2d(N, delta):
    """Tensor-mode coefficients placed so that a wrong grouping changes E:
    the top group gets modes at (N-1, N) and (N, 1) (max = N, i + j > N), the
    next-to-top group at (0, N-1) and (N-1, N-1)."""
    T = threshold(N)
    r, half = T * (1.0 + delta), 0.5 * T
    fill = {(0, 0): 1.0}
    if N >= 3:
        fill[(1, 0)] = 0.15
        fill[(1, 1)] = -0.1
    S = sum(v * v for v in fill.values())
    out = {}

    def top(e2):  # split the top energy 3:1 over (N-1, N) and (N, 1)
        return {(N - 1, N): math.sqrt(0.75 * e2), (N, 1): -math.sqrt(0.25 * e2)}

    def nxt(e2):
        return {(0, N - 1): math.sqrt(0.5 * e2), (N - 1, N - 1): math.sqrt(0.5 * e2)}

    out["top"] = {**fill, **top(_solve(r, S))}
    out["next"] = {**fill, **nxt(_solve(r, S))}
    b2 = _solve(r, S)
    out["both_next_fires"] = {**fill, **nxt(b2), **top(_solve(half, S + b2))}
    b2 = _solve(half, S)
    out["both_top_fires"] = {**fill, **nxt(b2), **top(_solve(r, S + b2))}
    return out


def _state(equation, dim, eps):
    """A state whose indicator variable is eps at every node (positive where a
    density): the scalar itself; Euler with p = 1, v = 0 (eps = rho p = rho);
    ten-moment with v = 0 and p11 + p22 = 2 (eps = rho (p11 + p22)/2 = rho)."""
    one = np.ones_like(eps)
    if equation == "linadv":
        return eps[None, :]
    if equation == "euler":
        return wl.euler_conservative(eps, 0 * one, 0 * one, one, 1.4, dim)
    return wl.tenmoment_conservative(eps, 0 * one, 0 * one, 1.2 * one, 0.3 * one, 0.8 * one)


DELTAS = [-0.05, 0.0, 0.05]


@pytest.mark.parametrize("N", [2, 3, 4])
@pytest.mark.parametrize("delta", DELTAS)
def test_indicator_1d_closed_form(N, delta):
    prob = wl.base_problem(dim=1, nx=1, degree=N, equation="linadv", limiter={"blend"})
    d = oracle_desc(prob)
    for name, c in cases_1d(N, delta).items():
        assert abs(ratio_1d(c, N) / threshold(N) - (1.0 + delta)) < 1e-12, name
        ue = eps_1d(c, N)[:, None]
        a = oracle.indicator(d, ue)
        assert abs(a - expected_alpha(delta)) < 1e-9, (name, a, expected_alpha(delta))


@pytest.mark.parametrize("N", [2, 3, 4])
@pytest.mark.parametrize("delta", DELTAS)
def test_indicator_2d_closed_form(N, delta):
    prob = wl.base_problem(dim=2, nx=1, ny=1, degree=N, equation="linadv", limiter={"blend"})
    d = oracle_desc(prob)
    for name, c in cases_2d(N, delta).items():
        assert abs(ratio_2d(c, N) / threshold(N) - (1.0 + delta)) < 1e-12, name
        ue = eps_2d(c, N)[:, None]
        a = oracle.indicator(d, ue)
        assert abs(a - expected_alpha(delta)) < 1e-9, (name, a, expected_alpha(delta))


@pytest.mark.parametrize("equation,dim", [("euler", 1), ("euler", 2), ("tenmoment", 2)])
def test_indicator_variable_of_systems(equation, dim):
    """The indicator variable of Euler is rho p and of ten-moment rho (p11 + p22)/2:
    states built so that it equals the Legendre combination give the same alpha
    as the scalar case."""
    N = 3
    prob = wl.base_problem(dim=dim, nx=1, ny=1, degree=N, equation=equation, limiter={"blend"})
    d = oracle_desc(prob)
    for delta in DELTAS:
        cs = cases_1d(N, delta) if dim == 1 else cases_2d(N, delta)
        for name, c in cs.items():
            eps = eps_1d(c, N) if dim == 1 else eps_2d(c, N)
            assert eps.min() > 0.3
            ue = _state(equation, dim, eps).T.copy()
            a = oracle.indicator(d, ue)
            assert abs(a - expected_alpha(delta)) < 1e-8, (name, delta, a)


def test_indicator_saturates_beyond_the_band():
    """E = T/5 and E = 2T clip to exactly 0 and 1 (the logistic is below 1e-3
    and above 1 - 1e-3 there)."""
    for N in (2, 3, 4):
        prob = wl.base_problem(dim=1, nx=1, degree=N, equation="linadv", limiter={"blend"})
        d = oracle_desc(prob)
        for delta, want in ((-0.8, 0.0), (1.0, 1.0)):
            c = cases_1d(N, delta)["top"]
            assert oracle.indicator(d, eps_1d(c, N)[:, None]) == want


def test_modal_energies_are_the_indicator_modes():
    """The learned alpha's inputs are the same normalised modes: for the 2D
    cases every c_ij^2 / sum c^2 appears at k = i + n j."""
    N = 3
    n = N + 1
    prob = wl.base_problem(dim=2, nx=1, ny=1, degree=N, equation="linadv")
    d = oracle_desc(prob)
    c = cases_2d(N, 0.0)["both_next_fires"]
    e = oracle.modal_energies(d, eps_2d(c, N)[:, None])
    tot = sum(v * v for v in c.values())
    want = np.zeros(n * n)
    for (i, j), v in c.items():
        want[i + n * j] = v * v / tot
    np.testing.assert_allclose(e, want, rtol=0, atol=1e-15)
