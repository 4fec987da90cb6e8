"""CFL(N) of Sec. 5 eq. (time.step.2d) by Fourier (von Neumann) analysis.

TEST INFRASTRUCTURE ONLY (part of the oracle).

The paper takes CFL(N) from the Fourier stability analysis of the linearly
equivalent Lax-Wendroff FR scheme (cited, not printed).  Reading: analyse the
cRKFR scheme itself on u_t + u_x = 0, periodic, with D2 dissipation (also
D-CSX, equivalent to D2 for linear problems) or with D1.  For a
linear flux the time averages are exact (App. A eq. (linear.avg)):
    U_e = T u_e,  T = sum_{m=0}^{N} (-nu)^m / (m+1)! D^m,  F = U,
with nu = dt/dx.  D2 gives the upwind flux F_{e+1/2} = l(1)^T U_e, so eq.
(crkfr.avg) becomes
    u_e^{n+1} = u_e - nu [ D T u_e + g_L' (l(1)^T T u_{e-1} - l(0)^T T u_e) ],
and a Fourier mode u_{e-1} = exp(-i k) u_e gives the amplification matrix
    G(k) = I - nu [ D T - g_L' l(0)^T T + exp(-i k) g_L' l(1)^T T ].
D1 (eq. (D1)) takes the jump of the u^n traces instead of the time-averaged
ones, F_{e+1/2} = (l(1)^T T u_e + l(0)^T T u_{e+1})/2 - (l(0)^T u_{e+1} -
l(1)^T u_e)/2, which is no longer upwind; in general, with V = T (D2) or
V = I (D1) and the correction derivatives g_L', g_R' at the solution points
(Radau with Gauss-Legendre points, g2 with Gauss-Lobatto points),
    G(k) = I - nu [ A_0 + exp(i k) A_+ + exp(-i k) A_- ],
    A_0 = D T + g_R' (l(1)^T V - l(1)^T T)/2 - g_L' (l(0)^T T + l(0)^T V)/2,
    A_+ = g_R' (l(0)^T T - l(0)^T V)/2,   A_- = g_L' (l(1)^T T + l(1)^T V)/2.
CFL(N) is the largest nu with spectral radius rho(G(k)) <= 1 + tol for all k,
found by bisection on a grid of wave numbers that contains k = pi.

Reading of the tolerance: for N = 4 the fifth-order time average has a weak
growth of about 5e-6 per step at mid wave numbers for every nu (it does not
grow with nu up to 0.069), while the genuine instability at k = pi jumps to
5e-3 within 0.001 of its onset.  tol = 1e-4 sits between the two, so the
result is the onset of the genuine instability; for N = 1..3 there is no weak
growth and tol raises the result by less than 2e-5 over the exact limit.
"""
import functools
import math

import numpy as np

from . import tables_corr


def amplification(N, nu, k, d1=False, points=0):
    xi, w, l0, l1, D, gL, gR = tables_corr(N, points)
    n = N + 1
    T = np.zeros((n, n))
    Dm = np.eye(n)
    for m in range(N + 1):
        T += (-nu) ** m / math.factorial(m + 1) * Dm
        Dm = Dm @ D
    V = np.eye(n) if d1 else T
    A0 = D @ T + 0.5 * np.outer(gR, l1 @ V - l1 @ T) - 0.5 * np.outer(gL, l0 @ T + l0 @ V)
    Ap = 0.5 * np.outer(gR, l0 @ T - l0 @ V)
    Am = 0.5 * np.outer(gL, l1 @ T + l1 @ V)
    return np.eye(n) - nu * (A0 + np.exp(1j * k) * Ap + np.exp(-1j * k) * Am)


def max_growth(N, nu, nk=721, d1=False, points=0):
    ks = np.linspace(0.0, 2.0 * np.pi, nk)
    return max(np.max(np.abs(np.linalg.eigvals(amplification(N, nu, k, d1, points)))) for k in ks)


@functools.lru_cache(maxsize=None)
def cfl_number(N, d1=False, tol=1e-4, iters=40, points=0):
    """CFL(N) for D2 (and D-CSX), or for D1 when d1 is true; Gauss-Legendre
    points with Radau correction (points 0) or Gauss-Lobatto with g2 (1)."""
    lo, hi = 0.0, 1.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if max_growth(N, mid, d1=d1, points=points) <= 1.0 + tol:
            lo = mid
        else:
            hi = mid
    return lo
