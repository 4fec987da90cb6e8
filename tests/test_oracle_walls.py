"""Pins of the solid-wall boundary (Sec. 3.3 eq. (reflect.time.avg)) in the
oracle, against things that hold independently of how the wall is coded:

* a domain closed by walls evolves exactly like the periodic domain of twice
  the size holding the mirror image of the data (velocity normal to the
  mirror reversed): the reflected ghost values are what the mirror element
  produces, and the indicator, the limiters and the time step are symmetric;
* in a box closed by walls on every side, mass and energy are conserved to
  round-off (no flux crosses a wall; momentum is not conserved: the walls
  push);
* a fluid at rest in a closed box stays at rest.
"""
import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc


def _euler1d(nx, N, seed):
    prob, u = wl.euler1d_riemann(nx=nx, degree=N, seed=seed)
    rng = np.random.default_rng(seed)
    # a smooth velocity and density variation on top of the two states
    x, _ = wl.node_coords(prob)
    rho, m, E = u
    f = 1.0 + 0.3 * np.sin(2 * np.pi * x + rng.uniform(0, 6.3))
    v = m / rho + 0.5 * np.cos(2 * np.pi * x)
    p = 0.4 * (E - 0.5 * m * m / rho)
    return prob, wl.euler_conservative(rho * f, v, None, p, 1.4, 1)


def _mirror_1d(u):
    """[M][ne][n] on [0, L] -> [M][2 ne][n] on [0, 2L]: element ne + i holds the
    mirror of element ne - 1 - i, nodes reversed, momentum negated."""
    m = u[:, ::-1, ::-1].copy()
    m[1] *= -1.0
    return np.concatenate([u, m], axis=1)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_wall_1d_equals_mirror_doubled_periodic(N):
    prob, u = _euler1d(23, N, seed=N)
    prob = dict(prob, bc_x="wall")
    d = oracle_desc(prob)
    dt = oracle.dt(d, u)
    wall = u
    big = _mirror_1d(u)
    pb = dict(prob, bc_x="periodic", nx=46, x1=2.0 * prob["x1"] - prob["x0"])
    db = oracle_desc(pb)
    for _ in range(3):
        wall, st = oracle.step(d, wall, dt)
        assert st == 0
        big, st = oracle.step(db, big, dt)
        assert st == 0
    for v in range(3):
        scale = np.abs(wall[v]).max()
        np.testing.assert_allclose(big[v, :23], wall[v], rtol=0, atol=1e-12 * scale)
    # and the walls were felt: an outflow domain gives something else
    out, _ = oracle.step(oracle_desc(dict(prob, bc_x="outflow")), u, dt)
    assert np.abs(out - oracle.step(d, u, dt)[0]).max() > 1e-6


def _box(nx, ny, N, seed, bcx="wall", bcy="wall"):
    prob, u = wl.euler2d_vortex_riemann(nx=nx, ny=ny, degree=N, seed=seed)
    prob = dict(prob, bc_x=bcx, bc_y=bcy)
    return prob, u


def _mirror_2d(u, nx, ny, n, axis):
    """Double a 2D state [M][ny*nx][n*n] along x (axis 0) or y (axis 1)."""
    M = u.shape[0]
    a = u.reshape(M, ny, nx, n, n)             # [v][iy][ix][q][p]
    if axis == 0:
        m = a[:, :, ::-1, :, ::-1].copy()
        m[1] *= -1.0
        b = np.concatenate([a, m], axis=2)
        return b.reshape(M, ny * 2 * nx, n * n)
    m = a[:, ::-1, :, ::-1, :].copy()
    m[2] *= -1.0
    b = np.concatenate([a, m], axis=1)
    return b.reshape(M, 2 * ny * nx, n * n)


@pytest.mark.parametrize("N,axis", [(3, 0), (4, 1), (2, 0)])
def test_wall_2d_equals_mirror_doubled_periodic(N, axis):
    nx, ny, n = 9, 7, N + 1
    prob, u = _box(nx, ny, N, seed=10 + N, bcx="wall" if axis == 0 else "periodic",
                   bcy="wall" if axis == 1 else "periodic")
    d = oracle_desc(prob)
    dt = oracle.dt(d, u)
    big = _mirror_2d(u, nx, ny, n, axis)
    if axis == 0:
        pb = dict(prob, bc_x="periodic", nx=2 * nx, x1=2 * prob["x1"] - prob["x0"])
    else:
        pb = dict(prob, bc_y="periodic", ny=2 * ny, y1=2 * prob["y1"] - prob["y0"])
    db = oracle_desc(pb)
    wall, st = oracle.step(d, u, dt)
    assert st == 0
    big, st = oracle.step(db, big, dt)
    assert st == 0
    M = u.shape[0]
    if axis == 0:
        half = big.reshape(M, ny, 2 * nx, n * n)[:, :, :nx].reshape(M, ny * nx, n * n)
    else:
        half = big[:, : ny * nx]
    for v in range(M):
        np.testing.assert_allclose(half[v], wall[v], rtol=0, atol=1e-12 * np.abs(wall[v]).max())


def test_closed_box_conserves_mass_and_energy():
    prob, u = _box(10, 8, 3, seed=3)
    d = oracle_desc(prob)
    tot0 = oracle.element_means(d, u).sum(axis=1)
    w = u
    for _ in range(4):
        w, st = oracle.step(d, w, oracle.dt(d, w))
        assert st == 0
    tot = oracle.element_means(d, w).sum(axis=1)
    for v in (0, 3):
        assert abs(tot[v] - tot0[v]) <= 1e-13 * abs(tot0[v])
    assert abs(tot[1] - tot0[1]) > 1e-8 * abs(tot0[3])  # the walls push


def test_fluid_at_rest_stays_at_rest():
    prob, _ = _box(6, 5, 4, seed=0)
    u = wl.uniform_state(prob, (1.3, 0.0, 0.0, 2.5))
    d = oracle_desc(prob)
    w, st = oracle.step(d, u, 1e-3)
    assert st == 0
    np.testing.assert_allclose(w, u, rtol=0, atol=1e-14 * np.abs(u).max())
