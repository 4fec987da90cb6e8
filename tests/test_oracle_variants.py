"""Pins of the oracle's other dissipation models and central fluxes
(Sec. 3.1: D1 eq. (D1), D-CSX eq. (dcsx), AE eq. (extrapolate)), each against
something the paper or the mathematics fixes independently of the code:

* for linear problems D-CSX equals D2 and AE equals EA (stated in Sec. 3.1),
  also with the blending limiter acting;
* on nonlinear Euler data every combination matches an independent numpy
  restatement of the unlimited step (tests/test_oracle_pins.np_euler_ho_step,
  extended here with the variants) in 1D and 2D;
* CFL(N) for D1 from the Fourier analysis is the stability limit of the
  computed scheme (0.99 CFL bounded, 1.05 CFL blows up) and lies below the
  D2 value, as the paper states (D1 gives lower CFL numbers);
* walls with every variant still evolve like the mirror-doubled periodic
  domain.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle.cfl import cfl_number
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc
from tests.test_oracle_pins import GOLDEN, np_tables

VARIANTS = [(oracle.DISS_D1, oracle.CENTRAL_EA), (oracle.DISS_DCSX, oracle.CENTRAL_EA),
            (oracle.DISS_D2, oracle.CENTRAL_AE), (oracle.DISS_D1, oracle.CENTRAL_AE),
            (oracle.DISS_DCSX, oracle.CENTRAL_AE)]
IDS = ["D1-EA", "DCSX-EA", "D2-AE", "D1-AE", "DCSX-AE"]


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("limited", [False, True])
def test_linear_equivalences(N, dim, limited):
    if dim == 1:
        prob, u = wl.linadv_random(nx=9, degree=N, seed=N, adv=(1.3, 0.0))
    else:
        prob, u = wl.linadv_random(nx=5, ny=4, dim=2, degree=N, seed=N, adv=(0.8, -1.1))
    if limited:
        prob = dict(prob, limiter=wl.LIMITER_ALL)
    base = oracle_desc(prob)
    dt = 0.5 * oracle.dt(base, u)
    ref, st = oracle.step(base, u, dt)
    assert st == 0
    for diss, cen in [(oracle.DISS_DCSX, oracle.CENTRAL_EA), (oracle.DISS_D2, oracle.CENTRAL_AE),
                      (oracle.DISS_DCSX, oracle.CENTRAL_AE)]:
        out, st = oracle.step(oracle_desc(prob, dissipation=diss, central=cen), u, dt)
        assert st == 0
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    if not limited:  # (random data make the blending pick the low-order scheme everywhere)
        # D1 is a different scheme even for linear data
        out, _ = oracle.step(oracle_desc(prob, dissipation=oracle.DISS_D1), u, dt)
        assert np.abs(out - ref).max() > 1e-8


def np_ho_step_variant(u, N, dx, dy, dt, gamma, A, b, dim, diss, central):
    """Unlimited periodic Euler step with any dissipation/central choice, written
    with numpy array operations (a second formulation, independent of the C
    oracle).  u is [M][nx][n] (1D) or [M][ny][nx][q][p] (2D)."""
    xi, w, l0, l1, D = np_tables(N)
    s = len(b)

    def pressure(U):
        ke = 0.5 * U[1] ** 2 / U[0] if dim == 1 else 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0]
        return (gamma - 1.0) * (U[-1] - ke)

    def flux(U, direction):
        p = pressure(U)
        vn = U[1 + direction] / U[0]
        f = [U[v] * vn for v in range(U.shape[0])]
        f[1 + direction] = f[1 + direction] + p
        f[-1] = (U[-1] + p) * vn
        return np.stack(f)

    def sigma(U, direction):
        return np.abs(U[1 + direction] / U[0]) + np.sqrt(gamma * pressure(U) / U[0])

    if dim == 1:
        ax = 1   # element axis of [v][e]
        tr = lambda X, l: np.einsum("p,vep->ve", l, X)
        dX = lambda f: np.einsum("pr,ver->vep", D, f) / dx
        Ls, stages = [], []
        for i in range(s):
            ui = u - dt * sum(A[i, j] * Ls[j] for j in range(i))
            stages.append(ui)
            Ls.append(dX(flux(ui, 0)))
        F = sum(b[i] * flux(stages[i], 0) for i in range(s))
        U = sum(b[i] * stages[i] for i in range(s))
        pairs = [(tr, 0, ax, F)]
    else:
        ax = 2
        trx = lambda X, l: np.einsum("p,vyxqp->vyxq", l, X)
        try_ = lambda X, l: np.einsum("q,vyxqp->vyxp", l, X)
        dXY = lambda f, g: (np.einsum("pr,vyxqr->vyxqp", D, f) / dx +
                            np.einsum("qr,vyxrp->vyxqp", D, g) / dy)
        Ls, stages = [], []
        for i in range(s):
            ui = u - dt * sum(A[i, j] * Ls[j] for j in range(i))
            stages.append(ui)
            Ls.append(dXY(flux(ui, 0), flux(ui, 1)))
        F = sum(b[i] * flux(stages[i], 0) for i in range(s))
        G = sum(b[i] * flux(stages[i], 1) for i in range(s))
        U = sum(b[i] * stages[i] for i in range(s))
        pairs = [(trx, 0, 2, F), (try_, 1, 1, G)]
    out = u.copy()
    for tr, d, axis, Fav in pairs:
        h = dx if d == 0 else dy
        if central == oracle.CENTRAL_EA:
            cR = sum(b[i] * flux(tr(stages[i], l1), d) for i in range(s))
            cL = sum(b[i] * flux(tr(stages[i], l0), d) for i in range(s))
        else:
            cR, cL = tr(Fav, l1), tr(Fav, l0)
        nxt = lambda X: np.roll(X, -1, axis=axis)
        if diss == oracle.DISS_DCSX:
            Dv = 0.0
            for i in range(s):
                if b[i] == 0.0:
                    continue
                sR, sL = tr(stages[i], l1), nxt(tr(stages[i], l0))
                lam = np.maximum(sigma(sR, d), sigma(sL, d))
                Dv = Dv + b[i] * 0.5 * lam * (sL - sR)
        else:
            lam = np.maximum(sigma(tr(u, l1), d), sigma(nxt(tr(u, l0)), d))
            J = u if diss == oracle.DISS_D1 else U
            Dv = 0.5 * lam * (nxt(tr(J, l0)) - tr(J, l1))
        Fr = 0.5 * (cR + nxt(cL)) - Dv       # face between an element (its right) and the next
        Fl = np.roll(Fr, 1, axis=axis)
        if dim == 1:
            R = (np.einsum("pr,ver->vep", D, Fav) + (Fr - tr(Fav, l1))[..., None] * (l1 / w)
                 + (Fl - tr(Fav, l0))[..., None] * (-l0 / w))
        elif d == 0:
            R = (np.einsum("pr,vyxqr->vyxqp", D, Fav) + (Fr - tr(Fav, l1))[..., None] * (l1 / w)
                 + (Fl - tr(Fav, l0))[..., None] * (-l0 / w))
        else:
            R = (np.einsum("qr,vyxrp->vyxqp", D, Fav) + (Fr - tr(Fav, l1))[..., None, :] * (l1 / w)[:, None]
                 + (Fl - tr(Fav, l0))[..., None, :] * (-l0 / w)[:, None])
        out = out - dt / h * R
    return out


@pytest.mark.parametrize("variant", VARIANTS + [(oracle.DISS_D2, oracle.CENTRAL_EA)],
                         ids=IDS + ["D2-EA"])
@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("dim", [1, 2])
def test_variants_match_numpy_formulation(variant, N, dim):
    diss, cen = variant
    gold = json.load(open(os.path.join(GOLDEN, "crk_tableaux.json")))
    A, b = np.array(gold[str(N)]["A"]), np.array(gold[str(N)]["b"])
    if dim == 1:
        prob, u = wl.euler1d_riemann(nx=4, degree=N, seed=3, limiter=())
        prob["bc_x"] = "periodic"
        x, _ = wl.node_coords(prob)
        rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.1 * np.cos(6 * np.pi * x)
        u = wl.euler_conservative(rho, 0.5 + 0.2 * np.cos(2 * np.pi * x), None,
                                  1.0 + 0.2 * np.sin(4 * np.pi * x), 1.4, 1)
    else:
        prob, u = wl.euler2d_vortex(nx=3, ny=2, degree=N, seed=1, limiter=())
    d = oracle_desc(prob, dissipation=diss, central=cen)
    dt = 0.5 * oracle.dt(d, u)
    new, st = oracle.step(d, u, dt)
    assert st == 0
    n = N + 1
    dx = (d.x1 - d.x0) / d.nx
    dy = (d.y1 - d.y0) / d.ny if dim == 2 else 1.0
    if dim == 1:
        ref = np_ho_step_variant(u, N, dx, dy, dt, 1.4, A, b, 1, diss, cen)
    else:
        M = u.shape[0]
        ref = np_ho_step_variant(u.reshape(M, d.ny, d.nx, n, n), N, dx, dy, dt, 1.4, A, b, 2,
                                 diss, cen).reshape(u.shape)
    np.testing.assert_allclose(new, ref, rtol=1e-12, atol=1e-12 * np.abs(u).max())


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_d1_cfl_is_the_stability_limit(N):
    cfl = cfl_number(N, True)
    assert cfl < cfl_number(N)
    peaks = []
    for frac in (0.99, 1.05):
        prob, u = wl.linadv_random(nx=16, degree=N, seed=5)
        d = oracle_desc(prob, cfl=cfl * frac, cfl_safety=1.0, dissipation=oracle.DISS_D1)
        out, t, steps, st = oracle.run(d, u, 3000, 1e9)
        peaks.append(np.abs(out).max() / np.abs(u).max())
    assert peaks[0] < 1.05, peaks
    assert peaks[1] > 10.0, peaks


@pytest.mark.parametrize("variant", VARIANTS, ids=IDS)
def test_walls_with_variants_equal_mirror_doubled_periodic(variant):
    from tests.test_oracle_walls import _euler1d, _mirror_1d
    diss, cen = variant
    prob, u = _euler1d(17, 3, seed=7)
    prob = dict(prob, bc_x="wall")
    d = oracle_desc(prob, dissipation=diss, central=cen)
    dt = oracle.dt(d, u)
    pb = dict(prob, bc_x="periodic", nx=34, x1=2.0 * prob["x1"] - prob["x0"])
    db = oracle_desc(pb, dissipation=diss, central=cen)
    wall, big = u, _mirror_1d(u)
    for _ in range(2):
        wall, st = oracle.step(d, wall, dt)
        assert st == 0
        big, st = oracle.step(db, big, dt)
        assert st == 0
    for v in range(3):
        np.testing.assert_allclose(big[v, :17], wall[v], rtol=0, atol=1e-12 * np.abs(wall[v]).max())
