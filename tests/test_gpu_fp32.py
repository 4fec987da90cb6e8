"""FP32_BULK mode: FP32 stage arithmetic with FP64 element means (eq. (upmean)
in FP64), FP64 flux-limiter and scaling-limiter theta.  Checked against the
FP64 oracle by the normalised L1 difference per variable, plus properties that
hold exactly: totals of the FP64 element means are conserved to FP64 round-off,
every point admissible."""
import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc

pytestmark = pytest.mark.gpu

# stated L1 bounds (normalised by the L1 norm of each variable's oracle value)
L1_ONE_STEP = 2e-7
L1_MULTI_STEP = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_07517_gb300 import build
    build.build()


def l1_rel(g, o):
    return np.array([np.abs(g[v] - o[v]).sum() / max(np.abs(o[v]).sum(), 1e-300)
                     for v in range(o.shape[0])])


def run32(prob, u, nsteps=1, dt_fixed=0.0, want_means=False):
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, precision=crkfr.CR_FP32_BULK))
    crkfr.cr_set_state(ctx, u)
    m0 = crkfr.cr_get_means(ctx, u.shape[0], u.shape[1])
    t, n = crkfr.cr_step(ctx, nsteps, 1e300, dt_fixed)
    g = crkfr.cr_get_state(ctx, shape=u.shape)
    if want_means:
        return g, t, n, m0, crkfr.cr_get_means(ctx, u.shape[0], u.shape[1])
    return g, t, n


@pytest.mark.parametrize("case", ["vortex4", "vortex3", "jumpy4", "riemann1d", "tenmoment"])
def test_fp32_one_step(case):
    if case.startswith("vortex"):
        prob, u = wl.euler2d_vortex(nx=24, ny=20, degree=int(case[-1]), seed=1)
    elif case == "jumpy4":
        prob, u = wl.euler2d_vortex(nx=16, ny=14, degree=4, seed=2)
        u = u * np.random.default_rng(2).uniform(0.5, 2.0, (1, u.shape[1], 1))
    elif case == "riemann1d":
        prob, u = wl.euler1d_riemann(nx=400, degree=4, seed=1)
    else:
        prob, u = wl.tenmoment2d_voronoi(nx=16, ny=12, degree=3, seed=1)
    d = oracle_desc(prob)
    dt = oracle.dt(d, u)
    ref, st = oracle.step(d, u, dt)
    assert st == 0
    g, t, n, m0, m1 = run32(prob, u, 1, dt, want_means=True)
    err = l1_rel(g, ref)
    print(case, "L1 rel", err)
    assert np.all(err < L1_ONE_STEP), err
    if prob["bc_x"] == "periodic" and prob.get("source") is None:
        t0, t1 = m0.sum(axis=1), m1.sum(axis=1)
        np.testing.assert_allclose(t1, t0, rtol=1e-13, atol=1e-13 * np.abs(t0).max())


def test_fp32_vortex_multi_step_conservative_and_admissible():
    prob, u = wl.euler2d_vortex(nx=32, ny=32, degree=4, seed=3)
    d = oracle_desc(prob)
    ref = u
    for _ in range(20):
        ref, st = oracle.step(d, ref, oracle.dt(d, ref))
    g, t, n, m0, m1 = run32(prob, u, 20, want_means=True)
    assert n == 20
    err = l1_rel(g, ref)
    print("20 steps L1 rel", err)
    assert np.all(err < L1_MULTI_STEP), err
    t0, t1 = m0.sum(axis=1), m1.sum(axis=1)
    np.testing.assert_allclose(t1, t0, rtol=1e-13, atol=1e-13 * np.abs(t0).max())
    rho = g[0]
    p = 0.4 * (g[3] - 0.5 * (g[1] ** 2 + g[2] ** 2) / g[0])
    assert rho.min() > 0 and p.min() > 0


@pytest.mark.parametrize("bcx,bcy", [("wall", "wall"), ("wall", "periodic"), ("periodic", "wall")])
def test_fp32_walls_conserve_and_match(bcx, bcy):
    """FP32 bulk with solid walls: L1 against the FP64 oracle, and mass and
    energy of the FP64 means conserved to FP64 round-off (no flux crosses a
    wall, interior face fluxes telescope)."""
    prob, u = wl.euler2d_vortex_riemann(nx=14, ny=12, degree=4, seed=5)
    prob = dict(prob, bc_x=bcx, bc_y=bcy)
    d = oracle_desc(prob)
    ref = u
    for _ in range(5):
        ref, st = oracle.step(d, ref, oracle.dt(d, ref))
        assert st == 0
    g, t, n, m0, m1 = run32(prob, u, 5, want_means=True)
    assert n == 5
    err = l1_rel(g, ref)
    assert np.all(err < L1_MULTI_STEP), err
    t0, t1 = m0.sum(axis=1), m1.sum(axis=1)
    for v in (0, 3):
        assert abs(t1[v] - t0[v]) <= 1e-13 * abs(t0[v]), (v, t1[v] - t0[v])


@pytest.mark.parametrize("diss,cen", [(1, 0), (2, 0), (0, 1), (2, 1)])
def test_fp32_variants_one_step(diss, cen):
    prob, u = wl.euler2d_vortex(nx=16, ny=14, degree=4, seed=2)
    u = u * np.random.default_rng(2).uniform(0.5, 2.0, (1, u.shape[1], 1))
    d = oracle_desc(prob, dissipation=diss, central=cen)
    dt = oracle.dt(d, u)
    ref, st = oracle.step(d, u, dt)
    assert st == 0
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, precision=crkfr.CR_FP32_BULK,
                                                     dissipation=diss, central=cen))
    crkfr.cr_set_state(ctx, u)
    crkfr.cr_step(ctx, 1, 1e300, dt)
    err = l1_rel(crkfr.cr_get_state(ctx, shape=u.shape), ref)
    assert np.all(err < L1_ONE_STEP), err
