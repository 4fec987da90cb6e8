"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle,
element by element on the same seeded inputs.

Tolerance (FP64 mode, the stated 1e-12 relative bar): for every variable v,
|gpu - oracle| <= 1e-12 * max(max |oracle_v|, flux increment of v), where the
flux increment is dt/dx max |F_v| + dt/dy max |G_v| over the oracle's face
fluxes (one-step checks).  The second term matters only for a variable that is
near zero but driven by O(1) fluxes (e.g. rho v2 in 1D ten-moment, moved by
p12): its absolute rounding is set by the flux size, not by its own size.
"""
import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_07517_gb300 import build
    build.build()


def assert_parity(g, o, rtol=RTOL, what="", extra_scale=None):
    assert g.shape == o.shape
    assert np.all(np.isfinite(g)), what
    for v in range(o.shape[0]):
        scale = np.abs(o[v]).max()
        if extra_scale is not None:
            scale = max(scale, extra_scale[v])
        err = np.abs(g[v] - o[v]).max()
        assert err <= rtol * max(scale, 1e-300), (what, v, err, scale, err / max(scale, 1e-300))


def gpu_run(prob, u, dt_fixed=0.0, nsteps=1, t_final=1e300, alpha_fixed=None,
            precision=crkfr.CR_FP64, **over):
    d = crkfr.desc_from_problem(prob, precision=precision, alpha_fixed=alpha_fixed, **over)
    ctx = crkfr.cr_init_mesh(d)
    crkfr.cr_set_state(ctx, u)
    t, n = crkfr.cr_step(ctx, nsteps, t_final, dt_fixed)
    out = crkfr.cr_get_state(ctx, shape=u.shape)
    alpha = crkfr.cr_get_alpha(ctx, u.shape[1])
    return out, alpha, t, n, ctx


def one_step_check(prob, u, alpha_fixed=None, over_oracle=None, over_gpu=None, frac=1.0):
    d = oracle_desc(prob, alpha_fixed=alpha_fixed, **(over_oracle or {}))
    dt = frac * oracle.dt(d, u)
    ref, st, dg = oracle.step(d, u, dt, want_diag=True)
    assert st == 0
    g, alpha, t, n, ctx = gpu_run(prob, u, dt_fixed=dt, alpha_fixed=alpha_fixed, **(over_gpu or {}))
    assert n == 1 and abs(t - dt) <= 1e-15 * dt
    assert_parity(g, ref, extra_scale=flux_increment(prob, dg, dt))
    np.testing.assert_allclose(alpha, dg["alpha"], rtol=0, atol=1e-12)
    return g, ref


def flux_increment(prob, dg, dt):
    dx = (prob["x1"] - prob["x0"]) / prob["nx"]
    inc = dt / dx * np.abs(dg["fnum_x"]).max(axis=(1, 2))
    if prob["dim"] == 2:
        dy = (prob["y1"] - prob["y0"]) / prob["ny"]
        inc = inc + dt / dy * np.abs(dg["fnum_y"]).max(axis=(1, 2))
    return inc


def _jumpy_2d(nx, ny, N, seed):
    prob, u = wl.euler2d_vortex(nx=nx, ny=ny, degree=N, seed=seed, perturb=0.01)
    rng = np.random.default_rng(seed)
    return prob, u * rng.uniform(0.5, 2.0, (1, nx * ny, 1))


# ------------------------------------------------------------ linear ------
def test_linear_advection_full_horizon():
    """64 elements, N = 3, CFL step, to t = 1 (last step clipped): same step count,
    same final time, same state as the oracle; optimal accuracy vs the exact solution."""
    prob, u = wl.linadv_sine(nx=64, degree=3, t_final=1.0)
    d = oracle_desc(prob)
    ref, t_o, n_o, st = oracle.run(d, u, 100000, 1.0)
    g, _, t_g, n_g, _ = gpu_run(prob, u, nsteps=100000, t_final=1.0)
    assert st == 0 and n_g == n_o and t_g == t_o == 1.0
    assert_parity(g, ref, rtol=1e-11)
    x, _ = wl.node_coords(prob)
    assert np.abs(g[0] - np.sin(2 * np.pi * (x - 1.0))).max() < 1e-6


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("bc", ["periodic", "outflow"])
@pytest.mark.parametrize("a", [1.0, -0.6])
def test_linear_advection_1d(N, bc, a):
    prob, u = wl.linadv_random(nx=37, degree=N, seed=N, adv=(a, 0.0), bc=bc)
    one_step_check(prob, u)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_linear_advection_2d(N):
    prob, u = wl.linadv_random(nx=11, ny=7, dim=2, degree=N, seed=3, adv=(0.7, -1.2))
    one_step_check(prob, u)


# ------------------------------------------------------------ Euler -------
@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("seed", [0, 1])
def test_euler1d_riemann_one_step(N, seed):
    prob, u = wl.euler1d_riemann(nx=53, degree=N, seed=seed)
    one_step_check(prob, u)


def test_euler1d_riemann_trajectory():
    """Shock case: per-step parity along the oracle trajectory (40 steps)."""
    prob, u = wl.euler1d_riemann(nx=200, degree=4, seed=3)
    d = oracle_desc(prob)
    dgpu = crkfr.desc_from_problem(prob)
    ctx = crkfr.cr_init_mesh(dgpu)
    for _ in range(40):
        dt = oracle.dt(d, u)
        ref, st = oracle.step(d, u, dt)
        assert st == 0
        crkfr.cr_set_state(ctx, u)
        assert abs(crkfr.cr_next_dt(ctx) - dt) <= 1e-14 * dt
        crkfr.cr_step(ctx, 1, 1e300, dt)
        g = crkfr.cr_get_state(ctx, shape=u.shape)
        assert_parity(g, ref)
        u = ref


@pytest.mark.parametrize("N", [3, 4])
def test_euler2d_vortex_multi_step(N):
    """Smooth case: 12 CFL steps on the GPU against 12 oracle steps."""
    prob, u = wl.euler2d_vortex(nx=14, ny=12, degree=N, seed=2)
    d = oracle_desc(prob)
    ref = u
    for _ in range(12):
        ref, st = oracle.step(d, ref, oracle.dt(d, ref))
        assert st == 0
    g, _, t, n, _ = gpu_run(prob, u, nsteps=12)
    assert n == 12
    assert_parity(g, ref, rtol=1e-11)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_euler2d_limited_one_step(N, bc):
    prob, u = _jumpy_2d(13, 11, N, seed=N)
    prob["bc_x"] = prob["bc_y"] = bc
    one_step_check(prob, u)


@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("mh", [True, False])
def test_euler2d_fixed_alpha(alpha, mh):
    prob, u = _jumpy_2d(9, 10, 3, seed=7)
    lim = {"mh", "flux", "scaling", "traces"} if mh else {"flux", "scaling", "traces"}
    prob["limiter"] = frozenset(lim)
    one_step_check(prob, u, alpha_fixed=alpha)


# ------------------------------------------------------- ten-moment -------
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_tenmoment2d_source_one_step(N):
    prob, u = wl.tenmoment2d_voronoi(nx=9, ny=7, degree=N, seed=N)
    one_step_check(prob, u)


def test_tenmoment2d_trajectory():
    prob, u = wl.tenmoment2d_voronoi(nx=12, ny=10, degree=3, seed=5)
    d = oracle_desc(prob)
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
    for _ in range(8):
        dt = oracle.dt(d, u)
        ref, st = oracle.step(d, u, dt)
        assert st == 0
        crkfr.cr_set_state(ctx, u)
        crkfr.cr_step(ctx, 1, 1e300, dt)
        assert_parity(crkfr.cr_get_state(ctx, shape=u.shape), ref)
        u = ref


@pytest.mark.parametrize("N", [3, 4])
def test_tenmoment1d(N):
    prob = wl.base_problem(dim=1, nx=41, degree=N, equation="tenmoment", bc_x="outflow",
                           limiter=wl.LIMITER_ALL, source=dict(amp=25.0, k=200.0, cx=0.4, cy=0.0))
    x, _ = wl.node_coords(prob)
    xc, _ = wl.element_centres(prob)
    left = np.broadcast_to((xc < 0.5)[:, None], x.shape)
    one = np.ones_like(x)
    u = wl.tenmoment_conservative(one, np.where(left, -1.0, 1.0), 0 * one, 9 * one, 7 * one, 9 * one)
    one_step_check(prob, u)


# ----------------------------------------------------- edge cases ---------
def test_single_element_and_single_row():
    prob, u = wl.euler1d_riemann(nx=1, degree=4, seed=0)
    prob["bc_x"] = "periodic"
    one_step_check(prob, u)
    prob, u = _jumpy_2d(17, 1, 3, seed=1)
    one_step_check(prob, u)


def test_invalid_state_rejected():
    prob, u = wl.euler1d_riemann(nx=20, degree=3, seed=0)
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
    bad = u.copy()
    bad[0, 7, 2] = -1.0
    with pytest.raises(crkfr.CrError) as ei:
        crkfr.cr_set_state(ctx, bad)
    assert ei.value.status == -2
    bad = u.copy()
    bad[2, 3, 1] = np.nan
    with pytest.raises(crkfr.CrError):
        crkfr.cr_set_state(ctx, bad)
    crkfr.cr_set_state(ctx, u)  # the context stays usable
    # an equation without admissibility constraints still refuses non-finite input
    prob, u = wl.linadv_random(nx=9, degree=2, seed=1)
    for value in (np.nan, np.inf):
        ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
        bad = u.copy()
        bad[0, 4, 1] = value
        with pytest.raises(crkfr.CrError) as ei:
            crkfr.cr_set_state(ctx, bad)
        assert ei.value.status == -2
        crkfr.cr_set_state(ctx, u)


def test_inadmissible_step_reported_like_the_oracle():
    """Pure high order (alpha = 0) without the flux limiter on two strong
    rarefactions: the oracle reports an inadmissible mean at some step; the
    library returns CR_E_INADMISSIBLE at the same step."""
    prob = wl.base_problem(dim=1, nx=50, degree=3, equation="euler", bc_x="outflow",
                           limiter={"mh", "scaling", "traces"})
    x, _ = wl.node_coords(prob)
    xc, _ = wl.element_centres(prob)
    left = np.broadcast_to((xc < 0.5)[:, None], x.shape)
    one = np.ones_like(x)
    u = wl.euler_conservative(one, np.where(left, -6.0, 6.0), None, 0.02 * one, 1.4, 1)
    d = oracle_desc(prob, alpha_fixed=0.0)
    _, t, steps, st = oracle.run(d, u, 300, 1e9)
    assert st == 1
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, alpha_fixed=0.0))
    crkfr.cr_set_state(ctx, u)
    with pytest.raises(crkfr.CrError) as ei:
        crkfr.cr_step(ctx, 300, 1e9)
    assert ei.value.status == -3
    import ctypes
    tt, nn = ctypes.c_double(), ctypes.c_int()
    assert crkfr.lib().cr_sync(ctx.handle, ctypes.byref(tt), ctypes.byref(nn)) == -3
    assert nn.value == steps


def test_clipped_final_step_and_dt():
    prob, u = wl.euler1d_riemann(nx=100, degree=4, seed=2, t_final=1e-3)
    d = oracle_desc(prob)
    ref, t_o, n_o, st = oracle.run(d, u, 1000, 1e-3)
    g, _, t_g, n_g, ctx = gpu_run(prob, u, nsteps=1000, t_final=1e-3)
    assert st == 0 and n_g == n_o and t_g == t_o == 1e-3
    assert_parity(g, ref, rtol=1e-11)
    # a further call does nothing once t_final is reached
    t2, n2 = crkfr.cr_step(ctx, 5, 1e-3)
    assert n2 == n_g and t2 == t_g


# ------------------------------------------------ full-size workloads -----
def test_euler2d_512_one_step_full_size():
    """2D Euler vortex + 1% perturbation, N = 4, 512 x 512, all limiters, the CFL step
    (the benchmark's workload and launch configuration): every output value."""
    prob, u = wl.euler2d_vortex(nx=512, degree=4, seed=0)
    d = oracle_desc(prob)
    dt = oracle.dt(d, u)
    ref, st = oracle.step(d, u, dt)
    assert st == 0
    g, _, t, n, ctx = gpu_run(prob, u, nsteps=1)
    assert n == 1 and abs(t - dt) <= 1e-14 * dt
    assert_parity(g, ref)


def test_tenmoment_256_one_step_full_size():
    prob, u = wl.tenmoment2d_voronoi(nx=256, degree=3, seed=0)
    one_step_check(prob, u)


def test_euler1d_4000_full_size():
    prob, u = wl.euler1d_riemann(nx=4000, degree=4, seed=0)
    one_step_check(prob, u)


def test_checkpoint_resume_is_bitwise():
    """cr_get_state / cr_set_state are a checkpoint: 3 + 3 steps through a fresh
    context equal 6 steps in one run, bit for bit (FP64, limiters acting)."""
    prob, u = _jumpy_2d(11, 9, 4, seed=9)
    d = crkfr.desc_from_problem(prob)
    a = crkfr.cr_init_mesh(d)
    crkfr.cr_set_state(a, u)
    crkfr.cr_step(a, 6, 1e300)
    full = crkfr.cr_get_state(a, shape=u.shape)
    b = crkfr.cr_init_mesh(d)
    crkfr.cr_set_state(b, u)
    crkfr.cr_step(b, 3, 1e300)
    mid = crkfr.cr_get_state(b, shape=u.shape)
    c = crkfr.cr_init_mesh(d)
    crkfr.cr_set_state(c, mid)
    crkfr.cr_step(c, 3, 1e300)
    np.testing.assert_array_equal(crkfr.cr_get_state(c, shape=u.shape), full)


# ------------------------------------------------------- solid walls ------
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_euler1d_walls_one_step(N):
    from tests.test_oracle_walls import _euler1d
    prob, u = _euler1d(31, N, seed=20 + N)
    one_step_check(dict(prob, bc_x="wall"), u)


@pytest.mark.parametrize("bcx,bcy", [("wall", "periodic"), ("periodic", "wall"), ("wall", "wall"),
                                     ("wall", "outflow")])
@pytest.mark.parametrize("N", [3, 4])
def test_euler2d_walls_one_step(N, bcx, bcy):
    prob, u = _jumpy_2d(12, 10, N, seed=30 + N)
    prob = dict(prob, bc_x=bcx, bc_y=bcy)
    one_step_check(prob, u)


def test_euler1d_walls_trajectory():
    """A Riemann problem between two walls: per-step parity along the oracle
    trajectory while the waves reflect off the walls (40 steps)."""
    from tests.test_oracle_walls import _euler1d
    prob, u = _euler1d(60, 4, seed=3)
    prob = dict(prob, bc_x="wall")
    d = oracle_desc(prob)
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
    for _ in range(40):
        dt = oracle.dt(d, u)
        ref, st = oracle.step(d, u, dt)
        assert st == 0
        crkfr.cr_set_state(ctx, u)
        crkfr.cr_step(ctx, 1, 1e300, dt)
        assert_parity(crkfr.cr_get_state(ctx, shape=u.shape), ref)
        u = ref


def test_walls_refused_for_other_equations():
    prob, u = wl.tenmoment2d_voronoi(nx=6, ny=5, degree=3, seed=0)
    with pytest.raises(crkfr.CrError) as ei:
        crkfr.cr_workspace_bytes(crkfr.desc_from_problem(dict(prob, bc_x="wall")))
    assert ei.value.status == -1


# ------------------------------------- dissipation models and central flux ------
VARIANTS = [(1, 0), (2, 0), (0, 1), (1, 1), (2, 1)]   # (dissipation, central): D1/D-CSX, AE
VIDS = ["D1-EA", "DCSX-EA", "D2-AE", "D1-AE", "DCSX-AE"]


def _variant_case(case):
    if case == "euler1d_outflow":
        return wl.euler1d_riemann(nx=41, degree=4, seed=4)
    if case == "euler2d_periodic":
        return _jumpy_2d(11, 9, 4, seed=5)
    if case == "euler2d_walls_N3":
        prob, u = _jumpy_2d(10, 8, 3, seed=6)
        return dict(prob, bc_x="wall", bc_y="outflow"), u
    if case == "tenmoment_N3":
        return wl.tenmoment2d_voronoi(nx=9, ny=7, degree=3, seed=3)
    return wl.linadv_random(nx=9, ny=7, dim=2, degree=3, seed=3, adv=(0.7, -1.2))


@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
@pytest.mark.parametrize("case", ["euler1d_outflow", "euler2d_periodic", "euler2d_walls_N3",
                                  "tenmoment_N3", "linadv2d"])
def test_variants_one_step(variant, case):
    diss, cen = variant
    prob, u = _variant_case(case)
    over = dict(dissipation=diss, central=cen)
    one_step_check(prob, u, over_oracle=over, over_gpu=over)


def test_d1_multi_step():
    """D1 over 12 CFL steps (its own, smaller CFL number) against 12 oracle steps."""
    from oracle.cfl import cfl_number
    prob, u = wl.euler2d_vortex(nx=12, ny=10, degree=4, seed=2)
    cfl = cfl_number(4, True)
    d = oracle_desc(prob, dissipation=1, cfl=cfl)
    ref = u
    for _ in range(12):
        ref, st = oracle.step(d, ref, oracle.dt(d, ref))
        assert st == 0
    g, _, t, n, _ = gpu_run(prob, u, nsteps=12, dissipation=1, cfl=cfl)
    assert n == 12
    assert_parity(g, ref, rtol=1e-11)
