"""GPU parity for the given-state boundaries (Sec. 3.3: Dirichlet ghost
values and the fully-inflow rule, per side) and the Euler gravity source
(Sec. 5.5), through the C ABI, against the FP64 oracle at the 1e-12 bar of
tests/test_gpu_parity.py; the Rayleigh-Taylor workload (walls in x, given
states at the bottom and top, gravity) along the oracle trajectory and run to
t = 2.5 on the GPU in FP64 and FP32 bulk; batches with these boundaries equal
single-problem steps bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc
from tests.test_gpu_parity import assert_parity, flux_increment, gpu_run, one_step_check
from tests.test_gpu_fp32 import L1_ONE_STEP, l1_rel, run32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_07517_gb300 import build
    build.build()


def _cons(rho, v1, v2, p, g=1.4):
    return [float(x) for x in wl.euler_conservative(np.array(rho), np.array(v1), np.array(v2),
                                                     np.array(p), g, 2)]


def _mixed_2d(N, seed):
    """2D Euler vortex-plus-jump data with all four side kinds: inflow at x-,
    outflow at x+, Dirichlet at y-, wall at y+."""
    prob, u = wl.euler2d_vortex_riemann(nx=13, ny=11, degree=N, seed=seed)
    prob = dict(prob, bc_x="outflow", bc_y="outflow",
                bc_side={"x-": "inflow", "x+": "outflow", "y-": "dirichlet", "y+": "wall"},
                bc_state={"x-": _cons(1.2, 2.5, 0.3, 1.1), "y-": _cons(0.8, -0.4, 0.6, 2.0)})
    return prob, u


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("seed", [0, 1])
def test_mixed_sides_one_step(N, seed):
    prob, u = _mixed_2d(N, seed)
    one_step_check(prob, u)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_euler1d_dirichlet_and_inflow_one_step(N):
    prob, u = wl.euler1d_riemann(nx=41, degree=N, seed=N)
    g = [1.1, 1.1 * 0.3, 2.0 / 0.4 + 0.5 * 1.1 * 0.09]
    one_step_check(dict(prob, bc_x="dirichlet", bc_state={"x-": g, "x+": g}), u)
    one_step_check(dict(prob, bc_side={"x-": "inflow"}, bc_state={"x-": g}), u)


@pytest.mark.parametrize("N", [1, 3])
def test_linear_advection_and_tenmoment_ghost_states(N):
    prob, u = wl.linadv_random(nx=23, degree=N, seed=4, adv=(1.3, 0.0), bc="outflow")
    one_step_check(dict(prob, bc_side={"x-": "inflow"}, bc_state={"x-": [0.4]}), u)
    one_step_check(dict(prob, bc_x="dirichlet", bc_state={"x-": [0.4], "x+": [-1.0]}), u)
    prob, u = wl.tenmoment2d_voronoi(nx=9, ny=7, degree=N, seed=N)
    gs = [float(x) for x in wl.tenmoment_conservative(np.array(1.5), np.array(0.2), np.array(-0.1),
                                                        np.array(2.0), np.array(0.3), np.array(1.0))]
    one_step_check(dict(prob, bc_x="dirichlet", bc_y="outflow",
                        bc_state={"x-": gs, "x+": gs}), u)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_hllc_sides_one_step(N):
    prob, u = _mixed_2d(N, 4)
    prob = dict(prob, bc_flux="hllc",
                bc_side={"x-": "dirichlet", "x+": "outflow", "y-": "dirichlet", "y+": "dirichlet"},
                bc_state={"x-": _cons(1.2, 2.5, 0.3, 1.1), "y-": _cons(0.8, -0.4, 0.6, 2.0),
                          "y+": _cons(2.0, 0.1, -0.9, 4.0)})
    one_step_check(prob, u)
    prob1, u1 = wl.euler1d_riemann(nx=31, degree=N, seed=N + 3)
    g = [1.1, 1.1 * 0.3, 2.0 / 0.4 + 0.5 * 1.1 * 0.09]
    one_step_check(dict(prob1, bc_x="dirichlet", bc_flux="hllc", bc_state={"x-": g, "x+": g}), u1)


def test_hllc_contact_at_rest_on_the_gpu():
    prob = wl.base_problem(dim=1, nx=10, degree=3, equation="euler", limiter=wl.LIMITER_ALL,
                           bc_x="dirichlet", bc_flux="hllc")
    u = wl.uniform_state(prob, (1.0, 0.0, 1.0))
    g = [3.0, 0.0, 1.0 / 0.4]
    prob["bc_state"] = {"x-": g, "x+": g}
    out, _, t, n, _ = gpu_run(prob, u, dt_fixed=1e-3)
    np.testing.assert_allclose(out, u, rtol=0, atol=1e-15)


@pytest.mark.parametrize("diss,cen", [(1, 0), (2, 0), (0, 1), (2, 1)])
def test_variants_with_ghost_states(diss, cen):
    prob, u = _mixed_2d(3, 5)
    over = dict(dissipation=diss, central=cen)
    one_step_check(prob, u, over_oracle=over, over_gpu=over)


@pytest.mark.parametrize("dim", [1, 2])
def test_gravity_one_step_and_closed_form(dim):
    if dim == 2:
        prob, u = wl.rayleigh_taylor(nx=8, ny=32, degree=3)
        one_step_check(prob, u)
    prob = wl.base_problem(dim=dim, nx=6, ny=5, degree=4, equation="euler",
                           source=dict(gravity=(0.7, -1.3) if dim == 2 else (-1.1, 0.0)))
    prim = (1.6, 0.4, -0.2, 2.0) if dim == 2 else (1.6, 0.4, 2.0)
    u = wl.uniform_state(prob, prim)
    d = oracle_desc(prob)
    dt = 0.8 * oracle.dt(d, u)
    g, _, t, n, _ = gpu_run(prob, u, dt_fixed=dt)
    gv = np.array(prob["source"]["gravity"][:dim])
    rho, m0, E0 = u[0, 0, 0], u[1:1 + dim, 0, 0], u[-1, 0, 0]
    scale = np.abs(u).max()
    np.testing.assert_allclose(g[0], rho, rtol=0, atol=1e-15 * scale)
    for i in range(dim):
        np.testing.assert_allclose(g[1 + i], m0[i] + rho * gv[i] * dt, rtol=0, atol=1e-14 * scale)
    np.testing.assert_allclose(g[-1], E0 + gv @ m0 * dt + 0.5 * rho * (gv @ gv) * dt * dt,
                               rtol=0, atol=1e-14 * scale)


def test_rayleigh_taylor_trajectory():
    prob, u = wl.rayleigh_taylor(nx=16, ny=64, degree=3)
    d = oracle_desc(prob)
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
    for _ in range(20):
        dt = oracle.dt(d, u)
        ref, st, dg = oracle.step(d, u, dt, want_diag=True)
        assert st == 0
        crkfr.cr_set_state(ctx, u)
        crkfr.cr_step(ctx, 1, 1e300, dt)
        assert_parity(crkfr.cr_get_state(ctx, shape=u.shape), ref, extra_scale=flux_increment(prob, dg, dt))
        np.testing.assert_allclose(crkfr.cr_get_alpha(ctx, u.shape[1]), dg["alpha"], rtol=0, atol=1e-12)
        u = ref


def _mirror(prob, g):
    nx, ny, n1 = prob["nx"], prob["ny"], prob["degree"] + 1
    G = g.reshape(4, ny, nx, n1, n1)
    F = G[:, :, ::-1, :, ::-1]
    return max(np.abs(G[v] - s * F[v]).max() / np.abs(G[v]).max() for v, s in enumerate((1, -1, 1, 1)))


def test_rayleigh_taylor_run():
    """The paper's 64 x 256, N = 3 mesh to t = 2.5 in FP64 and FP32 bulk:
    admissible means, and the mixing layer grown from the 2.5% perturbation:
    the heavy fluid's spike has risen along the centre line above y = 0.6 and
    the light fluid's bubbles have sunk below y = 0.45 at the walls, in both
    precisions within 3% of the height of each other.  Mirror symmetry about
    x = 0.125 holds only in exact arithmetic: the instability amplifies
    rounding, so it is reported, not asserted."""
    prob, u = wl.rayleigh_taylor()
    nx, ny = prob["nx"], prob["ny"]
    tips = {}
    for precision in (crkfr.CR_FP64, crkfr.CR_FP32_BULK):
        g, _, t, n, ctx = gpu_run(prob, u, nsteps=10 ** 7, t_final=prob["t_final"], precision=precision)
        assert t == prob["t_final"] and n > 1000
        mb = crkfr.cr_get_means(ctx, 4, u.shape[1])
        p = (5.0 / 3.0 - 1.0) * (mb[3] - 0.5 * (mb[1] ** 2 + mb[2] ** 2) / mb[0])
        assert mb[0].min() > 0 and p.min() > 0
        rho = mb[0].reshape(ny, nx)
        spike = (np.max(np.nonzero(rho[:, nx // 2] > 1.5)[0]) + 0.5) / ny
        bubble = (np.argmax(rho[:, 0] < 1.5) + 0.5) / ny
        tips[precision] = (spike, bubble)
        print("\nRT %s: %d steps, spike tip y = %.3f, bubble tip y = %.3f, asymmetry %.2e, rho [%.3f, %.3f]"
              % (precision, n, spike, bubble, _mirror(prob, g), mb[0].min(), mb[0].max()))
        assert spike > 0.6 and bubble < 0.45
    (s64, b64), (s32, b32) = tips[crkfr.CR_FP64], tips[crkfr.CR_FP32_BULK]
    assert abs(s64 - s32) <= 0.03 and abs(b64 - b32) <= 0.03


def test_fp32_ghost_states_one_step():
    prob, u = _mixed_2d(4, 3)
    d = oracle_desc(prob)
    dt = oracle.dt(d, u)
    ref, st = oracle.step(d, u, dt)
    assert st == 0
    g, t, n = run32(prob, u, 1, dt)
    assert np.all(l1_rel(g, ref) < L1_ONE_STEP), l1_rel(g, ref)


def test_batch_with_ghost_states_equals_single_steps():
    """Batches take ghost-state sides; gravity problems run alone (the batched
    kernels carry no source code)."""
    from tests.test_gpu_batch import _alone, _batched, _contexts, _same
    rt = lambda nx, ny, N: (lambda pu: (dict(pu[0], source=None), pu[1]))(
        wl.rayleigh_taylor(nx=nx, ny=ny, degree=N))
    probs = [_mixed_2d(4, 7), _mixed_2d(3, 8), rt(8, 32, 3), rt(12, 20, 4)]
    ref = _alone(probs, crkfr.CR_FP64, 3)
    for config in ((128, crkfr.CR_BATCH_PHASES), (256, crkfr.CR_BATCH_FUSED)):
        got, _ = _batched(probs, crkfr.CR_FP64, 3, config)
        _same(got, ref, crkfr.CR_FP64, "ghost states %s" % (config,))
    ctxs = _contexts([wl.rayleigh_taylor(nx=8, ny=32, degree=3)], crkfr.CR_FP64)
    with pytest.raises(crkfr.CrError):
        crkfr.cr_batch_init(ctxs)
