"""GPU parity and runs for Burgers' equation (Sec. 5.1) and the Sedov blasts
(Sec. 5.2 with solid walls, Sec. 5.3 periodic), through the C ABI, against
the FP64 oracle at the 1e-12 bar of tests/test_gpu_parity.py:

* Burgers: one step for every degree, dissipation model and central flux,
  with and without the limiters; the whole run to t = 2 (same step count and
  final time) for EA and AE; the EA flux's optimal order on the GPU against
  the exact characteristic solution; steps across the shock (t > 5)
  re-seeded from the oracle;
* 1D Sedov: steps along the oracle trajectory from the blast; the whole run
  to t = 0.001 in FP64 keeps mass and energy to rounding (the walls pass
  neither) and stays mirror symmetric, as the oracle's run does;
* 2D periodic Sedov: one step on a small mesh, a trajectory, and the whole
  run to t = 20 on the 64 x 64, N = 3 mesh in FP64 and FP32 bulk with
  admissible means and conserved mass, momentum and energy.
"""
import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc
from tests.test_gpu_parity import assert_parity, gpu_run, one_step_check
from tests.test_oracle_burgers import exact

pytestmark = pytest.mark.gpu

VARIANTS = [(oracle.DISS_D2, oracle.CENTRAL_EA), (oracle.DISS_D1, oracle.CENTRAL_EA),
            (oracle.DISS_DCSX, oracle.CENTRAL_EA), (oracle.DISS_D2, oracle.CENTRAL_AE),
            (oracle.DISS_D1, oracle.CENTRAL_AE), (oracle.DISS_DCSX, oracle.CENTRAL_AE)]
IDS = ["D2-EA", "D1-EA", "DCSX-EA", "D2-AE", "D1-AE", "DCSX-AE"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_07517_gb300 import build
    build.build()


def _burgers_random(nx, N, seed, limited):
    prob = wl.base_problem(dim=1, nx=nx, degree=N, equation="burgers",
                           limiter=wl.LIMITER_ALL if limited else frozenset())
    u = np.random.default_rng(seed).standard_normal((1, nx, N + 1))
    return prob, u


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("variant", VARIANTS, ids=IDS)
@pytest.mark.parametrize("limited", [False, True])
def test_burgers_one_step(N, variant, limited):
    diss, cen = variant
    prob, u = _burgers_random(29, N, seed=N + 10 * diss + 100 * cen, limited=limited)
    one_step_check(prob, u, over_oracle=dict(dissipation=diss, central=cen),
                   over_gpu=dict(dissipation=diss, central=cen))


@pytest.mark.parametrize("N", [3, 4])
@pytest.mark.parametrize("central", [oracle.CENTRAL_EA, oracle.CENTRAL_AE], ids=["EA", "AE"])
def test_burgers_full_horizon(N, central):
    prob, u = wl.burgers_sine(nx=48, degree=N, t_final=2.0)
    ref, t_o, n_o, st = oracle.run(oracle_desc(prob, central=central), u, 10 ** 6, 2.0)
    g, _, t_g, n_g, _ = gpu_run(prob, u, nsteps=10 ** 6, t_final=2.0, central=central)
    assert st == 0 and n_g == n_o and t_g == t_o == 2.0
    assert_parity(g, ref, rtol=1e-11)


def test_burgers_optimal_order_on_the_gpu():
    for N in (2, 3, 4):
        errs = []
        for nx in (32, 64, 128):
            prob, u = wl.burgers_sine(nx=nx, degree=N)
            g, _, t, _, _ = gpu_run(prob, u, nsteps=10 ** 6, t_final=2.0)
            assert t == 2.0
            x, _ = wl.node_coords(prob)
            _, w = wl.gl_nodes01(N)
            errs.append(np.sqrt(((g[0] - exact(x, 2.0)) ** 2 * w * 2 * np.pi / nx).sum()))
        assert np.log2(errs[1] / errs[2]) >= N + 1 - 0.25, (N, errs)


def test_burgers_across_the_shock():
    """From the oracle's state at t = 5.5 (shock formed), 30 steps with all
    limiters, each GPU step from the oracle's previous state."""
    prob, u = wl.burgers_sine(nx=64, degree=3)
    prob = dict(prob, limiter=wl.LIMITER_ALL)
    d = oracle_desc(prob)
    u, t, n, st = oracle.run(d, u, 10 ** 6, 5.5)
    assert st == 0
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
    blended = 0
    for _ in range(30):
        dt = oracle.dt(d, u)
        ref, st, dg = oracle.step(d, u, dt, want_diag=True)
        assert st == 0
        crkfr.cr_set_state(ctx, u)
        crkfr.cr_step(ctx, 1, 1e300, dt)
        assert_parity(crkfr.cr_get_state(ctx, shape=u.shape), ref)
        np.testing.assert_allclose(crkfr.cr_get_alpha(ctx, u.shape[1]), dg["alpha"], rtol=0, atol=1e-12)
        blended += int((dg["alpha"] > 0).sum())
        u = ref
    assert blended > 0


def test_burgers_refused_in_2d():
    prob = wl.base_problem(dim=2, nx=4, ny=4, degree=2, equation="burgers")
    with pytest.raises(crkfr.CrError):
        crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))


# ---------------------------------------------------------------- Sedov ----
def _means(prob, u):
    _, w = wl.gl_nodes01(prob["degree"])
    if prob["dim"] == 2:
        n = prob["degree"] + 1
        w = np.array([w[k % n] * w[k // n] for k in range(n * n)])
    return np.einsum("vek,k->ve", u, w)


def test_sedov1d_trajectory():
    """25 steps from the blast, each from the oracle's previous state.  The
    second step is ill-conditioned: input changes of one ulp move the oracle's
    own output momentum by up to ~5e-12 of its maximum next to the centre
    element.  The bar there is the larger of 1e-12 relative and twice the
    spread of the oracle's outputs over four inputs perturbed by at most one
    ulp (uniform relative factors), the rounding-level spread of the step
    itself."""
    prob, u = wl.sedov1d()
    d = oracle_desc(prob)
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
    rng = np.random.default_rng(7)
    for step in range(25):
        dt = oracle.dt(d, u)
        ref, st = oracle.step(d, u, dt)
        assert st == 0
        spread = np.zeros(3)
        for _ in range(4):
            alt, _ = oracle.step(d, u * (1.0 + rng.uniform(-1.0, 1.0, u.shape) * 2.0 ** -52), dt)
            spread = np.maximum(spread, np.abs(alt - ref).max(axis=(1, 2)))
        crkfr.cr_set_state(ctx, u)
        crkfr.cr_step(ctx, 1, 1e300, dt)
        g = crkfr.cr_get_state(ctx, shape=u.shape)
        for v in range(3):
            tol = max(1e-12 * np.abs(ref[v]).max(), 2.0 * spread[v])
            err = np.abs(g[v] - ref[v]).max()
            assert err <= tol, (step, v, err, tol, spread[v])
        u = ref


def _mirror_error(prob, g):
    """max relative asymmetry of a 1D state about x = 0: rho(x) = rho(-x),
    m(x) = -m(-x), E(x) = E(-x)."""
    flip = g[:, ::-1, ::-1]
    sgn = np.array([1.0, -1.0, 1.0])[:, None, None]
    return max(np.abs(g[v] - sgn[v] * flip[v]).max() / np.abs(g[v]).max() for v in range(3))


def test_sedov1d_full_run():
    """The whole run to t = 0.001 (about 6000 steps, the shock reflected from
    the walls) on the GPU and in the oracle: same step count, conserved mass
    and energy, mirror symmetry, and the two densities agree to well within
    the asymmetry that rounding grows over the run (the limiter's decisions
    amplify rounding; the oracle's own run is symmetric only to ~1e-4)."""
    prob, u = wl.sedov1d()
    ref, t_o, n_o, st = oracle.run(oracle_desc(prob), u, 10 ** 6, prob["t_final"])
    assert st == 0
    g, _, t, n, _ = gpu_run(prob, u, nsteps=10 ** 7, t_final=prob["t_final"])
    m0, m1 = _means(prob, u).sum(axis=1), _means(prob, g).sum(axis=1)
    mb = _means(prob, g)
    diff = np.abs(g[0] - ref[0])
    print("\nSedov 1D: %d steps (oracle %d); density max |gpu - oracle| %.2e, mean %.2e (max rho %.3f); "
          "asymmetry gpu %.2e oracle %.2e; mass drift %.2e energy drift %.2e"
          % (n, n_o, diff.max(), diff.mean(), ref[0].max(), _mirror_error(prob, g),
             _mirror_error(prob, ref), m1[0] - m0[0], (m1[2] - m0[2]) / m0[2]))
    assert t == t_o == prob["t_final"] and abs(n - n_o) <= 0.01 * n_o
    assert abs(m1[0] - m0[0]) <= 1e-14 * n * m0[0]
    assert abs(m1[2] - m0[2]) <= 1e-14 * n * m0[2]
    assert mb[0].min() > 0 and (0.4 * (mb[2] - 0.5 * mb[1] ** 2 / mb[0])).min() > 0
    assert _mirror_error(prob, g) < 1e-3
    assert diff.max() <= 0.05 * ref[0].max() and diff.mean() <= 1e-3 * ref[0].max()


def test_sedov2d_one_step_and_trajectory():
    prob, u = wl.sedov2d_periodic(nx=16, degree=3)
    one_step_check(prob, u)
    d = oracle_desc(prob)
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
    crkfr.cr_set_state(ctx, u)
    for _ in range(10):
        dt = oracle.dt(d, u)
        ref, st = oracle.step(d, u, dt)
        assert st == 0
        crkfr.cr_step(ctx, 1, 1e300, dt)
        assert_parity(crkfr.cr_get_state(ctx, shape=u.shape), ref, rtol=1e-11)
        u = ref


@pytest.mark.parametrize("precision", [crkfr.CR_FP64, crkfr.CR_FP32_BULK], ids=["fp64", "fp32"])
def test_sedov2d_periodic_to_t20(precision):
    prob, u = wl.sedov2d_periodic(nx=64, degree=3)
    g, _, t, n, ctx = gpu_run(prob, u, nsteps=10 ** 7, t_final=20.0, precision=precision)
    assert t == 20.0 and n > 1000
    # the library's element means (FP64 in both modes)
    m0 = _means(prob, u).sum(axis=1)
    m1 = crkfr.cr_get_means(ctx, 4, u.shape[1]).sum(axis=1)
    assert abs(m1[0] - m0[0]) <= 1e-13 * n * m0[0]
    assert abs(m1[3] - m0[3]) <= 1e-13 * n * m0[3]
    assert abs(m1[1]) <= 1e-10 * m0[0] and abs(m1[2]) <= 1e-10 * m0[0]
    mb = crkfr.cr_get_means(ctx, 4, u.shape[1])
    p = 0.4 * (mb[3] - 0.5 * (mb[1] ** 2 + mb[2] ** 2) / mb[0])
    assert mb[0].min() > 0 and p.min() > 0
    print("\nSedov 2D %s: %d steps, rho range [%.3g, %.3g]" % (precision, n, g[0].min(), g[0].max()))
