"""GPU parity with Gauss-Lobatto-Legendre solution points and the g2
correction (Sec. 5.1), through the C ABI, against the FP64 oracle at the
1e-12 bar of tests/test_gpu_parity.py: one step for Burgers, 1D and 2D Euler
(scaling limiter) and 2D linear advection with every dissipation model and
central flux; the evaluate and extrapolate fluxes give the same GPU step;
the whole Burgers run to t = 2 with the oracle's step count; FP32 bulk within
its L1 bound."""
import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc
from tests.test_gpu_fp32 import L1_ONE_STEP, l1_rel, run32
from tests.test_gpu_parity import assert_parity, gpu_run, one_step_check

pytestmark = pytest.mark.gpu

VARIANTS = [(0, 0), (1, 0), (2, 0), (0, 1)]
VIDS = ["D2-EA", "D1-EA", "DCSX-EA", "D2-AE"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_07517_gb300 import build
    build.build()


def _euler1d(N, seed):
    prob, _ = wl.euler1d_riemann(nx=37, degree=N, seed=seed, limiter=("scaling", "traces"))
    prob = dict(prob, points="gll")
    x, _ = wl.node_coords(prob)
    xc, _ = wl.element_centres(prob)
    r = prob["riemann"]
    right = np.broadcast_to((xc >= 0.5)[:, None], x.shape)
    pick = lambda k: np.where(right, r[k][1], r[k][0])
    return prob, wl.euler_conservative(pick("rho"), pick("v"), None, pick("p"), 1.4, 1)


def _euler2d(N, seed):
    prob, _ = wl.euler2d_vortex(nx=9, ny=8, degree=N, seed=seed, limiter=("scaling", "traces"))
    prob = dict(prob, points="gll")
    x, y = wl.node_coords(prob)
    rho, v1, v2, p = wl.isentropic_vortex(x, y, prob["gamma"])
    rho = rho * np.random.default_rng(seed).uniform(0.8, 1.25, (x.shape[0], 1))
    return prob, wl.euler_conservative(rho, v1, v2, p, prob["gamma"], 2)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
def test_one_step(N, variant):
    diss, cen = variant
    over = dict(dissipation=diss, central=cen)
    prob = wl.base_problem(dim=1, nx=19, degree=N, equation="burgers", points="gll")
    u = np.random.default_rng(N).standard_normal((1, 19, N + 1))
    one_step_check(prob, u, over_oracle=over, over_gpu=over)
    one_step_check(*_euler1d(N, N), over_oracle=over, over_gpu=over)
    if N >= 2:
        one_step_check(*_euler2d(N, N), over_oracle=over, over_gpu=over)
        prob, u = wl.linadv_random(nx=7, ny=6, dim=2, degree=N, seed=N, adv=(0.9, -0.6))
        one_step_check(dict(prob, points="gll"), u, over_oracle=over, over_gpu=over)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_evaluate_equals_extrapolate_on_the_gpu(N):
    prob, u = _euler2d(N, 11)
    dt = oracle.dt(oracle_desc(prob), u)
    a = gpu_run(prob, u, dt_fixed=dt)[0]
    b = gpu_run(prob, u, dt_fixed=dt, central=crkfr.CR_CENTRAL_AE)[0]
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13 * np.abs(a).max())


@pytest.mark.parametrize("N", [2, 3])
def test_burgers_full_horizon(N):
    prob, u = wl.burgers_sine(nx=40, degree=N, points="gll")
    ref, t_o, n_o, st = oracle.run(oracle_desc(prob), u, 10 ** 6, 2.0)
    g, _, t_g, n_g, _ = gpu_run(prob, u, nsteps=10 ** 6, t_final=2.0)
    assert st == 0 and n_g == n_o and t_g == t_o == 2.0
    assert_parity(g, ref, rtol=1e-11)


def test_fp32_bulk_one_step():
    prob, u = _euler2d(4, 3)
    d = oracle_desc(prob)
    dt = oracle.dt(d, u)
    ref, st = oracle.step(d, u, dt)
    assert st == 0
    g, t, n = run32(prob, u, 1, dt)
    assert np.all(l1_rel(g, ref) < L1_ONE_STEP), l1_rel(g, ref)


def test_static_and_batch_refuse_gll():
    prob, u = _euler2d(3, 1)
    import torch
    d = crkfr.desc_from_problem(prob)
    ut = torch.from_numpy(u).cuda()
    with pytest.raises(crkfr.CrError) as ei:
        crkfr.cr_step_static(d, ut, torch.empty_like(ut), 1e-3)
    assert ei.value.status == -7
    ctx = crkfr.cr_init_mesh(d)
    crkfr.cr_set_state(ctx, u)
    with pytest.raises(crkfr.CrError):
        crkfr.cr_batch_init([ctx])
