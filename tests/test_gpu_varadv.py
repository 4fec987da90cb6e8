"""GPU parity for variable advection u_t + (a(x) u)_x = 0 (Sec. 5.1, a(x) =
x^2 on [0.1, 1]) with the exact solution as time-dependent inflow data
(Chebyshev series in t, evaluated at the stage times) and outflow, through
the C ABI, against the FP64 oracle at the 1e-12 bar of
tests/test_gpu_parity.py: one step for every degree, dissipation model and
central flux, with and without the limiters; 25 CFL steps (the inflow data
then follow the device's own time); the whole run to t = 1 with the oracle's
step count and the EA flux's optimal order against the exact solution."""
import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc
from tests.test_gpu_parity import assert_parity, gpu_run, one_step_check

pytestmark = pytest.mark.gpu

VARIANTS = [(0, 0), (1, 0), (2, 0), (0, 1), (2, 1)]
VIDS = ["D2-EA", "D1-EA", "DCSX-EA", "D2-AE", "DCSX-AE"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_07517_gb300 import build
    build.build()


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
@pytest.mark.parametrize("limited", [False, True])
def test_one_step(N, variant, limited):
    diss, cen = variant
    prob, u = wl.varadv_x2(nx=23, degree=N)
    if limited:
        prob = dict(prob, limiter=wl.LIMITER_ALL)
        u = u * np.random.default_rng(N).uniform(0.5, 1.5, u.shape)
    over = dict(dissipation=diss, central=cen)
    one_step_check(prob, u, over_oracle=over, over_gpu=over)


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("side", ["dirichlet", "inflow"])
def test_trajectory(N, side):
    prob, u = wl.varadv_x2(nx=17, degree=N)
    prob = dict(prob, bc_side={"x-": side})
    ref, t_o, n_o, st = oracle.run(oracle_desc(prob), u, 25, 1e9)
    g, _, t_g, n_g, _ = gpu_run(prob, u, nsteps=25)
    assert st == 0 and n_o == n_g == 25 and abs(t_g - t_o) <= 1e-14 * t_o
    assert_parity(g, ref, rtol=1e-11)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("central", [oracle.CENTRAL_EA, oracle.CENTRAL_AE], ids=["EA", "AE"])
def test_full_horizon(N, central):
    prob, u = wl.varadv_x2(nx=20, degree=N)
    ref, t_o, n_o, st = oracle.run(oracle_desc(prob, central=central), u, 10 ** 6, 1.0)
    g, _, t_g, n_g, _ = gpu_run(prob, u, nsteps=10 ** 6, t_final=1.0, central=central)
    assert st == 0 and n_g == n_o and t_g == t_o == 1.0
    assert_parity(g, ref, rtol=1e-11)


def test_optimal_order_on_the_gpu():
    for N in (2, 3):
        errs = []
        for nx in (32, 64, 128):
            prob, u = wl.varadv_x2(nx=nx, degree=N)
            g, _, t, _, _ = gpu_run(prob, u, nsteps=10 ** 6, t_final=1.0)
            assert t == 1.0
            x, _ = wl.node_coords(prob)
            _, w = wl.nodes01(prob)
            errs.append(np.sqrt(((g[0] - wl.varadv_exact(x, 1.0)) ** 2 * w * 0.9 / nx).sum()))
        assert np.log2(errs[1] / errs[2]) >= N + 1 - 0.3, (N, errs)


def test_refusals():
    prob, u = wl.varadv_x2(nx=8, degree=3)
    d = crkfr.desc_from_problem(prob, precision=crkfr.CR_FP32_BULK)
    with pytest.raises(crkfr.CrError):
        crkfr.cr_init_mesh(d)
    d = crkfr.desc_from_problem(dict(prob, dim=2, ny=4))
    with pytest.raises(crkfr.CrError):
        crkfr.cr_init_mesh(d)
