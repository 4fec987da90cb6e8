"""Admissibility at every solution point after every step (Sec. 3.2: the
flux limiter keeps the means admissible and the scaling limiter the points):
shock workloads run on the GPU in FP64 and FP32 bulk one step at a time, and
after each step every node of the state has rho > 0 and p > 0 (Euler) or
rho > 0 and a positive-definite pressure tensor (ten-moment), and every value
is finite.  The checks are the constraints themselves, evaluated here in numpy
on the state the library returns."""
import numpy as np
import pytest

from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_07517_gb300 import build
    build.build()


def _min_constraints(prob, g):
    """Smallest rho and smallest second constraint over all nodes."""
    eq = prob["equation"]
    rho = g[0]
    if eq == "euler":
        gm1 = prob["gamma"] - 1.0
        kin = 0.5 * g[1] ** 2 / rho if prob["dim"] == 1 else 0.5 * (g[1] ** 2 + g[2] ** 2) / rho
        return rho.min(), (gm1 * (g[-1] - kin)).min()
    v1, v2 = g[1] / rho, g[2] / rho
    p11 = 2.0 * g[3] - rho * v1 * v1
    p12 = 2.0 * g[4] - rho * v1 * v2
    p22 = 2.0 * g[5] - rho * v2 * v2
    lam = 0.5 * (p11 + p22) - np.sqrt(0.25 * (p11 - p22) ** 2 + p12 ** 2)
    return rho.min(), lam.min()


# (name, workload, steps); the 1D Sedov blast runs its whole course to
# t = 0.001 (about 5,900 steps)
CASES = [
    ("euler1d_riemann_s0", lambda: wl.euler1d_riemann(nx=400, degree=4, seed=0), 150),
    ("euler1d_riemann_s5", lambda: wl.euler1d_riemann(nx=400, degree=4, seed=5), 150),
    ("euler2d_vortex_riemann", lambda: wl.euler2d_vortex_riemann(nx=64, degree=4, seed=3), 150),
    ("tenmoment2d_voronoi", lambda: wl.tenmoment2d_voronoi(nx=48, degree=3, seed=2), 150),
    ("sedov2d_periodic", lambda: wl.sedov2d_periodic(nx=32, degree=3), 150),
    ("sedov1d_walls", lambda: wl.sedov1d(), 6000),
    ("rayleigh_taylor", lambda: wl.rayleigh_taylor(nx=16, ny=64, degree=3), 150),
]


@pytest.mark.parametrize("precision", [crkfr.CR_FP64, crkfr.CR_FP32_BULK], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name,make,nsteps", CASES, ids=[c[0] for c in CASES])
def test_every_node_admissible(name, make, nsteps, precision):
    prob, u = make()
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, precision=precision))
    crkfr.cr_set_state(ctx, u)
    worst = (np.inf, np.inf)
    g = np.empty(u.shape)
    for k in range(nsteps):
        t, n = crkfr.cr_step(ctx, 1, 1e300)
        assert n == k + 1
        crkfr.cr_get_state(ctx, out=g)
        assert np.all(np.isfinite(g)), (name, k)
        r, c2 = _min_constraints(prob, g)
        worst = (min(worst[0], r), min(worst[1], c2))
        assert r > 0.0 and c2 > 0.0, (name, k, r, c2)
    print("\n%s %s: %d steps, min rho %.3e, min second constraint %.3e" % (name, precision, n, *worst))
