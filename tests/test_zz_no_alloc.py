"""cr_step_static, the entry point for callers that may not allocate device
memory (their device memory belongs to another allocator, or allocation's
implicit synchronisation or any allocation after start-up is not allowed):
two calls in a row must give what the context-based entry point gives, while
the fixed scratch array carries the previous call's contents into the next,
and one call must match the FP64 oracle directly.  Collected last on
purpose, so that a run stopping at the first failure has already run
everything else."""
import numpy as np
import pytest

from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _close(a, b, rtol=1e-12):
    for v in range(b.shape[0]):
        scale = max(np.abs(b[v]).max(), 1e-300)
        assert np.abs(a[v] - b[v]).max() <= rtol * scale, v


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_07517_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def test_static_scratch_step_matches_context_step_twice():
    import torch
    prob, u0 = wl.euler2d_vortex(nx=12, ny=10, degree=4, seed=4)
    u0 = u0 * np.random.default_rng(4).uniform(0.6, 1.6, (1, u0.shape[1], 1))  # limiters act
    desc = crkfr.desc_from_problem(prob)

    # reference: the context entry point, two steps of the same dt
    ctx = crkfr.cr_init_mesh(desc)
    crkfr.cr_set_state(ctx, u0)
    dt = crkfr.cr_next_dt(ctx)
    crkfr.cr_step(ctx, 1, 1e300, dt)
    ref1 = crkfr.cr_get_state(ctx, shape=u0.shape)
    crkfr.cr_step(ctx, 1, 1e300, dt)
    ref2 = crkfr.cr_get_state(ctx, shape=u0.shape)

    # the same two steps through the static-scratch entry point
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    crkfr.cr_step_static(desc, a, b, dt)
    torch.cuda.synchronize()
    _close(b.cpu().numpy(), ref1)
    crkfr.cr_step_static(desc, b, a, dt)
    torch.cuda.synchronize()
    _close(a.cpu().numpy(), ref2)

    # in place, and a mesh beyond the fixed scratch size is refused
    c = torch.from_numpy(u0).cuda()
    crkfr.cr_step_static(desc, c, c, dt)
    _close(c.cpu().numpy(), ref1)
    big, ubig = wl.euler2d_vortex(nx=96, ny=96, degree=4, seed=0)
    t_big = torch.from_numpy(ubig).cuda()
    with pytest.raises(crkfr.CrError) as ei:
        crkfr.cr_step_static(crkfr.desc_from_problem(big), t_big, t_big, dt)
    assert ei.value.status == -8


def _tenmoment_source():
    prob, u = wl.tenmoment2d_voronoi(nx=8, ny=8, degree=3, seed=3)
    return prob, u


CASES = {
    "euler1d_outflow_N4": lambda: wl.euler1d_riemann(nx=40, degree=4, seed=2),
    "tenmoment2d_source_N3": _tenmoment_source,
    "linadv1d_N3": lambda: wl.linadv_sine(nx=16, degree=3),
    "euler2d_walls_gravity_N3": lambda: wl.rayleigh_taylor(nx=4, ny=16, degree=3),
    "euler2d_N2_outflow": lambda: (lambda pu: (dict(pu[0], bc_x="outflow", bc_y="outflow"), pu[1]))(
        wl.euler2d_vortex(nx=7, ny=5, degree=2, seed=1)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_static_scratch_other_equations(name):
    """Other equations, dimensions, degrees, boundaries and sources: two
    static-scratch steps in a row equal two context steps of the same dt."""
    import torch
    prob, u0 = CASES[name]()
    desc = crkfr.desc_from_problem(prob)
    ctx = crkfr.cr_init_mesh(desc)
    crkfr.cr_set_state(ctx, u0)
    dt = crkfr.cr_next_dt(ctx)
    refs = []
    for _ in range(2):
        crkfr.cr_step(ctx, 1, 1e300, dt)
        refs.append(crkfr.cr_get_state(ctx, shape=u0.shape))
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    crkfr.cr_step_static(desc, a, b, dt)
    crkfr.cr_step_static(desc, b, a, dt)
    torch.cuda.synchronize()
    _close(b.cpu().numpy(), refs[0])
    _close(a.cpu().numpy(), refs[1])


@pytest.mark.parametrize("name", ["euler1d_outflow_N4", "tenmoment2d_source_N3"])
def test_static_scratch_step_matches_oracle(name):
    """One static-scratch step against the FP64 oracle directly, at the parity
    tests' tolerance (1e-12 of the larger of the variable's size and its flux
    increment)."""
    import torch
    import oracle
    from tests._oracle_util import oracle_desc
    prob, u0 = CASES[name]()
    d = oracle_desc(prob)
    dt = oracle.dt(d, u0)
    ref, st, dg = oracle.step(d, u0, dt, want_diag=True)
    assert st == 0
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    crkfr.cr_step_static(crkfr.desc_from_problem(prob), a, b, dt)
    g = b.cpu().numpy()
    dx = (prob["x1"] - prob["x0"]) / prob["nx"]
    inc = dt / dx * np.abs(dg["fnum_x"]).max(axis=(1, 2))
    if prob["dim"] == 2:
        inc = inc + dt / ((prob["y1"] - prob["y0"]) / prob["ny"]) * np.abs(dg["fnum_y"]).max(axis=(1, 2))
    for v in range(ref.shape[0]):
        scale = max(np.abs(ref[v]).max(), inc[v])
        assert np.abs(g[v] - ref[v]).max() <= 1e-12 * scale, v
