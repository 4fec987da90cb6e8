"""cr_set_state from pinned host memory: the prologue kernel reads the FP64
state over the host link and keeps the copy itself, instead of a copy followed
by the prologue.  The result must be the same, bit for bit, as setting the
same values from pageable host memory or from the device: the state, the raw
blending coefficients, the next time step and the state after steps; and a
non-finite or inadmissible value in pinned memory is refused the same way."""
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


def _cases():
    prob, u = wl.euler2d_vortex(nx=13, ny=11, degree=4, seed=3)
    yield "euler2d_N4", prob, u * np.random.default_rng(3).uniform(0.6, 1.6, (1, u.shape[1], 1))
    yield ("euler1d_N3",) + wl.euler1d_riemann(nx=37, degree=3, seed=2)
    yield ("tenmoment2d_N3",) + wl.tenmoment2d_voronoi(nx=9, ny=7, degree=3, seed=1)


@pytest.mark.parametrize("name,prob,u", list(_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_pinned_host_state_equals_pageable(name, prob, u):
    import torch
    pinned = torch.from_numpy(u).pin_memory()
    out = {}
    for src in ("pageable", "pinned", "device"):
        ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
        if src == "pageable":
            crkfr.cr_set_state(ctx, u)
        elif src == "pinned":
            crkfr._check(crkfr.lib().cr_set_state(ctx.handle, pinned.data_ptr(), 0), ctx.handle)
        else:
            crkfr._check(crkfr.lib().cr_set_state(ctx.handle, torch.from_numpy(u).cuda().data_ptr(), 1),
                         ctx.handle)
        s0 = crkfr.cr_get_state(ctx, shape=u.shape)
        _, a0 = crkfr.cr_get_features(ctx, u.shape[1], u.shape[2])
        dt = crkfr.cr_next_dt(ctx)
        crkfr.cr_step(ctx, 3, 1e300)
        out[src] = (s0, a0, dt, crkfr.cr_get_state(ctx, shape=u.shape))
    for src in ("pinned", "device"):
        for a, b in zip(out[src], out["pageable"]):
            np.testing.assert_array_equal(a, b, err_msg="%s %s" % (name, src))
    np.testing.assert_array_equal(out["pinned"][0], u)


def test_pinned_host_state_refuses_bad_input():
    import torch
    prob, u = wl.euler2d_vortex(nx=6, ny=5, degree=3, seed=0)
    ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
    for bad in (np.nan, -1.0):
        v = u.copy()
        v[0, 7, 3] = bad
        pinned = torch.from_numpy(v).pin_memory()
        st = crkfr.lib().cr_set_state(ctx.handle, pinned.data_ptr(), 0)
        assert st == -2, (bad, st)
    crkfr.cr_set_state(ctx, u)  # a good state afterwards is taken
    np.testing.assert_array_equal(crkfr.cr_get_state(ctx, shape=u.shape), u)
