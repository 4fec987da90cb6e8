"""Batched stepping (cr_batch_*): many independent 2D Euler problems of
uneven mesh size and degree 3/4 advanced together, in one launch per phase or
in one persistent cooperative launch.

A batched step runs the same per-block bodies as the single-problem kernels,
and no result depends on how elements are grouped into blocks, so in FP64
every problem's state must equal, bit for bit, what cr_step gives on that
problem alone, for every (threads, mode, tiles) configuration and with runs clipped
at t_final; in FP32 bulk (also with the learned alpha) it must agree to FP32
rounding and be reproducible bit for bit.  One batched FP64 step is also
compared with the FP64 oracle directly.
"""
import numpy as np
import pytest

import oracle
from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc

pytestmark = pytest.mark.gpu

# ragged meshes, both degrees, a single element and a single row
SHAPES = [((13, 11), 4), ((7, 5), 3), ((1, 1), 4), ((17, 1), 3), ((24, 20), 4), ((9, 16), 3)]
CONFIGS = [(128, crkfr.CR_BATCH_PHASES, 1), (128, crkfr.CR_BATCH_FUSED, 1),
           (256, crkfr.CR_BATCH_PHASES, 1), (256, crkfr.CR_BATCH_FUSED, 1),
           (256, crkfr.CR_BATCH_FUSED, 2), (128, crkfr.CR_BATCH_FUSED, 4)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_07517_gb300 import build
    build.build()


def _problems(seed, shapes=SHAPES):
    out = []
    for i, ((nx, ny), N) in enumerate(shapes):
        prob, u = wl.euler2d_vortex_riemann(nx=nx, ny=ny, degree=N, seed=seed + i)
        out.append((prob, u))
    return out


def _contexts(probs, precision, **over):
    ctxs = []
    for prob, u in probs:
        c = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, precision=precision, **over))
        crkfr.cr_set_state(c, u)
        ctxs.append(c)
    return ctxs


def _alone(probs, precision, nsteps, t_final=1e300, params=None, **over):
    out = []
    for (prob, u), c in zip(probs, _contexts(probs, precision, **over)):
        if params is not None:
            crkfr.cr_mlp_load(c, params[u.shape[2]])
            crkfr.cr_set_state(c, u)
        crkfr.cr_step(c, nsteps, t_final)
        out.append(crkfr.cr_get_state(c, shape=u.shape))
    return out


def _batched(probs, precision, nsteps, config=None, t_final=1e300, params=None, **over):
    ctxs = _contexts(probs, precision, **over)
    if params is not None:
        for (prob, u), c in zip(probs, ctxs):
            crkfr.cr_mlp_load(c, params[u.shape[2]])
            crkfr.cr_set_state(c, u)
    b = crkfr.cr_batch_init(ctxs)
    if config is not None:
        crkfr.cr_batch_config(b, *config)
    crkfr.cr_batch_step(b, nsteps, t_final)
    return [crkfr.cr_get_state(c, shape=u.shape) for (prob, u), c in zip(probs, ctxs)], ctxs


def _same(got, ref, precision, what=""):
    """FP64: bit for bit.  FP32 bulk: the batched kernels inline the same bodies
    into other kernels, where the compiler may contract a * b + c into a fused
    multiply-add at other places; the results then differ by FP32 rounding, so
    they are compared with a bound well below the FP32 bulk error (2e-7 L1)."""
    for i, (g, r) in enumerate(zip(got, ref)):
        if precision == crkfr.CR_FP64:
            np.testing.assert_array_equal(g, r, err_msg="%s problem %d" % (what, i))
        else:
            for v in range(r.shape[0]):
                scale = np.abs(r[v]).max()
                assert np.abs(g[v] - r[v]).max() <= 2e-6 * scale, (what, i, v)
                assert np.abs(g[v] - r[v]).sum() <= 1e-7 * np.abs(r[v]).sum(), (what, i, v)


@pytest.mark.parametrize("precision", [crkfr.CR_FP64, crkfr.CR_FP32_BULK], ids=["fp64", "fp32"])
@pytest.mark.parametrize("config", CONFIGS, ids=["%d-%s-%d" % (t, "fused" if m else "phases", k)
                                                 for t, m, k in CONFIGS])
def test_batch_equals_single_problem_steps(precision, config):
    probs = _problems(10)
    ref = _alone(probs, precision, 5)
    got, _ = _batched(probs, precision, 5, config)
    _same(got, ref, precision, str(config))
    again, _ = _batched(probs, precision, 5, config)   # deterministic: bit for bit run to run
    for i, (g, a) in enumerate(zip(got, again)):
        np.testing.assert_array_equal(g, a, err_msg="problem %d" % i)


def test_batch_t_final_clipping_and_step_counts():
    probs = _problems(20)
    # a final time some problems reach within the 12 steps and others do not
    dts = []
    for c in _contexts(probs, crkfr.CR_FP64):
        dts.append(crkfr.cr_next_dt(c))
    t_final = 6.5 * float(np.median(dts))
    ref = _alone(probs, crkfr.CR_FP64, 12, t_final)
    got, ctxs = _batched(probs, crkfr.CR_FP64, 12, (256, crkfr.CR_BATCH_FUSED), t_final)
    steps = []
    for i, (g, r, c) in enumerate(zip(got, ref, ctxs)):
        np.testing.assert_array_equal(g, r, err_msg="problem %d" % i)
        t, n = crkfr.cr_sync(c)
        steps.append(n)
        assert t <= t_final
    assert min(steps) < 12 and max(steps) >= 7


def test_batch_learned_alpha_equals_single_problem_steps():
    from oracle import mlp
    rng = np.random.default_rng(3)
    params = {}
    for npts in (16, 25):
        p = rng.normal(0.0, 0.6, mlp.param_count(npts)).astype(np.float32)
        p[-1] = 1.0
        params[npts] = p
    probs = _problems(30)
    ref = _alone(probs, crkfr.CR_FP32_BULK, 4, params=params, alpha_mode=crkfr.CR_ALPHA_MLP)
    got, ctxs = _batched(probs, crkfr.CR_FP32_BULK, 4, (128, crkfr.CR_BATCH_FUSED), params=params,
                         alpha_mode=crkfr.CR_ALPHA_MLP)
    _same(got, ref, crkfr.CR_FP32_BULK)
    a = np.concatenate([crkfr.cr_get_alpha(c, u.shape[1]) for (prob, u), c in zip(probs, ctxs)])
    assert a.max() > 0.0  # the network's alpha is in play


def test_batched_step_matches_oracle():
    from tests.test_gpu_parity import assert_parity, flux_increment
    probs = _problems(40, shapes=[((9, 8), 4), ((6, 7), 3), ((5, 3), 4)])
    got, ctxs = _batched(probs, crkfr.CR_FP64, 1, (128, crkfr.CR_BATCH_FUSED))
    for (prob, u), g, c in zip(probs, got, ctxs):
        d = oracle_desc(prob)
        dt = oracle.dt(d, u)
        ref, st, dg = oracle.step(d, u, dt, want_diag=True)
        assert st == 0
        t, n = crkfr.cr_sync(c)
        assert n == 1 and abs(t - dt) <= 1e-14 * dt
        assert_parity(g, ref, extra_scale=flux_increment(prob, dg, dt))


def test_autotune_then_step():
    probs = _problems(50)
    ctxs = _contexts(probs, crkfr.CR_FP32_BULK)
    b = crkfr.cr_batch_init(ctxs)
    threads, mode, tiles, ms = crkfr.cr_batch_autotune(b, 2)
    assert len(ms) == 8 and np.all(ms > 0) and np.all(ms < 1e300)
    assert ms[crkfr.BATCH_CANDIDATES.index((threads, mode, tiles))] == ms.min()
    for (prob, u), c in zip(probs, ctxs):  # the tuning advanced the problems: start again
        crkfr.cr_set_state(c, u)
    crkfr.cr_batch_step(b, 3)
    got = [crkfr.cr_get_state(c, shape=u.shape) for (prob, u), c in zip(probs, ctxs)]
    ref = _alone(probs, crkfr.CR_FP32_BULK, 3)
    _same(got, ref, crkfr.CR_FP32_BULK)


def test_batch_rejects_unsupported_problems():
    prob, u = wl.euler1d_riemann(nx=20, degree=4, seed=0)
    c = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
    with pytest.raises(crkfr.CrError) as ei:
        crkfr.cr_batch_init([c])
    assert ei.value.status == -7
    probs = _problems(60, shapes=[((5, 5), 3), ((5, 5), 4)])
    c64 = _contexts(probs[:1], crkfr.CR_FP64)
    c32 = _contexts(probs[1:], crkfr.CR_FP32_BULK)
    with pytest.raises(crkfr.CrError) as ei:
        crkfr.cr_batch_init(c64 + c32)
    assert ei.value.status == -1


def test_fused_wait_timeout_is_reported_and_recoverable():
    """Waits of the fused kernel that require completions that never come
    (fault injection): the first wait gives up after its budget, every block
    returns, cr_batch_step reports CR_E_TIMEOUT, and after the states are set
    again the batch steps exactly like the single-problem path.  No block
    traps or hangs."""
    import time
    probs = _problems(70, shapes=[((13, 11), 4), ((7, 5), 3)])
    ctxs = _contexts(probs, crkfr.CR_FP64)
    b = crkfr.cr_batch_init(ctxs)
    crkfr.cr_batch_config(b, 256, crkfr.CR_BATCH_FUSED, 1)
    crkfr.cr_batch_barrier_test(b, 20000, 1)
    t0 = time.perf_counter()
    with pytest.raises(crkfr.CrError) as ei:
        crkfr.cr_batch_step(b, 1)
    assert ei.value.status == -4
    assert time.perf_counter() - t0 < 30.0
    crkfr.cr_batch_barrier_test(b, 0, 0)
    for (prob, u), c in zip(probs, ctxs):
        crkfr.cr_set_state(c, u)
    crkfr.cr_batch_step(b, 3)
    got = [crkfr.cr_get_state(c, shape=u.shape) for (prob, u), c in zip(probs, ctxs)]
    _same(got, _alone(probs, crkfr.CR_FP64, 3), crkfr.CR_FP64, "after timeout")


def test_batch_with_walls_equals_single_problem_steps():
    probs = [(dict(p, bc_x="wall"), u) for p, u in _problems(80, shapes=[((11, 9), 4), ((8, 6), 3)])]
    probs += [(dict(p, bc_y="wall", bc_x="outflow"), u) for p, u in _problems(90, shapes=[((7, 9), 4)])]
    ref = _alone(probs, crkfr.CR_FP64, 4)
    for config in ((128, crkfr.CR_BATCH_PHASES, 1), (256, crkfr.CR_BATCH_FUSED, 2)):
        got, _ = _batched(probs, crkfr.CR_FP64, 4, config)
        _same(got, ref, crkfr.CR_FP64, "walls %s" % (config,))


@pytest.mark.parametrize("diss,cen", [(1, 0), (2, 1)])
def test_batch_with_variants_equals_single_problem_steps(diss, cen):
    probs = _problems(100, shapes=[((11, 9), 4), ((8, 6), 3), ((5, 7), 4)])
    ref = _alone(probs, crkfr.CR_FP64, 3, dissipation=diss, central=cen)
    got, _ = _batched(probs, crkfr.CR_FP64, 3, (128, crkfr.CR_BATCH_FUSED, 2), dissipation=diss, central=cen)
    _same(got, ref, crkfr.CR_FP64, "variant %d %d" % (diss, cen))
