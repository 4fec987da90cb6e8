"""What the learned blending coefficient gains, measured against exact
solutions: seeded 1D Euler Riemann problems (the 1D Euler workload recipe,
N = 4, 400 elements, all limiters on) are run until just before the fastest
wave reaches the boundary, and the L1 error of the density against the exact
Riemann solution is compared for

* alpha from the smoothness indicator (the method of Sec. 4),
* alpha from the network trained on the GPU on the indicator's alpha of other
  seeds (served by the fused inference kernel),
* no blending at all (alpha = 0: the unlimited high-order scheme, with only
  the flux and scaling limiters keeping the solution admissible).

The network is trained to imitate the indicator, so it cannot beat it on
accuracy; what it offers over the method without it (no blending) is the
indicator's shock capturing with the indicator kept as fallback.  A run whose
step turns out inadmissible stops there and is counted as failed.  The test
asserts that the learned alpha fails no more often than the indicator, that
its error relative to the indicator's has a median within 10% and a geometric
mean within 25% over the problems, and that it beats the unblended scheme
(which either fails or is less accurate), and prints all of it.
"""
import json
import os

import numpy as np
import pytest

from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl
from tests import _riemann_exact as rx

pytestmark = pytest.mark.gpu

NX, N = 400, 4
TRAIN_SEEDS = range(100, 148)
TEST_SEEDS = range(0, 10)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_07517_gb300 import build
    build.build()


def _states(prob):
    r = prob["riemann"]
    return (r["rho"][0], r["v"][0], r["p"][0]), (r["rho"][1], r["v"][1], r["p"][1])


def _usable(seed):
    prob, u = wl.euler1d_riemann(nx=NX, degree=N, seed=seed)
    L, R = _states(prob)
    return (not rx.vacuum(L, R)), prob, u


def _t_end(prob):
    L, R = _states(prob)
    return min(0.2, 0.4 / rx.max_speed(L, R))


def _train():
    import torch
    X, T = [], []
    for seed in TRAIN_SEEDS:
        ok, prob, u = _usable(seed)
        if not ok:
            continue
        ctx = crkfr.cr_init_mesh(crkfr.desc_from_problem(prob))
        crkfr.cr_set_state(ctx, u)
        t_end = _t_end(prob)
        for frac in (0.0, 0.02, 0.05, 0.1, 0.2, 0.35, 0.5, 0.75, 1.0):
            if frac > 0:
                crkfr.cr_step(ctx, 10 ** 7, frac * t_end)
            f, a = crkfr.cr_get_features(ctx, NX, N + 1)
            X.append(f)
            T.append(a)
    X, T = np.concatenate(X), np.concatenate(T).astype(np.float32)
    nin = N + 1
    p = torch.from_numpy(np.random.default_rng(0).normal(0, 0.2, crkfr.cr_mlp_param_count(nin))
                         .astype(np.float32)).cuda()
    crkfr.cr_mlp_train(nin, p, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), batch=256,
                       epochs=60, lr=3e-3, seed=3)
    return p.cpu().numpy(), X.shape[0]


def _l1_rho(prob, g, t):
    x, _ = wl.node_coords(prob)
    _, w = wl.gl_nodes01(N)
    dx = (prob["x1"] - prob["x0"]) / prob["nx"]
    L, R = _states(prob)
    x_face = prob["x0"] + (prob["nx"] // 2) * dx
    ex = rx.sample(L, R, (x - x_face) / t)[0]
    return float((np.abs(g[0] - ex) * w[None, :] * dx).sum())


def test_learned_alpha_gain_on_exact_riemann_solutions():
    params, nsamples = _train()
    rows = []
    for seed in TEST_SEEDS:
        ok, prob, u = _usable(seed)
        if not ok:
            continue
        t_end = _t_end(prob)
        res = {}
        for name in ("indicator", "learned", "no_blend"):
            if name == "no_blend":
                p2 = dict(prob, limiter=frozenset({"flux", "scaling", "traces"}))
                d = crkfr.desc_from_problem(p2)
            else:
                mode = crkfr.CR_ALPHA_MLP if name == "learned" else crkfr.CR_ALPHA_INDICATOR
                d = crkfr.desc_from_problem(prob, alpha_mode=mode)
            ctx = crkfr.cr_init_mesh(d)
            crkfr.cr_set_state(ctx, u)
            if name == "learned":
                crkfr.cr_mlp_load(ctx, params)
            try:
                t, n = crkfr.cr_step(ctx, 10 ** 7, t_end)
            except crkfr.CrError as err:     # a step produced an inadmissible state
                assert err.status == -3
                res[name] = None
                res[name + "_failed_at_t"] = _time_reached(ctx)
                continue
            assert t == t_end
            g = crkfr.cr_get_state(ctx, shape=u.shape)
            assert np.all(np.isfinite(g))
            res[name] = _l1_rho(prob, g, t_end)
            res[name + "_steps"] = n
        rows.append(dict(seed=seed, **res))
    names = ("indicator", "learned", "no_blend")
    failed = {k: sum(r[k] is None for r in rows) for k in names}
    ratio = np.array([r["learned"] / r["indicator"] for r in rows
                      if r["learned"] is not None and r["indicator"] is not None])
    both = [r for r in rows if r["indicator"] is not None and r["learned"] is not None]
    mean = {k: float(np.mean([r[k] for r in both])) for k in ("indicator", "learned")}
    nb = [r for r in both if r["no_blend"] is not None]
    mean_nb = {k: float(np.mean([r[k] for r in nb])) for k in names} if nb else None
    print("\ntrained on %d samples; %d problems; failed runs %s" % (nsamples, len(rows), failed))
    print("mean L1(rho), indicator vs learned over %d problems: %s" % (len(both), mean))
    print("L1(learned)/L1(indicator) per problem: median %.3f, geometric mean %.3f, max %.3f"
          % (np.median(ratio), np.exp(np.log(ratio).mean()), ratio.max()))
    print("mean L1(rho) where the unblended scheme finished (%d): %s" % (len(nb), mean_nb))
    for r in rows:
        print(r)
    out = os.environ.get("CR_GAIN_JSON")
    if out:
        with open(out, "w") as fh:
            json.dump({"samples": nsamples, "failed": failed, "mean": mean, "mean_where_no_blend_ran": mean_nb,
                       "ratio_median": float(np.median(ratio)),
                       "ratio_geomean": float(np.exp(np.log(ratio).mean())), "ratio_max": float(ratio.max()),
                       "rows": rows}, fh, indent=1)
    assert len(rows) >= 6
    assert failed["learned"] <= failed["indicator"]
    # per problem, the learned alpha's error against the indicator's: typically equal, with
    # the occasional problem more sensitive to alpha; no single problem dominates the check
    assert np.median(ratio) <= 1.1 and np.exp(np.log(ratio).mean()) <= 1.25
    # what it gains over the method without it: the unblended scheme fails, or is less accurate
    assert failed["no_blend"] > 0 or mean_nb["learned"] < mean_nb["no_blend"]


def _time_reached(ctx):
    import ctypes
    t, n = ctypes.c_double(), ctypes.c_int()
    crkfr.lib().cr_sync(ctx.handle, ctypes.byref(t), ctypes.byref(n))
    return t.value
