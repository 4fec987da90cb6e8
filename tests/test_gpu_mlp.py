"""Learned blending coefficient on the GPU, checked against the FP64 CPU
reference (oracle/mlp.py, oracle.modal_energies):

* the network inputs (normalised modal energies of the indicator variable,
  Sec. 4) the fused inference kernel computes, element by element;
* the network output with BF16 weights and FP32 arithmetic against the FP64
  forward pass on the same BF16-rounded weights and the same inputs;
* one whole cRKFR step with the learned alpha against the oracle step given
  the same raw alpha (1e-12 relative, as every FP64 step);
* the fallbacks to the indicator (no network loaded, a non-finite output);
* the training kernels: cross-entropy loss and gradient against the
  hand-derived FP64 backward pass, and Adam training that fits the
  indicator's alpha.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2502_07517_gb300 import crkfr
from paper_2502_07517_gb300 import workloads as wl
from tests._oracle_util import oracle_desc

pytestmark = pytest.mark.gpu

FEATURE_ATOL = 2e-6   # FP32 energy ratio and log10f of an FP64 modal energy
ALPHA_ATOL = 1e-5     # FP32 network arithmetic vs FP64 on the same BF16 weights


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_07517_gb300 import build
    build.build()


def _cases():
    out = []
    prob, u = wl.euler2d_vortex(nx=13, ny=11, degree=3, seed=5)
    out.append(("euler2d_N3", prob, u * np.random.default_rng(5).uniform(0.5, 2.0, (1, u.shape[1], 1))))
    out.append(("tenmoment2d_N3",) + wl.tenmoment2d_voronoi(nx=12, ny=10, degree=3, seed=6))
    out.append(("euler1d_N4",) + wl.euler1d_riemann(nx=61, degree=4, seed=7))
    prob, u = wl.euler2d_vortex(nx=9, ny=8, degree=4, seed=8)
    out.append(("euler2d_N4", prob, u * np.random.default_rng(8).uniform(0.5, 2.0, (1, u.shape[1], 1))))
    return out


CASES = _cases()


def _params(nin, seed, scale=0.6):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, scale, mlp.param_count(nin))
    p[-1] = -0.5
    return p.astype(np.float32)


def _ctx(prob, mode=crkfr.CR_ALPHA_MLP, precision=crkfr.CR_FP64):
    return crkfr.cr_init_mesh(crkfr.desc_from_problem(prob, precision=precision, alpha_mode=mode))


def _oracle_features(prob, u):
    d = oracle_desc(prob)
    return np.stack([mlp.encode(oracle.modal_energies(d, u[:, e, :].T)) for e in range(u.shape[1])])


@pytest.mark.parametrize("name,prob,u", CASES, ids=[c[0] for c in CASES])
def test_features_match_oracle(name, prob, u):
    ctx = _ctx(prob)
    crkfr.cr_set_state(ctx, u)
    f, _ = crkfr.cr_get_features(ctx, u.shape[1], u.shape[2])
    ref = _oracle_features(prob, u)
    assert np.abs(f - ref).max() <= FEATURE_ATOL, np.abs(f - ref).max()


def _centred_params(prob, u, seed):
    """Random weights with the output bias set so that the median element sits
    at z = 0: the outputs then spread over (0, 1) instead of saturating."""
    p = _params(u.shape[2], seed)
    p[-1] = 0.0
    y, _ = mlp.forward(mlp.bf16_round(p).astype(np.float64), _oracle_features(prob, u))
    z = np.log(y / (1.0 - y))
    p[-1] = -np.median(z)
    return p


def _wiggle(u, seed):
    """Scale every node's conserved variables by its own factor in [0.7, 1.4]:
    stays admissible, and every element gets its own modal energies."""
    return u * np.random.default_rng(seed).uniform(0.7, 1.4, (1,) + u.shape[1:])


@pytest.mark.parametrize("name,prob,u", CASES, ids=[c[0] for c in CASES])
def test_learned_alpha_matches_fp64_forward(name, prob, u):
    npts = u.shape[2]
    u = _wiggle(u, npts)
    p = _centred_params(prob, u, seed=npts)
    ctx = _ctx(prob)
    crkfr.cr_set_state(ctx, u)
    crkfr.cr_mlp_load(ctx, p)
    f, a = crkfr.cr_get_features(ctx, u.shape[1], npts)
    y, _ = mlp.forward(mlp.bf16_round(p).astype(np.float64), f.astype(np.float64))
    ref = mlp.alpha_from_output(y)
    near = (np.abs(y - 1e-3) < 1e-5) | (np.abs(y - (1 - 1e-3)) < 1e-5)  # clip decided either way
    err = np.abs(a - ref)[~near]
    assert err.max() <= ALPHA_ATOL, err.max()
    assert np.mean((ref > 0.05) & (ref < 0.95)) > 0.3  # a spread of alphas, not a constant


@pytest.mark.parametrize("name,prob,u", CASES, ids=[c[0] for c in CASES])
def test_step_with_learned_alpha_matches_oracle(name, prob, u):
    from tests.test_gpu_parity import assert_parity, flux_increment
    npts = u.shape[2]
    u = _wiggle(u, npts + 1)
    ctx = _ctx(prob)
    crkfr.cr_set_state(ctx, u)
    crkfr.cr_mlp_load(ctx, _centred_params(prob, u, seed=npts + 1))
    _, a = crkfr.cr_get_features(ctx, u.shape[1], npts)
    d = oracle_desc(prob, alpha_given=a)
    dt = oracle.dt(d, u)
    ref, st, dg = oracle.step(d, u, dt, want_diag=True)
    assert st == 0
    crkfr.cr_step(ctx, 1, 1e300, dt)
    g = crkfr.cr_get_state(ctx, shape=u.shape)
    assert_parity(g, ref, extra_scale=flux_increment(prob, dg, dt))
    np.testing.assert_allclose(crkfr.cr_get_alpha(ctx, u.shape[1]), dg["alpha"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("precision", [crkfr.CR_FP64, crkfr.CR_FP32_BULK])
def test_fallback_to_indicator(precision):
    """No network loaded, or a network whose output is NaN: the step is the
    indicator's step, bit for bit."""
    name, prob, u = CASES[0]
    npts = u.shape[2]

    def run(mode, params=None):
        ctx = _ctx(prob, mode, precision)
        crkfr.cr_set_state(ctx, u)
        if params is not None:
            crkfr.cr_mlp_load(ctx, params)
        crkfr.cr_step(ctx, 3, 1e300)
        return crkfr.cr_get_state(ctx, shape=u.shape)

    ref = run(crkfr.CR_ALPHA_INDICATOR)
    np.testing.assert_array_equal(run(crkfr.CR_ALPHA_MLP), ref)
    p = np.zeros(mlp.param_count(npts), dtype=np.float32)
    H = mlp.H
    o_b2 = H * npts + H + H * H
    p[o_b2:o_b2 + H] = -1.0               # every second-layer unit is off ...
    p[o_b2 + H:o_b2 + 2 * H] = np.inf     # ... and inf * 0 makes the output NaN
    np.testing.assert_array_equal(run(crkfr.CR_ALPHA_MLP, p), ref)
    y, _ = mlp.forward(p.astype(np.float64), np.zeros((1, npts)))
    assert np.isnan(y[0])


def test_load_rejects_bad_parameters():
    name, prob, u = CASES[0]
    ctx = _ctx(prob)
    n = mlp.param_count(u.shape[2])
    assert crkfr.cr_mlp_param_count(u.shape[2]) == n
    assert crkfr.cr_mlp_param_count(7) == -1
    with pytest.raises(crkfr.CrError):
        crkfr.cr_mlp_load(ctx, np.zeros(n - 1, dtype=np.float32))
    bad = np.zeros(n, dtype=np.float32)
    bad[3] = np.nan
    with pytest.raises(crkfr.CrError):
        crkfr.cr_mlp_load(ctx, bad)


@pytest.mark.parametrize("nin,n", [(16, 1000), (25, 333), (5, 64), (16, 1)])
def test_gradient_matches_fp64_backward(nin, n):
    import torch
    rng = np.random.default_rng(nin + n)
    p = _params(nin, seed=nin, scale=0.4)
    X = rng.uniform(0.0, 1.0, (n, nin)).astype(np.float32)
    t = rng.uniform(0.0, 1.0, n).astype(np.float32)
    dev = lambda a: torch.from_numpy(a).cuda()
    grad = torch.full((p.size,), 7.0, device="cuda")   # overwritten, not accumulated
    loss = torch.full((1,), 7.0, device="cuda")
    crkfr.cr_mlp_grad(nin, dev(p), dev(X), dev(t), grad, loss)
    torch.cuda.synchronize()
    p64, X64, t64 = p.astype(np.float64), X.astype(np.float64), t.astype(np.float64)
    g_ref = mlp.grad(p64, X64, t64)
    l_ref = mlp.loss(p64, X64, t64)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - l_ref) <= 1e-5 * l_ref
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max(), np.abs(g - g_ref).max()


def _indicator_samples(seeds, nx=48, steps=(0, 6, 12)):
    """Network inputs and the indicator's raw alpha harvested along GPU runs of
    the ten-moment workload recipe (N = 3, 16 inputs)."""
    X, T = [], []
    for seed in seeds:
        prob, u = wl.tenmoment2d_voronoi(nx=nx, ny=nx, degree=3, seed=seed)
        ctx = _ctx(prob, crkfr.CR_ALPHA_INDICATOR)
        crkfr.cr_set_state(ctx, u)
        done = 0
        for s in steps:
            if s > done:
                crkfr.cr_step(ctx, s - done, 1e300)
                done = s
            f, a = crkfr.cr_get_features(ctx, u.shape[1], u.shape[2])
            X.append(f)
            T.append(a)
    return np.concatenate(X), np.concatenate(T)


def test_training_fits_the_indicator():
    import torch
    X, T = _indicator_samples(range(4))
    assert 0.02 < T.mean() < 0.9
    nin = X.shape[1]
    p = torch.from_numpy(_params(nin, seed=0, scale=0.2)).cuda()
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T.astype(np.float32)).cuda()
    g, l0 = torch.empty_like(p), torch.empty(1, device="cuda")
    crkfr.cr_mlp_grad(nin, p, Xd, Td, g, l0)
    first = l0.item()
    loss = crkfr.cr_mlp_train(nin, p, Xd, Td, batch=256, epochs=30, lr=3e-3, seed=1)
    crkfr.cr_mlp_grad(nin, p, Xd, Td, g, l0)
    assert l0.item() < first
    y, _ = mlp.forward(p.cpu().numpy().astype(np.float64), X.astype(np.float64))
    mse, var = float(np.mean((y - T) ** 2)), T.var()
    print("samples", T.size, "target var %.4f, trained mse %.5f (cross-entropy %.4f -> %.4f, last epoch %.4f)"
          % (var, mse, first, l0.item(), loss))
    assert mse < 0.1 * var
    # served by the fused inference kernel on an unseen seed
    Xv, Tv = _indicator_samples([11], steps=(0, 8))
    prob, u = wl.tenmoment2d_voronoi(nx=48, ny=48, degree=3, seed=11)
    ctx = _ctx(prob)
    crkfr.cr_set_state(ctx, u)
    crkfr.cr_mlp_load(ctx, p.cpu().numpy())
    _, a = crkfr.cr_get_features(ctx, u.shape[1], u.shape[2])
    t0 = Tv[:u.shape[1]]
    print("unseen seed: mean |alpha_mlp - alpha_indicator| %.4f" % np.abs(a - t0).mean())
    assert np.abs(a - t0).mean() < 0.05
