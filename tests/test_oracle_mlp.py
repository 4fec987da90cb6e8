"""Pins of the learned blending coefficient's CPU reference (oracle/mlp.py and
oracle.modal_energies), each against something other than the reference
itself: finite differences of its own loss, networks whose output is known
in closed form, pure Legendre modes, and torch's bfloat16 rounding."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp


def _params(nin, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, mlp.param_count(nin))


@pytest.mark.parametrize("nin", [5, 16, 25])
def test_grad_matches_central_differences(nin):
    rng = np.random.default_rng(nin)
    p = _params(nin, nin)
    X = rng.uniform(0.0, 1.0, (9, nin))
    t = rng.uniform(0.0, 1.0, 9)
    g = mlp.grad(p, X, t)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        a, b = p.copy(), p.copy()
        a[i] += h
        b[i] -= h
        fd[i] = (mlp.loss(a, X, t) - mlp.loss(b, X, t)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-9 * np.abs(fd).max())


def test_zero_network_is_sigmoid_of_output_bias():
    p = np.zeros(mlp.param_count(16))
    p[-1] = 0.7
    y, _ = mlp.forward(p, np.random.default_rng(0).uniform(size=(4, 16)))
    np.testing.assert_allclose(y, 1.0 / (1.0 + math.exp(-0.7)), rtol=1e-15)


def test_cross_entropy_of_a_constant_output():
    """Zero weights and output bias b: y = 1/(1 + e^-b) for every sample, so the
    loss is -(t log y + (1 - t) log(1 - y)) averaged over the targets."""
    p = np.zeros(mlp.param_count(5))
    p[-1] = -1.3
    t = np.array([0.0, 1.0, 0.25, 0.9])
    y = 1.0 / (1.0 + math.exp(1.3))
    ref = -np.mean(t * math.log(y) + (1 - t) * math.log(1 - y))
    assert abs(mlp.loss(p, np.ones((4, 5)), t) - ref) < 1e-15
    # and the output-bias gradient is mean(y - t)
    assert abs(mlp.grad(p, np.ones((4, 5)), t)[-1] - np.mean(y - t)) < 1e-15


def test_hand_built_network():
    """Hidden unit j of layer 1 reads input (3j mod nin) with weight j+1 and bias
    -0.25; layer 2 is the identity; the output sums the units with weights
    (-1)^j and bias 0.1: y = sigmoid(0.1 + sum_j (-1)^j relu((j+1) x_(3j mod nin) - 0.25))."""
    nin, H = 16, mlp.H
    W1 = np.zeros((H, nin))
    for j in range(H):
        W1[j, (3 * j) % nin] = j + 1
    b1 = np.full(H, -0.25)
    W2, b2 = np.eye(H), np.zeros(H)
    w3 = np.array([(-1.0) ** j for j in range(H)])
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [0.1]])
    x = np.linspace(0.05, 0.8, nin)
    z = 0.1
    for j in range(H):
        z += (-1.0) ** j * max((j + 1) * x[(3 * j) % nin] - 0.25, 0.0)
    y, _ = mlp.forward(p, x[None, :])
    assert abs(y[0] - 1.0 / (1.0 + math.exp(-z))) < 1e-15


def test_encoding_and_clip():
    np.testing.assert_allclose(mlp.encode([0.0, 1.0, 1e-5]), [0.0, 1.0 + math.log10(1 + 1e-10) / 10,
                                                             0.5 + math.log10(1 + 1e-5) / 10], rtol=1e-14)
    np.testing.assert_array_equal(mlp.alpha_from_output([5e-4, 0.5, 0.9995, 1.0]), [0.0, 0.5, 1.0, 1.0])


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.normal(0, 1, 4000).astype(np.float32),
                        np.float32([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0])])
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(a), ref)


def _legendre01(j, x):
    return np.polynomial.legendre.Legendre.basis(j)(2 * x - 1)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_modal_energies_of_pure_modes_1d(N):
    d = oracle.make_desc(dim=1, nx=1, degree=N)
    xi = oracle.tables(N)[0]
    for j in range(N + 1):
        ue = (_legendre01(j, xi) * 2.5)[:, None]
        e = oracle.modal_energies(d, ue)
        ref = np.zeros(N + 1)
        ref[j] = 1.0
        np.testing.assert_allclose(e, ref, atol=1e-13)


@pytest.mark.parametrize("N", [3, 4])
def test_modal_energies_2d_mode_index_and_mix(N):
    n = N + 1
    d = oracle.make_desc(dim=2, nx=1, ny=1, degree=N)
    xi = oracle.tables(N)[0]
    X, Y = xi[None, :], xi[:, None]          # node k = p + n q: x varies fastest
    i, j = 1, N                              # distinct x and y indices catch a transpose
    ue = (_legendre01(i, X) * _legendre01(j, Y)).reshape(-1)[:, None]
    e = oracle.modal_energies(d, ue)
    assert abs(e[i + n * j] - 1.0) < 1e-13 and abs(e.sum() - 1.0) < 1e-13
    # a mix 3 + 2 L_1(x): coefficients 3 and 2 -> energies 9/13, 4/13
    ue = (3.0 + 2.0 * _legendre01(1, X) + 0 * Y).reshape(-1)[:, None]
    e = oracle.modal_energies(d, ue)
    np.testing.assert_allclose([e[0], e[1]], [9 / 13, 4 / 13], atol=1e-13)
    assert abs(e.sum() - 1.0) < 1e-13


def test_modal_energies_euler_constant_pressure_density():
    d = oracle.make_desc(dim=2, nx=1, ny=1, degree=3, equation=oracle.EQ_EULER)
    ue = np.tile([2.0, 0.4, -0.2, 5.0], (16, 1))
    e = oracle.modal_energies(d, ue)
    ref = np.zeros(16)
    ref[0] = 1.0
    np.testing.assert_allclose(e, ref, atol=1e-13)
