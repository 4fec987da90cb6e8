"""FP64 reference of the learned blending coefficient.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark may use it; the CUDA library never does.

The paper's alpha comes from the smoothness indicator (Sec. 4).  The learned
variant replaces the indicator's last step by a small network: inputs are the
element's normalised modal energies e_k = m_k^2 / sum m^2 (the indicator's
own modes), encoded as x_k = log10(e_k + 1e-10) / 10 + 1; two hidden layers
of 32 ReLU units; a sigmoid output.  It is trained on the indicator's alpha
with the cross-entropy loss -mean(t log y + (1 - t) log(1 - y)), alpha in
[0, 1] taken as a probability: unlike the squared error, its gradient with
respect to the output logit, (y - t)/n, does not vanish where y saturates,
so alpha = 1 regions (shocks) are learned as 1.  This module is the plain
definition: forward pass, loss and the hand-derived backward pass, in FP64.

Pinned (tests/test_oracle_mlp.py) by central finite differences of the loss
(the backward pass against the forward pass), hand-built networks with a
closed-form output, and torch's own bfloat16 rounding.  The modal energies
come from oracle.modal_energies (the indicator's modes, pinned by pure
Legendre modes).

Parameter vector layout (float): W1 [H][nin], b1 [H], W2 [H][H], b2 [H],
w3 [H], b3 [1], with H = 32.
"""
import numpy as np

H = 32


def param_count(nin):
    return H * nin + H + H * H + H + H + 1


def unpack(params, nin):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * nin].reshape(H, nin); o += H * nin
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def encode(e):
    """Network input from normalised modal energies."""
    return np.log10(np.asarray(e, dtype=np.float64) + 1e-10) / 10.0 + 1.0


def forward(params, X):
    """X [B][nin] -> (y [B], cache)."""
    X = np.asarray(X, dtype=np.float64)
    W1, b1, W2, b2, w3, b3 = unpack(params, X.shape[1])
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w3 + b3
    y = 1.0 / (1.0 + np.exp(-z))
    return y, (X, a1, h1, a2, h2, y)


def _softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def logits(params, X):
    """Output before the sigmoid."""
    X = np.asarray(X, dtype=np.float64)
    W1, b1, W2, b2, w3, b3 = unpack(params, X.shape[1])
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss(params, X, t):
    """Cross-entropy, with log y = -softplus(-z) and log(1 - y) = -softplus(z)."""
    z = logits(params, X)
    t = np.asarray(t, dtype=np.float64)
    return float(np.mean(t * _softplus(-z) + (1.0 - t) * _softplus(z)))


def grad(params, X, t):
    """Gradient of the cross-entropy loss, same layout as params."""
    y, (X, a1, h1, a2, h2, y) = forward(params, X)
    W1, b1, W2, b2, w3, b3 = unpack(params, X.shape[1])
    B = X.shape[0]
    dz = (y - np.asarray(t, dtype=np.float64)) / B
    dw3 = h2.T @ dz
    db3 = dz.sum()
    da2 = np.outer(dz, w3) * (a2 > 0.0)
    dW2 = da2.T @ h1
    db2 = da2.sum(axis=0)
    da1 = (da2 @ W2) * (a1 > 0.0)
    dW1 = da1.T @ X
    db1 = da1.sum(axis=0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])


def alpha_from_output(y):
    """Clip of the indicator applied to the network output: below 1e-3 -> 0,
    above 1 - 1e-3 -> 1."""
    y = np.asarray(y, dtype=np.float64).copy()
    y[y < 1e-3] = 0.0
    y[y > 1.0 - 1e-3] = 1.0
    return np.minimum(y, 1.0)


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)
