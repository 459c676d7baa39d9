"""FP64 numpy oracle of the learned interface-placement network.

TEST INFRASTRUCTURE (see oracle/__init__.py): used only by tests/, the smoke check and
the benchmark's CPU-baseline leg.

The network is not in the paper (it extends the switching-criterion discussion of
Sec. 2.2, which leaves the criterion open): 8 normalised local features -> 64 -> 64 -> 1
with GELU hidden activations (exact, erf form) and a sigmoid output giving
p(high-order set needed); loss = mean binary cross-entropy; optimiser = Adam.

Parameter vector layout (4801 values), shared by both implementations as a data format:
W1 [64][8], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1].
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

NF, NH = 8, 64
SIZES = (("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)), ("b3", (1,)))
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, k = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SIZES])


def init_params(seed=1007):
    """He-style normal initialisation (scale sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = {"W1": rng.standard_normal((NH, NF)) * math.sqrt(2.0 / NF), "b1": np.zeros(NH),
             "W2": rng.standard_normal((NH, NH)) * math.sqrt(2.0 / NH), "b2": np.zeros(NH),
             "W3": rng.standard_normal(NH) * math.sqrt(2.0 / NH), "b3": np.zeros(1)}
    return pack(parts)


def gelu(a):
    return 0.5 * a * (1.0 + erf(a / math.sqrt(2.0)))


def gelu_grad(a):
    return 0.5 * (1.0 + erf(a / math.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(theta, x):
    """x [B][8] (already normalised) -> p [B], plus the intermediates."""
    P = unpack(theta)
    a1 = x @ P["W1"].T + P["b1"]
    h1 = gelu(a1)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = gelu(a2)
    z = h2 @ P["W3"] + P["b3"][0]
    return sigmoid(z), (x, a1, h1, a2, h2, z)


def forward_bf16_operands(theta, x):
    """The forward pass with the precision of a tensor-core inference: BF16-rounded
    weights and biases, and the inputs of the first two layers (the normalised features
    and the first hidden activations) rounded to BF16 before each product; sums, GELU and
    the output layer in FP64. x [B][8] (normalised) -> p [B]."""
    P = unpack(round_bf16(theta))
    xr = round_bf16(x)
    a1 = xr @ P["W1"].T + P["b1"]
    h1 = round_bf16(gelu(a1))
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = gelu(a2)
    z = h2 @ P["W3"] + P["b3"][0]
    return sigmoid(z)


def loss(theta, x, y):
    p, _ = forward(theta, x)
    p = np.clip(p, 1e-300, 1.0 - 1e-16)
    return float(-np.mean(y * np.log(p) + (1.0 - y) * np.log(1.0 - p)))


def grad(theta, x, y):
    """Analytic gradient of the mean cross-entropy, packed like theta."""
    P = unpack(theta)
    p, (x, a1, h1, a2, h2, z) = forward(theta, x)
    B = x.shape[0]
    dz = (p - y) / B
    g = {"W3": h2.T @ dz, "b3": np.array([dz.sum()])}
    dh2 = np.outer(dz, P["W3"])
    da2 = dh2 * gelu_grad(a2)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ P["W2"]
    da1 = dh1 * gelu_grad(a1)
    g["W1"] = da1.T @ x
    g["b1"] = da1.sum(axis=0)
    return pack(g)


def adam_step(theta, m, v, g, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) at step t >= 1; returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def round_bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
