"""Pins of the FP64 MLP oracle: the analytic gradient against central finite
differences, closed forms of GELU / sigmoid / cross-entropy, the Adam update against a
hand-evaluated first step, and BF16 rounding against its definition."""
import math

import numpy as np

from oracle import mlp


def batch(n=12, seed=3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, mlp.NF)), (rng.random(n) < 0.4).astype(np.float64)


def test_parameter_count():
    assert mlp.NPARAM == 8 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4801


def test_gelu_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(mlp.gelu_grad(np.array([0.0])), [0.5], rtol=0, atol=1e-15)
    # large |a|: GELU -> relu
    np.testing.assert_allclose(mlp.gelu(np.array([8.0, -8.0])), [8.0, 0.0], atol=1e-12)
    # derivative against central differences
    a = np.linspace(-3, 3, 13)
    hh = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(a), (mlp.gelu(a + hh) - mlp.gelu(a - hh)) / (2 * hh), rtol=1e-8,
                               atol=1e-9)


def test_gradient_matches_finite_differences():
    x, y = batch()
    theta = mlp.init_params(5)
    g = mlp.grad(theta, x, y)
    rng = np.random.default_rng(9)
    idx = np.concatenate([rng.choice(mlp.NPARAM, 60, replace=False), [0, 512, 576, 4672, 4800]])
    hh = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += hh
        tm[i] -= hh
        fd = (mlp.loss(tp, x, y) - mlp.loss(tm, x, y)) / (2 * hh)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_output_gradient_closed_form():
    # with every hidden weight zero, z = b3 for all samples: dL/db3 = mean(p - y)
    x, y = batch()
    parts = mlp.unpack(np.zeros(mlp.NPARAM))
    parts["b3"] = np.array([0.3])
    theta = mlp.pack(parts)
    g = mlp.unpack(mlp.grad(theta, x, y))
    p = 1.0 / (1.0 + math.exp(-0.3))
    np.testing.assert_allclose(g["b3"][0], np.mean(p - y), rtol=1e-14)
    assert np.all(g["W1"] == 0) and np.all(g["W2"] == 0)


def test_adam_first_step_is_signed_lr():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.1, 0.0])
    t1, m, v = mlp.adam_step(theta, np.zeros(3), np.zeros(3), g, 1, lr=0.01)
    # bias-corrected first step: -lr * g / (|g| + eps)
    np.testing.assert_allclose(t1, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-14)


def test_bf16_rounding_definition():
    # bfloat16 keeps 8 significant bits: next to 1.0 the spacing is 2^-7
    v = np.array([1.0, 1.00390625, 1.001953125, 1.005859375, -3.14159, 65504.0, 1e-20, 1.01171875],
                 dtype=np.float32)
    r = mlp.round_bf16(v)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to the even mantissa (1.0);
    # 1 + 2^-9 rounds down; 1 + 3 * 2^-9 rounds up; 1 + 2^-7 + 2^-8 ties up to the even 1 + 2^-6
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 and r[3] == 1.0078125 and r[7] == 1.015625
    # every result has at most 8 significant bits
    for x in r:
        if x != 0:
            m, _ = math.frexp(x)
            assert abs(m * 256 - round(m * 256)) < 1e-12
    assert abs(r[4] - (-3.140625)) < 1e-12


def test_training_lowers_the_loss():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((400, mlp.NF))
    y = (x[:, 0] + 0.5 * x[:, 3] > 0.2).astype(np.float64)
    theta = mlp.init_params(2)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    l0 = mlp.loss(theta, x, y)
    for t in range(1, 201):
        theta, m, v = mlp.adam_step(theta, m, v, mlp.grad(theta, x, y), t, lr=1e-2)
    assert mlp.loss(theta, x, y) < 0.3 * l0
