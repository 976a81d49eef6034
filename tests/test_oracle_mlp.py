"""Pins of the FP64 MLP oracle (learned initialiser): bfloat16 rounding, backward pass, Adam."""
import numpy as np
import pytest
import torch

from oracle import mlp

DIMS = [6, 16, 16, 5]


def _params(seed=0):
    rng = np.random.default_rng(seed)
    n = sum(a * b + b for a, b in zip(DIMS[:-1], DIMS[1:]))
    return rng.uniform(-0.5, 0.5, n)


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(1).normal(0, 100, 10000)
    x = np.concatenate([x, [0.0, -0.0, 1.0, 3.0e38, 1e-40, 1.00390625, 1.01171875]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_backward_matches_finite_differences():
    p = _params()
    rng = np.random.default_rng(2)
    x = rng.normal(size=(7, DIMS[0])); t = rng.normal(size=(7, DIMS[-1]))
    loss, g = mlp.loss_and_grad(p, DIMS, x, t, bf16_ops=False)
    h = 1e-6
    for i in rng.choice(len(p), 40, replace=False):
        e = np.zeros_like(p); e[i] = h
        fd = (mlp.loss_and_grad(p + e, DIMS, x, t, False)[0] - mlp.loss_and_grad(p - e, DIMS, x, t, False)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_backward_matches_torch_autograd():
    p = _params(3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(9, DIMS[0])); t = rng.normal(size=(9, DIMS[-1]))
    loss, g = mlp.loss_and_grad(p, DIMS, x, t, bf16_ops=False)
    tp = torch.tensor(p, requires_grad=True)
    h = torch.tensor(x)
    o = 0
    n_layers = len(DIMS) - 1
    for l, (a, b) in enumerate(zip(DIMS[:-1], DIMS[1:])):
        W = tp[o:o + a * b].view(a, b); o += a * b
        bb = tp[o:o + b]; o += b
        h = h @ W + bb
        if l + 1 < n_layers:
            h = torch.nn.functional.silu(h)
    tl = torch.mean((h - torch.tensor(t)) ** 2)
    tl.backward()
    assert loss == pytest.approx(tl.item(), rel=1e-13)
    assert np.allclose(g, tp.grad.numpy(), rtol=1e-11, atol=1e-14)


def test_adam_first_step_is_sign_step():
    # after one step from zero moments, the update is lr * g / (|g| + eps) ~ lr * sign(g)
    p = np.zeros(5); g = np.array([1.0, -2.0, 0.5, -1e-3, 3.0])
    p1, m, v = mlp.adam(p, g, np.zeros(5), np.zeros(5), 1, lr=0.01)
    assert np.allclose(p1, -0.01 * np.sign(g), rtol=1e-4)


def test_magnitude_sums_equal_the_values_when_every_term_is_non_negative():
    # with non-negative inputs, weights and biases every term of every product is non-negative, so
    # the scale of the output (the sum of |terms|) is the output itself (the last layer's input is
    # a SiLU output, non-negative for non-negative pre-activations)
    rng = np.random.default_rng(4)
    dims = [3, 5, 4]
    n = sum(a * b + b for a, b in zip(dims[:-1], dims[1:]))
    p = rng.uniform(0.0, 1.0, n)
    x = rng.uniform(0.0, 1.0, (7, 3))
    y, _, _ = mlp.forward(p, dims, x, bf16_ops=False)
    sy, sg = mlp.magnitude_sums(p, dims, x, np.zeros((7, 4)), bf16_ops=False)
    np.testing.assert_allclose(sy, y, rtol=1e-14)
    # y > 0 = target, so every output error and hence every gradient term of the last layer is positive
    _, g = mlp.loss_and_grad(p, dims, x, np.zeros((7, 4)), bf16_ops=False)
    last = slice(n - (5 * 4 + 4), n)
    np.testing.assert_allclose(sg[last], g[last], rtol=1e-14)
