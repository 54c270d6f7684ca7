"""Pins for the numpy oracle of the CG preconditioner network (a project addition)."""
import numpy as np
import pytest
import torch

from oracle import convnet


def _weights(seed=0, scale=0.2):
    return np.random.default_rng(seed).standard_normal(convnet.NPARAM) * scale


def test_forward_matches_torch_conv2d():
    w = _weights(1)
    x = np.random.default_rng(2).standard_normal((3, 11, 13))
    o, _ = convnet.forward(w, x)
    W1, W2, W3 = [torch.tensor(t) for t in convnet.split(convnet.bf16_round(w))]
    t = torch.tensor(x)[:, None]
    t = torch.relu(torch.nn.functional.conv2d(t, W1, padding=1))
    t = torch.relu(torch.nn.functional.conv2d(t, W2, padding=1))
    t = torch.nn.functional.conv2d(t, W3, padding=1)[:, 0]
    np.testing.assert_allclose(o, t.numpy(), rtol=1e-12, atol=1e-12)


def test_bf16_rounding_matches_torch():
    w = np.random.default_rng(3).standard_normal(1000).astype(np.float32) * 7
    ref = torch.tensor(w).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(convnet.bf16_round(w), ref)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    w = _weights(5)
    x = rng.standard_normal((2, 9, 10))
    e = rng.standard_normal((2, 9, 10))
    _, g = convnet.loss_and_grad(w, x, e, margin=1, round_bf16=False)
    for k in rng.choice(convnet.NPARAM, size=40, replace=False):
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        lp, _ = convnet.loss_and_grad(wp, x, e, margin=1, round_bf16=False)
        lm, _ = convnet.loss_and_grad(wm, x, e, margin=1, round_bf16=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_adam_first_step_is_signed_lr():
    w = np.zeros(5)
    g = np.array([1.0, -2.0, 0.5, 0.0, 3.0])
    w1, m, v = convnet.adam(w, g, np.zeros(5), np.zeros(5), 1, 0.01)
    np.testing.assert_allclose(w1[g != 0], -0.01 * np.sign(g[g != 0]), rtol=1e-6)
    assert w1[3] == 0.0
