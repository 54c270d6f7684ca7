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


def _dense(fn, N):
    return np.stack([fn(np.eye(N)[k]) for k in range(N)], axis=1)


def test_two_level_map_is_symmetric_positive_definite_and_restrict_is_adjoint():
    n, b = 7, 3                                         # ragged last block
    rng = np.random.default_rng(8)
    w = _weights(9)
    dinv = rng.uniform(0.5, 2.0, n * n)
    N = n * n
    # R^T = P: <R x, y> = <x, P y>
    x = rng.standard_normal(N)
    y = rng.standard_normal((3, 3))
    assert abs(np.sum(convnet.restrict(x, n, b) * y) - x @ convnet.prolong(y, n, b)) < 1e-12
    # an explicit block-sum matrix for R
    Rm = np.zeros((9, N))
    for k in range(N):
        Rm[(k // n // b) * 3 + (k % n) // b, k] = 1.0
    np.testing.assert_allclose(convnet.restrict(x, n, b).ravel(), Rm @ x, atol=1e-12)
    M = _dense(lambda v: convnet.apply_two_level(w, v, dinv, n, b), N)
    np.testing.assert_allclose(M, M.T, atol=1e-10 * np.abs(M).max())
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
    # and it is D^{-1} + gamma R^T (K^T K) R with K the dense linear chain
    Ws = convnet.split(convnet.bf16_round(w))
    K = _dense(lambda v: convnet.linear_chain(Ws, v.reshape(1, 3, 3))[0].ravel(), 9)
    ref = np.diag(dinv) + convnet.two_level_gamma(dinv, b) * Rm.T @ (K.T @ K) @ Rm
    np.testing.assert_allclose(M, ref, atol=1e-10 * np.abs(ref).max())


def test_linear_chain_matches_torch_and_adjoint():
    w = _weights(10)
    x = np.random.default_rng(11).standard_normal((2, 6, 5))
    Ws = convnet.split(w)
    u, _ = convnet.linear_chain(Ws, x)
    W1, W2, W3 = [torch.tensor(t) for t in Ws]
    t = torch.nn.functional.conv2d(torch.tensor(x)[:, None], W1, padding=1)
    t = torch.nn.functional.conv2d(t, W2, padding=1)
    t = torch.nn.functional.conv2d(t, W3, padding=1)[:, 0]
    np.testing.assert_allclose(u, t.numpy(), rtol=1e-12, atol=1e-12)
    y = np.random.default_rng(12).standard_normal((2, 6, 5))
    lhs = np.sum(u * y)
    rhs = np.sum(x * convnet.linear_chain_adjoint(Ws, y))
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_two_level_gradient_matches_finite_differences():
    n, b = 6, 2
    rng = np.random.default_rng(13)
    N = n * n
    Q = rng.standard_normal((N, N))
    A = Q @ Q.T + N * np.eye(N)                          # an SPD stand-in for -L
    apply_A = lambda v: v @ A.T
    dinv = 1.0 / np.diag(A)
    e = rng.standard_normal((2, N))
    r = apply_A(e)
    w = _weights(14, 0.3)
    _, g = convnet.two_level_energy_loss_and_grad(w, r, e, dinv, n, b, apply_A, round_bf16=False)
    for k in rng.choice(convnet.NPARAM, size=40, replace=False):
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        lp, _ = convnet.two_level_energy_loss_and_grad(wp, r, e, dinv, n, b, apply_A, False)
        lm, _ = convnet.two_level_energy_loss_and_grad(wm, r, e, dinv, n, b, apply_A, False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])
