"""Pins of the kappa part of the splitting of Sec. 3 in the FP64 oracle.

The profile gamma(s) = s^{-alpha} chi(s < 1) splits as kappa(s) + p^{2K}(s) chi(s < 1) (Sec. 3),
with p^{2K} the even polynomial matching gamma and its first K derivatives at s = 1, so that
kappa vanishes to order K + 1 at the horizon (smooth there) while keeping the singularity at 0.
"""
import numpy as np
import pytest

import oracle
from paper_1905_08375_gb300 import synth

# gamma = 1/s: kappa_K(s) = (1 - s)^{K+1} q_K(s) / s, q_K from the polynomial division of
# 1 - s p^{2K}(s) by (1 - s)^{K+1} (K = 3 with the Hermite p^6, reading A8), lowest power first
Q = {0: [1.0], 1: [1.0, 0.5], 2: [1.0, 9 / 8, 3 / 8], 3: [1.0, 29 / 16, 5 / 4, 5 / 16]}


def kappa_closed(K, s):
    q = sum(c * s ** m for m, c in enumerate(Q[K]))
    return (1.0 - s) ** (K + 1) * q / s


@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_weights_equal_the_factorised_closed_form(K):
    # 1-D, C = 1, sigma = 1: (L e_j)_i = h delta^-3 kappa(|x_j - x_i| / delta) for j != i
    n, i, rho = 128, 64, 20.5
    h = 1.0 / n
    delta = rho * h
    for m in range(1, 21):
        u = np.zeros(n)
        u[i + m] = 1.0
        Lu = oracle.direct_scalar(u, 1, n, delta, family=oracle.KAPPA, alpha=1.0, K=K,
                                  normalize=False, idx=[i])
        w = Lu[0] / h * delta ** 3
        assert w == pytest.approx(kappa_closed(K, m / rho), rel=1e-11, abs=1e-13), m


@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_second_moment_continuum_limit(K):
    # 1-D, gamma = 1/s, sigma = 1: L[x^2] -> int_{-1}^{1} kappa(|s|) s^2 ds
    #   = int |s| ds - 2 sum_m p_m / (2m + 3) = 1 - (2K + 2)/(2K + 3) = 1/(2K + 3)
    n, delta = 4096, 0.25
    x = (np.arange(n) + 0.5) / n
    i = n // 2
    Lu = oracle.direct_scalar(x ** 2, 1, n, delta, family=oracle.KAPPA, alpha=1.0, K=K,
                              normalize=False, idx=[i])
    assert Lu[0] == pytest.approx(1.0 / (2 * K + 3), rel=1e-4)


@pytest.mark.parametrize("K", [0, 1, 3])
def test_splitting_identity_variable_horizon(K):
    # Sec. 3: gamma chi = kappa + p^{2K} chi, so on one quadrature set (the direct sum over the
    # open ball) L^gamma = L^kappa + L^P, here with a variable horizon and C = a(x) a(y)
    n = 24
    f = synth.heterogeneous_2d(n=n, seed=3, nrhs=1, rmin=2.0, rspan=5.0)
    kw = dict(alpha=1.5, K=K, coef=oracle.COEF_XY, a=f["a"])
    g = oracle.direct_scalar(f["u"][0], 2, n, f["delta"], family=oracle.POWER, **kw)
    k = oracle.direct_scalar(f["u"][0], 2, n, f["delta"], family=oracle.KAPPA, **kw)
    p = oracle.direct_scalar(f["u"][0], 2, n, f["delta"], family=oracle.POLY, **kw)
    assert np.linalg.norm(g - (k + p)) <= 1e-13 * np.linalg.norm(g)
    # kappa is not zero and not the whole kernel
    assert 0.05 * np.linalg.norm(g) < np.linalg.norm(k) < 0.95 * np.linalg.norm(g)


def test_kappa_annihilates_constants_and_linear_fields_in_the_interior():
    n, delta = 40, 6.5 / 40
    X, Y = synth.node_coords(2, n)
    for u in (np.ones((n, n)), 0.3 * X - 1.7 * Y):
        Lu = oracle.direct_scalar(u.reshape(-1), 2, n, delta, family=oracle.KAPPA, alpha=1.0,
                                  K=2).reshape(n, n)
        assert np.abs(Lu[8:-8, 8:-8]).max() <= 1e-9 * np.abs(Lu).max() + 1e-10
