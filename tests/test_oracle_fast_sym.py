"""Pins of the oracle's symmetrised leaf-set operator (the divergence-type form of the Sec. 3
polynomial operator, a project extension): it reduces to the one-sided leaf-set operator for a
constant horizon (globally, and locally where every node that reaches a node has its
horizon), its matrix is symmetric and negative semi-definite, and its transpose half equals a scatter over each node's leaf rows (the form
a fast kernel would use)."""
import numpy as np
import pytest

import oracle
from paper_1905_08375_gb300 import synth


def smooth_delta(n, lo, hi, seed):
    s = synth.fourier_modes_field(np.random.default_rng(seed), 2, n, modes=4, kmax=2)
    return (lo + (hi - lo) * s).reshape(-1) / n


@pytest.mark.parametrize("d,L,K,coef", [(1, 6, 0, oracle.COEF_NONE), (1, 6, 2, oracle.COEF_XY),
                                        (2, 4, 0, oracle.COEF_XY), (2, 4, 1, oracle.COEF_NONE)])
def test_constant_horizon_reduces_to_one_sided(d, L, K, coef):
    n = 1 << L
    rng = np.random.default_rng(L + K)
    u = rng.standard_normal((2, n ** d))
    a = np.exp(0.3 * rng.standard_normal(n ** d)) if coef == oracle.COEF_XY else None
    delta = 3.3 / n
    kw = dict(K=K, alpha=1.0, coef=coef, a=a)
    sym = oracle.fast_sym_leafset(u, d, L, delta, **kw)
    one = oracle.fast_leafset(u, d, L, delta, **kw)
    assert np.abs(sym - one).max() <= 1e-12 * np.abs(one).max()


def assembled(n, delta, a, K):
    N = n * n
    A = np.zeros((N, N))
    E = np.eye(N)
    for j0 in range(0, N, 64):
        cols = oracle.fast_sym_leafset(E[j0:j0 + 64], 2, int(np.log2(n)), delta, K=K, alpha=1.0,
                                       coef=oracle.COEF_XY, a=a)
        A[:, j0:j0 + 64] = cols.T
    return A


@pytest.mark.parametrize("K", [0, 2])
def test_matrix_symmetric_negative_semidefinite(K):
    n = 16
    delta = smooth_delta(n, 1.5, 4.5, seed=K)
    a = np.exp(0.4 * np.random.default_rng(3).standard_normal(n * n))
    A = assembled(n, delta, a, K)
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() <= 1e-12 * np.abs(ev).max()
    # one-sided operator with the same horizons is not symmetric (the check has teeth)
    B = np.zeros_like(A)
    E = np.eye(n * n)
    for j0 in range(0, n * n, 64):
        B[:, j0:j0 + 64] = oracle.fast_leafset(E[j0:j0 + 64], 2, 4, delta, K=K, alpha=1.0,
                                               coef=oracle.COEF_XY, a=a).T
    assert np.abs(B - B.T).max() > 1e-3 * np.abs(B).max()


@pytest.mark.parametrize("K", [0, 1])
def test_locally_constant_horizon_matches_one_sided(K):
    # horizon 2.5h for x < 1/2 and 4.5h beyond: every node k whose leaf set reaches a node i
    # with x_i < 1/2 - 6h has the horizon of i (exterior cells take it too), so there both
    # halves of the symmetrised weights equal the one-sided ones and the operators agree on a
    # field that the weights do not annihilate; near the jump they differ
    n, L = 32, 5
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    delta = np.where(X < 0.5, 2.5 * h, 4.5 * h).reshape(-1)
    a = np.exp(0.2 * np.random.default_rng(7).standard_normal(n * n))
    u = (X ** 2 + 0.5 * Y ** 2 + X * Y).reshape(-1)
    kw = dict(K=K, alpha=1.0, coef=oracle.COEF_XY, a=a)
    sym = oracle.fast_sym_leafset(u, 2, L, delta, **kw).reshape(n, n)
    one = oracle.fast_leafset(u, 2, L, delta, **kw).reshape(n, n)
    left = x < 0.5 - 6 * h
    assert np.abs(one[:, left]).min() > 0.0
    assert np.abs(sym[:, left] - one[:, left]).max() <= 1e-12 * np.abs(one[:, left]).max()
    jump = np.abs(x - 0.5) < 2 * h
    assert np.abs(sym[:, jump] - one[:, jump]).max() > 1e-3 * np.abs(one).max()


def leaf_run(X, R2x4, dy2):
    """Cells kx (units of h) of one leaf row whose cell [2kx, 2kx + 2] (half units) meets the open
    ball of radius^2 R2x4 (quarter units) around the node at half-unit abscissa X, given the
    row's squared vertical gap dy2: the run kx0..kx1, or None."""
    rem = R2x4 - dy2
    if rem <= 0:
        return None
    r = int(np.floor(np.sqrt(rem)))
    while r * r >= rem:
        r -= 1
    while (r + 1) * (r + 1) < rem:
        r += 1
    return -((r - X) // 2) - 1, (X + r) // 2      # cells with |gap| < sqrt(rem) along x


def test_transpose_half_is_a_leaf_row_scatter():
    # K = 0, C = a_i a_k: L_i = h^2/2 [one-sided sum over LS(i)] + h^2/2 [sum over the k with
    # i in LS(k)], the second half scattered by each k along its leaf rows with difference arrays
    L = 4
    n = 1 << L
    h = 1.0 / n
    delta = smooth_delta(n, 1.5, 4.5, seed=9)
    rng = np.random.default_rng(10)
    a = np.exp(0.3 * rng.standard_normal(n * n))
    u = rng.standard_normal(n * n)
    one = oracle.fast_leafset(u, 2, L, delta, K=0, alpha=1.0, normalize=False,
                              coef=oracle.COEF_XY, a=a) / h ** 2
    D = np.zeros((n, n + 1))
    E = np.zeros((n, n + 1))
    ext = np.zeros(n * n)              # exterior cells in each node's own leaf set
    for k in range(n * n):
        kx, ky = k % n, k // n
        X, Y = 2 * kx + 1, 2 * ky + 1
        R2x4 = 4.0 * (delta[k] * n) ** 2
        c = a[k] * delta[k] ** -4.0
        for y in range(-2 * n, 3 * n):
            y0, y1 = 2 * y, 2 * y + 2
            dy2 = (y0 - Y) ** 2 if y0 > Y else ((y1 - Y) ** 2 if y1 < Y else 0)
            run = leaf_run(X, R2x4, dy2)
            if run is None:
                continue
            x0, x1 = run
            inside_row = 0 <= y < n
            lo, hi = max(x0, 0), min(x1, n - 1)
            ext[k] += (x1 - x0 + 1) - ((hi - lo + 1) if (inside_row and lo <= hi) else 0)
            if inside_row and lo <= hi:
                D[y, lo] += c * u[k]
                D[y, hi + 1] -= c * u[k]
                E[y, lo] += c
                E[y, hi + 1] -= c
    S = np.cumsum(D, axis=1)[:, :n].reshape(-1)
    T = np.cumsum(E, axis=1)[:, :n].reshape(-1)
    half2 = a * (S - u * T) - u * a * a * delta ** -4.0 * ext
    want = 0.5 * h ** 2 * (one + half2)
    got = oracle.fast_sym_leafset(u, 2, L, delta, K=0, alpha=1.0, normalize=False,
                                  coef=oracle.COEF_XY, a=a)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
