"""Pins for the oracle of the fast-path peridynamic operator: the bond tensor
xi xi^T p(|xi|/delta)/delta^3, p = 1 (K = 0) or the polynomial p^{2K} matched to s^-3 at the
horizon (K >= 1), summed over the leaf set of Algorithm 1."""
import itertools
import numpy as np
import pytest

import oracle
from paper_1905_08375_gb300 import synth


def _interior(d, n, R):
    idx = np.arange(n ** d)
    ok = np.ones(n ** d, dtype=bool)
    rest = idx.copy()
    for _ in range(d):
        c = rest % n
        rest //= n
        ok &= (c >= R) & (c < n - R)
    return idx[ok]


def test_rigid_motions_annihilated():
    """Constant displacements and u = W x with W antisymmetric stretch no bond:
    xi^T W xi = 0 term by term, for any c."""
    n, L = 32, 5
    f = synth.pd_2d(n=n, seed=2)
    X = synth.node_coords(2, n)
    x, y = X[0].reshape(-1), X[1].reshape(-1)
    inner = _interior(2, n, 6)
    for u in (np.stack([np.full(n * n, 0.7), np.full(n * n, -1.3)]),
              np.stack([-0.4 * y, 0.4 * x])):
        Lu = oracle.fast_pd_leafset(u, 2, L, 4.0 / n, f["c"], idx=inner)
        assert np.abs(Lu).max() < 1e-10


def test_quadratic_field_continuum_limit():
    """c = 1, delta fixed: for u = (x^2, 0) the x-component tends to
    delta^-3 int_{B_delta} xi_x^4 = pi delta^3 / 8, for u = (x y, 0) the y-component to
    delta^-3 int xi_x^2 xi_y^2 = pi delta^3 / 24; the leaf set exceeds the ball by a rim of
    cells, so the error falls like h."""
    delta = 0.25
    errs = []
    for L in (6, 7, 8):
        n = 1 << L
        X = synth.node_coords(2, n)
        x, y = X[0].reshape(-1), X[1].reshape(-1)
        c = np.ones(n * n)
        node = np.array([(n // 2) * n + n // 2])
        Lu = oracle.fast_pd_leafset(np.stack([x * x, 0 * x]), 2, L, delta, c, idx=node)
        e1 = abs(Lu[0, 0] - np.pi * delta ** 3 / 8) / (np.pi * delta ** 3 / 8)
        Lu = oracle.fast_pd_leafset(np.stack([x * y, 0 * x]), 2, L, delta, c, idx=node)
        e2 = abs(Lu[1, 0] - np.pi * delta ** 3 / 24) / (np.pi * delta ** 3 / 24)
        errs.append(max(e1, e2))
    assert errs[-1] < 0.08
    for k in (1, 2):                                    # first order: halves per doubling
        assert 0.4 < errs[k] / errs[k - 1] < 0.6, errs


def test_symmetric_negative_semidefinite():
    """Constant delta: cell k meets the ball of x_i iff cell i meets the ball of x_k, and
    c_ik = c_ki, so the operator is symmetric; each bond adds -c (xi.v)^2 to <L v, v>."""
    n, L = 8, 3
    rng = np.random.default_rng(5)
    c = rng.uniform(1.0, 10.0, n * n)
    N2 = 2 * n * n
    A = np.zeros((N2, N2))
    for k in range(N2):
        e = np.zeros(N2)
        e[k] = 1.0
        A[:, k] = oracle.fast_pd_leafset(e.reshape(2, -1), 2, L, 2.5 / n, c).reshape(-1)
    np.testing.assert_allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).max() < 1e-12 * np.abs(A).max()


def test_leaf_set_is_the_fast_scalar_set():
    """The sum runs over the leaf cells the scalar fast oracle counts: with u = (e_k, 0) the
    x-component at x_i is non-zero iff cell k is in the leaf set and xi_x != 0, with
    u = (0, e_k) the y-component iff xi_y != 0; together, every leaf cell but x_i's own."""
    n, L = 16, 4
    rng = np.random.default_rng(6)
    delta = np.ascontiguousarray(rng.uniform(1.2, 3.5, n * n) / n)
    node = 5 * n + 7
    _, cnt = oracle.fast_leafset(np.zeros(n * n), 2, L, delta, idx=np.array([node]),
                                 return_counts=True)
    support = 0
    for k in range(n * n):
        ux = np.zeros((2, n * n))
        ux[0, k] = 1.0
        uy = np.zeros((2, n * n))
        uy[1, k] = 1.0
        a = oracle.fast_pd_leafset(ux, 2, L, delta, np.ones(n * n), idx=np.array([node]))
        b = oracle.fast_pd_leafset(uy, 2, L, delta, np.ones(n * n), idx=np.array([node]))
        if k != node and (a[0, 0] != 0 or b[1, 0] != 0):
            support += 1
    assert support == cnt[0] - 1


@pytest.mark.parametrize("K", [1, 2, 3])
def test_micromodulus_polynomial_matches_s_minus_3(K):
    """p^{2K} agrees with s^-3 in value and first K derivatives at s = 1 (checked by
    differentiating the polynomial and the power independently)."""
    p = oracle.poly_coeffs(K, 3.0)
    poly = np.polynomial.Polynomial(np.ravel(np.column_stack([p, np.zeros_like(p)]))[:2 * K + 1])
    for j in range(K + 1):
        want = np.prod([-3 - i for i in range(j)]) if j else 1.0       # d^j s^-3 at s = 1
        assert abs(poly.deriv(j)(1.0) - want) < 1e-11 * max(1.0, abs(want))


@pytest.mark.parametrize("K", [1, 2])
def test_polynomial_continuum_limit(K):
    """c = 1: u = (x^2, 0) tends to delta^-3 int_{B_delta} xi_x^4 p(|xi|/delta) =
    (3 pi / 4) delta^3 sum_m p_m / (2m + 6), u = (x y, 0) (y-component) to
    (pi / 4) delta^3 sum_m p_m / (2m + 6); first order in h (the rim cells of the leaf set)."""
    delta = 0.25
    p = oracle.poly_coeffs(K, 3.0)
    rad = sum(p[m] / (2 * m + 6) for m in range(K + 1))
    want1, want2 = 0.75 * np.pi * delta ** 3 * rad, 0.25 * np.pi * delta ** 3 * rad
    errs = []
    for L in (6, 7, 8):
        n = 1 << L
        X = synth.node_coords(2, n)
        x, y = X[0].reshape(-1), X[1].reshape(-1)
        c = np.ones(n * n)
        node = np.array([(n // 2) * n + n // 2])
        Lu = oracle.fast_pd_leafset(np.stack([x * x, 0 * x]), 2, L, delta, c, K=K, idx=node)
        e1 = abs(Lu[0, 0] - want1) / abs(want1)
        Lu = oracle.fast_pd_leafset(np.stack([x * y, 0 * x]), 2, L, delta, c, K=K, idx=node)
        e2 = abs(Lu[1, 0] - want2) / abs(want2)
        errs.append(max(e1, e2))
    assert errs[-1] < 0.1
    for k in (1, 2):
        assert 0.35 < errs[k] / errs[k - 1] < 0.65, errs


def _brute(u, n, delta, c, K):
    """Plain numpy restatement on a tiny grid: every lattice cell k within the padded box,
    kept when its cell meets the open ball of x_i, weight p(|xi|/delta_i)."""
    h = 1.0 / n
    p = oracle.poly_coeffs(K, 3.0)
    out = np.zeros((2, n * n))
    B = int(np.ceil(delta.max() * n)) + 1
    for iy, ix in itertools.product(range(n), range(n)):
        i = iy * n + ix
        di = delta[i]
        acc = np.zeros(2)
        for oy, ox in itertools.product(range(-B, B + 1), repeat=2):
            if ox == 0 and oy == 0:
                continue
            gx = max(abs(ox) - 0.5, 0.0) * h
            gy = max(abs(oy) - 0.5, 0.0) * h
            if not gx * gx + gy * gy < di * di:
                continue
            kx, ky = ix + ox, iy + oy
            inside = 0 <= kx < n and 0 <= ky < n
            k = ky * n + kx if inside else None
            xi = np.array([ox * h, oy * h])
            s2 = (xi @ xi) / di ** 2
            w = sum(p[m] * s2 ** m for m in range(K + 1))
            uk = u[:, k] if inside else np.zeros(2)
            cik = 0.5 * (c[i] + (c[k] if inside else c[i]))
            acc += cik * w * (xi @ (uk - u[:, i])) * xi / di ** 3
        out[:, i] = h ** 2 * acc
    return out


@pytest.mark.parametrize("K", [0, 2])
def test_matches_brute_force_on_a_tiny_grid(K):
    n, L = 8, 3
    rng = np.random.default_rng(11 + K)
    delta = rng.uniform(1.3, 3.1, n * n) / n
    c = rng.uniform(1.0, 10.0, n * n)
    u = rng.standard_normal((2, n * n))
    got = oracle.fast_pd_leafset(u, 2, L, delta, c, K=K)
    want = _brute(u, n, delta, c, K)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("K", [1, 3])
def test_polynomial_rigid_motions_and_symmetry(K):
    n, L = 8, 3
    rng = np.random.default_rng(21 + K)
    c = rng.uniform(1.0, 10.0, n * n)
    N2 = 2 * n * n
    A = np.zeros((N2, N2))
    for k in range(N2):
        e = np.zeros(N2)
        e[k] = 1.0
        A[:, k] = oracle.fast_pd_leafset(e.reshape(2, -1), 2, L, 2.5 / n, c, K=K).reshape(-1)
    np.testing.assert_allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).max() < 1e-12 * np.abs(A).max()
    X = synth.node_coords(2, n)
    x, y = X[0].reshape(-1), X[1].reshape(-1)
    inner = _interior(2, n, 3)
    for u in (np.stack([np.full(n * n, 0.7), np.full(n * n, -1.3)]), np.stack([-0.4 * y, 0.4 * x])):
        Lu = oracle.fast_pd_leafset(u, 2, L, 2.5 / n, c, K=K, idx=inner)
        assert np.abs(Lu).max() < 1e-10


# ---------------------------------------------------------------------------
# 3-D: the same operator with xi in R^3 (u with three components)
# ---------------------------------------------------------------------------
def test_3d_rigid_motions_annihilated():
    """Constant displacements and u = W x, W antisymmetric (3 x 3), stretch no bond."""
    n, L = 16, 4
    rng = np.random.default_rng(31)
    c = rng.uniform(1.0, 10.0, n ** 3)
    delta = rng.uniform(1.5, 3.0, n ** 3) / n
    X = [x.reshape(-1) for x in synth.node_coords(3, n)]
    W = np.array([[0.0, 0.3, -0.7], [-0.3, 0.0, 0.45], [0.7, -0.45, 0.0]])
    inner = _interior(3, n, 5)
    for u in (np.stack([np.full(n ** 3, v) for v in (0.7, -1.3, 0.25)]),
              np.stack([sum(W[a, b] * X[b] for b in range(3)) for a in range(3)])):
        Lu = oracle.fast_pd_leafset(u, 3, L, delta, c, idx=inner)
        assert np.abs(Lu).max() < 1e-10


@pytest.mark.parametrize("K", [0, 1])
def test_3d_quadratic_field_continuum_limit(K):
    """c = 1: u = (x^2, 0, 0) (x-component) tends to delta^-3 int_{B_delta} xi_x^4 p(|xi|/delta)
    = (4 pi / 5) delta^4 sum_m p_m / (2m + 7) and u = (x y, 0, 0) (y-component) to
    delta^-3 int xi_x^2 xi_y^2 p = (4 pi / 15) delta^4 sum_m p_m / (2m + 7) (the sphere
    averages of x^4 and x^2 y^2 are 1/5 and 1/15); first order in h (the rim cells), so the
    errors halve per doubling and the Richardson value 2 v(2n) - v(n) is close to the limit."""
    delta = 0.25
    p = oracle.poly_coeffs(K, 3.0)
    rad = sum(p[m] / (2 * m + 7) for m in range(K + 1))
    want1, want2 = 0.8 * np.pi * delta ** 4 * rad, (4 * np.pi / 15) * delta ** 4 * rad
    errs, v1, v2 = [], [], []
    for L in (5, 6, 7):
        n = 1 << L
        x, y, _ = (v.reshape(-1) for v in synth.node_coords(3, n))
        c = np.ones(n ** 3)
        node = np.array([((n // 2) * n + n // 2) * n + n // 2])
        z = np.zeros(n ** 3)
        v1.append(oracle.fast_pd_leafset(np.stack([x * x, z, z]), 3, L, delta, c, K=K,
                                         idx=node)[0, 0])
        v2.append(oracle.fast_pd_leafset(np.stack([x * y, z, z]), 3, L, delta, c, K=K,
                                         idx=node)[1, 0])
        errs.append(max(abs(v1[-1] - want1) / abs(want1), abs(v2[-1] - want2) / abs(want2)))
    assert errs[-1] < 0.25, errs
    for k in (1, 2):
        assert 0.35 < errs[k] / errs[k - 1] < 0.65, errs
    r1, r2 = 2 * v1[2] - v1[1], 2 * v2[2] - v2[1]
    assert abs(r1 - want1) / abs(want1) < 0.05 and abs(r2 - want2) / abs(want2) < 0.05, (r1, r2)


def test_3d_symmetric_negative_semidefinite():
    """Constant delta, any c: symmetric, and <L v, v> = -sum of c (xi.v)^2 terms <= 0."""
    n, L = 4, 2
    rng = np.random.default_rng(33)
    c = rng.uniform(1.0, 10.0, n ** 3)
    N3 = 3 * n ** 3
    A = np.zeros((N3, N3))
    for k in range(N3):
        e = np.zeros(N3)
        e[k] = 1.0
        A[:, k] = oracle.fast_pd_leafset(e.reshape(3, -1), 3, L, 1.6 / n, c).reshape(-1)
    np.testing.assert_allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).max() < 1e-12 * np.abs(A).max()


def _brute3(u, n, delta, c, K):
    """Plain numpy restatement in 3-D: every cell of the padded box whose cell meets the open
    ball of x_i (per-axis gap max(|o| - 1/2, 0) h), weight p(|xi|/delta_i)."""
    h = 1.0 / n
    p = oracle.poly_coeffs(K, 3.0)
    out = np.zeros((3, n ** 3))
    B = int(np.ceil(delta.max() * n)) + 1
    for iz, iy, ix in itertools.product(range(n), repeat=3):
        i = (iz * n + iy) * n + ix
        di = delta[i]
        acc = np.zeros(3)
        for oz, oy, ox in itertools.product(range(-B, B + 1), repeat=3):
            if ox == 0 and oy == 0 and oz == 0:
                continue
            g2 = sum((max(abs(o) - 0.5, 0.0) * h) ** 2 for o in (ox, oy, oz))
            if not g2 < di * di:
                continue
            kx, ky, kz = ix + ox, iy + oy, iz + oz
            inside = 0 <= kx < n and 0 <= ky < n and 0 <= kz < n
            k = (kz * n + ky) * n + kx if inside else None
            xi = np.array([ox * h, oy * h, oz * h])
            s2 = (xi @ xi) / di ** 2
            w = sum(p[m] * s2 ** m for m in range(K + 1))
            uk = u[:, k] if inside else np.zeros(3)
            cik = 0.5 * (c[i] + (c[k] if inside else c[i]))
            acc += cik * w * (xi @ (uk - u[:, i])) * xi / di ** 3
        out[:, i] = h ** 3 * acc
    return out


@pytest.mark.parametrize("K", [0, 1])
def test_3d_matches_brute_force_on_a_tiny_grid(K):
    n, L = 4, 2
    rng = np.random.default_rng(41 + K)
    delta = rng.uniform(1.1, 2.2, n ** 3) / n
    c = rng.uniform(1.0, 10.0, n ** 3)
    u = rng.standard_normal((3, n ** 3))
    got = oracle.fast_pd_leafset(u, 3, L, delta, c, K=K)
    want = _brute3(u, n, delta, c, K)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
