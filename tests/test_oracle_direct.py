"""Pins for the oracle's direct scalar operator, Eq. (2.1)-(2.2).

Each test checks the oracle against something other than itself: a closed
form, an exact lattice identity, a continuum limit, or a linear-algebra fact.
"""
import numpy as np
import pytest

import oracle
from paper_1905_08375_gb300 import synth


def _interior(d, n, R):
    """Flat indices of nodes whose whole ball (radius R cells) stays inside Omega."""
    idx = np.arange(n ** d)
    ok = np.ones(n ** d, dtype=bool)
    rest = idx.copy()
    for _ in range(d):
        c = rest % n
        rest //= n
        ok &= (c >= R) & (c < n - R)
    return idx[ok]


def test_config1_quadratic_closed_form():
    """1-D, delta = 0.05, gamma = 3/delta^3 (alpha = 0, normalised), u = x^2.
    Away from the boundary: (L u)_i = h^3 m(m+1)(2m+1)/delta^3 with m = #{o>0: o < delta/h}."""
    n, delta = 4096, 0.05
    x = (np.arange(n) + 0.5) / n
    rho = delta * n                      # 204.8
    m = int(np.ceil(rho)) - 1            # 204
    expect = (1.0 / n) ** 3 * m * (m + 1) * (2 * m + 1) / delta ** 3
    assert abs(expect - 1.99121) < 1e-5
    inner = _interior(1, n, m + 1)
    Lu = oracle.direct_scalar(x ** 2, 1, n, delta, family=oracle.POWER, alpha=0.0, idx=inner)
    np.testing.assert_allclose(Lu, expect, rtol=1e-12)


def test_config1_sine_dirichlet_kernel():
    """u = sin(2 pi x): (L u)_i = (3/delta^3) h sin(2 pi x_i) [D_m(2 pi h) - (2m+1)],
    D_m(t) = sin((m + 1/2) t)/sin(t/2) (Dirichlet kernel)."""
    n, delta = 4096, 0.05
    x = (np.arange(n) + 0.5) / n
    m = int(np.ceil(delta * n)) - 1
    t = 2 * np.pi / n
    D = np.sin((m + 0.5) * t) / np.sin(t / 2)
    inner = _interior(1, n, m + 1)
    expect = 3.0 / delta ** 3 / n * np.sin(2 * np.pi * x[inner]) * (D - (2 * m + 1))
    Lu = oracle.direct_scalar(np.sin(2 * np.pi * x), 1, n, delta, alpha=0.0, idx=inner)
    np.testing.assert_allclose(Lu, expect, rtol=1e-9, atol=1e-9 * np.abs(expect).max())


def test_boundary_rows_see_zero_exterior():
    """Volume constraint: at the first node of a 1-D grid with u = 1 only the exterior
    neighbours contribute, each (0 - 1) w: (L 1)_0 = -h (3/delta^3) #{o < 0 : |o| < rho}."""
    n, delta = 256, 10.5 / 256
    u = np.ones(n)
    Lu = oracle.direct_scalar(u, 1, n, delta, alpha=0.0)
    assert abs(Lu[0] - (-(1.0 / n) * 3 / delta ** 3 * 10)) < 1e-10 * abs(Lu[0])
    assert abs(Lu[n // 2]) < 1e-9


@pytest.mark.parametrize("d,n,rho,alpha", [(2, 96, 24.0, 1.5), (3, 40, 10.0, 1.0), (1, 1024, 300.0, 0.0)])
def test_quadratic_continuum_limit(d, n, rho, alpha):
    """Normalised kernels: L -> Laplacian.  L[x^2] -> 2 (d/dx^2 of x^2) within the lattice
    (Gauss-circle) error; L[x y] and L[x^2 - y^2] vanish exactly by lattice symmetry."""
    X = synth.node_coords(d, n)
    x = X[0].reshape(-1)
    inner = _interior(d, n, int(np.ceil(rho)) + 1)[::97]
    Lx2 = oracle.direct_scalar(x ** 2, d, n, rho / n, alpha=alpha, idx=inner)
    tol = {1: 1e-2, 2: 3e-2, 3: 8e-2}[d]
    assert np.all(np.abs(Lx2 - 2.0) < tol), (Lx2.min(), Lx2.max())
    if d >= 2:
        y = X[1].reshape(-1)
        Lxy = oracle.direct_scalar(x * y, d, n, rho / n, alpha=alpha, idx=inner)
        Ld = oracle.direct_scalar(x ** 2 - y ** 2, d, n, rho / n, alpha=alpha, idx=inner)
        assert np.abs(Lxy).max() < 1e-9 and np.abs(Ld).max() < 1e-9


def test_horizon_power_scaling():
    """Unnormalised kernel: raw L[x^2] = 2/sigma at every horizon, because the only
    horizon dependence is delta^{-(d+2)} (|xi|/delta)^{-alpha}, which the second moment
    cancels exactly.  A wrong power of delta would make raw * sigma drift with rho."""
    d, n, alpha = 2, 160, 1.5
    x = synth.node_coords(d, n)[0].reshape(-1)
    vals = []
    for rho in (16.0, 32.0):
        inner = _interior(d, n, int(rho) + 2)[::211]
        raw = oracle.direct_scalar(x ** 2, d, n, rho / n, alpha=alpha, normalize=False, idx=inner)
        vals.append(raw.mean())
    sg = oracle.sigma(d, alpha)
    assert abs(vals[0] * sg - 2) < 0.04 and abs(vals[1] * sg - 2) < 0.02


def test_linear_field_annihilated_variable_horizon():
    """Centred balls are symmetric under o -> -o, so linear u is annihilated at interior
    nodes for any per-node horizon (coefficient NONE or X)."""
    f = synth.heterogeneous_2d(n=64, seed=3)
    n, d = 64, 2
    X = synth.node_coords(d, n)
    u = (0.3 * X[0] - 1.7 * X[1] + 0.25).reshape(-1)
    inner = _interior(d, n, 17)
    for coef in (oracle.COEF_NONE, oracle.COEF_X):
        Lu = oracle.direct_scalar(u, d, n, f["delta"], alpha=1.5, coef=coef, a=f["a"], idx=inner)
        assert np.abs(Lu).max() < 1e-9


def test_divergence_form_limit_with_product_coefficient():
    """C(x,y) = a(x) a(y), constant delta: L u -> div(a^2 grad u).  For u = x and
    a = 1 + x/2 this is 2 a a_x = 1 + x/2 (a dropped a(y) would give 0)."""
    d, n, rho = 2, 128, 24.0
    X = synth.node_coords(d, n)
    x = X[0].reshape(-1)
    a = 1.0 + 0.5 * x
    inner = _interior(d, n, int(rho) + 1)[::53]
    Lu = oracle.direct_scalar(x, d, n, rho / n, alpha=1.5, coef=oracle.COEF_XY, a=a, idx=inner)
    np.testing.assert_allclose(Lu, 1.0 + 0.5 * x[inner], rtol=3e-2)


def _dense(d, n, delta, **kw):
    N = n ** d
    A = np.zeros((N, N))
    E = np.eye(N)
    for j in range(N):
        A[:, j] = oracle.direct_scalar(E[j], d, n, delta, **kw)
    return A


def test_symmetric_variant_is_symmetric_negative_definite():
    f = synth.heterogeneous_2d(n=16, seed=1)
    kw = dict(alpha=1.5, coef=oracle.COEF_XY, a=f["a"], symmetric=True)
    A = _dense(2, 16, f["delta"], **kw)
    np.testing.assert_allclose(A, A.T, atol=1e-10 * np.abs(A).max())
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() < 0
    # the one-sided (non-divergence) operator with a variable horizon is not symmetric
    A1 = _dense(2, 16, f["delta"], alpha=1.5, coef=oracle.COEF_XY, a=f["a"])
    assert np.abs(A1 - A1.T).max() > 1e-3 * np.abs(A1).max()
    # diagonal helper agrees with the assembled matrix
    dg = oracle.direct_diag(2, 16, f["delta"], **kw)
    np.testing.assert_allclose(-np.diag(A), dg, rtol=1e-12)


def test_poly_family_with_unit_polynomial_counts_ball():
    """POLY, K = 0 (p = 1), unnormalised: (L 1_{j})_i sums h^d delta^{-(d+2)} over the ball.
    For u = 1 at interior nodes L u = 0; for u = delta_{i0} the row i0 is -h^d delta^{-(d+2)} #ball."""
    d, n, rho = 2, 40, 6.3
    N = n * n
    e = np.zeros(N)
    i0 = 20 * n + 20
    e[i0] = 1.0
    Lu = oracle.direct_scalar(e, d, n, rho / n, family=oracle.POLY, K=0, normalize=False)
    o = np.arange(-7, 8)
    cnt = sum(1 for a in o for b in o if 0 < a * a + b * b < rho * rho)
    h = 1.0 / n
    assert abs(Lu[i0] - (-(h ** 2) * (rho / n) ** -4 * cnt)) < 1e-9 * abs(Lu[i0])
