"""Pins for the oracle's linear bond-based peridynamic operator, Eq. (1.1)-(1.2)."""
import numpy as np

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
    """Constant displacements and infinitesimal rotations u = W x (W antisymmetric)
    stretch no bond: e.(u_j - u_i) = xi^T W xi / |xi| = 0, for any micromodulus."""
    n = 48
    f = synth.pd_2d(n=n, seed=2)
    X = synth.node_coords(2, n)
    x, y = X[0].reshape(-1), X[1].reshape(-1)
    inner = _interior(2, n, 9)
    for u in (np.stack([np.full(n * n, 0.7), np.full(n * n, -1.3)]),
              np.stack([-0.4 * y, 0.4 * x])):
        Lu = oracle.pd_direct(u, 2, n, 8.0 / n, f["c"], idx=inner)
        assert np.abs(Lu).max() < 1e-9


def test_quadratic_fields_continuum_limit():
    """c = 1, constant delta.  Continuum values: for u = (x y, 0),
    (L u)_y = int xi_x^2 xi_y^2/|xi|^3 = pi delta^3/12 and (L u)_x = 0;
    for u = (x^2, 0), (L u)_x = int xi_x^4/|xi|^3 = pi delta^3/4.  The first checks the
    off-diagonal of xi xi^T, the second the diagonal and the |xi|^-3 power."""
    n, rho = 128, 24.0
    delta = rho / n
    X = synth.node_coords(2, n)
    x, y = X[0].reshape(-1), X[1].reshape(-1)
    inner = _interior(2, n, int(rho) + 1)[::61]
    z = np.zeros(n * n)
    L1 = oracle.pd_direct(np.stack([x * y, z]), 2, n, delta, 1.0, idx=inner)
    np.testing.assert_allclose(L1[1], np.pi * delta ** 3 / 12, rtol=4e-2)
    assert np.abs(L1[0]).max() < 1e-12
    L2 = oracle.pd_direct(np.stack([x * x, z]), 2, n, delta, 1.0, idx=inner)
    np.testing.assert_allclose(L2[0], np.pi * delta ** 3 / 4, rtol=4e-2)
    assert np.abs(L2[1]).max() < 1e-12


def test_one_dimensional_reduces_to_scalar_power_kernel():
    """In 1-D, xi xi^T/|xi|^3 = 1/|xi|: PD with c = 1 equals the scalar operator with
    gamma(s) = s^{-1}, unnormalised, scale delta^2 (w = delta^{-3} (|xi|/delta)^{-1})."""
    n, delta = 512, 20.5 / 512
    rng = np.random.default_rng(0)
    u = rng.standard_normal(n)
    Lpd = oracle.pd_direct(u.reshape(1, n), 1, n, delta, 1.0)
    Ls = oracle.direct_scalar(u, 1, n, delta, alpha=1.0, normalize=False, scale=delta ** 2)
    np.testing.assert_allclose(Lpd[0], Ls, rtol=1e-12, atol=1e-12 * np.abs(Ls).max())


def test_symmetric_negative_definite_two_phase():
    n = 12
    f = synth.pd_2d(n=n, seed=5, radius_cells=3)
    N = 2 * n * n
    A = np.zeros((N, N))
    E = np.eye(N)
    for j in range(N):
        A[:, j] = oracle.pd_direct(E[j].reshape(2, -1), 2, n, f["delta"], f["c"]).reshape(-1)
    np.testing.assert_allclose(A, A.T, atol=1e-10 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).max() < 0
    np.testing.assert_allclose(-np.diag(A), oracle.pd_diag(2, n, f["delta"], f["c"]), rtol=1e-12)
