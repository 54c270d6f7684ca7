"""Pins for the oracle's Hermite-matched polynomial p^{2K} (Sec. 3) and constants."""
import os
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import polynomial as P

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "p2K_gamma_inv_s.txt")


def _printed():
    rows = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        parts = line.split()
        rows[int(parts[0])] = [float(Fraction(t)) for t in parts[1:]]
    return rows


def _as_power_series(p):
    """p_m s^{2m} -> ordinary coefficients in s."""
    c = np.zeros(2 * len(p) - 1)
    c[::2] = p
    return c


def _falling(x, j):
    r = 1.0
    for t in range(j):
        r *= x - t
    return r


@pytest.mark.parametrize("K", [0, 1, 2])
def test_matches_printed_table(K):
    np.testing.assert_allclose(oracle.poly_coeffs(K, 1.0), _printed()[K], rtol=0, atol=1e-14)


def test_printed_K3_fails_third_derivative_and_oracle_passes():
    printed = _as_power_series(_printed()[3])
    d3 = P.polyval(1.0, P.polyder(printed, 3))
    assert abs(d3 - (-3.0)) < 1e-12          # printed row: p'''(1) = -3
    ours = _as_power_series(oracle.poly_coeffs(3, 1.0))
    assert abs(P.polyval(1.0, P.polyder(ours, 3)) - (-6.0)) < 1e-12
    # and the derived row in exact rationals: (35 - 35 s^2 + 21 s^4 - 5 s^6)/16
    np.testing.assert_allclose(oracle.poly_coeffs(3, 1.0),
                               [35 / 16, -35 / 16, 21 / 16, -5 / 16], atol=1e-14)


@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0, 1.5, 2.0])
@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_hermite_conditions(K, alpha):
    c = _as_power_series(oracle.poly_coeffs(K, alpha))
    for j in range(K + 1):
        lhs = P.polyval(1.0, P.polyder(c, j)) if j else P.polyval(1.0, c)
        rhs = _falling(-alpha, j)                # d^j/ds^j s^{-alpha} at s = 1
        assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(rhs)), (K, alpha, j, lhs, rhs)


def test_sphere_area_and_normalisation():
    assert oracle.sphere_area(1) == 2.0
    assert abs(oracle.sphere_area(2) - 2 * np.pi) < 1e-15
    assert abs(oracle.sphere_area(3) - 4 * np.pi) < 1e-15
    # sigma delta^{-(d+2)} |xi/delta|^{-alpha}: the second moment over the unit ball is 2d.
    # Check by independent radial quadrature (scipy) for a few (d, alpha).
    from scipy.integrate import quad
    for d, alpha in [(1, 0.0), (2, 1.5), (3, 1.0), (2, 0.0)]:
        radial, _ = quad(lambda r: r ** (2 - alpha) * r ** (d - 1), 0, 1)
        assert abs(oracle.sigma(d, alpha) * oracle.sphere_area(d) * radial - 2 * d) < 1e-10
    # the closed forms of the three workloads: 3/delta^3, 5/(pi delta^2.5), 6/(pi delta^4)
    assert abs(oracle.sigma(1, 0.0) - 3.0) < 1e-15
    assert abs(oracle.sigma(2, 1.5) - 5.0 / np.pi) < 1e-14
    assert abs(oracle.sigma(3, 1.0) - 6.0 / np.pi) < 1e-14
