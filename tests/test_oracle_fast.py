"""Pins for the oracle's fast algorithm (Sec. 3: Algorithms 1-2, Steps 1-3, Eq. (3.3)-(3.5))."""
import numpy as np
import pytest

import oracle
from paper_1905_08375_gb300 import synth


def _coords(d, n, f):
    c = []
    for _ in range(d):
        c.append(f % n)
        f //= n
    return c


@pytest.mark.parametrize("d,L,K", [(1, 9, 0), (1, 9, 3), (2, 5, 0), (2, 5, 1), (2, 5, 3),
                                   (3, 3, 0), (3, 3, 2)])
@pytest.mark.parametrize("coef,self_mode", [(oracle.COEF_NONE, oracle.SELF_PAPER),
                                            (oracle.COEF_X, oracle.SELF_DISCRETE),
                                            (oracle.COEF_XY, oracle.SELF_DISCRETE)])
def test_tree_equals_leafset(d, L, K, coef, self_mode):
    """O1 (recur + moment pyramid + Eq. (3.5)) and O2 (plain leaf-set sum) are two
    independent routes to the same number."""
    n = 1 << L
    rng = np.random.default_rng(10 * d + K)
    N = n ** d
    rho = rng.uniform(1.2, 0.3 * n, size=N) if d < 3 else rng.uniform(1.2, 3.5, size=N)
    delta = rho / n
    a = np.exp(0.3 * rng.standard_normal(N))
    u = rng.standard_normal((2, N))
    o1 = oracle.fast_tree(u, d, L, delta, K=K, alpha=1.0, coef=coef, a=a, self_mode=self_mode)
    o2 = oracle.fast_leafset(u, d, L, delta, K=K, alpha=1.0, coef=coef, a=a, self_mode=self_mode)
    err = np.linalg.norm(o1 - o2) / np.linalg.norm(o2)
    assert err < 1e-13, err


@pytest.mark.parametrize("d,L,rho", [(1, 8, 13.7), (2, 6, 9.3), (2, 6, 20.1), (3, 4, 3.6)])
def test_decomposition_is_disjoint_cover_of_leafset(d, L, rho):
    """The panels Algorithm 1 includes are disjoint and their union is exactly the set of
    leaf cells meeting the open ball (leaf cells that only touch it are not included)."""
    n = 1 << L
    rng = np.random.default_rng(d)
    for node in rng.integers(0, n ** d, size=6):
        lev, pk, _ = oracle.tree_decompose(d, L, rho / n, node)
        cover = np.zeros((n,) * d, dtype=np.int64)
        for l, k in zip(lev, pk):
            kc = _coords(d, 1 << l, int(k))
            s = n >> l
            sl = tuple(slice(kc[j] * s, (kc[j] + 1) * s) for j in reversed(range(d)))
            cover[sl] += 1
        assert cover.max() == 1
        ci = _coords(d, n, int(node))
        # leaf cell k meets the ball iff sum over dims of the squared gap (in half-units)
        # is below (2 rho)^2
        grids = np.meshgrid(*([np.arange(n)] * d), indexing="ij")[::-1]
        gap2 = np.zeros((n,) * d)
        for j in range(d):
            g = np.abs(2 * grids[j] + 1 - (2 * ci[j] + 1)) - 1
            gap2 += np.maximum(g, 0) ** 2
        expect = gap2 < 4 * rho * rho
        np.testing.assert_array_equal(cover.astype(bool), expect)


def test_whole_domain_ball_is_single_root_panel_and_top_sum():
    """If the ball contains all of Omega, recur includes only the root, and Step 3 reduces
    to h^d times the total sum stored at the top of the pyramid (Fig. of Step 2)."""
    d, L = 2, 5
    n = 1 << L
    rng = np.random.default_rng(3)
    u = rng.standard_normal(n * n)
    node = 7 * n + 3
    lev, pk, _ = oracle.tree_decompose(d, L, 1.5, node)
    assert list(lev) == [0] and list(pk) == [0]
    out = oracle.fast_tree(u, d, L, 1.5, K=0, normalize=False, self_mode=oracle.SELF_PAPER,
                           idx=[node])
    expect = 1.5 ** -4 * (u.sum() / n ** 2 - u[node] * np.pi * 1.5 ** 2)
    assert abs(out[0] - expect) < 1e-12 * abs(expect)


def test_1d_constant_horizon_is_sliding_window():
    """1-D, K = 0, constant delta: the included cells are |o| < rho + 1/2, so the panel sum
    is a moving-window sum (np.convolve) of u."""
    L, rho = 10, 37.3
    n = 1 << L
    rng = np.random.default_rng(7)
    u = rng.standard_normal(n)
    m = int(np.ceil(rho + 0.5)) - 1
    win = np.convolve(np.concatenate([np.zeros(m), u, np.zeros(m)]), np.ones(2 * m + 1), "valid")
    S_paper = 2 * (rho / n)
    out = oracle.fast_tree(u, 1, L, rho / n, K=0, normalize=False, self_mode=oracle.SELF_PAPER)
    expect = (rho / n) ** -3 * (win / n - u * S_paper)
    np.testing.assert_allclose(out, expect, rtol=1e-11, atol=1e-11 * np.abs(expect).max())


def _disk_square_overlap(cx, cy, r, m=4000):
    """|B_r(c) cap [0,1]^2| by a fine midpoint rule in x of the chord length (independent
    of the lattice)."""
    xs = cx - r + (np.arange(m) + 0.5) * (2 * r / m)
    half = np.sqrt(np.maximum(r * r - (xs - cx) ** 2, 0.0))
    lo = np.maximum(cy - half, 0.0)
    hi = np.minimum(cy + half, 1.0)
    inside = (xs >= 0) & (xs <= 1)
    return np.sum(np.where(inside, np.maximum(hi - lo, 0.0), 0.0)) * (2 * r / m)


def test_example1_closed_form_converges():
    """Sec. 4 Example 1: d = 2, K = 0, p = 1, delta = 1/2, C = 1:
    L^P u = delta^{-4} int_{B cap Omega} u - |B_1| delta^{-2} u.  For u = 1 this is
    -|B_delta(x) \\ Omega| / delta^4.  The leaf-set quadrature converges to it at O(h): the
    cells that meet the ball without lying inside it fit in a band of width sqrt(2) h outside
    the circle, so the error is at most 2 pi (delta + sqrt(2) h) sqrt(2) h / delta^4."""
    errs, bounds = [], []
    for L in (4, 5, 6):
        n = 1 << L
        idx = np.array([0, n // 3 * n + n // 5, (n - 1) * n + n // 2, n * n // 2 + n // 2])
        u = np.ones(n * n)
        out = oracle.fast_tree(u, 2, L, 0.5, K=0, normalize=False,
                               self_mode=oracle.SELF_PAPER, idx=idx)
        e = []
        for q, f in enumerate(idx):
            ix, iy = f % n, f // n
            cx, cy = (ix + 0.5) / n, (iy + 0.5) / n
            exact = -(np.pi * 0.25 - _disk_square_overlap(cx, cy, 0.5)) / 0.5 ** 4
            e.append(abs(out[q] - exact))
        errs.append(max(e))
        h = 1.0 / n
        bounds.append(2 * np.pi * (0.5 + np.sqrt(2) * h) * np.sqrt(2) * h / 0.5 ** 4)
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.35 * errs[0]
    assert all(e <= b for e, b in zip(errs, bounds)), (errs, bounds)


def test_panel_counts_follow_complexity_estimate():
    """Eq. (3.4): panels per node stay O(1) per level in 1-D, so the count grows by a
    bounded amount per level; in 2-D at fixed delta they grow ~ n^{1/2} per node per
    doubling of N, i.e. x2 per doubling of n."""
    c1 = []
    for L in (8, 10, 12):
        n = 1 << L
        lev, _, _ = oracle.tree_decompose(1, L, 0.2, n // 2)
        c1.append(len(lev))
    assert c1[1] - c1[0] <= 8 and c1[2] - c1[1] <= 8
    c2 = []
    for L in (6, 7, 8):
        n = 1 << L
        node = (n // 2) * n + n // 2
        lev, _, _ = oracle.tree_decompose(2, L, 0.23, node)
        c2.append(len(lev))
    r1, r2 = c2[1] / c2[0], c2[2] / c2[1]
    assert 1.6 < r1 < 2.4 and 1.6 < r2 < 2.4, c2


def test_discrete_self_term_annihilates_constants():
    """With the discrete self term (every cell meeting the ball, inside or outside Omega,
    weighted like the summed field), L^P 1 = 0 at nodes whose leaf set lies inside Omega."""
    d, L = 2, 6
    n = 1 << L
    f = synth.heterogeneous_2d(n=n, seed=4)
    u = np.ones(n * n)
    out = oracle.fast_leafset(u, d, L, f["delta"], K=2, alpha=1.5, coef=oracle.COEF_XY,
                              a=f["a"], self_mode=oracle.SELF_DISCRETE)
    ix, iy = np.arange(n * n) % n, np.arange(n * n) // n
    R = np.ceil(f["delta"] * n) + 1
    inner = (ix >= R) & (ix < n - R) & (iy >= R) & (iy < n - R)
    assert inner.sum() > 100
    assert np.abs(out[inner]).max() < 1e-9 * np.abs(out).max()
