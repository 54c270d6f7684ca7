"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the operator itself: it only draws the
fields (horizons, coefficients, right-hand sides) that both the CUDA path and
the FP64 oracle consume.  Everything is generated on the host in FP64 with
``numpy.random.default_rng(seed)`` and cast by the caller.

Workloads (grid: n nodes per dimension, h = 1/n, x_i = (i + 1/2) h):

* ``diffusion_1d``: Sec. 2 homogeneous 1-D case -- constant horizon delta,
  u = sin(2 pi x) + 0.01 N(0,1).
* ``example2_1d``: Sec. 4 Example 2 -- delta(x) = delta0 (1 + exp(-20 (x-1/2)^2)).
* ``heterogeneous_2d``: variable horizon delta = h (4 + 12 s(x)), s a smooth
  field of 8 random Fourier modes rescaled to [0,1]; coefficient a lognormal
  (sigma 0.5) smoothed over 8h; u a Gaussian random field.
* ``pd_2d``: two-phase material from a seeded Voronoi partition of 64 cells,
  c in {1, 10}; u a pair of Gaussian random fields.
* ``diffusion_3d``: constant horizon, lognormal (sigma 0.3) coefficient,
  several right-hand sides.
"""
from __future__ import annotations

import numpy as np


def node_coords(d: int, n: int) -> list[np.ndarray]:
    """Cell-centred coordinates, one array per dimension, shape (n,)*d (z, y, x order)."""
    x = (np.arange(n) + 0.5) / n
    return list(np.meshgrid(*([x] * d), indexing="ij"))[::-1]  # [x, y, z] arrays


def _smooth_noise(rng, d, n, width_cells):
    """White noise convolved (periodically) with a Gaussian of std `width_cells` cells,
    normalised to zero mean and unit variance."""
    w = rng.standard_normal((n,) * d)
    k = np.fft.fftfreq(n) * n  # integer wavenumbers
    kr = np.fft.rfftfreq(n) * n
    ks = np.meshgrid(*([k] * (d - 1) + [kr]), indexing="ij", sparse=True)
    k2 = sum(kk.astype(np.float64) ** 2 for kk in ks)
    filt = np.exp(-2.0 * (np.pi * width_cells / n) ** 2 * k2)
    axes = list(range(d))
    g = np.fft.irfftn(np.fft.rfftn(w, axes=axes) * filt, s=w.shape, axes=axes)
    g -= g.mean()
    sd = g.std()
    return g / sd if sd > 0 else g


def gaussian_field(rng, d, n, corr_cells=None):
    """Stationary Gaussian random field (spectral filter of white noise), unit variance."""
    if corr_cells is None:
        corr_cells = max(2.0, n / 32.0)
    return _smooth_noise(rng, d, n, corr_cells)


def fourier_modes_field(rng, d, n, modes=8, kmax=4):
    """Sum of `modes` cosines with random nonzero integer wavevectors (|k|_inf <= kmax) and
    seeded phases, rescaled to [0, 1]."""
    X = node_coords(d, n)
    s = np.zeros((n,) * d)
    for _ in range(modes):
        while True:
            kv = rng.integers(-kmax, kmax + 1, size=d)
            if np.any(kv != 0):
                break
        phase = rng.uniform(0, 2 * np.pi)
        arg = sum(2 * np.pi * kv[j] * X[j] for j in range(d))
        s += np.cos(arg + phase)
    s -= s.min()
    mx = s.max()
    return s / mx if mx > 0 else s


def diffusion_1d(n=4096, delta=0.05, seed=0):
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    u = np.sin(2 * np.pi * x) + 0.01 * rng.standard_normal(n)
    return dict(d=1, n=n, delta=np.full(n, float(delta)), u=u)


def example2_1d(n=4096, delta0=0.25, seed=0):
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    delta = delta0 * (1.0 + np.exp(-20.0 * (x - 0.5) ** 2))
    u = gaussian_field(rng, 1, n, corr_cells=n / 64.0)
    return dict(d=1, n=n, delta=delta, u=u)


def heterogeneous_2d(n=1024, seed=0, nrhs=1, rmin=4.0, rspan=12.0, sigma_a=0.5,
                     smooth_cells=8.0):
    """Config: delta = h (rmin + rspan s), a = exp(sigma_a g), u Gaussian random field."""
    rng = np.random.default_rng(seed)
    s = fourier_modes_field(rng, 2, n)
    delta = (rmin + rspan * s) / n
    g = _smooth_noise(rng, 2, n, smooth_cells)
    a = np.exp(sigma_a * g)
    u = np.stack([gaussian_field(rng, 2, n) for _ in range(nrhs)])
    return dict(d=2, n=n, delta=delta.reshape(-1), a=a.reshape(-1),
                u=u.reshape(nrhs, -1))


def voronoi_phase(rng, d, n, cells=64, values=(1.0, 10.0)):
    sites = rng.uniform(0, 1, size=(cells, d))
    phase = rng.integers(0, 2, size=cells)
    X = node_coords(d, n)
    pts = np.stack([x.reshape(-1) for x in X], axis=1)
    best = np.full(pts.shape[0], np.inf)
    lab = np.zeros(pts.shape[0], dtype=np.int64)
    for c in range(cells):
        dist = ((pts - sites[c]) ** 2).sum(axis=1)
        m = dist < best
        best[m] = dist[m]
        lab[m] = c
    vals = np.asarray(values, dtype=np.float64)
    return vals[phase[lab]]


def pd_2d(n=512, seed=0, radius_cells=8, nrhs=1):
    rng = np.random.default_rng(seed)
    c = voronoi_phase(rng, 2, n)
    u = np.stack([np.stack([gaussian_field(rng, 2, n).reshape(-1) for _ in range(2)])
                  for _ in range(nrhs)])
    return dict(d=2, n=n, delta=np.full(n * n, radius_cells / n), c=c, u=u)


def pd_batch_sizes(count=64, nmin=128, nmax=512):
    """Uneven instance sizes n_k = nmin + round((nmax - nmin) k / (count - 1))."""
    if count == 1:
        return [nmin]
    return [int(nmin + round((nmax - nmin) * k / (count - 1))) for k in range(count)]


def diffusion_3d(n=256, seed=0, nrhs=8, radius_cells=4, sigma_a=0.3, smooth_cells=4.0):
    rng = np.random.default_rng(seed)
    g = _smooth_noise(rng, 3, n, smooth_cells)
    a = np.exp(sigma_a * g)
    u = np.stack([gaussian_field(rng, 3, n).reshape(-1) for _ in range(nrhs)])
    return dict(d=3, n=n, delta=np.full(n ** 3, radius_cells / n), a=a.reshape(-1), u=u)


def cg_rhs(n, seed=0, count=1):
    rng = np.random.default_rng(seed)
    return np.stack([gaussian_field(rng, 2, n).reshape(-1) for _ in range(count)])
