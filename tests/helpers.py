"""Shared helpers for the GPU parity tests (no operator arithmetic here)."""
import numpy as np


def rel_l2(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))


def sample_idx(N, count, seed=0, extra=()):
    """Sampled node indices: random ones plus the first/last nodes and any extras."""
    rng = np.random.default_rng(seed)
    idx = set(rng.choice(N, size=min(count, N), replace=False).tolist())
    idx.update([0, N - 1, *extra])
    return np.array(sorted(idx), dtype=np.int64)


def boundary_idx(d, n, width, count, seed=0):
    """Sample of nodes within `width` cells of the boundary (where the exterior matters)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        c = rng.integers(0, n, size=d)
        k = rng.integers(0, d)
        c[k] = rng.integers(0, width) if rng.random() < 0.5 else n - 1 - rng.integers(0, width)
        f = 0
        for j in reversed(range(d)):
            f = f * n + int(c[j])
        out.append(f)
    return np.array(sorted(set(out)), dtype=np.int64)
