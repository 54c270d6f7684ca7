"""FP64 CPU oracle for the nonlocal operator library.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or execute anything
under ``oracle/``.  The product path (``paper_1905_08375_gb300``) never does,
and the two share no code: this package holds its own C source
(``nl_oracle.c``), its own constants and its own polynomial solver, written
from the paper (Tian & Engquist, arXiv 1905.08375):

* ``direct_scalar``  -- Eq. (2.1)-(2.2), nodal Riemann sum over the open ball, for the
  profiles s^-alpha (POWER), p^{2K} (POLY) and the Sec. 3 splitting remainder
  kappa = s^-alpha - p^{2K} (KAPPA).
* ``pd_direct``      -- Eq. (1.1)-(1.2), linear bond-based peridynamics.
* ``fast_tree``      -- Sec. 3: Algorithm 1 (recur) with Algorithm 2, the Step 2
  moment pyramid and the Step 3 sum of Eq. (3.5), then Eq. (3.3).
* ``fast_leafset``   -- the same quantity as a plain sum over the leaf cells
  that meet the ball (the union of the panels Algorithm 1 includes).
* ``fast_sym_leafset`` -- the symmetrised (divergence-type) form of that operator, each half
  of a pair's weight over its own node's leaf set (a project extension; no fast kernel yet).
* ``poly_coeffs``    -- the Hermite-matched even polynomial p^{2K} of Sec. 3.
* ``cg``             -- plain conjugate gradients on -L x = f (Sec. 4 remark).
* ``convnet``        -- the CG preconditioner network (a project addition the
  paper has no counterpart for); see ``oracle/convnet.py``.

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
against closed forms, the paper's printed polynomials, invariants (constants
and linear fields annihilated, symmetry, definiteness), continuum limits and
two independent implementations of the fast algorithm.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_SRC = os.path.join(_HERE, "nl_oracle.c")

POWER, POLY, KAPPA = 0, 1, 2   # KAPPA: kappa = s^-alpha - p^{2K} (Sec. 3 splitting)
COEF_NONE, COEF_X, COEF_XY = 0, 1, 2
SELF_DISCRETE, SELF_PAPER = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, OpenMP over nodes)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i, i64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        L.or_num_threads.restype = i
        L.or_set_threads.restype = None
        L.or_set_threads.argtypes = [i]
        L.or_sphere_area.restype = d
        L.or_sphere_area.argtypes = [i]
        L.or_sigma.restype = d
        L.or_sigma.argtypes = [i, d, d, i]
        L.or_poly_coeffs.restype = i
        L.or_poly_coeffs.argtypes = [i, d, vp]
        L.or_direct_scalar.restype = i
        L.or_direct_scalar.argtypes = [i, i, vp, i, d, i, vp, d, i, vp, i, i, vp, vp, vp, i64]
        L.or_direct_diag.restype = i
        L.or_direct_diag.argtypes = [i, i, vp, i, d, i, vp, d, i, vp, i, vp]
        L.or_pd_direct.restype = i
        L.or_pd_direct.argtypes = [i, i, vp, vp, d, i, vp, vp, vp, i64]
        L.or_fast_pd_leafset.restype = i
        L.or_fast_pd_leafset.argtypes = [i, i, vp, vp, d, i, vp, i, vp, vp, vp, i64]
        L.or_tree_decompose.restype = i64
        L.or_tree_decompose.argtypes = [i, i, d, i64, vp, vp, i64, vp]
        L.or_fast_tree.restype = i
        L.or_fast_tree.argtypes = [i, i, vp, i, vp, d, i, vp, i, i, vp, vp, vp, i64, vp]
        L.or_fast_leafset.restype = i
        L.or_fast_leafset.argtypes = [i, i, vp, i, vp, d, i, vp, i, i, vp, vp, vp, i64, vp]
        L.or_fast_sym_leafset.restype = i
        L.or_fast_sym_leafset.argtypes = [i, i, vp, i, vp, d, i, vp, i, vp, vp, vp, i64]
        L.or_cg.restype = i
        L.or_cg.argtypes = [i, i, i, vp, i, d, i, vp, d, i, vp, vp, vp, vp, vp, d, i,
                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        _lib = L
    return _lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _ptr(x):
    return None if x is None else x.ctypes.data


def num_threads() -> int:
    return lib().or_num_threads()


def set_threads(t: int) -> None:
    """OpenMP threads of later oracle calls (for timing; the results do not depend on it)."""
    lib().or_set_threads(int(t))


def sphere_area(d: int) -> float:
    return lib().or_sphere_area(d)


def sigma(d: int, alpha: float, scale: float = 1.0, normalize: bool = True) -> float:
    """Kernel constant: scale * 2d(d+2-alpha)/|S^{d-1}| when normalised (L -> Laplacian)."""
    return lib().or_sigma(d, alpha, scale, int(normalize))


def poly_coeffs(K: int, alpha: float = 1.0) -> np.ndarray:
    """Coefficients p_m of p^{2K}(s) = sum_m p_m s^{2m} (Sec. 3, Hermite matching)."""
    p = np.zeros(K + 1)
    rc = lib().or_poly_coeffs(K, float(alpha), p.ctypes.data)
    if rc:
        raise ValueError(f"or_poly_coeffs failed ({rc})")
    return p


def _delta_field(delta, d, n):
    N = n ** d
    if np.isscalar(delta):
        return np.full(N, float(delta))
    out = _f64(delta).reshape(-1)
    assert out.size == N
    return out


def _idx(idx):
    if idx is None:
        return None, 0
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    return idx, idx.size


def direct_scalar(u, d, n, delta, family=POWER, alpha=0.0, K=0, scale=1.0, normalize=True,
                  coef=COEF_NONE, a=None, symmetric=False, idx=None):
    """(L u)_i = h^d sum_{j != i, |x_j-x_i|<delta} w_ij c_ij (u_j - u_i).

    u: [nrhs, N] or [N].  Returns the same leading shape (or [nrhs, len(idx)])."""
    u = _f64(u)
    squeeze = u.ndim == 1
    u2 = u.reshape(1, -1) if squeeze else u.reshape(u.shape[0], -1)
    nrhs = u2.shape[0]
    dl = _delta_field(delta, d, n)
    p = poly_coeffs(K, alpha) if family in (POLY, KAPPA) else np.zeros(1)
    sg = sigma(d, alpha, scale, normalize)
    a_ = None if a is None else _f64(a).reshape(-1)
    ix, nix = _idx(idx)
    M = nix if ix is not None else n ** d
    out = np.zeros((nrhs, M))
    rc = lib().or_direct_scalar(d, n, _ptr(dl), family, float(alpha), K, _ptr(p), sg, coef,
                                _ptr(a_), int(symmetric), nrhs, _ptr(u2), _ptr(out), _ptr(ix), nix)
    if rc:
        raise ValueError(f"or_direct_scalar failed ({rc})")
    return out[0] if squeeze else out


def direct_diag(d, n, delta, family=POWER, alpha=0.0, K=0, scale=1.0, normalize=True,
                coef=COEF_NONE, a=None, symmetric=False):
    """Diagonal of -L (h^d sum_j w_ij c_ij)."""
    dl = _delta_field(delta, d, n)
    p = poly_coeffs(K, alpha) if family in (POLY, KAPPA) else np.zeros(1)
    sg = sigma(d, alpha, scale, normalize)
    a_ = None if a is None else _f64(a).reshape(-1)
    out = np.zeros(n ** d)
    rc = lib().or_direct_diag(d, n, _ptr(dl), family, float(alpha), K, _ptr(p), sg, coef,
                              _ptr(a_), int(symmetric), _ptr(out))
    if rc:
        raise ValueError(f"or_direct_diag failed ({rc})")
    return out


def pd_direct(u, d, n, delta, c, scale=1.0, idx=None):
    """Linear bond-based PD: h^d sum scale c_ij xi xi^T/|xi|^3 (u_j - u_i).

    u: [nrhs, d, N] or [d, N]."""
    u = _f64(u)
    squeeze = u.ndim == 2
    u3 = u.reshape(1, d, -1) if squeeze else u.reshape(u.shape[0], d, -1)
    nrhs = u3.shape[0]
    dl = _delta_field(delta, d, n)
    c_ = _delta_field(c, d, n)
    ix, nix = _idx(idx)
    M = nix if ix is not None else n ** d
    out = np.zeros((nrhs, d, M))
    rc = lib().or_pd_direct(d, n, _ptr(dl), _ptr(c_), float(scale), nrhs, _ptr(u3), _ptr(out),
                            _ptr(ix), nix)
    if rc:
        raise ValueError(f"or_pd_direct failed ({rc})")
    return out[0] if squeeze else out


def tree_decompose(d, L, delta_i, node):
    """Step 1 for one node: arrays (levels, flat panel indices), recur-call count."""
    cap = 1 << 16
    lev = np.zeros(cap, dtype=np.int64)
    pk = np.zeros(cap, dtype=np.int64)
    calls = np.zeros(1, dtype=np.int64)
    cnt = lib().or_tree_decompose(d, L, float(delta_i), int(node), _ptr(lev), _ptr(pk), cap,
                                  _ptr(calls))
    assert cnt <= cap
    return lev[:cnt].copy(), pk[:cnt].copy(), int(calls[0])


def _fast(fn, u, d, L, delta, K, alpha, scale, normalize, coef, a, self_mode, idx):
    u = _f64(u)
    n = 1 << L
    squeeze = u.ndim == 1
    u2 = u.reshape(1, -1) if squeeze else u.reshape(u.shape[0], -1)
    nrhs = u2.shape[0]
    dl = _delta_field(delta, d, n)
    p = poly_coeffs(K, alpha)
    sg = sigma(d, alpha, scale, normalize)
    a_ = None if a is None else _f64(a).reshape(-1)
    ix, nix = _idx(idx)
    M = nix if ix is not None else n ** d
    out = np.zeros((nrhs, M))
    cnt = np.zeros(M, dtype=np.int64)
    rc = fn(d, L, _ptr(dl), K, _ptr(p), sg, coef, _ptr(a_), self_mode, nrhs, _ptr(u2),
            _ptr(out), _ptr(ix), nix, _ptr(cnt))
    if rc:
        raise ValueError(f"oracle fast path failed ({rc})")
    return (out[0] if squeeze else out), cnt


def fast_tree(u, d, L, delta, K=0, alpha=1.0, scale=1.0, normalize=True, coef=COEF_NONE,
              a=None, self_mode=SELF_DISCRETE, idx=None, return_counts=False):
    """O1: Algorithm 1 + Step 2 pyramid + Step 3 + Eq. (3.3)."""
    out, cnt = _fast(lib().or_fast_tree, u, d, L, delta, K, alpha, scale, normalize, coef, a,
                     self_mode, idx)
    return (out, cnt) if return_counts else out


def fast_leafset(u, d, L, delta, K=0, alpha=1.0, scale=1.0, normalize=True, coef=COEF_NONE,
                 a=None, self_mode=SELF_DISCRETE, idx=None, return_counts=False):
    """O2: plain sum over the leaf cells meeting the open ball, then Eq. (3.3)."""
    out, cnt = _fast(lib().or_fast_leafset, u, d, L, delta, K, alpha, scale, normalize, coef, a,
                     self_mode, idx)
    return (out, cnt) if return_counts else out


def fast_sym_leafset(u, d, L, delta, K=0, alpha=1.0, scale=1.0, normalize=True,
                     coef=COEF_NONE, a=None, idx=None):
    """Symmetrised leaf-set operator of the polynomial kernel (divergence type, a project
    extension of Sec. 3): sigma h^d sum_k (w_i(k) + w_k(i))/2 (u_k - u_i), each half over its
    own node's leaf set.  u: [nrhs, N] or [N]."""
    u = _f64(u)
    n = 1 << L
    squeeze = u.ndim == 1
    u2 = u.reshape(1, -1) if squeeze else u.reshape(u.shape[0], -1)
    nrhs = u2.shape[0]
    dl = _delta_field(delta, d, n)
    p = poly_coeffs(K, alpha)
    sg = sigma(d, alpha, scale, normalize)
    a_ = None if a is None else _f64(a).reshape(-1)
    ix, nix = _idx(idx)
    M = nix if ix is not None else n ** d
    out = np.zeros((nrhs, M))
    rc = lib().or_fast_sym_leafset(d, L, _ptr(dl), K, _ptr(p), sg, coef, _ptr(a_), nrhs,
                                   _ptr(u2), _ptr(out), _ptr(ix), nix)
    if rc:
        raise ValueError(f"or_fast_sym_leafset failed ({rc})")
    return out[0] if squeeze else out


def fast_pd_leafset(u, d, L, delta, c, scale=1.0, K=0, idx=None):
    """Fast-path peridynamics over the leaf set of Algorithm 1 with the polynomial
    micromodulus p^{2K} matched to gamma(s) = s^-3 (K = 0: p = 1):
    h^d sum_{k in LS(i)} scale c_ik p(|xi|/delta_i) (xi xi^T / delta_i^3) (u_k - u_i).
    u: [nrhs, d, N] or [d, N]."""
    u = _f64(u)
    n = 1 << L
    squeeze = u.ndim == 2
    u3 = u.reshape(1, d, -1) if squeeze else u.reshape(u.shape[0], d, -1)
    nrhs = u3.shape[0]
    dl = _delta_field(delta, d, n)
    c_ = _delta_field(c, d, n)
    pc = poly_coeffs(K, 3.0)
    ix, nix = _idx(idx)
    M = nix if ix is not None else n ** d
    out = np.zeros((nrhs, d, M))
    rc = lib().or_fast_pd_leafset(d, L, _ptr(dl), _ptr(c_), float(scale), int(K), _ptr(pc),
                                  nrhs, _ptr(u3), _ptr(out), _ptr(ix), nix)
    if rc != 0:
        raise ValueError(f"or_fast_pd_leafset failed ({rc})")
    return out[0] if squeeze else out


def cg(f, d, n, delta, kind="scalar", family=POWER, alpha=0.0, K=0, scale=1.0, normalize=True,
       coef=COEF_NONE, a=None, c=None, jacobi=True, rtol=1e-8, maxit=10000):
    """Plain PCG on -L x = f (x0 = 0).  Returns (x, iterations, true relative residual)."""
    f = _f64(f).reshape(-1)
    dl = _delta_field(delta, d, n)
    k = 0 if kind == "scalar" else 1
    p = poly_coeffs(K, alpha) if family in (POLY, KAPPA) else np.zeros(1)
    sg = sigma(d, alpha, scale, normalize) if k == 0 else float(scale)
    a_ = None if a is None else _f64(a).reshape(-1)
    c_ = None if c is None else _delta_field(c, d, n)
    dinv = None
    if jacobi:
        if k == 0:
            dinv = 1.0 / direct_diag(d, n, dl, family, alpha, K, scale, normalize, coef, a_, True)
        else:
            dinv = 1.0 / pd_diag(d, n, dl, c_, scale)
        dinv = _f64(dinv)
    x = np.zeros_like(f)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    lib().or_cg(k, d, n, _ptr(dl), family, float(alpha), K, _ptr(p), sg, coef, _ptr(a_),
                _ptr(c_), _ptr(dinv), _ptr(f), _ptr(x), float(rtol), int(maxit),
                ctypes.byref(it), ctypes.byref(rr))
    return x, it.value, rr.value


def pd_diag(d, n, delta, c, scale=1.0):
    """Diagonal of -L_PD, component-major [d, N]: h^d sum scale c_ij xi_k^2/|xi|^3."""
    N = n ** d
    dl = _delta_field(delta, d, n)
    c_ = _delta_field(c, d, n)
    diag = np.zeros((d, N))
    h = 1.0 / n
    rmax = float(np.max(dl)) * n
    B = int(np.ceil(rmax))
    rng = np.arange(-B, B + 1)
    grids = np.meshgrid(*([rng] * d), indexing="ij")
    offs = np.stack([g.reshape(-1) for g in grids[::-1]], axis=1)  # columns: x, y, z
    o2 = (offs ** 2).sum(axis=1)
    coords = np.stack(np.unravel_index(np.arange(N), (n,) * d)[::-1], axis=1)  # x fastest
    for i in range(N):
        R2 = (dl[i] * n) * (dl[i] * n)
        sel = (o2 > 0) & (o2.astype(np.float64) < R2)
        o = offs[sel]
        cj = coords[i] + o
        inside = np.all((cj >= 0) & (cj < n), axis=1)
        fj = np.zeros(len(o), dtype=np.int64)
        mult = 1
        for k in range(d):
            fj += np.where(inside, cj[:, k], 0) * mult
            mult *= n
        cij = 0.5 * (c_[i] + np.where(inside, c_[fj], c_[i]))
        xi = o * h
        L = np.sqrt((xi ** 2).sum(axis=1))
        for k in range(d):
            diag[k, i] = h ** d * np.sum(scale * cij * xi[:, k] ** 2 / L ** 3)
    return diag.reshape(-1)
