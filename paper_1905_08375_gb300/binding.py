"""Thin ctypes binding over the C-ABI in ``include/nl.h`` (same entry-point names).

Argument marshalling only: every step of an apply runs in ``_lib/libnl.so``.
Device buffers are torch CUDA tensors (PyTorch is used for device memory and
streams); host-side plan inputs are numpy arrays.  There is no fallback: if
the library has not been built, or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libnl.so")

NL_OK, NL_EINVAL, NL_EUNSUPPORTED, NL_ENOMEM, NL_ECUDA, NL_ENOTCONV, NL_ETIMEOUT = range(7)
NL_F32, NL_F64, NL_F64_PAIRS = 0, 1, 2
NL_POWER, NL_POLY, NL_PD_BOND, NL_KAPPA = 0, 1, 2, 3
NL_COEF_NONE, NL_COEF_X, NL_COEF_XY, NL_COEF_MEAN = 0, 1, 2, 3
NL_SELF_DISCRETE, NL_SELF_PAPER = 0, 1
NL_FAST_AUTO, NL_FAST_PANELS, NL_FAST_ROWPREFIX, NL_FAST_FP64_PANELS, NL_FAST_LEAFROWS = 0, 1, 2, 3, 4
NL_PRECOND_NONE, NL_PRECOND_JACOBI = 0, 1

_STATUS = {0: "NL_OK", 1: "NL_EINVAL", 2: "NL_EUNSUPPORTED", 3: "NL_ENOMEM", 4: "NL_ECUDA",
           5: "NL_ENOTCONV", 6: "NL_ETIMEOUT"}


class NlError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class nl_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int)]


class nl_horizon(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("delta_field", ctypes.c_void_p),
                ("symmetric", ctypes.c_int)]


class nl_kernel(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int), ("alpha", ctypes.c_double), ("K", ctypes.c_int),
                ("scale", ctypes.c_double), ("normalize", ctypes.c_int), ("coef", ctypes.c_int),
                ("a", ctypes.c_void_p), ("self_term", ctypes.c_int),
                ("fast_variant", ctypes.c_int)]


class nl_cg_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("converged", ctypes.c_int)]


class nl_plan_info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("levels", ctypes.c_int),
                ("max_radius", ctypes.c_int), ("num_offsets", ctypes.c_int),
                ("moments", ctypes.c_int), ("sigma", ctypes.c_double),
                ("poly", ctypes.c_double * 8), ("device_bytes", ctypes.c_size_t),
                ("step1_bytes", ctypes.c_size_t)]


ENTRY_POINTS = ("nl_plan_create", "nl_plan_destroy", "nl_apply", "nl_apply_fast", "nl_cg_solve",
                "nl_get_plan_info", "nl_last_error", "nl_batch_create", "nl_batch_destroy",
                "nl_batch_layout", "nl_batch_apply", "nl_batch_cg_solve")

_lib = None


def lib():
    """Load libnl.so (built by ``build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.nl_plan_create.restype = i
    L.nl_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(nl_grid),
                                 ctypes.POINTER(nl_horizon), ctypes.POINTER(nl_kernel), vp]
    L.nl_plan_destroy.restype = i
    L.nl_plan_destroy.argtypes = [vp]
    for name in ("nl_apply", "nl_apply_fast"):
        fn = getattr(L, name)
        fn.restype = i
        fn.argtypes = [vp, vp, vp, i, i, vp]
    L.nl_cg_solve.restype = i
    L.nl_cg_solve.argtypes = [vp, vp, vp, i, d, i, i, ctypes.POINTER(nl_cg_stats), vp]
    L.nl_get_plan_info.restype = i
    L.nl_get_plan_info.argtypes = [vp, ctypes.POINTER(nl_plan_info)]
    L.nl_last_error.restype = ctypes.c_char_p
    L.nl_last_error.argtypes = []
    _lib = L
    return L


def nl_last_error() -> str:
    return lib().nl_last_error().decode()


def _check(status):
    if status != NL_OK:
        raise NlError(status, nl_last_error())


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(t):
    import torch
    if t.dtype == torch.float32:
        return NL_F32
    if t.dtype == torch.float64:
        return NL_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


class Plan:
    """Owns an ``nl_plan*``; freed by ``close()`` or garbage collection."""

    def __init__(self, handle, dim, n, family):
        self.handle = handle
        self.dim, self.n, self.family = dim, n, family

    @property
    def N(self):
        return self.n ** self.dim

    def close(self):
        if self.handle:
            lib().nl_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return nl_get_plan_info(self)


def nl_plan_create(dim, n, delta, family=NL_POWER, alpha=0.0, K=0, scale=1.0, normalize=True,
                   coef=NL_COEF_NONE, a=None, symmetric=False, self_term=NL_SELF_DISCRETE,
                   fast_variant=NL_FAST_AUTO, stream=None) -> Plan:
    """Create a plan.  `delta`: scalar or host array of n^dim values; `a`: host array or None."""
    g = nl_grid(dim, n)
    keep = []
    if np.isscalar(delta):
        hz = nl_horizon(float(delta), None, int(bool(symmetric)))
    else:
        dl = np.ascontiguousarray(delta, dtype=np.float64).reshape(-1)
        if dl.size != n ** dim:
            raise ValueError("delta field must have n^dim values")
        keep.append(dl)
        hz = nl_horizon(0.0, dl.ctypes.data, int(bool(symmetric)))
    ap = None
    if a is not None:
        aa = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        if aa.size != n ** dim:
            raise ValueError("coefficient field must have n^dim values")
        keep.append(aa)
        ap = aa.ctypes.data
    k = nl_kernel(int(family), float(alpha), int(K), float(scale), int(bool(normalize)),
                  int(coef), ap, int(self_term), int(fast_variant))
    h = ctypes.c_void_p()
    st = _stream_ptr(stream) if _cuda_ready() else ctypes.c_void_p(None)
    _check(lib().nl_plan_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(hz),
                                ctypes.byref(k), st))
    return Plan(h, dim, n, family)


def _cuda_ready():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def _apply(fn, plan, u, Lu, nrhs, stream, dtype=None):
    if not (u.is_cuda and Lu.is_cuda):
        raise ValueError("u and Lu must be CUDA tensors")
    if not (u.is_contiguous() and Lu.is_contiguous()) or u.dtype != Lu.dtype:
        raise ValueError("u and Lu must be contiguous with the same dtype")
    comps = plan.dim if plan.family == NL_PD_BOND else 1
    per = plan.N * comps
    if nrhs is None:
        nrhs = u.numel() // per
    if u.numel() != nrhs * per or Lu.numel() != nrhs * per:
        raise ValueError("u/Lu size does not match nrhs * n^d (* d)")
    code = _dtype_code(u) if dtype is None else dtype
    _check(fn(plan.handle, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(Lu.data_ptr()),
              int(nrhs), code, _stream_ptr(stream)))
    return Lu


def nl_apply(plan: Plan, u, Lu, nrhs=None, stream=None, pairs=False):
    """Direct apply on device tensors; returns Lu.  pairs=True (FP64 tensors): the
    FP32-pair arithmetic of NL_F64_PAIRS."""
    if pairs:
        import torch
        if u.dtype != torch.float64:
            raise ValueError("pairs=True takes FP64 tensors")
        return _apply(lib().nl_apply, plan, u, Lu, nrhs, stream, NL_F64_PAIRS)
    return _apply(lib().nl_apply, plan, u, Lu, nrhs, stream)


def nl_apply_fast(plan: Plan, u, Lu, nrhs=None, stream=None):
    """Fast (Sec. 3) apply on device tensors; returns Lu."""
    return _apply(lib().nl_apply_fast, plan, u, Lu, nrhs, stream)


def nl_cg_solve(plan: Plan, f, x, nrhs=None, rtol=1e-8, maxit=10000, precond=NL_PRECOND_JACOBI,
                stream=None) -> dict:
    """CG on -L x = f (FP64 device tensors).  Returns the stats as a dict."""
    comps = plan.dim if plan.family == NL_PD_BOND else 1
    per = plan.N * comps
    if nrhs is None:
        nrhs = f.numel() // per
    st = nl_cg_stats()
    status = lib().nl_cg_solve(plan.handle, ctypes.c_void_p(f.data_ptr()),
                               ctypes.c_void_p(x.data_ptr()), int(nrhs), float(rtol), int(maxit),
                               int(precond), ctypes.byref(st), _stream_ptr(stream))
    out = dict(iterations=st.iterations, rel_residual=st.rel_residual,
               converged=bool(st.converged), status=status)
    if status not in (NL_OK, NL_ENOTCONV):
        _check(status)
    return out


def nl_get_plan_info(plan: Plan) -> dict:
    info = nl_plan_info()
    _check(lib().nl_get_plan_info(plan.handle, ctypes.byref(info)))
    return dict(dim=info.dim, n=info.n, levels=info.levels, max_radius=info.max_radius,
                num_offsets=info.num_offsets, moments=info.moments, sigma=info.sigma,
                poly=list(info.poly), device_bytes=int(info.device_bytes),
                step1_bytes=int(info.step1_bytes))


def nl_apply_fast_noalloc(dim, n, delta, u, Lu, alpha=0.0, scale=1.0, normalize=True,
                          self_term=NL_SELF_DISCRETE, nrhs=None, stream=None):
    """The allocation-free fast apply (p = 1, C = 1).  `delta`: a float (constant horizon) or
    a CUDA float64 tensor of n^dim horizons.  u, Lu: CUDA tensors.  Returns Lu."""
    L = lib()
    fn = L.nl_apply_fast_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                   ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    N = int(n) ** int(dim)
    if isinstance(delta, (int, float)):
        dconst, dptr = float(delta), None
    else:
        import torch
        if not (delta.is_cuda and delta.dtype == torch.float64 and delta.is_contiguous()):
            raise ValueError("delta field must be a contiguous CUDA float64 tensor")
        if delta.numel() != N:
            raise ValueError(f"delta field has {delta.numel()} values, expected n^dim = {N}")
        dconst, dptr = 0.0, ctypes.c_void_p(delta.data_ptr())
    if not (u.is_cuda and Lu.is_cuda and u.is_contiguous() and Lu.is_contiguous()):
        raise ValueError("u and Lu must be contiguous CUDA tensors")
    if u.dtype != Lu.dtype:
        raise ValueError(f"u ({u.dtype}) and Lu ({Lu.dtype}) must have the same dtype")
    if nrhs is None:
        nrhs = u.numel() // N if N > 0 else 0
    if u.numel() != nrhs * N or Lu.numel() != nrhs * N:
        raise ValueError(f"u and Lu need nrhs * n^dim = {nrhs * N} elements "
                         f"(got {u.numel()} and {Lu.numel()})")
    _check(fn(int(dim), int(n), dconst, dptr, float(alpha), float(scale), int(bool(normalize)),
              int(self_term), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(Lu.data_ptr()),
              int(nrhs), _dtype_code(u), _stream_ptr(stream)))
    return Lu


# ---------------------------------------------------------------------------
# learned CG preconditioner
# ---------------------------------------------------------------------------
NL_PRECOND_LEARNED = 2
NL_NET_PARAMS = 9792


def _net_fns():
    L = lib()
    if getattr(L, "_net_ready", False):
        return L
    vp, i, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    L.nl_net_create.restype = i
    L.nl_net_create.argtypes = [ctypes.POINTER(vp), vp, vp]
    L.nl_net_destroy.restype = i
    L.nl_net_destroy.argtypes = [vp]
    L.nl_net_get_weights.restype = i
    L.nl_net_get_weights.argtypes = [vp, vp, vp]
    L.nl_net_gradient.restype = i
    L.nl_net_gradient.argtypes = [vp, vp, vp]
    L.nl_net_forward.restype = i
    L.nl_net_forward.argtypes = [vp, vp, vp, i, i, i, vp]
    L.nl_net_train_step.restype = i
    L.nl_net_train_step.argtypes = [vp, vp, vp, i, i, vp, i, i, i, f, ctypes.POINTER(f), vp]
    L.nl_net_train_step_energy.restype = i
    L.nl_net_train_step_energy.argtypes = [vp, vp, vp, vp, i, vp, i, f, ctypes.POINTER(f), vp]
    L.nl_net_prepare_pairs.restype = i
    L.nl_net_prepare_pairs.argtypes = [vp, vp, vp, i, vp, vp, vp]
    L.nl_net_apply.restype = i
    L.nl_net_apply.argtypes = [vp, vp, vp, vp, i, vp]
    L.nl_plan_set_net.restype = i
    L.nl_plan_set_net.argtypes = [vp, vp]
    L.nl_net_set_coarse.restype = i
    L.nl_net_set_coarse.argtypes = [vp, i]
    L.nl_cg_history.restype = i
    L.nl_cg_history.argtypes = [vp, vp, vp, ctypes.c_double, i, i, vp, i,
                                ctypes.POINTER(i), ctypes.POINTER(nl_cg_stats), vp]
    L._net_ready = True
    return L


class Net:
    """Owns an ``nl_net*``."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            _net_fns().nl_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nl_net_set_coarse(net: Net, block: int):
    """0: the local form; block >= 2: the two-level form on ceil(n/block)^2 coarse cells."""
    _check(_net_fns().nl_net_set_coarse(net.handle, int(block)))


def nl_net_create(weights, stream=None) -> Net:
    w = np.ascontiguousarray(weights, dtype=np.float32).reshape(-1)
    if w.size != NL_NET_PARAMS:
        raise ValueError(f"need {NL_NET_PARAMS} weights")
    h = ctypes.c_void_p()
    _check(_net_fns().nl_net_create(ctypes.byref(h), w.ctypes.data, _stream_ptr(stream)))
    return Net(h)


def nl_net_get_weights(net: Net, stream=None) -> np.ndarray:
    w = np.zeros(NL_NET_PARAMS, dtype=np.float32)
    _check(_net_fns().nl_net_get_weights(net.handle, w.ctypes.data, _stream_ptr(stream)))
    return w


def nl_net_gradient(net: Net, stream=None) -> np.ndarray:
    g = np.zeros(NL_NET_PARAMS, dtype=np.float32)
    _check(_net_fns().nl_net_gradient(net.handle, g.ctypes.data, _stream_ptr(stream)))
    return g


def nl_net_forward(net: Net, x, o, stream=None):
    """x, o: CUDA float32 [batch, H, W]."""
    B, H, W = x.shape
    _check(_net_fns().nl_net_forward(net.handle, ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(o.data_ptr()), B, H, W,
                                     _stream_ptr(stream)))
    return o


def nl_net_train_step(net: Net, x, e, crops, S, margin, lr, want_loss=True, stream=None):
    """x, e: CUDA float32 [nfields, n, n]; crops: CUDA int32 [batch, 3].  Returns the loss."""
    nf, n, _ = x.shape
    loss = ctypes.c_float(0.0)
    _check(_net_fns().nl_net_train_step(net.handle, ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(e.data_ptr()), nf, n,
                                        ctypes.c_void_p(crops.data_ptr()), crops.shape[0], S,
                                        margin, float(lr),
                                        ctypes.byref(loss) if want_loss else None,
                                        _stream_ptr(stream)))
    return float(loss.value) if want_loss else None


def nl_net_train_step_energy(net: Net, plan: Plan, x, e, fields, lr, want_loss=True,
                             stream=None):
    """x, e: CUDA float32 [nfields, N]; fields: CUDA int32 [batch].  Returns the loss."""
    loss = ctypes.c_float(0.0)
    _check(_net_fns().nl_net_train_step_energy(
        net.handle, plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(e.data_ptr()),
        x.shape[0], ctypes.c_void_p(fields.data_ptr()), fields.shape[0], float(lr),
        ctypes.byref(loss) if want_loss else None, _stream_ptr(stream)))
    return float(loss.value) if want_loss else None


def nl_net_prepare_pairs(plan: Plan, r, e, xo, eo, stream=None):
    """r, e: CUDA float64 [count, N]; xo, eo: CUDA float32 [count, N]."""
    _check(_net_fns().nl_net_prepare_pairs(plan.handle, ctypes.c_void_p(r.data_ptr()),
                                           ctypes.c_void_p(e.data_ptr()), r.shape[0],
                                           ctypes.c_void_p(xo.data_ptr()),
                                           ctypes.c_void_p(eo.data_ptr()), _stream_ptr(stream)))


def nl_net_history_pairs(plan: Plan, f, x, history, count, xo, eo, stream=None):
    """f, x: CUDA float64 [N]; history: CUDA float64 [>= count, N] (CG iterates);
    xo, eo: CUDA float32 [count, N].  r_k = f + L x_k and e_k = x - x_k are formed by the
    library, then scaled as by nl_net_prepare_pairs."""
    L = _net_fns()
    fn = L.nl_net_history_pairs
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int] + [ctypes.c_void_p] * 3
    N = plan.N
    if f.numel() != N or x.numel() != N or history.numel() < count * N:
        raise ValueError("f, x need n^2 values and history count * n^2")
    if xo.numel() < count * N or eo.numel() < count * N:
        raise ValueError("xo, eo need count * n^2 values")
    _check(fn(plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(x.data_ptr()),
              ctypes.c_void_p(history.data_ptr()), int(count), ctypes.c_void_p(xo.data_ptr()),
              ctypes.c_void_p(eo.data_ptr()), _stream_ptr(stream)))


def nl_net_apply(net: Net, plan: Plan, r, z, nrhs=None, stream=None):
    if nrhs is None:
        nrhs = r.numel() // plan.N
    _check(_net_fns().nl_net_apply(net.handle, plan.handle, ctypes.c_void_p(r.data_ptr()),
                                   ctypes.c_void_p(z.data_ptr()), int(nrhs), _stream_ptr(stream)))
    return z


def nl_plan_set_net(plan: Plan, net):
    _check(_net_fns().nl_plan_set_net(plan.handle, net.handle if net is not None else None))
    plan._net = net      # keep the network alive while attached


def nl_cg_history(plan: Plan, f, x, history, rtol=1e-8, maxit=10000,
                  precond=NL_PRECOND_JACOBI, stream=None):
    """CG for one right-hand side recording x every 16 iterations into history [cap, N]."""
    cnt = ctypes.c_int(0)
    st = nl_cg_stats()
    status = _net_fns().nl_cg_history(plan.handle, ctypes.c_void_p(f.data_ptr()),
                                      ctypes.c_void_p(x.data_ptr()), float(rtol), int(maxit),
                                      int(precond), ctypes.c_void_p(history.data_ptr()),
                                      history.shape[0], ctypes.byref(cnt), ctypes.byref(st),
                                      _stream_ptr(stream))
    if status not in (NL_OK, NL_ENOTCONV):
        _check(status)
    return cnt.value, dict(iterations=st.iterations, rel_residual=st.rel_residual,
                           converged=bool(st.converged), status=status)


def nl_plan_profile(plan: Plan, enable=True):
    L = lib()
    L.nl_plan_profile.restype = ctypes.c_int
    L.nl_plan_profile.argtypes = [ctypes.c_void_p, ctypes.c_int]
    _check(L.nl_plan_profile(plan.handle, int(bool(enable))))


def nl_plan_profile_read(plan: Plan) -> dict:
    """Summed Step 2 / Step 3 milliseconds of the fast applies since the last read."""
    L = lib()
    L.nl_plan_profile_read.restype = ctypes.c_int
    L.nl_plan_profile_read.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int)]
    a, b, c = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_int(0)
    _check(L.nl_plan_profile_read(plan.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return dict(step2_ms=a.value, step3_ms=b.value, applies=c.value)


NL_TILE_AUTO, NL_TILE_32x4, NL_TILE_32x8, NL_TILE_32x16 = -1, 0, 1, 2


class Batch:
    """Owns an ``nl_batch*`` (many uneven 2-D instances applied and solved together)."""

    def __init__(self, handle, sizes, family, offsets, tile_shape):
        self.handle = handle
        self.sizes = list(sizes)
        self.family = family
        self.offsets = offsets
        self.tile_shape = tile_shape

    @property
    def total(self):
        return int(self.offsets[-1])

    def close(self):
        if self.handle:
            lib().nl_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batch_sigs(L):
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.nl_batch_create.restype = i
    L.nl_batch_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(nl_grid),
                                  ctypes.POINTER(nl_horizon), ctypes.POINTER(nl_kernel), i, vp]
    L.nl_batch_destroy.restype = i
    L.nl_batch_destroy.argtypes = [vp]
    L.nl_batch_layout.restype = i
    L.nl_batch_layout.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(i)]
    L.nl_batch_apply.restype = i
    L.nl_batch_apply.argtypes = [vp, vp, vp, i, vp]
    L.nl_batch_cg_solve.restype = i
    L.nl_batch_cg_solve.argtypes = [vp, vp, vp, d, i, i, ctypes.POINTER(nl_cg_stats), vp]


def nl_batch_create(instances, family=NL_POWER, alpha=0.0, scale=1.0, normalize=True,
                    coef=NL_COEF_NONE, symmetric=False, tile_shape=NL_TILE_AUTO,
                    stream=None) -> Batch:
    """instances: list of (n, delta, a) with delta a float or a host array of n*n horizons and
    a None or a host array of n*n coefficient values (all instances 2-D).  tile_shape:
    NL_TILE_AUTO (time the three shapes and keep the fastest) or 0, 1, 2 (32x4, 32x8, 32x16)."""
    L = lib()
    _batch_sigs(L)
    cnt = len(instances)
    grids = (nl_grid * cnt)()
    hzs = (nl_horizon * cnt)()
    kers = (nl_kernel * cnt)()
    keep = []
    for k, (n, delta, a) in enumerate(instances):
        grids[k] = nl_grid(2, int(n))
        if np.isscalar(delta):
            hzs[k] = nl_horizon(float(delta), None, int(bool(symmetric)))
        else:
            dl = np.ascontiguousarray(delta, dtype=np.float64).reshape(-1)
            if dl.size != n * n:
                raise ValueError("delta field must have n*n values")
            keep.append(dl)
            hzs[k] = nl_horizon(0.0, dl.ctypes.data, int(bool(symmetric)))
        ap = None
        if a is not None:
            aa = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
            if aa.size != n * n:
                raise ValueError("coefficient field must have n*n values")
            keep.append(aa)
            ap = aa.ctypes.data
        kers[k] = nl_kernel(int(family), float(alpha), 0, float(scale), int(bool(normalize)),
                            int(coef) if a is not None else NL_COEF_NONE, ap,
                            NL_SELF_DISCRETE, NL_FAST_AUTO)
    h = ctypes.c_void_p()
    _check(L.nl_batch_create(ctypes.byref(h), cnt, grids, hzs, kers, int(tile_shape),
                             _stream_ptr(stream)))
    offs = (ctypes.c_int64 * (cnt + 1))()
    shape = ctypes.c_int()
    _check(L.nl_batch_layout(h, offs, ctypes.byref(shape)))
    return Batch(h, [inst[0] for inst in instances], family, np.array(list(offs), dtype=np.int64),
                 shape.value)


def nl_batch_apply(batch: Batch, u, Lu, stream=None):
    """Direct apply of every instance in one launch (concatenated device tensors)."""
    L = lib()
    _batch_sigs(L)
    if not (u.is_cuda and Lu.is_cuda and u.is_contiguous() and Lu.is_contiguous()):
        raise ValueError("u and Lu must be contiguous CUDA tensors")
    if u.dtype != Lu.dtype or u.numel() != batch.total or Lu.numel() != batch.total:
        raise ValueError("u/Lu must hold the batch's concatenated fields (same dtype)")
    _check(L.nl_batch_apply(batch.handle, ctypes.c_void_p(u.data_ptr()),
                            ctypes.c_void_p(Lu.data_ptr()), _dtype_code(u), _stream_ptr(stream)))
    return Lu


def nl_batch_cg_solve(batch: Batch, f, x, rtol=1e-8, maxit=10000, precond=NL_PRECOND_JACOBI,
                      stream=None) -> dict:
    """CG on -L_k x_k = f_k for every instance together (FP64 device tensors)."""
    L = lib()
    _batch_sigs(L)
    if f.numel() != batch.total or x.numel() != batch.total:
        raise ValueError("f/x must hold the batch's concatenated fields")
    st = nl_cg_stats()
    status = L.nl_batch_cg_solve(batch.handle, ctypes.c_void_p(f.data_ptr()),
                                 ctypes.c_void_p(x.data_ptr()), float(rtol), int(maxit),
                                 int(precond), ctypes.byref(st), _stream_ptr(stream))
    out = dict(iterations=st.iterations, rel_residual=st.rel_residual,
               converged=bool(st.converged), status=status)
    if status not in (NL_OK, NL_ENOTCONV):
        _check(status)
    return out


# ---------------------------------------------------------------------------
# host-side failure handling
# ---------------------------------------------------------------------------
WAIT_POLL_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p)


def nl_set_wait_limit(seconds: float):
    """Limit (s) of the library's bounded host waits (CG chunks); 600 s by default."""
    fn = lib().nl_set_wait_limit
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_double]
    _check(fn(float(seconds)))


def nl_wait_poll(poll, seconds: float) -> int:
    """Run the library's bounded wait on a Python condition: poll() -> 1 done, 0 not yet,
    < 0 error.  Returns the status code (NL_OK, NL_ETIMEOUT or NL_ECUDA)."""
    fn = lib().nl_wait_poll
    fn.restype = ctypes.c_int
    fn.argtypes = [WAIT_POLL_FN, ctypes.c_void_p, ctypes.c_double]
    cb = WAIT_POLL_FN(lambda _ctx: int(poll()))
    return int(fn(cb, None, float(seconds)))


def nl_debug_fail_host_alloc(after: int):
    """Make the host allocation after `after` successful ones in nl_plan_create fail once
    (after < 0 disarms)."""
    fn = lib().nl_debug_fail_host_alloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int]
    _check(fn(int(after)))


def nl_measure_peaks(stream=None) -> dict:
    """Measured FMA peaks of the current device in TFLOP/s (fp32, fp32x2, fp64)."""
    fn = lib().nl_measure_peaks
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(ctypes.c_double)] * 3 + [ctypes.c_void_p]
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(fn(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), _stream_ptr(stream)))
    return {"fp32_tflops": a.value, "fp32x2_tflops": b.value, "fp64_tflops": c.value}
