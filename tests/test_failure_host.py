"""Failure handling of the C-ABI library, exercised on the host only (no GPU is faulted, hung
or even needed): the bounded host wait that CG uses runs out and reports NL_ETIMEOUT, an
injected host-allocation failure inside nl_plan_create comes back as NL_ENOMEM, and corrupted
plan, batch and network handles are rejected with NL_EINVAL before any device work."""
import ctypes
import time

import numpy as np
import pytest


@pytest.fixture(scope="module")
def nl():
    from paper_1905_08375_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def test_bounded_wait_runs_out(nl):
    t0 = time.perf_counter()
    st = nl.nl_wait_poll(lambda: 0, 0.05)
    dt = time.perf_counter() - t0
    assert st == nl.NL_ETIMEOUT
    assert 0.05 <= dt < 5.0
    assert "gave up" in nl.nl_last_error()


def test_bounded_wait_returns_when_the_condition_holds(nl):
    calls = []

    def poll():
        calls.append(1)
        return 1 if len(calls) >= 3 else 0
    assert nl.nl_wait_poll(poll, 10.0) == nl.NL_OK
    assert len(calls) == 3


def test_bounded_wait_reports_a_failed_condition(nl):
    assert nl.nl_wait_poll(lambda: -1, 10.0) == nl.NL_ECUDA


def test_wait_limit_is_settable_and_validated(nl):
    try:
        nl.nl_set_wait_limit(0.03)
        t0 = time.perf_counter()
        assert nl.nl_wait_poll(lambda: 0, 0.0) == nl.NL_ETIMEOUT    # 0: the library limit
        assert time.perf_counter() - t0 < 5.0
        for bad in (0.0, -1.0, float("nan"), 1e7):
            with pytest.raises(nl.NlError, match="NL_EINVAL"):
                nl.nl_set_wait_limit(bad)
    finally:
        nl.nl_set_wait_limit(600.0)


@pytest.mark.parametrize("after", [0, 1])
def test_injected_host_allocation_failure(nl, after):
    try:
        nl.nl_debug_fail_host_alloc(after)
        with pytest.raises(nl.NlError) as ei:
            nl.nl_plan_create(2, 8, 0.3)
        assert str(ei.value).startswith("NL_ENOMEM"), str(ei.value)
        assert "host allocation" in str(ei.value)
    finally:
        nl.nl_debug_fail_host_alloc(-1)


def test_injected_failure_fires_once(nl):
    nl.nl_debug_fail_host_alloc(0)
    with pytest.raises(nl.NlError, match="NL_ENOMEM"):
        nl.nl_plan_create(2, 8, 0.3)
    # disarmed after firing: a bad argument is reported as such again
    with pytest.raises(nl.NlError, match="NL_EINVAL"):
        nl.nl_plan_create(2, 8, -0.3)


def _fake_handle(magic=None, version=None, seed=0):
    rng = np.random.default_rng(seed)
    buf = (ctypes.c_ubyte * 65536)(*rng.integers(0, 256, 65536).tolist())
    if magic is not None:
        ctypes.memmove(buf, ctypes.byref(ctypes.c_uint32(magic)), 4)
    if version is not None:
        ctypes.memmove(ctypes.addressof(buf) + 4, ctypes.byref(ctypes.c_int32(version)), 4)
    return buf, ctypes.c_void_p(ctypes.addressof(buf))


@pytest.mark.parametrize("magic,version", [(None, None), (0x4E4C504C, 99), (0, 1)])
def test_corrupted_plan_handle_rejected(nl, magic, version):
    lib = nl.lib()
    buf, h = _fake_handle(magic, version)
    dummy = ctypes.c_void_p(ctypes.addressof(buf))        # never dereferenced as data
    assert lib.nl_apply(h, dummy, dummy, 1, 0, None) == nl.NL_EINVAL
    assert lib.nl_apply_fast(h, dummy, dummy, 1, 0, None) == nl.NL_EINVAL
    st = nl.nl_cg_stats()
    assert lib.nl_cg_solve(h, dummy, dummy, 1, 1e-8, 10, 1, ctypes.byref(st), None) == nl.NL_EINVAL
    info = nl.nl_plan_info()
    assert lib.nl_get_plan_info(h, ctypes.byref(info)) == nl.NL_EINVAL
    assert lib.nl_plan_destroy(h) == nl.NL_EINVAL
    assert "plan" in nl.nl_last_error()


def test_corrupted_batch_and_network_handles_rejected(nl):
    lib = nl.lib()
    nl._net_fns()
    buf, h = _fake_handle(seed=3)
    dummy = ctypes.c_void_p(ctypes.addressof(buf))
    for fn, args in (("nl_batch_apply", (h, dummy, dummy, 0, None)),
                     ("nl_batch_destroy", (h,)),
                     ("nl_net_destroy", (h,)),
                     ("nl_net_set_coarse", (h, 4)),
                     ("nl_plan_set_net", (h, None))):
        f = getattr(lib, fn)
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p if isinstance(a, ctypes.c_void_p) or a is None
                                          else ctypes.c_int for a in args[1:]]
        assert f(*args) == nl.NL_EINVAL, fn
