"""CPU-side checks of the C-ABI library: it loads, exports every entry point that
include/nl.h declares, and rejects invalid plans before touching the GPU."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nl.h")


@pytest.fixture(scope="module")
def nl():
    from paper_1905_08375_gb300 import build, binding
    build.build()
    binding.lib()
    return binding


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nl_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("nl_plan_create", "nl_plan_destroy", "nl_apply", "nl_apply_fast", "nl_cg_solve",
              "nl_last_error", "nl_get_plan_info"):
        assert n in names


def test_library_exports_every_declared_symbol(nl):
    out = subprocess.run(["nm", "-D", "--defined-only", nl.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = nl.lib()
    for n in declared_functions():
        assert hasattr(lib, n)


@pytest.mark.parametrize("kw,status", [
    (dict(dim=4, n=8, delta=0.1), "NL_EINVAL"),
    (dict(dim=2, n=0, delta=0.1), "NL_EINVAL"),
    (dict(dim=2, n=8, delta=-0.1), "NL_EINVAL"),
    (dict(dim=2, n=8, delta=float("nan")), "NL_EINVAL"),
    (dict(dim=2, n=8, delta=0.1, family=1, K=7), "NL_EINVAL"),
    (dict(dim=2, n=8, delta=0.1, coef=2), "NL_EINVAL"),                     # XY without a
    (dict(dim=2, n=8, delta=0.1, coef=2, a=-np.ones(64)), "NL_EINVAL"),     # a <= 0
    (dict(dim=3, n=8, delta=0.1, family=2, K=1), "NL_EUNSUPPORTED"),        # 3-D PD: K = 0
    (dict(dim=3, n=12, delta=0.1, family=2), "NL_EUNSUPPORTED"),            # 3-D PD: n = 2^L
    (dict(dim=2, n=8, delta=0.1, family=1, K=1, symmetric=True, self_term=1),
     "NL_EUNSUPPORTED"),                                                   # paper self term
    (dict(dim=2, n=8, delta=0.1, family=1, coef=1, a=np.ones(64), symmetric=True),
     "NL_EUNSUPPORTED"),
    (dict(dim=2, n=8, delta=0.1, alpha=4.5), "NL_EINVAL"),
    (dict(dim=2, n=8, delta=0.1, family=3, K=4), "NL_EINVAL"),              # kappa: K 0..3
    (dict(dim=2, n=8, delta=0.1, family=3, symmetric=True), "NL_EUNSUPPORTED"),
    (dict(dim=2, n=8, delta=0.1, family=4), "NL_EINVAL"),                   # unknown family
])
def test_plan_validation_errors(nl, kw, status):
    with pytest.raises(nl.NlError) as ei:
        nl.nl_plan_create(**kw)
    assert str(ei.value).startswith(status), str(ei.value)
    assert nl.nl_last_error()


def test_null_plan_calls_are_rejected(nl):
    import ctypes
    lib = nl.lib()
    assert lib.nl_apply(None, None, None, 1, 0, None) == nl.NL_EINVAL
    assert lib.nl_apply_fast(None, None, None, 1, 0, None) == nl.NL_EINVAL
    assert lib.nl_plan_destroy(None) == nl.NL_OK
    info = nl.nl_plan_info()
    assert lib.nl_get_plan_info(None, ctypes.byref(info)) == nl.NL_EINVAL
