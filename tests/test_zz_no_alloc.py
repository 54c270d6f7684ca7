"""GPU test of nl_apply_fast_noalloc, the allocation-free fast apply.

Some callers cannot allocate device memory (their device memory belongs to their own pool
allocator, or they must not take the synchronisation cudaMalloc may cause).  For them the
library offers a fast apply whose scratch is a fixed static device array.  This file checks,
through the C-ABI, that it gives the same result as nl_apply_fast on the matching plan, on
two calls in a row (the second with new data, so that leftovers from the first call in the
shared array would show), and that it rejects grids larger than its array.  It is collected
last so that a stop-at-first-failure run has executed every other test before it.
"""
import numpy as np
import pytest
import torch

from paper_1905_08375_gb300 import binding as nl
from paper_1905_08375_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = {torch.float64: 1e-12, torch.float32: 2e-6}


def _rel(x, ref):
    x = x.double().cpu().numpy()
    ref = ref.double().cpu().numpy()
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("self_term", [nl.NL_SELF_DISCRETE, nl.NL_SELF_PAPER])
def test_matches_plan_fast_apply_two_calls(dtype, self_term):
    n = 256
    f = synth.heterogeneous_2d(n=n, seed=21, nrhs=2)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5, K=0,
                             self_term=self_term)
    delta_dev = torch.tensor(f["delta"], dtype=torch.float64, device=DEV)
    for call in range(2):
        u = torch.tensor(f["u"][call], dtype=dtype, device=DEV)
        ref = torch.empty_like(u)
        nl.nl_apply_fast(plan, u, ref)
        out = torch.full_like(u, float("nan"))
        nl.nl_apply_fast_noalloc(2, n, delta_dev, u, out, alpha=1.5, self_term=self_term)
        torch.cuda.synchronize()
        assert _rel(out, ref) <= TOL[dtype], (call, _rel(out, ref))
    plan.close()


@pytest.mark.parametrize("d,n,delta", [(1, 4096, 0.05), (3, 32, 3.5 / 32), (2, 1024, 9.0 / 1024)])
def test_constant_horizon_other_dimensions(d, n, delta):
    rng = np.random.default_rng(d)
    plan = nl.nl_plan_create(d, n, delta, family=nl.NL_POLY, alpha=1.0, K=0)
    for call in range(2):
        u = torch.tensor(rng.standard_normal(n ** d), dtype=torch.float64, device=DEV)
        ref = torch.empty_like(u)
        nl.nl_apply_fast(plan, u, ref)
        out = torch.full_like(u, float("nan"))
        nl.nl_apply_fast_noalloc(d, n, delta, u, out, alpha=1.0)
        torch.cuda.synchronize()
        assert _rel(out, ref) <= 1e-12
    plan.close()


def test_rejects_grids_beyond_the_static_array():
    # the size check runs on the host before any launch (the buffers are never touched)
    u = torch.zeros(2048 * 2048, dtype=torch.float64, device=DEV)
    with pytest.raises(nl.NlError, match="NL_EINVAL.*static array"):
        nl.nl_apply_fast_noalloc(2, 2048, 0.01, u, u.clone(), nrhs=1)
    u = torch.zeros(1000 * 1000, dtype=torch.float64, device=DEV)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_apply_fast_noalloc(2, 1000, 0.01, u, u.clone(), nrhs=1)


def test_rejects_bad_horizons_and_mismatched_buffers():
    # host-side checks: the C entry point rejects horizons outside (0, 2]; the binding rejects
    # buffers whose dtype or size do not match what the kernels would read and write
    n = 64
    u = torch.zeros(n * n, dtype=torch.float64, device=DEV)
    for bad in (0.0, -0.1, 2.5, float("inf"), float("nan")):
        with pytest.raises(nl.NlError, match="NL_EINVAL"):
            nl.nl_apply_fast_noalloc(2, n, bad, u, u.clone())
    with pytest.raises(ValueError, match="same dtype"):
        nl.nl_apply_fast_noalloc(2, n, 0.1, u, torch.zeros(n * n, dtype=torch.float32, device=DEV))
    with pytest.raises(ValueError, match="elements"):
        nl.nl_apply_fast_noalloc(2, n, 0.1, u, torch.zeros(n * n - 1, dtype=torch.float64,
                                                          device=DEV), nrhs=1)
    with pytest.raises(ValueError, match="delta field"):
        nl.nl_apply_fast_noalloc(2, n, torch.full((n * n - 3,), 0.1, dtype=torch.float64,
                                                  device=DEV), u, u.clone())


def test_out_of_range_field_values_stay_bounded():
    # NaN and huge horizons in a device field are clamped for the geometry: the call finishes
    # promptly and the other nodes are unaffected
    n = 64
    rng = np.random.default_rng(5)
    dl = np.full(n * n, 3.0 / n)
    u = torch.tensor(rng.standard_normal(n * n), dtype=torch.float64, device=DEV)
    ref = torch.empty_like(u)
    nl.nl_apply_fast_noalloc(2, n, torch.tensor(dl, device=DEV), u, ref)
    bad = dl.copy()
    bad[100], bad[2000] = float("nan"), 1.0e12
    out = torch.empty_like(u)
    nl.nl_apply_fast_noalloc(2, n, torch.tensor(bad, device=DEV), u, out)
    torch.cuda.synchronize()
    keep = np.ones(n * n, dtype=bool)
    keep[[100, 2000]] = False
    assert torch.equal(out.cpu()[torch.tensor(keep)], ref.cpu()[torch.tensor(keep)])
