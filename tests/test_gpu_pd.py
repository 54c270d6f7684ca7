"""GPU parity of the peridynamic direct apply (NL_PD_BOND) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_08375_gb300 import binding as nl
from paper_1905_08375_gb300 import synth
from helpers import boundary_idx, rel_l2, sample_idx

pytestmark = pytest.mark.gpu
TOL = {torch.float64: 1e-12, torch.float32: 2e-6}
DEV = "cuda:0"


def run(plan, u, dtype):
    ut = torch.tensor(np.asarray(u), dtype=dtype, device=DEV).contiguous()
    out = torch.full_like(ut, float("nan"))
    nl.nl_apply(plan, ut, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n", [70, 128])
def test_two_phase_ragged(dtype, n):
    f = synth.pd_2d(n=n, seed=n, radius_cells=8, nrhs=2)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN,
                             a=f["c"])
    ref = oracle.pd_direct(f["u"], 2, n, f["delta"], f["c"])
    assert rel_l2(run(plan, f["u"], dtype), ref) <= TOL[dtype]


def test_full_size_512_sampled():
    n = 512
    f = synth.pd_2d(n=n, seed=0, radius_cells=8)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN,
                             a=f["c"])
    got = run(plan, f["u"], torch.float32).reshape(1, 2, -1)
    idx = np.concatenate([sample_idx(n * n, 1500, seed=7), boundary_idx(2, n, 9, 500, seed=8)])
    ref = oracle.pd_direct(f["u"], 2, n, f["delta"], f["c"], idx=idx)
    assert rel_l2(got[:, :, idx], ref) <= 2e-6


# ---------------------------------------------------------------------------
# fast-path peridynamics of degree 0 (nl_apply_fast on an NL_PD_BOND plan)
# ---------------------------------------------------------------------------
def run_fast(plan, u):
    ut = torch.tensor(np.asarray(u), dtype=torch.float32, device=DEV).contiguous()
    out = torch.full_like(ut, float("nan"))
    nl.nl_apply_fast(plan, ut, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("n,rho,variable", [(64, 8.0, False), (32, 3.0, True), (128, 8.0, True),
                                            (8, 2.2, False), (2, 1.4, False)])
def test_fast_pd_matches_oracle(n, rho, variable):
    L = int(np.log2(n))
    f = synth.pd_2d(n=n, seed=n + 1, radius_cells=rho, nrhs=2)
    delta = f["delta"]
    if variable:
        delta = delta * np.random.default_rng(n).uniform(0.6, 1.3, n * n)
    plan = nl.nl_plan_create(2, n, delta, family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN,
                             a=f["c"])
    got = run_fast(plan, f["u"])
    ref = oracle.fast_pd_leafset(f["u"], 2, L, delta, f["c"])
    assert rel_l2(got, ref) <= 2e-6, rel_l2(got, ref)


def test_fast_pd_512_sampled_and_rejections():
    n, L = 512, 9
    f = synth.pd_2d(n=n, seed=0, radius_cells=8)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN,
                             a=f["c"])
    got = run_fast(plan, f["u"][0]).reshape(2, -1)
    idx = np.concatenate([sample_idx(n * n, 1500, seed=9), boundary_idx(2, n, 10, 500, seed=10)])
    ref = oracle.fast_pd_leafset(f["u"][0], 2, L, f["delta"], f["c"], idx=idx)
    assert rel_l2(got[:, idx], ref) <= 2e-6
    u64 = torch.zeros(2 * n * n, dtype=torch.float64, device=DEV)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_apply_fast(plan, u64, torch.empty_like(u64))
    p2 = nl.nl_plan_create(2, 48, 0.1, family=nl.NL_PD_BOND)
    u2 = torch.zeros(2 * 48 * 48, dtype=torch.float32, device=DEV)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_apply_fast(p2, u2, torch.empty_like(u2))


@pytest.mark.parametrize("K", [1, 2])
@pytest.mark.parametrize("n,rho,variable", [(64, 8.0, False), (32, 3.0, True), (128, 6.0, True),
                                            (8, 2.2, False)])
def test_fast_pd_polynomial_micromodulus(K, n, rho, variable):
    """The polynomial micromodulus p^{2K} (matched to s^-3 at the horizon) over the leaf set,
    from exact 64-bit moments of o_x up to 2K + 2, against the oracle."""
    L = int(np.log2(n))
    f = synth.pd_2d(n=n, seed=n + 7, radius_cells=rho, nrhs=2)
    delta = f["delta"]
    if variable:
        delta = delta * np.random.default_rng(n + K).uniform(0.6, 1.3, n * n)
    plan = nl.nl_plan_create(2, n, delta, family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN,
                             a=f["c"], K=K)
    got = run_fast(plan, f["u"])
    ref = oracle.fast_pd_leafset(f["u"], 2, L, delta, f["c"], K=K)
    assert rel_l2(got, ref) <= 2e-6, rel_l2(got, ref)


def test_fast_pd_polynomial_512_sampled():
    n, L, K = 512, 9, 2
    f = synth.pd_2d(n=n, seed=3, radius_cells=8)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN,
                             a=f["c"], K=K)
    got = run_fast(plan, f["u"][0]).reshape(2, -1)
    idx = np.concatenate([sample_idx(n * n, 1500, seed=4), boundary_idx(2, n, 10, 500, seed=5)])
    ref = oracle.fast_pd_leafset(f["u"][0], 2, L, f["delta"], f["c"], K=K, idx=idx)
    assert rel_l2(got[:, idx], ref) <= 2e-6
    p3 = nl.nl_plan_create(2, 64, 0.1, family=nl.NL_PD_BOND, K=3)
    u3 = torch.zeros(2 * 64 * 64, dtype=torch.float32, device=DEV)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_apply_fast(p3, u3, torch.empty_like(u3))
