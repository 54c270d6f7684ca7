"""GPU parity of the kappa part of the splitting of Sec. 3 (NL_KAPPA, the direct sum with the
profile kappa(s) = s^-alpha - p^{2K}(s)) against the FP64 oracle, through the C-ABI, and the
splitting identity L^gamma = L^kappa + L^P computed entirely on the GPU.

Tolerances (rel-L2 over the compared nodes): FP64 <= 1e-12, FP32 <= 2e-6."""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_08375_gb300 import binding as nl
from paper_1905_08375_gb300 import synth
from helpers import rel_l2, sample_idx

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
@pytest.mark.parametrize("K", [0, 1, 2, 3])
@pytest.mark.parametrize("n", [77, 203])
def test_2d_variable_horizon_ragged(dtype, K, n):
    # ragged against every block shape; 77^2 nodes take the small-grid kernel (a lane group
    # per node), 203^2 the staged-tile kernel
    f = synth.heterogeneous_2d(n=n, seed=11, nrhs=2)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_KAPPA, alpha=1.5, K=K,
                             coef=nl.NL_COEF_XY, a=f["a"])
    ref = oracle.direct_scalar(f["u"], 2, n, f["delta"], family=oracle.KAPPA, alpha=1.5, K=K,
                               coef=oracle.COEF_XY, a=f["a"])
    got = run(plan, f["u"], dtype)
    assert not np.isnan(got).any()
    assert rel_l2(got, ref) <= TOL[dtype]
    plan.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("d,n,delta", [(1, 4096, 0.05), (1, 300, 0.2), (3, 21, 3.5 / 21),
                                     (3, 35, 3.5 / 35), (1, 40000, 7.5 / 40000)])
def test_other_dimensions(dtype, d, n, delta):
    rng = np.random.default_rng(d * 1000 + n)
    u = rng.standard_normal(n ** d)
    plan = nl.nl_plan_create(d, n, delta, family=nl.NL_KAPPA, alpha=1.0, K=1)
    ref = oracle.direct_scalar(u, d, n, delta, family=oracle.KAPPA, alpha=1.0, K=1)
    assert rel_l2(run(plan, u, dtype), ref) <= TOL[dtype]
    plan.close()


@pytest.mark.parametrize("K", [0, 2])
def test_splitting_identity_on_the_gpu(K):
    # Sec. 3: with one sigma, nl_apply on NL_POWER equals NL_KAPPA + NL_POLY (FP64, one
    # quadrature set: the open ball of each node)
    n = 128
    f = synth.heterogeneous_2d(n=n, seed=5)
    kw = dict(alpha=1.5, K=K, coef=nl.NL_COEF_XY, a=f["a"])
    plans = {fam: nl.nl_plan_create(2, n, f["delta"], family=fam, **kw)
             for fam in (nl.NL_POWER, nl.NL_KAPPA, nl.NL_POLY)}
    out = {fam: run(p, f["u"][0], torch.float64) for fam, p in plans.items()}
    g = out[nl.NL_POWER]
    assert rel_l2(out[nl.NL_KAPPA] + out[nl.NL_POLY], g) <= 1e-12
    for p in plans.values():
        p.close()


def test_full_size_config2_sampled_fp32():
    n = 1024
    f = synth.heterogeneous_2d(n=n, seed=0)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_KAPPA, alpha=1.5, K=1,
                             coef=nl.NL_COEF_XY, a=f["a"])
    got = run(plan, f["u"][0], torch.float32)
    idx = sample_idx(n * n, 3000, seed=4)
    ref = oracle.direct_scalar(f["u"][0], 2, n, f["delta"], family=oracle.KAPPA, alpha=1.5,
                               K=1, coef=oracle.COEF_XY, a=f["a"], idx=idx)
    assert rel_l2(got[idx], ref) <= 2e-6
    plan.close()


def test_fast_apply_rejects_kappa_plans():
    plan = nl.nl_plan_create(2, 64, 0.1, family=nl.NL_KAPPA, alpha=1.0, K=1)
    u = torch.zeros(64 * 64, dtype=torch.float64, device=DEV)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_apply_fast(plan, u, u.clone())
    plan.close()
