"""GPU parity of the 3-D fast-path peridynamic operator (nl_apply_fast on a 3-D NL_PD_BOND
plan, K = 0: the bond tensor xi xi^T / delta_i^3 over the leaf set of Algorithm 1) against
the FP64 oracle's plain sum over the leaf set."""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_08375_gb300 import binding as nl
from paper_1905_08375_gb300 import synth
from helpers import boundary_idx, rel_l2, sample_idx

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def fields(n, seed, nrhs):
    rng = np.random.default_rng(seed)
    c = synth.voronoi_phase(rng, 3, n, cells=16)
    u = np.stack([np.stack([synth.gaussian_field(rng, 3, n).reshape(-1) for _ in range(3)])
                  for _ in range(nrhs)])
    return c, u


def run_fast(plan, u):
    ut = torch.tensor(np.asarray(u), dtype=torch.float32, device=DEV).contiguous()
    out = torch.full_like(ut, float("nan"))
    nl.nl_apply_fast(plan, ut, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("n,rho,variable", [(2, 1.1, False), (4, 1.2, False), (8, 1.6, False),
                                            (16, 2.5, True), (32, 4.0, False), (32, 3.0, True)])
def test_fast_pd3_matches_oracle(n, rho, variable):
    L = int(np.log2(n))
    c, u = fields(n, seed=n + 3, nrhs=2)
    delta = np.full(n ** 3, rho / n)
    if variable:
        delta = delta * np.random.default_rng(n).uniform(0.6, 1.3, n ** 3)
    plan = nl.nl_plan_create(3, n, delta, family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN, a=c)
    got = run_fast(plan, u)
    ref = oracle.fast_pd_leafset(u, 3, L, delta, c)
    assert rel_l2(got, ref) <= 2e-6, rel_l2(got, ref)
    assert np.array_equal(got, run_fast(plan, u))           # exact integer sums: repeatable
    plan.close()


def test_fast_pd3_128_sampled():
    n, L = 128, 7
    c, u = fields(n, seed=5, nrhs=1)
    delta = np.full(n ** 3, 4.0 / n)
    plan = nl.nl_plan_create(3, n, delta, family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN, a=c)
    got = run_fast(plan, u[0]).reshape(3, -1)
    idx = np.concatenate([sample_idx(n ** 3, 1500, seed=2), boundary_idx(3, n, 5, 500, seed=3)])
    ref = oracle.fast_pd_leafset(u[0], 3, L, delta, c, idx=idx)
    assert rel_l2(got[:, idx], ref) <= 2e-6
    plan.close()


def test_fast_pd3_rejections():
    n = 16
    c, u = fields(n, seed=1, nrhs=1)
    plan = nl.nl_plan_create(3, n, 2.0 / n, family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN, a=c)
    u64 = torch.zeros(3 * n ** 3, dtype=torch.float64, device=DEV)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):        # FP32 data only
        nl.nl_apply_fast(plan, u64, torch.empty_like(u64))
    u32 = torch.zeros(3 * n ** 3, dtype=torch.float32, device=DEV)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):        # no 3-D direct operator
        nl.nl_apply(plan, u32, torch.empty_like(u32))
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):        # nor CG on it
        nl.nl_cg_solve(plan, u64, torch.empty_like(u64), rtol=1e-8, maxit=10)
    plan.close()
    for kw in (dict(K=1), dict(n=12), dict(n=512)):
        m = kw.pop("n", n)
        with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
            nl.nl_plan_create(3, m, 2.0 / m, family=nl.NL_PD_BOND, **kw)
