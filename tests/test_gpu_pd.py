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
