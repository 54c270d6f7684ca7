"""GPU parity of the FP32-pair symmetric operator (nl_apply with NL_F64_PAIRS).

The operator of Eq. (2.1)-(2.2) in divergence form, FP64 data, arithmetic on hi + lo pairs of
FP32 numbers with error-free sums and products.  Compared element by element with the FP64
oracle (the point-in-ball double loop) and with the library's own FP64 apply: the pairs carry
48 significant bits, so the result is within ~1e-13 of the FP64 one relative to the size of
the terms (the bounds below leave a factor of ten).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_08375_gb300 import binding as nl
from paper_1905_08375_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _plan(n, fld, coef):
    return nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POWER, alpha=1.5, coef=coef,
                             a=fld["a"] if coef != nl.NL_COEF_NONE else None, symmetric=True)


def _term_scale(u, n, fld, coef):
    """An upper bound of sum_j |w_ij c_ij| |u_j - u_i| over the nodes: 2 max |u| times the
    largest diagonal entry of -L, taken from the oracle on unit vectors at sampled nodes."""
    rng = np.random.default_rng(3)
    idx = rng.choice(n * n, size=min(64, n * n), replace=False)
    e = np.zeros(n * n)
    diag = 0.0
    for i in idx:
        e[:] = 0.0
        e[i] = 1.0
        Le = oracle.direct_scalar(e, 2, n, fld["delta"], alpha=1.5, coef=coef,
                                  a=fld["a"] if coef != oracle.COEF_NONE else None,
                                  symmetric=True, idx=np.array([i]))
        diag = max(diag, -float(np.ravel(Le)[0]))
    return 2.0 * float(np.abs(u).max()) * diag


@pytest.mark.parametrize("n,nrhs,coef", [(64, 1, nl.NL_COEF_XY), (100, 3, nl.NL_COEF_XY),
                                         (96, 2, nl.NL_COEF_NONE), (33, 1, nl.NL_COEF_XY)])
def test_pairs_match_fp64_oracle(n, nrhs, coef):
    fld = synth.heterogeneous_2d(n=n, seed=31 + n, nrhs=nrhs)
    u = fld["u"].reshape(nrhs, -1)
    plan = _plan(n, fld, coef)
    ut = torch.tensor(u, dtype=torch.float64, device=DEV)
    lp = torch.full_like(ut, float("nan"))
    l64 = torch.empty_like(ut)
    nl.nl_apply(plan, ut, lp, pairs=True)
    nl.nl_apply(plan, ut, l64)
    torch.cuda.synchronize()
    ref = oracle.direct_scalar(u, 2, n, fld["delta"], alpha=1.5, coef=coef,
                               a=fld["a"] if coef != nl.NL_COEF_NONE else None, symmetric=True)
    got = lp.cpu().numpy()
    assert np.all(np.isfinite(got))
    scale = _term_scale(u, n, fld, coef)
    err_o = np.abs(got - ref).max()
    err_64 = np.abs(got - l64.cpu().numpy()).max()
    assert err_o <= 1e-12 * scale, (err_o, scale)
    assert err_64 <= 1e-12 * scale, (err_64, scale)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 1e-11, rel
    plan.close()


def test_pairs_offset_field_and_smooth_field():
    # a large constant offset (the differences u_j - u_i come from the low words) and a smooth
    # field (the terms cancel: |L u| is far below the sum of |terms|)
    n = 64
    fld = synth.heterogeneous_2d(n=n, seed=5)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    smooth = np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    plan = _plan(n, fld, nl.NL_COEF_XY)
    for u in (100.0 + fld["u"].reshape(-1), smooth.reshape(-1)):
        ut = torch.tensor(u, dtype=torch.float64, device=DEV)
        lp = torch.empty_like(ut)
        nl.nl_apply(plan, ut, lp, pairs=True)
        torch.cuda.synchronize()
        ref = oracle.direct_scalar(u, 2, n, fld["delta"], alpha=1.5, coef=oracle.COEF_XY,
                                   a=fld["a"], symmetric=True)
        scale = _term_scale(u, n, fld, oracle.COEF_XY)
        assert np.abs(lp.cpu().numpy() - ref).max() <= 1e-12 * scale
    plan.close()


def test_pairs_large_horizon_and_constant_field():
    # Rmax between 16 and 24 (the next tile halo), and L 1 = 0 up to the pair rounding
    n = 128
    rng = np.random.default_rng(9)
    delta = (10.0 + 10.0 * rng.random(n * n)) / n
    fld = dict(delta=delta, a=np.exp(0.3 * rng.standard_normal(n * n)))
    plan = _plan(n, fld, nl.NL_COEF_XY)
    assert nl.nl_get_plan_info(plan)["max_radius"] > 16
    u = rng.standard_normal(n * n)
    ut = torch.tensor(u, dtype=torch.float64, device=DEV)
    lp = torch.empty_like(ut)
    l64 = torch.empty_like(ut)
    nl.nl_apply(plan, ut, lp, pairs=True)
    nl.nl_apply(plan, ut, l64)
    torch.cuda.synchronize()
    rel = float(torch.linalg.norm(lp - l64) / torch.linalg.norm(l64))
    assert rel <= 1e-11, rel
    one = torch.ones(n * n, dtype=torch.float64, device=DEV)
    nl.nl_apply(plan, one, lp, pairs=True)
    nl.nl_apply(plan, one, l64)
    torch.cuda.synchronize()
    # interior nodes: exactly the FP64 result (every difference is zero); near the boundary
    # only the exterior term u_i ext_i remains, computed in FP64 on both paths
    assert torch.equal(lp, l64)
    plan.close()


def test_pairs_rejected_where_not_built():
    n = 32
    fld = synth.heterogeneous_2d(n=n, seed=2)
    u = torch.zeros(n * n, dtype=torch.float64, device=DEV)
    one_sided = nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POWER, alpha=1.5)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_apply(one_sided, u, u.clone(), pairs=True)
    sym1 = nl.nl_plan_create(1, 256, np.full(256, 0.02), family=nl.NL_POWER, alpha=1.5,
                             symmetric=True)
    u1 = torch.zeros(256, dtype=torch.float64, device=DEV)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_apply(sym1, u1, u1.clone(), pairs=True)
    with pytest.raises(ValueError, match="FP64"):
        nl.nl_apply(one_sided, u.float(), u.float().clone(), pairs=True)
    one_sided.close()
    sym1.close()
