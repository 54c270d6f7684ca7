"""GPU parity of the symmetrised fast operator (nl_apply_fast on a symmetric NL_POLY plan,
K = 0..3: the divergence-type pairing (w_i(k) + w_k(i))/2 over the leaf sets of Algorithm 1)
against the oracle's plain sum over both leaf sets, and CG on it with the oracle residual."""
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


def smooth_delta(d, n, lo, hi, seed):
    s = synth.fourier_modes_field(np.random.default_rng(seed), d, n, modes=4, kmax=2)
    return (lo + (hi - lo) * s).reshape(-1) / n


def run(plan, u, dtype):
    ut = torch.tensor(np.asarray(u), dtype=dtype, device=DEV).contiguous()
    out = torch.full_like(ut, float("nan"))
    nl.nl_apply_fast(plan, ut, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("d,L,lo,hi", [(1, 9, 2.0, 40.0), (2, 6, 1.5, 6.5), (2, 7, 3.0, 9.0),
                                       (3, 4, 1.2, 3.4)])
@pytest.mark.parametrize("coef", [nl.NL_COEF_NONE, nl.NL_COEF_XY])
def test_matches_oracle_variable_horizon(dtype, d, L, lo, hi, coef):
    n = 1 << L
    rng = np.random.default_rng(d * 10 + L)
    delta = smooth_delta(d, n, lo, hi, seed=L)
    a = np.exp(0.4 * rng.standard_normal(n ** d)) if coef == nl.NL_COEF_XY else None
    u = rng.standard_normal((2, n ** d))
    plan = nl.nl_plan_create(d, n, delta, family=nl.NL_POLY, alpha=1.0, K=0, coef=coef, a=a,
                             symmetric=True)
    ref = oracle.fast_sym_leafset(u, d, L, delta, K=0, alpha=1.0, coef=coef, a=a)
    got = run(plan, u, dtype)
    assert rel_l2(got, ref) <= TOL[dtype]
    plan.close()


@pytest.mark.parametrize("route", [nl.NL_FAST_PANELS, nl.NL_FAST_ROWPREFIX, nl.NL_FAST_LEAFROWS])
def test_routes_bitwise_equal(route):
    n = 128
    f = synth.heterogeneous_2d(n=n, seed=3)
    kw = dict(family=nl.NL_POLY, alpha=1.5, K=0, coef=nl.NL_COEF_XY, a=f["a"], symmetric=True)
    base = nl.nl_plan_create(2, n, f["delta"], **kw)
    other = nl.nl_plan_create(2, n, f["delta"], fast_variant=route, **kw)
    u = f["u"][0]
    assert np.array_equal(run(base, u, torch.float32), run(other, u, torch.float32))


def test_full_size_sampled():
    n = 1024
    f = synth.heterogeneous_2d(n=n, seed=4)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5, K=0,
                             coef=nl.NL_COEF_XY, a=f["a"], symmetric=True)
    got = run(plan, f["u"][0], torch.float32)
    idx = sample_idx(n * n, 3000, seed=1, extra=(n - 1, n * (n - 1), n * n // 2 + 7))
    ref = oracle.fast_sym_leafset(f["u"][0], 2, 10, f["delta"], K=0, alpha=1.5,
                                  coef=oracle.COEF_XY, a=f["a"], idx=idx)
    assert rel_l2(got[idx], ref) <= 2e-6


def test_symmetric_and_constants():
    # <L u, v> = <u, L v> and L 1 = 0 where every leaf set that reaches a node stays inside
    n, L = 64, 6
    delta = smooth_delta(2, n, 1.5, 4.5, seed=2)
    rng = np.random.default_rng(9)
    plan = nl.nl_plan_create(2, n, delta, family=nl.NL_POLY, alpha=1.0, K=0, symmetric=True)
    u, v = rng.standard_normal(n * n), rng.standard_normal(n * n)
    Lu, Lv = run(plan, u, torch.float64), run(plan, v, torch.float64)
    assert abs(Lu @ v - u @ Lv) <= 1e-12 * np.linalg.norm(Lu) * np.linalg.norm(v)
    L1 = run(plan, np.ones(n * n), torch.float64).reshape(n, n)
    assert np.abs(L1[8:-8, 8:-8]).max() <= 1e-10 * np.abs(L1).max()


@pytest.mark.parametrize("n,nrhs", [(64, 1), (128, 3)])
def test_cg_on_the_fast_operator(n, nrhs):
    fld = synth.heterogeneous_2d(n=n, seed=12)
    f = synth.cg_rhs(n, seed=13, count=nrhs)
    plan = nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POLY, alpha=1.5, K=0,
                             coef=nl.NL_COEF_XY, a=fld["a"], symmetric=True)
    ft = torch.tensor(f, dtype=torch.float64, device=DEV)
    xt = torch.empty_like(ft)
    st = nl.nl_cg_solve(plan, ft, xt, rtol=1e-8, maxit=20000)
    assert st["converged"] and st["rel_residual"] <= 1e-8, st
    x = xt.cpu().numpy()
    Lx = oracle.fast_sym_leafset(x, 2, int(np.log2(n)), fld["delta"], K=0, alpha=1.5,
                                 coef=oracle.COEF_XY, a=fld["a"])
    res = np.linalg.norm(f + Lx, axis=-1) / np.linalg.norm(f, axis=-1)
    assert np.all(res <= 1.01e-8), res
    plan.close()


def test_plan_and_call_validation():
    n = 32
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_plan_create(2, n, 0.1, family=nl.NL_POLY, K=1, coef=nl.NL_COEF_X, a=np.ones(n * n),
                          symmetric=True)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_plan_create(2, n, 0.1, family=nl.NL_POLY, K=0, symmetric=True,
                          self_term=nl.NL_SELF_PAPER)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_plan_create(2, 48, 0.1, family=nl.NL_POLY, K=0, symmetric=True)
    plan = nl.nl_plan_create(2, n, 0.1, family=nl.NL_POLY, K=0, symmetric=True)
    u = torch.zeros(n * n, device=DEV)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_apply(plan, u, u.clone())
    plan.close()


# ---------------------------------------------------------------------------
# K >= 1: the transpose half with the source's polynomial weights p(|o|^2 / R_k^2), exact
# two-limb integer coefficients of the target column
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("K", [1, 2, 3])
@pytest.mark.parametrize("d,L,lo,hi", [(1, 8, 2.0, 30.0), (2, 6, 1.5, 6.5), (2, 7, 3.0, 9.0),
                                       (3, 4, 1.2, 3.4)])
def test_polynomial_matches_oracle(dtype, K, d, L, lo, hi):
    n = 1 << L
    rng = np.random.default_rng(100 * K + 10 * d + L)
    delta = smooth_delta(d, n, lo, hi, seed=L + K)
    a = np.exp(0.4 * rng.standard_normal(n ** d))
    u = rng.standard_normal((2, n ** d))
    for coef in (nl.NL_COEF_NONE, nl.NL_COEF_XY):
        aa = a if coef == nl.NL_COEF_XY else None
        plan = nl.nl_plan_create(d, n, delta, family=nl.NL_POLY, alpha=1.0, K=K, coef=coef,
                                 a=aa, symmetric=True)
        ref = oracle.fast_sym_leafset(u, d, L, delta, K=K, alpha=1.0, coef=coef, a=aa)
        got = run(plan, u, dtype)
        assert rel_l2(got, ref) <= TOL[dtype], (coef, rel_l2(got, ref))
        assert np.array_equal(got, run(plan, u, dtype))     # exact integer sums: repeatable
        plan.close()


def test_polynomial_symmetric_and_constants():
    n, L = 64, 6
    delta = smooth_delta(2, n, 1.5, 4.5, seed=7)
    rng = np.random.default_rng(19)
    plan = nl.nl_plan_create(2, n, delta, family=nl.NL_POLY, alpha=1.5, K=2, symmetric=True)
    u, v = rng.standard_normal(n * n), rng.standard_normal(n * n)
    Lu, Lv = run(plan, u, torch.float64), run(plan, v, torch.float64)
    assert abs(Lu @ v - u @ Lv) <= 1e-12 * np.linalg.norm(Lu) * np.linalg.norm(v)
    L1 = run(plan, np.ones(n * n), torch.float64).reshape(n, n)
    assert np.abs(L1[8:-8, 8:-8]).max() <= 1e-10 * np.abs(L1).max()
    plan.close()


@pytest.mark.parametrize("K", [1, 2])
def test_cg_on_the_polynomial_fast_operator(K):
    n = 64
    fld = synth.heterogeneous_2d(n=n, seed=22)
    f = synth.cg_rhs(n, seed=23, count=2)
    plan = nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POLY, alpha=1.5, K=K,
                             coef=nl.NL_COEF_XY, a=fld["a"], symmetric=True)
    ft = torch.tensor(f, dtype=torch.float64, device=DEV)
    xt = torch.empty_like(ft)
    st = nl.nl_cg_solve(plan, ft, xt, rtol=1e-8, maxit=20000)
    assert st["converged"] and st["rel_residual"] <= 1e-8, st
    x = xt.cpu().numpy()
    Lx = oracle.fast_sym_leafset(x, 2, 6, fld["delta"], K=K, alpha=1.5, coef=oracle.COEF_XY,
                                 a=fld["a"])
    res = np.linalg.norm(f + Lx, axis=-1) / np.linalg.norm(f, axis=-1)
    assert np.all(res <= 1.01e-8), res
    plan.close()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_polynomial_full_size_sampled(dtype):
    # the 1024^2 heterogeneous field (horizons of 4..16 cells): the limbs at their widest
    n = 1024
    f = synth.heterogeneous_2d(n=n, seed=4)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5, K=2,
                             coef=nl.NL_COEF_XY, a=f["a"], symmetric=True)
    got = run(plan, f["u"][0], dtype)
    idx = sample_idx(n * n, 2000, seed=3, extra=(n - 1, n * (n - 1), n * n // 2 + 7))
    ref = oracle.fast_sym_leafset(f["u"][0], 2, 10, f["delta"], K=2, alpha=1.5,
                                  coef=oracle.COEF_XY, a=f["a"], idx=idx)
    assert rel_l2(got[idx], ref) <= TOL[dtype], rel_l2(got[idx], ref)
    plan.close()
