"""GPU parity of the fast algorithm (nl_apply_fast, Sec. 3) against the FP64 oracle.

The fast result is exact with respect to its own quadrature (the leaf cells that meet
the ball), so it is gated against the oracle's leaf-set sum O2 (itself pinned to the
literal tree algorithm O1) at the direct path's tolerances."""
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


def run_fast(plan, u, dtype):
    ut = torch.tensor(np.asarray(u), dtype=dtype, device=DEV).contiguous()
    out = torch.full_like(ut, float("nan"))
    nl.nl_apply_fast(plan, ut, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_example2_1d_variable_horizon(dtype, K):
    n = 512
    f = synth.example2_1d(n=n, delta0=0.25, seed=0)
    plan = nl.nl_plan_create(1, n, f["delta"], family=nl.NL_POLY, alpha=1.0, K=K)
    ref = oracle.fast_leafset(f["u"], 1, 9, f["delta"], K=K, alpha=1.0)
    assert rel_l2(run_fast(plan, f["u"], dtype), ref) <= TOL[dtype]


@pytest.mark.parametrize("K", [0, 1, 2, 3])
@pytest.mark.parametrize("coef,self_mode", [(nl.NL_COEF_NONE, nl.NL_SELF_PAPER),
                                            (nl.NL_COEF_X, nl.NL_SELF_DISCRETE),
                                            (nl.NL_COEF_XY, nl.NL_SELF_DISCRETE)])
def test_2d_all_orders(K, coef, self_mode):
    n, L = 64, 6
    f = synth.heterogeneous_2d(n=n, seed=5, nrhs=2)
    a = None if coef == nl.NL_COEF_NONE else f["a"]
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5, K=K, coef=coef,
                             a=a, self_term=self_mode)
    ref = oracle.fast_leafset(f["u"], 2, L, f["delta"], K=K, alpha=1.5, coef=coef, a=a,
                              self_mode=self_mode)
    ut = torch.tensor(f["u"], dtype=torch.float64, device=DEV)
    out = torch.empty_like(ut)
    nl.nl_apply_fast(plan, ut, out)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), ref) <= 1e-12


def test_2d_literal_tree_agrees():
    """Also against O1 (Algorithm 1 + pyramid) directly."""
    n, L = 32, 5
    rng = np.random.default_rng(11)
    delta = rng.uniform(1.5, 9.0, size=n * n) / n
    u = rng.standard_normal(n * n)
    plan = nl.nl_plan_create(2, n, delta, family=nl.NL_POLY, alpha=1.0, K=2)
    ref = oracle.fast_tree(u, 2, L, delta, K=2, alpha=1.0)
    assert rel_l2(run_fast(plan, u, torch.float64), ref) <= 1e-12


@pytest.mark.parametrize("n", [1, 2, 4, 16])
def test_3d_k0_and_tiny(n):
    L = int(np.log2(n))
    rng = np.random.default_rng(n)
    delta = rng.uniform(0.6, 3.5, size=n ** 3) / n
    a = np.exp(0.3 * rng.standard_normal(n ** 3))
    u = rng.standard_normal(n ** 3)
    plan = nl.nl_plan_create(3, n, delta, family=nl.NL_POLY, alpha=1.0, K=0,
                             coef=nl.NL_COEF_XY, a=a)
    ref = oracle.fast_leafset(u, 3, L, delta, K=0, alpha=1.0, coef=oracle.COEF_XY, a=a)
    got = run_fast(plan, u, torch.float64)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_example1_2d_full():
    """Example 1 of Sec. 4: 128^2, delta = 1/2, K = 0, C = 1, continuous self term."""
    n, L = 128, 7
    rng = np.random.default_rng(12)
    u = rng.standard_normal(n * n)
    plan = nl.nl_plan_create(2, n, 0.5, family=nl.NL_POLY, K=0, normalize=False,
                             self_term=nl.NL_SELF_PAPER)
    ref = oracle.fast_tree(u, 2, L, 0.5, K=0, normalize=False, self_mode=oracle.SELF_PAPER)
    assert rel_l2(run_fast(plan, u, torch.float64), ref) <= 1e-12


def test_example2_1d_4096_k3():
    n, L = 4096, 12
    f = synth.example2_1d(n=n, delta0=0.25, seed=1)
    plan = nl.nl_plan_create(1, n, f["delta"], family=nl.NL_POLY, alpha=1.0, K=3,
                             normalize=False)
    ref = oracle.fast_tree(f["u"], 1, L, f["delta"], K=3, alpha=1.0, normalize=False)
    assert rel_l2(run_fast(plan, f["u"], torch.float64), ref) <= 1e-12


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_config2_full_size_sampled(dtype):
    n, L = 1024, 10
    f = synth.heterogeneous_2d(n=n, seed=0)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5, K=0,
                             coef=nl.NL_COEF_XY, a=f["a"])
    got = run_fast(plan, f["u"][0], dtype)
    idx = np.concatenate([sample_idx(n * n, 1500, seed=5), boundary_idx(2, n, 18, 500, seed=6)])
    ref = oracle.fast_leafset(f["u"][0], 2, L, f["delta"], K=0, alpha=1.5, coef=oracle.COEF_XY,
                              a=f["a"], idx=idx)
    assert rel_l2(got[idx], ref) <= TOL[dtype]
    assert np.isfinite(got).all()


def test_unsupported_requests():
    rng = np.random.default_rng(0)
    u = torch.zeros(24 * 24, dtype=torch.float64, device=DEV)
    out = torch.empty_like(u)
    p1 = nl.nl_plan_create(2, 24, 0.1, family=nl.NL_POLY, K=0)       # n not a power of 2
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_apply_fast(p1, u, out)
    p2 = nl.nl_plan_create(2, 16, 0.1, family=nl.NL_POWER, alpha=1.0)
    u2 = torch.zeros(256, dtype=torch.float64, device=DEV)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_apply_fast(p2, u2, torch.empty_like(u2))


@pytest.mark.parametrize("d,n", [(1, 2048), (2, 128), (2, 256), (3, 32)])
def test_integer_routes_bitwise_equal_and_match_oracle(d, n):
    """FP32, K = 0: the row-prefix, leaf-row and panel-by-panel fixed-point routes add the
    same integers, so their outputs are bitwise equal; all match the FP64 oracle."""
    L = int(np.log2(n))
    rng = np.random.default_rng(40 + d)
    N = n ** d
    rho = rng.uniform(1.5, 0.25 * n if d < 3 else 3.5, size=N)
    a = np.exp(0.3 * rng.standard_normal(N))
    u = rng.standard_normal(N)
    outs = []
    for variant in (nl.NL_FAST_ROWPREFIX, nl.NL_FAST_PANELS, nl.NL_FAST_FP64_PANELS,
                    nl.NL_FAST_LEAFROWS):
        plan = nl.nl_plan_create(d, n, rho / n, family=nl.NL_POLY, alpha=1.0, K=0,
                                 coef=nl.NL_COEF_XY, a=a, fast_variant=variant)
        outs.append(run_fast(plan, u, torch.float32))
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[3], outs[1])
    ref = oracle.fast_leafset(u, d, L, rho / n, K=0, alpha=1.0, coef=oracle.COEF_XY, a=a)
    for o in outs:
        assert rel_l2(o, ref) <= 2e-6


@pytest.mark.parametrize("d,n", [(1, 2), (1, 8192), (2, 2), (2, 8), (2, 32), (2, 1024),
                                 (2, 4096), (3, 2), (3, 8), (3, 64)])
def test_fused_step2_bitwise_equal_to_panels(d, n):
    """The fused Step 2 build (one launch for every level; for 2-D 4096^2 the coarse levels
    come from per-level launches) gives the row-prefix gather the same integers as the
    panel-by-panel route, at band and level edge cases; sampled against the oracle."""
    L = int(np.log2(n))
    rng = np.random.default_rng(7 * n + d)
    N = n ** d
    rho = rng.uniform(0.6, max(0.7, min(6.0, n / 4)), size=N)
    a = np.exp(0.3 * rng.standard_normal(N))
    u = rng.standard_normal(N)
    outs = []
    for variant in (nl.NL_FAST_ROWPREFIX, nl.NL_FAST_PANELS, nl.NL_FAST_LEAFROWS):
        plan = nl.nl_plan_create(d, n, rho / n, family=nl.NL_POLY, alpha=1.0, K=0,
                                 coef=nl.NL_COEF_XY, a=a, fast_variant=variant)
        outs.append(run_fast(plan, u, torch.float32))
        plan.close()
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[2], outs[1])
    idx = sample_idx(N, 400, seed=d) if N > 4096 else np.arange(N)
    ref = oracle.fast_leafset(u, d, L, rho / n, K=0, alpha=1.0, coef=oracle.COEF_XY, a=a,
                              idx=idx)
    assert rel_l2(outs[0][idx], ref) <= 2e-6


@pytest.mark.parametrize("d,n,nrhs", [(2, 64, 3), (2, 128, 9), (3, 16, 5), (1, 1024, 2),
                                      (2, 256, 2), (3, 128, 3)])
def test_multi_rhs_leafrows_bitwise_equal_to_single(d, n, nrhs):
    """Several FP32 right-hand sides share one gather launch (per-row run bounds computed once);
    each output is bitwise the one-right-hand-side apply, and matches the oracle."""
    rng = np.random.default_rng(100 * d + n)
    N = n ** d
    rho = rng.uniform(0.6, max(0.7, min(5.0, n / 4)), size=N)
    a = np.exp(0.3 * rng.standard_normal(N))
    u = rng.standard_normal((nrhs, N))
    plan = nl.nl_plan_create(d, n, rho / n, family=nl.NL_POLY, alpha=1.0, K=0,
                             coef=nl.NL_COEF_XY, a=a)
    many = run_fast(plan, u, torch.float32)
    for r in range(nrhs):
        np.testing.assert_array_equal(many[r], run_fast(plan, u[r], torch.float32))
    L = int(np.log2(n))
    idx = sample_idx(N, 3000, seed=n) if N > 100000 else np.arange(N)
    ref = oracle.fast_leafset(u[-1], d, L, rho / n, K=0, alpha=1.0, coef=oracle.COEF_XY, a=a,
                              idx=idx)
    assert rel_l2(many[-1][idx], ref) <= 2e-6


@pytest.mark.parametrize("n,rho,nrhs", [(32, 4.0, 1), (32, 2.3, 3), (64, 4.0, 8),
                                          (64, 5.7, 2), (32, 1.2, 1)])
def test_3d_constant_horizon_staged_rows_bitwise(n, rho, nrhs):
    """3-D constant horizon (the staged leaf-row gather: one tile of prefix rows per block,
    every node the same run pattern): bitwise equal to the row-prefix and panel routes, for one
    and several right-hand sides, and against the FP64 oracle."""
    L = int(np.log2(n))
    N = n ** 3
    rng = np.random.default_rng(int(10 * rho) + n + nrhs)
    a = np.exp(0.3 * rng.standard_normal(N))
    u = rng.standard_normal((nrhs, N))
    outs = {}
    for name, variant in (("leaf", nl.NL_FAST_LEAFROWS), ("prefix", nl.NL_FAST_ROWPREFIX),
                          ("panels", nl.NL_FAST_PANELS)):
        plan = nl.nl_plan_create(3, n, rho / n, family=nl.NL_POLY, alpha=1.0, K=0,
                                 coef=nl.NL_COEF_XY, a=a, fast_variant=variant)
        outs[name] = run_fast(plan, u, torch.float32)
        if name == "leaf" and nrhs > 1:
            for r in (0, nrhs - 1):
                np.testing.assert_array_equal(outs[name][r], run_fast(plan, u[r], torch.float32))
        plan.close()
    np.testing.assert_array_equal(outs["leaf"], outs["prefix"])
    np.testing.assert_array_equal(outs["leaf"], outs["panels"])
    idx = sample_idx(N, 2000, seed=n)
    ref = oracle.fast_leafset(u[-1], 3, L, rho / n, K=0, alpha=1.0, coef=oracle.COEF_XY, a=a,
                              idx=idx)
    assert rel_l2(outs["leaf"].reshape(nrhs, N)[-1][idx], ref) <= 2e-6


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("K", [1, 2, 3])
@pytest.mark.parametrize("coef", [nl.NL_COEF_NONE, nl.NL_COEF_XY])
def test_3d_polynomial_orders(dtype, K, coef):
    """3-D with K > 0: moments of degree <= 2K in three variables (C(2K+3, 3) per panel)."""
    n, L = 16, 4
    rng = np.random.default_rng(30 + K)
    s = synth.fourier_modes_field(rng, 3, n, modes=4, kmax=2).reshape(-1)
    delta = (1.3 + 2.4 * s) / n
    a = np.exp(0.3 * rng.standard_normal(n ** 3)) if coef == nl.NL_COEF_XY else None
    u = rng.standard_normal((2, n ** 3))
    plan = nl.nl_plan_create(3, n, delta, family=nl.NL_POLY, alpha=1.0, K=K, coef=coef, a=a)
    ref = oracle.fast_leafset(u, 3, L, delta, K=K, alpha=1.0, coef=coef, a=a)
    assert rel_l2(run_fast(plan, u, dtype), ref) <= TOL[dtype]
    if dtype == torch.float64 and coef == nl.NL_COEF_NONE:
        idx = sample_idx(n ** 3, 300, seed=K)
        tree = oracle.fast_tree(u[0], 3, L, delta, K=K, alpha=1.0, idx=idx)
        assert rel_l2(run_fast(plan, u[0], dtype)[idx], tree) <= 1e-12
    plan.close()


def test_3d_polynomial_large_ball_and_boundary():
    """A ball larger than Omega (a root-level panel) and a constant horizon, K = 2."""
    n, L = 8, 3
    rng = np.random.default_rng(41)
    u = rng.standard_normal(n ** 3)
    for delta in (0.3, 1.9):
        plan = nl.nl_plan_create(3, n, delta, family=nl.NL_POLY, alpha=1.0, K=2)
        ref = oracle.fast_tree(u, 3, L, delta, K=2, alpha=1.0)
        assert rel_l2(run_fast(plan, u, torch.float64), ref) <= 1e-12
        plan.close()


# ---------------------------------------------------------------------------
# K >= 1, FP32 data, the default (leaf-row) variant: exact integer run sums of o_x^{2j} q from
# prefix sums of k^e q; the panel variant keeps the FP64 moment pyramid
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("K", [1, 2, 3])
@pytest.mark.parametrize("d,n", [(1, 512), (2, 64), (2, 128)])
@pytest.mark.parametrize("coef,self_mode", [(nl.NL_COEF_NONE, nl.NL_SELF_PAPER),
                                            (nl.NL_COEF_XY, nl.NL_SELF_DISCRETE)])
def test_integer_leafrows_k_matches_oracle_and_moments(K, d, n, coef, self_mode):
    L = int(np.log2(n))
    if d == 1:
        f = synth.example2_1d(n=n, delta0=0.25, seed=K)
        u = np.stack([f["u"], np.sin(np.arange(n) * 0.37)])
        a = np.exp(0.3 * np.cos(np.arange(n) * 0.11)) if coef == nl.NL_COEF_XY else None
    else:
        f = synth.heterogeneous_2d(n=n, seed=5 + K, nrhs=2)
        u = f["u"]
        a = f["a"] if coef == nl.NL_COEF_XY else None
    kw = dict(family=nl.NL_POLY, alpha=1.5, K=K, coef=coef, a=a, self_term=self_mode)
    plan = nl.nl_plan_create(d, n, f["delta"], **kw)
    mom = nl.nl_plan_create(d, n, f["delta"], fast_variant=nl.NL_FAST_PANELS, **kw)
    ref = oracle.fast_leafset(u, d, L, f["delta"], K=K, alpha=1.5, coef=coef, a=a,
                              self_mode=self_mode)
    got = run_fast(plan, u, torch.float32)
    assert rel_l2(got, ref) <= 2e-6, rel_l2(got, ref)
    assert rel_l2(run_fast(mom, u, torch.float32), ref) <= 2e-6
    assert np.array_equal(got, run_fast(plan, u, torch.float32))
    plan.close()
    mom.close()


def test_integer_leafrows_k2_full_size_sampled():
    n = 1024
    f = synth.heterogeneous_2d(n=n, seed=9)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5, K=2,
                             coef=nl.NL_COEF_XY, a=f["a"])
    got = run_fast(plan, f["u"][0], torch.float32)
    idx = sample_idx(n * n, 2000, seed=4, extra=(n - 1, n * (n - 1), n * n // 2 + 7))
    ref = oracle.fast_leafset(f["u"][0], 2, 10, f["delta"], K=2, alpha=1.5, coef=oracle.COEF_XY,
                              a=f["a"], idx=idx)
    assert rel_l2(got[idx], ref) <= 2e-6
    plan.close()
