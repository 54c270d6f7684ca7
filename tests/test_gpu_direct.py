"""GPU parity of the direct apply (nl_apply) against the FP64 oracle, through the C-ABI.

Tolerances (rel-L2 over the compared nodes): FP64 <= 1e-12, FP32 <= 2e-6."""
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


def run_direct(plan, u, dtype, nrhs=None):
    ut = torch.tensor(np.asarray(u), dtype=dtype, device=DEV).contiguous()
    out = torch.full_like(ut, float("nan"))
    nl.nl_apply(plan, ut, out, nrhs=nrhs)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_config1_1d_full(dtype):
    f = synth.diffusion_1d(n=4096, delta=0.05, seed=0)
    plan = nl.nl_plan_create(1, 4096, 0.05, family=nl.NL_POWER, alpha=0.0)
    ref = oracle.direct_scalar(f["u"], 1, 4096, 0.05, alpha=0.0)
    assert rel_l2(run_direct(plan, f["u"], dtype), ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("coef", [nl.NL_COEF_NONE, nl.NL_COEF_X, nl.NL_COEF_XY])
def test_2d_heterogeneous_ragged(dtype, coef):
    n = 203                                   # ragged against the 32x8 block in x and y
    f = synth.heterogeneous_2d(n=n, seed=1, nrhs=2)
    a = f["a"] if coef != nl.NL_COEF_NONE else None
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POWER, alpha=1.5, coef=coef, a=a)
    ref = oracle.direct_scalar(f["u"], 2, n, f["delta"], alpha=1.5, coef=coef, a=a)
    got = run_direct(plan, f["u"], dtype)
    assert rel_l2(got, ref) <= TOL[dtype]
    assert not np.isnan(got).any()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_2d_polynomial_kernel(dtype, K):
    n = 96
    f = synth.heterogeneous_2d(n=n, seed=2)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POLY, alpha=1.5, K=K,
                             coef=nl.NL_COEF_XY, a=f["a"])
    ref = oracle.direct_scalar(f["u"][0], 2, n, f["delta"], family=oracle.POLY, alpha=1.5, K=K,
                               coef=oracle.COEF_XY, a=f["a"])
    assert rel_l2(run_direct(plan, f["u"][0], dtype), ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_2d_symmetric_variant(dtype):
    n = 77
    f = synth.heterogeneous_2d(n=n, seed=3)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=f["a"], symmetric=True)
    ref = oracle.direct_scalar(f["u"][0], 2, n, f["delta"], alpha=1.5, coef=oracle.COEF_XY,
                               a=f["a"], symmetric=True)
    assert rel_l2(run_direct(plan, f["u"][0], dtype), ref) <= TOL[dtype]


@pytest.mark.parametrize("n,nrhs", [(203, 2), (181, 1), (77, 8), (256, 5)])
def test_2d_symmetric_paired_columns_fp32(n, nrhs):
    """Grids large enough for the paired-column symmetrised kernel, ragged tails, several
    right-hand sides (pairs of them take the two-right-hand-side kernel, an odd last one the
    single kernel): against the FP64 oracle, and each right-hand side bit for bit its own
    single apply where one right-hand side also takes the paired-column path (n^2 >= 32768;
    smaller single applies split each ball over a group of lanes instead)."""
    f = synth.heterogeneous_2d(n=n, seed=n, nrhs=nrhs)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=f["a"], symmetric=True)
    ref = oracle.direct_scalar(f["u"], 2, n, f["delta"], alpha=1.5, coef=oracle.COEF_XY,
                               a=f["a"], symmetric=True)
    got = run_direct(plan, f["u"], torch.float32)
    assert rel_l2(got, ref) <= 2e-6
    if nrhs > 1 and n * n >= 32 * 1024:
        for r in range(nrhs):
            one = run_direct(plan, f["u"][r], torch.float32)
            assert np.array_equal(one.reshape(-1), got[r].reshape(-1)), r


@pytest.mark.parametrize("n,rmin,rspan", [(190, 2.0, 19.0), (184, 9.0, 0.0), (200, 19.0, 1.5)])
def test_2d_symmetric_paired_columns_horizon_mixes(n, rmin, rspan):
    """Horizons from 2 to 21 cells (most rows need masks), a constant horizon (no masks) and
    radii above 16 cells (the 24-cell halo); FP32 against the FP64 oracle and each right-hand
    side of a batch equal bit for bit to its own apply (n^2 > 32768 nodes, so that one
    right-hand side takes the same kernel as three)."""
    f = synth.heterogeneous_2d(n=n, seed=n + 7, nrhs=3, rmin=rmin, rspan=rspan)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=f["a"], symmetric=True)
    ref = oracle.direct_scalar(f["u"], 2, n, f["delta"], alpha=1.5, coef=oracle.COEF_XY,
                               a=f["a"], symmetric=True)
    got = run_direct(plan, f["u"], torch.float32)
    assert rel_l2(got, ref) <= 2e-6
    for r in range(3):
        one = run_direct(plan, f["u"][r], torch.float32)
        assert np.array_equal(one.reshape(-1), got[r].reshape(-1))


def test_2d_symmetric_fp32_operator_is_symmetric():
    """<v, L u> = <u, L v> for the divergence-form operator, up to FP32 rounding."""
    n = 140
    f = synth.heterogeneous_2d(n=n, seed=5, nrhs=2)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=f["a"], symmetric=True)
    Lw = run_direct(plan, f["u"], torch.float32)
    u, v = f["u"][0], f["u"][1]
    a, b = float(np.dot(v, Lw[0])), float(np.dot(u, Lw[1]))
    assert abs(a - b) <= 1e-5 * np.linalg.norm(Lw) * np.linalg.norm(u), (a, b)


def test_2d_symmetric_512_sampled():
    n = 512
    f = synth.heterogeneous_2d(n=n, seed=1)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=f["a"], symmetric=True)
    got = run_direct(plan, f["u"][0], torch.float32)
    idx = np.concatenate([sample_idx(n * n, 1500, seed=3), boundary_idx(2, n, 18, 500, seed=4)])
    ref = oracle.direct_scalar(f["u"][0], 2, n, f["delta"], alpha=1.5, coef=oracle.COEF_XY,
                               a=f["a"], symmetric=True, idx=idx)
    assert rel_l2(got[idx], ref) <= 2e-6


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_3d_multi_rhs_ragged(dtype):
    n = 29
    f = synth.diffusion_3d(n=n, seed=4, nrhs=3, radius_cells=4)
    plan = nl.nl_plan_create(3, n, f["delta"], family=nl.NL_POWER, alpha=1.0,
                             coef=nl.NL_COEF_XY, a=f["a"])
    ref = oracle.direct_scalar(f["u"], 3, n, f["delta"], alpha=1.0, coef=oracle.COEF_XY, a=f["a"])
    assert rel_l2(run_direct(plan, f["u"], dtype), ref) <= TOL[dtype]


@pytest.mark.parametrize("d,n,delta", [(1, 1, 0.3), (2, 1, 0.7), (2, 3, 0.2), (1, 17, 0.01),
                                       (2, 9, 5.0), (3, 5, 0.5), (1, 64, 3.0)])
def test_degenerate_sizes(d, n, delta):
    """Single node, empty ball (delta < h), ball larger than the domain."""
    rng = np.random.default_rng(d * 100 + n)
    u = rng.standard_normal(n ** d)
    a = np.exp(0.2 * rng.standard_normal(n ** d))
    plan = nl.nl_plan_create(d, n, delta, family=nl.NL_POWER, alpha=0.5, coef=nl.NL_COEF_XY, a=a)
    ref = oracle.direct_scalar(u, d, n, delta, alpha=0.5, coef=oracle.COEF_XY, a=a)
    got = run_direct(plan, u, torch.float64)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(ref).max()))


def test_global_memory_variant_large_ball():
    """A horizon whose halo tile would not fit in shared memory takes the unstaged kernel."""
    n = 128
    rng = np.random.default_rng(9)
    u = rng.standard_normal(n * n)
    plan = nl.nl_plan_create(2, n, 0.5, family=nl.NL_POLY, K=0, normalize=False)
    ref = oracle.direct_scalar(u, 2, n, 0.5, family=oracle.POLY, K=0, normalize=False)
    assert rel_l2(run_direct(plan, u, torch.float64), ref) <= 1e-12


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_config2_full_size_sampled(dtype):
    """1024^2, delta = h (4 + 12 s), a lognormal, POWER 1.5: the launch the bench times;
    compared on sampled interior and boundary nodes."""
    n = 1024
    f = synth.heterogeneous_2d(n=n, seed=0)
    plan = nl.nl_plan_create(2, n, f["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=f["a"])
    got = run_direct(plan, f["u"][0], dtype)
    idx = np.concatenate([sample_idx(n * n, 1500, seed=1), boundary_idx(2, n, 17, 500, seed=2)])
    ref = oracle.direct_scalar(f["u"][0], 2, n, f["delta"], alpha=1.5, coef=oracle.COEF_XY,
                               a=f["a"], idx=idx)
    assert rel_l2(got[idx], ref) <= TOL[dtype]
    assert np.isfinite(got).all()


def test_config5_3d_full_size_sampled():
    n = 256
    f = synth.diffusion_3d(n=n, seed=0, nrhs=8, radius_cells=4)
    plan = nl.nl_plan_create(3, n, f["delta"], family=nl.NL_POWER, alpha=1.0,
                             coef=nl.NL_COEF_XY, a=f["a"])
    got = run_direct(plan, f["u"], torch.float32).reshape(8, -1)
    idx = np.concatenate([sample_idx(n ** 3, 400, seed=3), boundary_idx(3, n, 5, 200, seed=4)])
    ref = oracle.direct_scalar(f["u"], 3, n, f["delta"], alpha=1.0, coef=oracle.COEF_XY,
                               a=f["a"], idx=idx)
    assert rel_l2(got[:, idx], ref) <= 2e-6
