"""GPU parity of the batched apply (uneven 2-D instances in one persistent launch) and of the
batched CG, against the FP64 oracle."""
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


def scalar_instances(sizes, seed=0):
    out = []
    for k, n in enumerate(sizes):
        f = synth.heterogeneous_2d(n=n, seed=seed + k)
        out.append((n, f["delta"], f["a"], f["u"][0]))
    return out


def pd_instances(sizes, seed=0):
    out = []
    for k, n in enumerate(sizes):
        f = synth.pd_2d(n=n, seed=seed + k, radius_cells=8)
        out.append((n, f["delta"], f["c"], f["u"][0].reshape(-1)))
    return out


def run_batch(b, fields, dtype):
    u = torch.tensor(np.concatenate(fields), dtype=dtype, device=DEV)
    out = torch.full_like(u, float("nan"))
    nl.nl_batch_apply(b, u, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", [nl.NL_TILE_32x4, nl.NL_TILE_32x8, nl.NL_TILE_32x16])
@pytest.mark.parametrize("symmetric", [False, True])
def test_scalar_uneven(dtype, shape, symmetric):
    inst = scalar_instances([40, 70, 33, 96, 57], seed=3)
    b = nl.nl_batch_create([(n, d, a) for n, d, a, _ in inst], family=nl.NL_POWER, alpha=1.5,
                           coef=nl.NL_COEF_XY, symmetric=symmetric, tile_shape=shape)
    assert b.tile_shape == shape
    assert list(np.diff(b.offsets)) == [n * n for n, *_ in inst]
    got = run_batch(b, [u for *_, u in inst], dtype)
    for k, (n, d, a, u) in enumerate(inst):
        ref = oracle.direct_scalar(u[None], 2, n, d, alpha=1.5, coef=oracle.COEF_XY, a=a,
                                   symmetric=symmetric)[0]
        seg = got[b.offsets[k]:b.offsets[k + 1]]
        assert rel_l2(seg, ref) <= TOL[dtype], (k, n)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_pd_uneven_autotuned(dtype):
    inst = pd_instances([24, 61, 45, 80], seed=11)
    b = nl.nl_batch_create([(n, d, c) for n, d, c, _ in inst], family=nl.NL_PD_BOND,
                           coef=nl.NL_COEF_MEAN, tile_shape=nl.NL_TILE_AUTO)
    assert b.tile_shape in (0, 1, 2)
    assert list(np.diff(b.offsets)) == [2 * n * n for n, *_ in inst]
    got = run_batch(b, [u for *_, u in inst], dtype)
    for k, (n, d, c, u) in enumerate(inst):
        ref = oracle.pd_direct(u.reshape(1, 2, -1), 2, n, d, c).reshape(-1)
        seg = got[b.offsets[k]:b.offsets[k + 1]]
        assert rel_l2(seg, ref) <= TOL[dtype], (k, n)


def test_batch_matches_plans_fp64():
    """Every instance of a batch gives the same FP64 values as its own plan's generic
    staged kernel up to summation order (checked here at 1e-14)."""
    inst = scalar_instances([64, 31], seed=5)
    b = nl.nl_batch_create([(n, d, a) for n, d, a, _ in inst], alpha=1.5, coef=nl.NL_COEF_XY,
                           tile_shape=nl.NL_TILE_32x8)
    got = run_batch(b, [u for *_, u in inst], torch.float64)
    for k, (n, d, a, u) in enumerate(inst):
        p = nl.nl_plan_create(2, n, d, alpha=1.5, coef=nl.NL_COEF_XY, a=a)
        ut = torch.tensor(u, dtype=torch.float64, device=DEV)
        lo = torch.empty_like(ut)
        nl.nl_apply(p, ut, lo)
        torch.cuda.synchronize()
        assert rel_l2(got[b.offsets[k]:b.offsets[k + 1]], lo.cpu().numpy()) <= 1e-14


def test_pd_64_instances_full_sizes_sampled():
    """64 peridynamic instances, 128^2 .. 512^2, FP32, one launch; sampled against the oracle."""
    sizes = synth.pd_batch_sizes(64, 128, 512)
    inst = pd_instances(sizes, seed=0)
    b = nl.nl_batch_create([(n, d, c) for n, d, c, _ in inst], family=nl.NL_PD_BOND,
                           coef=nl.NL_COEF_MEAN)
    got = run_batch(b, [u for *_, u in inst], torch.float32)
    for k in (0, 1, 31, 62, 63):
        n, d, c, u = inst[k]
        idx = sample_idx(n * n, 300, seed=k)
        ref = oracle.pd_direct(u.reshape(1, 2, -1), 2, n, d, c, idx=idx)
        seg = got[b.offsets[k]:b.offsets[k + 1]].reshape(1, 2, -1)
        assert rel_l2(seg[:, :, idx], ref) <= 2e-6, (k, n)


def oracle_residual_pd(n, d, c, f, x):
    Lx = oracle.pd_direct(x.reshape(1, 2, -1), 2, n, d, c).reshape(-1)
    return np.linalg.norm(f + Lx) / np.linalg.norm(f)


def test_batch_cg_pd_uneven():
    sizes = [32, 48, 40, 64, 57]
    inst = pd_instances(sizes, seed=21)
    b = nl.nl_batch_create([(n, d, c) for n, d, c, _ in inst], family=nl.NL_PD_BOND,
                           coef=nl.NL_COEF_MEAN)
    f = torch.tensor(np.concatenate([u for *_, u in inst]), dtype=torch.float64, device=DEV)
    x = torch.zeros_like(f)
    st = nl.nl_batch_cg_solve(b, f, x, rtol=1e-8, maxit=20000)
    assert st["converged"] and st["rel_residual"] <= 1e-8
    xs = x.cpu().numpy()
    fs = f.cpu().numpy()
    for k, (n, d, c, _) in enumerate(inst):
        sl = slice(b.offsets[k], b.offsets[k + 1])
        assert oracle_residual_pd(n, d, c, fs[sl], xs[sl]) <= 1.5e-8, (k, n)


def test_batch_cg_equals_per_instance_cg():
    """A batch of one instance and that instance's own plan run the same CG: same iterations."""
    (n, d, c, u), = pd_instances([72], seed=4)
    b = nl.nl_batch_create([(n, d, c)], family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN)
    f = torch.tensor(u, dtype=torch.float64, device=DEV)
    x1 = torch.zeros_like(f)
    s1 = nl.nl_batch_cg_solve(b, f, x1, rtol=1e-8)
    p = nl.nl_plan_create(2, n, d, family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN, a=c)
    x2 = torch.zeros_like(f)
    s2 = nl.nl_cg_solve(p, f, x2, rtol=1e-8)
    assert s1["converged"] and s2["converged"]
    assert abs(s1["iterations"] - s2["iterations"]) <= 2
    assert rel_l2(x1.cpu().numpy(), x2.cpu().numpy()) <= 1e-6


def test_batch_rejects_unsupported_family():
    with pytest.raises(nl.NlError):
        nl.nl_batch_create([(32, 0.1, None)], family=nl.NL_POLY)
