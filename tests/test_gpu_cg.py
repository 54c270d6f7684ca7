"""GPU conjugate gradients (nl_cg_solve) on -L x = f, checked by the FP64 oracle residual."""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_08375_gb300 import binding as nl
from paper_1905_08375_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def oracle_residual_scalar(x, f, n, fld):
    Lx = oracle.direct_scalar(x, 2, n, fld["delta"], alpha=1.5, coef=oracle.COEF_XY, a=fld["a"],
                              symmetric=True)
    return np.linalg.norm(f + Lx, axis=-1) / np.linalg.norm(f, axis=-1)


@pytest.mark.parametrize("n,nrhs", [(64, 1), (96, 3)])
def test_scalar_symmetric_jacobi(n, nrhs):
    fld = synth.heterogeneous_2d(n=n, seed=7)
    f = synth.cg_rhs(n, seed=8, count=nrhs)
    plan = nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=fld["a"], symmetric=True)
    ft = torch.tensor(f, dtype=torch.float64, device=DEV)
    xt = torch.empty_like(ft)
    st = nl.nl_cg_solve(plan, ft, xt, rtol=1e-8, maxit=20000)
    assert st["converged"] and st["rel_residual"] <= 1e-8, st
    res = oracle_residual_scalar(xt.cpu().numpy(), f, n, fld)
    assert np.all(res <= 1.01e-8), res
    # same number of iterations as the oracle's FP64 Jacobi-PCG, up to the restarts
    _, it_o, _ = oracle.cg(f[0], 2, n, fld["delta"], alpha=1.5, coef=oracle.COEF_XY, a=fld["a"],
                           rtol=1e-8)
    assert st["iterations"] <= 1.5 * it_o + 32, (st["iterations"], it_o)


def test_unpreconditioned_and_not_converged():
    n = 48
    fld = synth.heterogeneous_2d(n=n, seed=9)
    f = synth.cg_rhs(n, seed=10)
    plan = nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=fld["a"], symmetric=True)
    ft = torch.tensor(f, dtype=torch.float64, device=DEV)
    xt = torch.empty_like(ft)
    st = nl.nl_cg_solve(plan, ft, xt, rtol=1e-8, maxit=20000, precond=nl.NL_PRECOND_NONE)
    assert st["converged"]
    assert oracle_residual_scalar(xt.cpu().numpy(), f, n, fld)[0] <= 1.01e-8
    st2 = nl.nl_cg_solve(plan, ft, xt, rtol=1e-12, maxit=16)
    assert not st2["converged"] and st2["status"] == nl.NL_ENOTCONV


def test_solves_in_sequence_match_solves_on_fresh_plans():
    # the Jacobi factors are formed once per workspace and kept: a sequence of solves that
    # changes the preconditioner and the number of right-hand sides (so that the workspace
    # layout moves) gives the iterations and solutions of solves on fresh plans
    n = 64
    fld = synth.heterogeneous_2d(n=n, seed=12)
    f = synth.cg_rhs(n, seed=13, count=3)

    def make():
        return nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POWER, alpha=1.5,
                                 coef=nl.NL_COEF_XY, a=fld["a"], symmetric=True)

    shared = make()
    for nrhs, pc in [(3, nl.NL_PRECOND_JACOBI), (3, nl.NL_PRECOND_NONE), (1, nl.NL_PRECOND_JACOBI),
                     (3, nl.NL_PRECOND_JACOBI), (1, nl.NL_PRECOND_NONE)]:
        ft = torch.tensor(f[:nrhs], dtype=torch.float64, device=DEV)
        xs = torch.empty_like(ft)
        xf = torch.empty_like(ft)
        st_s = nl.nl_cg_solve(shared, ft, xs, rtol=1e-8, maxit=20000, precond=pc)
        fresh = make()
        st_f = nl.nl_cg_solve(fresh, ft, xf, rtol=1e-8, maxit=20000, precond=pc)
        fresh.close()
        assert st_s["converged"] and st_f["converged"]
        assert st_s["iterations"] == st_f["iterations"], (nrhs, pc, st_s, st_f)
        assert torch.equal(xs, xf), (nrhs, pc)
    shared.close()


def test_non_symmetric_plan_rejected():
    n = 32
    fld = synth.heterogeneous_2d(n=n, seed=11)
    plan = nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POWER, alpha=1.5)
    ft = torch.ones(n * n, dtype=torch.float64, device=DEV)
    with pytest.raises(nl.NlError, match="NL_EUNSUPPORTED"):
        nl.nl_cg_solve(plan, ft, torch.empty_like(ft))


def test_peridynamics_two_phase():
    n = 40
    fld = synth.pd_2d(n=n, seed=12, radius_cells=6)
    rng = np.random.default_rng(13)
    f = rng.standard_normal((2, 2, n * n))
    plan = nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_PD_BOND, coef=nl.NL_COEF_MEAN,
                             a=fld["c"])
    ft = torch.tensor(f, dtype=torch.float64, device=DEV)
    xt = torch.empty_like(ft)
    st = nl.nl_cg_solve(plan, ft, xt, rtol=1e-8, maxit=20000)
    assert st["converged"], st
    x = xt.cpu().numpy()
    Lx = oracle.pd_direct(x, 2, n, fld["delta"], fld["c"])
    res = np.linalg.norm((f + Lx).reshape(2, -1), axis=1) / np.linalg.norm(f.reshape(2, -1), axis=1)
    assert np.all(res <= 1.01e-8), res


@pytest.mark.parametrize("n", [256, 512])
def test_config4_sizes(n):
    """Learned-preconditioner workload sizes, Jacobi-CG to 1e-8 with the FP64 oracle residual."""
    fld = synth.heterogeneous_2d(n=n, seed=0)
    f = synth.cg_rhs(n, seed=1)
    plan = nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=fld["a"], symmetric=True)
    ft = torch.tensor(f, dtype=torch.float64, device=DEV)
    xt = torch.empty_like(ft)
    st = nl.nl_cg_solve(plan, ft, xt, rtol=1e-8, maxit=50000)
    assert st["converged"] and st["rel_residual"] <= 1e-8, st
    assert oracle_residual_scalar(xt.cpu().numpy(), f, n, fld)[0] <= 1.01e-8


def test_wait_limit_runs_out_and_the_plan_recovers():
    # the host gives up on the first chunk (a wait limit far below one chunk's run time) and
    # returns NL_ETIMEOUT; the chunk's kernels finish on their own, and after a device
    # synchronisation the same plan solves normally with the default limit
    n = 256
    fld = synth.heterogeneous_2d(n=n, seed=17)
    f = synth.cg_rhs(n, seed=18, count=4)
    plan = nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=fld["a"], symmetric=True)
    ft = torch.tensor(f, dtype=torch.float64, device=DEV)
    xt = torch.empty_like(ft)
    try:
        nl.nl_set_wait_limit(1e-6)
        with pytest.raises(nl.NlError) as ei:
            nl.nl_cg_solve(plan, ft, xt, rtol=1e-8, maxit=20000)
        assert str(ei.value).startswith("NL_ETIMEOUT"), str(ei.value)
    finally:
        torch.cuda.synchronize()
        nl.nl_set_wait_limit(600.0)
    st = nl.nl_cg_solve(plan, ft, xt, rtol=1e-8, maxit=20000)
    assert st["converged"] and st["rel_residual"] <= 1e-8, st
    res = oracle_residual_scalar(xt.cpu().numpy(), f, n, fld)
    assert np.all(res <= 1.01e-8), res
    plan.close()
