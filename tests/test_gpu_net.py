"""GPU parity of the learned-preconditioner kernels against the numpy oracle, and
flexible CG with the network (the FP64 oracle residual decides convergence)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import convnet
from paper_1905_08375_gb300 import binding as nl
from paper_1905_08375_gb300 import precond, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _w(seed, scale=0.15):
    return (np.random.default_rng(seed).standard_normal(convnet.NPARAM) * scale).astype(np.float32)


@pytest.mark.parametrize("H,W", [(16, 16), (37, 50)])
def test_forward_matches_oracle(H, W):
    w = _w(1)
    x = np.random.default_rng(2).standard_normal((3, H, W)).astype(np.float32)
    net = nl.nl_net_create(w)
    xt = torch.tensor(x, device=DEV)
    ot = torch.full_like(xt, float("nan"))
    nl.nl_net_forward(net, xt, ot)
    torch.cuda.synchronize()
    ref, _ = convnet.forward(w, x.astype(np.float64))
    err = np.abs(ot.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 2e-5, err


def test_train_step_gradient_and_adam_match_oracle():
    n, S, B, margin, lr = 40, 32, 5, 3, 1e-3
    rng = np.random.default_rng(3)
    w = _w(4)
    x = rng.standard_normal((2, n, n)).astype(np.float32)
    e = rng.standard_normal((2, n, n)).astype(np.float32)
    crops = np.array([[0, 0, 0], [1, 8, 3], [0, 5, 8], [1, 0, 8], [0, 8, 8]], dtype=np.int32)
    net = nl.nl_net_create(w)
    loss = nl.nl_net_train_step(net, torch.tensor(x, device=DEV), torch.tensor(e, device=DEV),
                                torch.tensor(crops, device=DEV), S, margin, lr)
    g = nl.nl_net_gradient(net)
    xb = np.stack([x[f, y0:y0 + S, x0:x0 + S] for f, y0, x0 in crops]).astype(np.float64)
    eb = np.stack([e[f, y0:y0 + S, x0:x0 + S] for f, y0, x0 in crops]).astype(np.float64)
    ref_loss, ref_g = convnet.loss_and_grad(w, xb, eb, margin=margin)
    assert abs(loss - ref_loss) < 1e-5 * max(1.0, ref_loss)
    assert np.linalg.norm(g - ref_g) / np.linalg.norm(ref_g) < 1e-4
    w1 = nl.nl_net_get_weights(net)
    ref_w1, _, _ = convnet.adam(w.astype(np.float64), g.astype(np.float64), np.zeros_like(g),
                                np.zeros_like(g), 1, lr)
    np.testing.assert_allclose(w1, ref_w1, rtol=0, atol=1e-6)


def test_apply_matches_oracle_preconditioner():
    n = 64
    fld = synth.heterogeneous_2d(n=n, seed=5)
    plan = nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=fld["a"], symmetric=True)
    w = _w(6, 0.1)
    net = nl.nl_net_create(w)
    r = synth.cg_rhs(n, seed=7, count=2)
    rt = torch.tensor(r, device=DEV)
    zt = torch.empty_like(rt)
    nl.nl_net_apply(net, plan, rt, zt)
    torch.cuda.synchronize()
    dinv = 1.0 / oracle.direct_diag(2, n, fld["delta"], alpha=1.5, coef=oracle.COEF_XY,
                                    a=fld["a"], symmetric=True)
    for k in range(2):
        ref = convnet.apply_preconditioner(w, r[k], dinv, n)
        err = np.linalg.norm(zt[k].cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err < 2e-5, err


def test_flexible_cg_with_trained_network_converges():
    n = 64
    fld = synth.heterogeneous_2d(n=n, seed=8)
    plan = nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=fld["a"], symmetric=True)
    x, e = precond.collect_pairs(plan, n, seeds=range(100, 106), cap=32)
    net = nl.nl_net_create(precond.init_weights(0))
    hist = precond.train(net, x, e, pairs=2048, crop=32, batch=32, epochs=2, lr=2e-3,
                         log_every=16)
    assert hist[-1][2] < hist[0][2]                    # the loss went down
    nl.nl_plan_set_net(plan, net)
    f = synth.cg_rhs(n, seed=999, count=2)
    ft = torch.tensor(f, device=DEV)
    xt = torch.empty_like(ft)
    st = nl.nl_cg_solve(plan, ft, xt, rtol=1e-8, maxit=20000, precond=nl.NL_PRECOND_LEARNED)
    assert st["converged"], st
    Lx = oracle.direct_scalar(xt.cpu().numpy(), 2, n, fld["delta"], alpha=1.5,
                              coef=oracle.COEF_XY, a=fld["a"], symmetric=True)
    res = np.linalg.norm(f + Lx, axis=1) / np.linalg.norm(f, axis=1)
    assert np.all(res <= 1.01e-8), res


# ---------------------------------------------------------------------------
# two-level form: M = D^-1 + gamma P K^T K R
# ---------------------------------------------------------------------------
def _sym_plan(n, seed):
    fld = synth.heterogeneous_2d(n=n, seed=seed)
    plan = nl.nl_plan_create(2, n, fld["delta"], family=nl.NL_POWER, alpha=1.5,
                             coef=nl.NL_COEF_XY, a=fld["a"], symmetric=True)
    dinv = 1.0 / oracle.direct_diag(2, n, fld["delta"], alpha=1.5, coef=oracle.COEF_XY,
                                    a=fld["a"], symmetric=True)
    return fld, plan, dinv


@pytest.mark.parametrize("n,block", [(50, 8), (64, 16), (33, 2)])
def test_two_level_apply_matches_oracle(n, block):
    fld, plan, dinv = _sym_plan(n, 21)
    w = precond.init_weights(3, two_level=True)
    net = nl.nl_net_create(w)
    nl.nl_net_set_coarse(net, block)
    r = synth.cg_rhs(n, seed=22, count=2)
    rt = torch.tensor(r, device=DEV)
    zt = torch.full_like(rt, float("nan"))
    nl.nl_net_apply(net, plan, rt, zt)
    torch.cuda.synchronize()
    ref = convnet.apply_two_level(w, r, dinv, n, block)
    err = np.linalg.norm(zt.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < 1e-5, err


def test_two_level_energy_gradient_matches_oracle():
    n, block, B = 32, 4, 3
    fld, plan, dinv = _sym_plan(n, 23)
    apply_A = lambda v: -oracle.direct_scalar(v, 2, n, fld["delta"], alpha=1.5,
                                              coef=oracle.COEF_XY, a=fld["a"], symmetric=True)
    rng = np.random.default_rng(24)
    e64 = np.stack([synth.gaussian_field(rng, 2, n).reshape(-1) for _ in range(B)])
    r64 = apply_A(e64)
    xo = torch.empty((B, n * n), dtype=torch.float32, device=DEV)
    eo = torch.empty_like(xo)
    nl.nl_net_prepare_pairs(plan, torch.tensor(r64, device=DEV), torch.tensor(e64, device=DEV),
                            xo, eo)
    w = precond.init_weights(5, two_level=True)
    net = nl.nl_net_create(w)
    nl.nl_net_set_coarse(net, block)
    idx = torch.arange(B, dtype=torch.int32, device=DEV)
    loss = nl.nl_net_train_step_energy(net, plan, xo, eo, idx, 1e-9)
    g = nl.nl_net_gradient(net)
    x = xo.double().cpu().numpy()
    ref_loss, ref_g = convnet.two_level_energy_loss_and_grad(w, x / dinv, eo.double().cpu().numpy(),
                                                             dinv, n, block, apply_A)
    assert abs(loss - ref_loss) < 1e-4 * max(1.0, abs(ref_loss)), (loss, ref_loss)
    assert np.linalg.norm(g - ref_g) / np.linalg.norm(ref_g) < 2e-3


def test_two_level_learned_cg_fewer_iterations_than_jacobi():
    n = 128
    fld, plan, dinv = _sym_plan(n, 0)
    x, e = precond.collect_pairs(plan, n, seeds=range(100, 112), cap=64)
    net = nl.nl_net_create(precond.init_weights(0, two_level=True))
    nl.nl_net_set_coarse(net, precond.coarse_block(n))
    precond.train_energy(net, plan, x, e, pairs=3200, batch=8, lr=3e-3)
    f = synth.cg_rhs(n, seed=998, count=3)
    ft = torch.tensor(f, device=DEV)
    xt = torch.empty_like(ft)
    sj = nl.nl_cg_solve(plan, ft, xt, rtol=1e-8, maxit=20000, precond=nl.NL_PRECOND_JACOBI)
    nl.nl_plan_set_net(plan, net)
    sl = nl.nl_cg_solve(plan, ft, xt, rtol=1e-8, maxit=20000, precond=nl.NL_PRECOND_LEARNED)
    assert sj["converged"] and sl["converged"], (sj, sl)
    assert sl["iterations"] < 0.75 * sj["iterations"], (sl, sj)
    Lx = oracle.direct_scalar(xt.cpu().numpy(), 2, n, fld["delta"], alpha=1.5,
                              coef=oracle.COEF_XY, a=fld["a"], symmetric=True)
    res = np.linalg.norm(f + Lx, axis=1) / np.linalg.norm(f, axis=1)
    assert np.all(res <= 1.01e-8), res


def test_two_level_cg_follows_buffer_moves_and_weight_updates():
    """A captured CG chunk must not outlive the network's buffers or weights: growing the
    apply workspace between solves gives the same solve bit for bit, and after a training
    step the solve equals that of a fresh network holding the updated weights."""
    n, block = 64, 8
    fld, plan, dinv = _sym_plan(n, 31)
    net = nl.nl_net_create(precond.init_weights(2, two_level=True))
    nl.nl_net_set_coarse(net, block)
    nl.nl_plan_set_net(plan, net)
    ft = torch.tensor(synth.cg_rhs(n, seed=32, count=2), device=DEV)
    x1 = torch.empty_like(ft)
    s1 = nl.nl_cg_solve(plan, ft, x1, rtol=1e-8, maxit=5000, precond=nl.NL_PRECOND_LEARNED)
    big = torch.tensor(synth.cg_rhs(n, seed=33, count=6), device=DEV)
    nl.nl_net_apply(net, plan, big, torch.empty_like(big))          # moves the workspace
    x2 = torch.empty_like(ft)
    s2 = nl.nl_cg_solve(plan, ft, x2, rtol=1e-8, maxit=5000, precond=nl.NL_PRECOND_LEARNED)
    assert s1["converged"] and s1["iterations"] == s2["iterations"], (s1, s2)
    assert torch.equal(x1, x2)
    xp, ep = precond.collect_pairs(plan, n, seeds=range(40, 42), cap=8)
    precond.train_energy(net, plan, xp, ep, pairs=16, batch=8, lr=1e-2)
    x3 = torch.empty_like(ft)
    s3 = nl.nl_cg_solve(plan, ft, x3, rtol=1e-8, maxit=5000, precond=nl.NL_PRECOND_LEARNED)
    net2 = nl.nl_net_create(nl.nl_net_get_weights(net))
    nl.nl_net_set_coarse(net2, block)
    nl.nl_plan_set_net(plan, net2)
    x4 = torch.empty_like(ft)
    s4 = nl.nl_cg_solve(plan, ft, x4, rtol=1e-8, maxit=5000, precond=nl.NL_PRECOND_LEARNED)
    assert s3["converged"] and s3["iterations"] == s4["iterations"], (s3, s4)
    assert torch.equal(x3, x4)
    assert not torch.equal(x1, x3)                                 # the weights did change


def test_history_pairs_match_pairs_from_oracle_residuals():
    # nl_net_history_pairs forms r_k = f + L x_k and e_k = x - x_k itself; the same pairs from
    # the oracle's FP64 residuals through nl_net_prepare_pairs must agree
    n, count = 32, 3
    fld, plan, dinv = _sym_plan(n, 31)
    rng = np.random.default_rng(32)
    f = synth.gaussian_field(rng, 2, n).reshape(-1)
    x = synth.gaussian_field(rng, 2, n).reshape(-1)
    H = np.stack([synth.gaussian_field(rng, 2, n).reshape(-1) for _ in range(count + 1)])
    Lh = oracle.direct_scalar(H[:count], 2, n, fld["delta"], alpha=1.5, coef=oracle.COEF_XY,
                              a=fld["a"], symmetric=True)
    r64 = f[None, :] + Lh
    e64 = x[None, :] - H[:count]
    xo_ref = torch.empty((count, n * n), dtype=torch.float32, device=DEV)
    eo_ref = torch.empty_like(xo_ref)
    nl.nl_net_prepare_pairs(plan, torch.tensor(r64, device=DEV), torch.tensor(e64, device=DEV),
                            xo_ref, eo_ref)
    xo = torch.full_like(xo_ref, float("nan"))
    eo = torch.full_like(xo_ref, float("nan"))
    nl.nl_net_history_pairs(plan, torch.tensor(f, device=DEV), torch.tensor(x, device=DEV),
                            torch.tensor(H, device=DEV), count, xo, eo)
    for got, ref in ((xo, xo_ref), (eo, eo_ref)):
        g, r = got.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.linalg.norm(g - r) / np.linalg.norm(r) < 1e-6
