"""Training the learned CG preconditioner from the solver's own Jacobi-CG runs.

Host-side orchestration only: every numerical step (CG with iterate history, residuals,
pair preparation, crop gathering, forward/backward/Adam) is a call into the C-ABI library.

Pairs: for a right-hand side f, Jacobi-CG records its iterate x_k every 16 iterations; with
x* the converged solution, e_k = x* - x_k is the error and r_k = f + L x_k the residual of
the iterate (-L e_k = r_k).  The network learns x = D^{-1} r_k / s -> e_k / s.
"""
from __future__ import annotations

import numpy as np

from . import binding as nl
from . import synth


def init_weights(seed=0, two_level=False, scale=1.0):
    """Seeded initial weights.  Local form: He-style, the last layer zero (the preconditioner
    starts as plain Jacobi).  Two-level form: variance-preserving for a linear chain in every
    layer (K = 0 would be a stationary point of the K^T K loss), times `scale`."""
    rng = np.random.default_rng(seed)
    if two_level:
        w1 = rng.standard_normal(32 * 1 * 9) * np.sqrt(1.0 / 9) * scale
        w2 = rng.standard_normal(32 * 32 * 9) * np.sqrt(1.0 / (32 * 9)) * scale
        w3 = rng.standard_normal(32 * 9) * np.sqrt(1.0 / (32 * 9)) * scale
        return np.concatenate([w1, w2, w3]).astype(np.float32)
    w1 = rng.standard_normal(32 * 1 * 9) * np.sqrt(2.0 / 9)
    w2 = rng.standard_normal(32 * 32 * 9) * np.sqrt(2.0 / (32 * 9))
    w3 = np.zeros(32 * 9)
    return np.concatenate([w1, w2, w3]).astype(np.float32)


def coarse_block(n, cells=16):
    """Block size giving about `cells` x `cells` coarse cells."""
    return max(2, -(-n // cells))


def collect_pairs(plan, n, seeds, cap=64, rtol=1e-10, device="cuda"):
    """Run Jacobi-CG for each seed; return CUDA tensors (x, e) [count, n, n] float32."""
    import torch
    xs, es = [], []
    for sd in seeds:
        f = torch.tensor(synth.cg_rhs(n, seed=sd)[0], dtype=torch.float64, device=device)
        x = torch.empty_like(f)
        hist = torch.empty((cap, n * n), dtype=torch.float64, device=device)
        cnt, st = nl.nl_cg_history(plan, f, x, hist, rtol=rtol, maxit=100000)
        if cnt < 2:
            continue
        count = cnt - 1                          # drop the last snapshot (~ converged)
        xo = torch.empty((count, n * n), dtype=torch.float32, device=device)
        eo = torch.empty_like(xo)
        nl.nl_net_history_pairs(plan, f, x, hist, count, xo, eo)
        xs.append(xo)
        es.append(eo)
    x = torch.cat(xs).reshape(-1, n, n).contiguous()
    e = torch.cat(es).reshape(-1, n, n).contiguous()
    return x, e


def train_energy(net, plan, x, e, pairs=20000, batch=8, lr=1e-3, seed=0, log_every=0):
    """Adam on the energy-norm loss over whole fields; `pairs` field samples in total."""
    import torch
    rng = np.random.default_rng(seed)
    nf = x.shape[0]
    xf = x.reshape(nf, -1)
    ef = e.reshape(nf, -1)
    losses = []
    steps = max(1, pairs // batch)
    for s in range(steps):
        idx = torch.tensor(rng.integers(0, nf, batch).astype(np.int32), device=x.device)
        want = log_every and (s % log_every == 0 or s == steps - 1)
        loss = nl.nl_net_train_step_energy(net, plan, xf, ef, idx, lr, want_loss=bool(want))
        if want:
            losses.append((0, s, loss))
    return losses


def train(net, x, e, pairs=20000, crop=64, margin=3, batch=64, epochs=2, lr=1e-3, seed=0,
          log_every=0):
    """Adam on `pairs` random crops (field, y0, x0) per epoch; returns the loss history."""
    import torch
    rng = np.random.default_rng(seed)
    nf, n, _ = x.shape
    losses = []
    steps = max(1, pairs // batch)
    for ep in range(epochs):
        for s in range(steps):
            c = np.stack([rng.integers(0, nf, batch), rng.integers(0, n - crop + 1, batch),
                          rng.integers(0, n - crop + 1, batch)], axis=1).astype(np.int32)
            ct = torch.tensor(c, device=x.device)
            want = log_every and (s % log_every == 0 or s == steps - 1)
            loss = nl.nl_net_train_step(net, x, e, ct, crop, margin, lr, want_loss=bool(want))
            if want:
                losses.append((ep, s, loss))
    return losses
