"""Plain numpy reference of the CG preconditioner network.  TEST INFRASTRUCTURE ONLY.

The paper has no counterpart for this network (it only remarks, in its conclusion, that
the fast product can serve a Krylov method); it is a project addition.  Definition:

    x   = D^{-1} r / s            (Jacobi-scaled residual, s its RMS)
    y1  = relu(conv1(x))          conv1: 1 -> 32 channels, 3x3, zero padding, no bias
    y2  = relu(conv2(y1))         conv2: 32 -> 32
    o   = conv3(y2)               conv3: 32 -> 1
    M(r) = s (x + o)              (Jacobi plus a learned correction)

Weights use the [out][in][3][3] layout and are rounded to bfloat16 before use
(round to nearest even); sums are in float64 here.  conv(x)[o, y, x'] =
sum_{c, dy, dx} W[o, c, dy, dx] * x[c, y + dy - 1, x' + dx - 1].

Training loss per sample b over the interior (a margin of `margin` pixels dropped):
    L_b = sum (x + o - e)^2 / sum e^2,  loss = mean_b L_b.
Gradients are the adjoint of each step, written out below; Adam is the usual update.

Two-level form (the preconditioner the CG uses with a coarse block size b >= 2).  The same
three layers without activations make one linear map K (1 -> 32 -> 32 -> 1 channels) applied
on a coarse grid of ceil(n/b)^2 cells; with R the sum over each b x b block (cells cut by the
grid edge sum what they hold) and P = R^T the piecewise-constant prolongation,
    M(r) = D^{-1} r + gamma P K^T K R r,    gamma = 1 / (b^2 mean(diag A)),   A = -L,
which is symmetric positive definite for any weights (K^T K is positive semi-definite).
Training minimises the energy norm of the preconditioned step's error over pairs (r, e),
A e = r:  loss = (z - e)^T A (z - e) / e^T A e  with z = M r, averaged over the batch.

Parity pins (tests/test_oracle_convnet.py): forward against torch.nn.functional.conv2d
(an independent library routine), the gradients against central finite differences, the
two-level map against a dense matrix built from its definition (symmetry, definiteness).
"""
from __future__ import annotations

import numpy as np

SHAPES = [(32, 1), (32, 32), (1, 32)]
NPARAM = sum(o * i * 9 for o, i in SHAPES)


def split(w):
    """Flat weight vector -> [W1, W2, W3] in [out][in][3][3]."""
    out, k = [], 0
    for o, i in SHAPES:
        out.append(np.asarray(w[k:k + o * i * 9], dtype=np.float64).reshape(o, i, 3, 3))
        k += o * i * 9
    return out


def bf16_round(w):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (a >> 16) & 1
    a = ((a + 0x7FFF + lsb) >> 16) << 16
    return a.astype(np.uint32).view(np.float32).astype(np.float64)


def conv(x, W):
    """x: [B, C, H, W]; W: [O, C, 3, 3] -> [B, O, H, W], zero padding."""
    B, C, H, Wd = x.shape
    xp = np.zeros((B, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.zeros((B, W.shape[0], H, Wd))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + H, dx:dx + Wd]
            out += np.einsum("bchw,oc->bohw", patch, W[:, :, dy, dx])
    return out


def conv_adjoint_input(g, W):
    """Adjoint of conv w.r.t. its input: g [B, O, H, W] -> [B, C, H, W]."""
    B, O, H, Wd = g.shape
    out = np.zeros((B, W.shape[1], H + 2, Wd + 2))
    for dy in range(3):
        for dx in range(3):
            out[:, :, dy:dy + H, dx:dx + Wd] += np.einsum("bohw,oc->bchw", g, W[:, :, dy, dx])
    return out[:, :, 1:-1, 1:-1]


def conv_adjoint_weight(x, g):
    """Gradient of sum(g * conv(x, W)) w.r.t. W: [O, C, 3, 3]."""
    B, C, H, Wd = x.shape
    xp = np.zeros((B, C, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    dW = np.zeros((g.shape[1], C, 3, 3))
    for dy in range(3):
        for dx in range(3):
            dW[:, :, dy, dx] = np.einsum("bohw,bchw->oc", g, xp[:, :, dy:dy + H, dx:dx + Wd])
    return dW


def forward(w, x, round_bf16=True):
    """x: [B, H, W] scaled input.  Returns o [B, H, W] and the activations."""
    Ws = split(bf16_round(w) if round_bf16 else np.asarray(w, dtype=np.float64))
    a0 = np.asarray(x, dtype=np.float64)[:, None]
    y1 = np.maximum(conv(a0, Ws[0]), 0.0)
    y2 = np.maximum(conv(y1, Ws[1]), 0.0)
    o = conv(y2, Ws[2])[:, 0]
    return o, (a0, y1, y2, Ws)


def loss_and_grad(w, x, e, margin=3, round_bf16=True):
    """Mean over samples of sum_int (x + o - e)^2 / sum_int e^2, and its gradient."""
    o, (a0, y1, y2, Ws) = forward(w, x, round_bf16)
    B, H, Wd = o.shape
    m = np.zeros((H, Wd))
    m[margin:H - margin, margin:Wd - margin] = 1.0
    diff = (x + o - e) * m
    ee = ((e * m) ** 2).sum(axis=(1, 2))
    loss = float(np.mean((diff ** 2).sum(axis=(1, 2)) / ee))
    go = 2.0 * diff / ee[:, None, None] / B                 # d loss / d o
    g3 = go[:, None]
    dW3 = conv_adjoint_weight(y2, g3)
    g2 = conv_adjoint_input(g3, Ws[2]) * (y2 > 0)
    dW2 = conv_adjoint_weight(y1, g2)
    g1 = conv_adjoint_input(g2, Ws[1]) * (y1 > 0)
    dW1 = conv_adjoint_weight(a0, g1)
    grad = np.concatenate([dW1.ravel(), dW2.ravel(), dW3.ravel()])
    return loss, grad


def adam(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1).  Returns new (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def apply_preconditioner(w, r, dinv, n):
    """M(r) for one field r [n*n] with inverse diagonal dinv [n*n]."""
    xin = dinv * r
    s = np.sqrt(np.mean(xin * xin))
    if s == 0:
        return np.zeros_like(r)
    o, _ = forward(w, (xin / s).reshape(1, n, n))
    return s * (xin / s + o.reshape(-1))


# ---------------------------------------------------------------------------
# two-level form
# ---------------------------------------------------------------------------
def coarse_size(n, b):
    return -(-n // b)


def restrict(r, n, b):
    """R r: sums over b x b blocks.  r: [..., n*n] -> [..., nc, nc]."""
    nc = coarse_size(n, b)
    r = np.asarray(r, dtype=np.float64)
    lead = r.shape[:-1]
    pad = np.zeros(lead + (nc * b, nc * b))
    pad[..., :n, :n] = r.reshape(lead + (n, n))
    return pad.reshape(lead + (nc, b, nc, b)).sum(axis=(-3, -1))


def prolong(zc, n, b):
    """P zc = R^T zc: each fine node takes its block's value.  [..., nc, nc] -> [..., n*n]."""
    zc = np.asarray(zc, dtype=np.float64)
    full = np.repeat(np.repeat(zc, b, axis=-2), b, axis=-1)
    return full[..., :n, :n].reshape(zc.shape[:-2] + (n * n,))


def linear_chain(Ws, x):
    """K x for x [B, H, W] (no activations); returns the activations too."""
    a0 = np.asarray(x, dtype=np.float64)[:, None]
    a1 = conv(a0, Ws[0])
    a2 = conv(a1, Ws[1])
    u = conv(a2, Ws[2])
    return u[:, 0], (a0, a1, a2)


def linear_chain_adjoint(Ws, y):
    """K^T y for y [B, H, W]."""
    g = np.asarray(y, dtype=np.float64)[:, None]
    g = conv_adjoint_input(g, Ws[2])
    g = conv_adjoint_input(g, Ws[1])
    g = conv_adjoint_input(g, Ws[0])
    return g[:, 0]


def chain_weight_grad(Ws, acts, gy):
    """Gradient of sum(gy * K x) w.r.t. the three weights, given the chain's activations."""
    a0, a1, a2 = acts
    g3 = np.asarray(gy, dtype=np.float64)[:, None]
    dW3 = conv_adjoint_weight(a2, g3)
    g2 = conv_adjoint_input(g3, Ws[2])
    dW2 = conv_adjoint_weight(a1, g2)
    g1 = conv_adjoint_input(g2, Ws[1])
    dW1 = conv_adjoint_weight(a0, g1)
    return np.concatenate([dW1.ravel(), dW2.ravel(), dW3.ravel()])


def two_level_gamma(dinv, b):
    """gamma = 1 / (b^2 mean(diag A)) from the inverse diagonal."""
    return 1.0 / (b * b * float(np.mean(1.0 / np.asarray(dinv, dtype=np.float64))))


def apply_two_level(w, r, dinv, n, b, round_bf16=True):
    """M(r) = D^{-1} r + gamma P K^T K R r for r [..., n*n]."""
    Ws = split(bf16_round(w) if round_bf16 else np.asarray(w, dtype=np.float64))
    r = np.asarray(r, dtype=np.float64)
    lead = r.shape[:-1]
    rc = restrict(r.reshape((-1, n * n)), n, b)
    u, _ = linear_chain(Ws, rc)
    zc = linear_chain_adjoint(Ws, u)
    z = np.asarray(dinv) * r.reshape((-1, n * n)) + two_level_gamma(dinv, b) * prolong(zc, n, b)
    return z.reshape(lead + (n * n,))


def two_level_energy_loss_and_grad(w, r, e, dinv, n, b, apply_A, round_bf16=True):
    """Mean over samples of (z - e)^T A (z - e) / e^T r with z = M r, A e = r, and its
    gradient.  r, e: [B, n*n]; apply_A(v) applies A = -L to [B, n*n]."""
    Ws = split(bf16_round(w) if round_bf16 else np.asarray(w, dtype=np.float64))
    r = np.asarray(r, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    B = r.shape[0]
    gam = two_level_gamma(dinv, b)
    rc = restrict(r, n, b)
    u, acts_r = linear_chain(Ws, rc)
    zc = linear_chain_adjoint(Ws, u)
    z = np.asarray(dinv) * r + gam * prolong(zc, n, b)
    Az = apply_A(z)
    er = np.sum(e * r, axis=1)
    loss = float(np.mean((np.sum(z * Az, axis=1) - 2 * np.sum(z * r, axis=1) + er) / er))
    go = 2.0 * (Az - r) / er[:, None] / B                 # d loss / d z (A symmetric)
    g = gam * restrict(go, n, b)                          # d loss / d (K^T K rc)
    v, acts_g = linear_chain(Ws, g)
    # d <g, K^T K rc> = <v, dK rc> + <u, dK g>
    grad = chain_weight_grad(Ws, acts_r, v) + chain_weight_grad(Ws, acts_g, u)
    return loss, grad
