"""FP64 oracle of the per-element MLP preconditioner (test infrastructure).

Network: x (n_in) -> relu(W1 x + b1) (h) -> relu(W2 . + b2) (h) -> W3 . + b3 + Ws x_v (n_out),
where x_v is the first n_out entries of x (the scaled vector block) and Ws a learned
linear skip map.
Its input is an element block scaled to unit 2-norm, followed (when state features
are used) by the element's state block: x = [v_K / ||v_K||, u_K], and
    M(v)_K = ||v_K|| * net(v_K / ||v_K||, u_K).
Training pairs (v_K, z_K, u_K): the loss is the mean over valid pairs of
||net(v/||v||, u) - z/||v|| ||^2.
Parameter order (flat vector): W1 [h][n_in], b1 [h], W2 [h][h], b2 [h], W3 [n_out][h], b3 [n_out],
Ws [n_out][n_out].

Plain numpy, written from the definitions (forward pass, chain rule, Adam).
"""
from __future__ import annotations

import numpy as np


def shapes(n_in: int, hidden: int, n_out: int):
    return [(hidden, n_in), (hidden,), (hidden, hidden), (hidden,), (n_out, hidden), (n_out,), (n_out, n_out)]


def unflatten(theta, n_in, hidden, n_out):
    out, o = [], 0
    for s in shapes(n_in, hidden, n_out):
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    return out


def normalise(X, T, tiny=1e-30, U=None):
    """Row-wise scaling by ||x|| (state rows U appended unscaled); rows with
    ||x|| <= tiny are dropped (mask 0)."""
    nrm = np.linalg.norm(X, axis=1)
    mask = nrm > tiny
    s = np.where(mask, 1.0 / np.where(mask, nrm, 1.0), 0.0)
    Xn = X * s[:, None]
    if U is not None:
        Xn = np.hstack([Xn, U])
    return Xn, T * s[:, None], mask


def round_bf16(x):
    """Nearest BF16 value (8-bit significand, ties to even) of each entry, via its FP32
    bit pattern, returned as FP64."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    f = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000
    return f.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, Xn, n_in, hidden, n_out, act_round=None):
    """act_round (optional) is applied to the network input and to both hidden
    activations before they enter the next layer (storage precision of a kernel)."""
    W1, b1, W2, b2, W3, b3, Ws = unflatten(theta, n_in, hidden, n_out)
    r = act_round if act_round is not None else (lambda a: a)
    Xr = r(Xn)
    Z1 = Xr @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    H1r = r(H1)
    Z2 = H1r @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    Y = r(H2) @ W3.T + b3 + Xr[:, :n_out] @ Ws.T
    return Y, (Z1, H1, Z2, H2)


def loss_grad(theta, X, T, n_in, hidden, n_out, U=None):
    """Mean squared error over the valid pairs and its gradient (chain rule)."""
    Xn, Tn, mask = normalise(X, T, U=U)
    cnt = max(int(mask.sum()), 1)
    W1, b1, W2, b2, W3, b3, Ws = unflatten(theta, n_in, hidden, n_out)
    Y, (Z1, H1, Z2, H2) = forward(theta, Xn, n_in, hidden, n_out)
    E = (Y - Tn) * mask[:, None]
    loss = float((E * E).sum() / cnt)
    dY = 2.0 * E / cnt
    gW3 = dY.T @ H2
    gb3 = dY.sum(0)
    dH2 = (dY @ W3) * (Z2 > 0)
    gW2 = dH2.T @ H1
    gb2 = dH2.sum(0)
    dH1 = (dH2 @ W2) * (Z1 > 0)
    gW1 = dH1.T @ Xn
    gb1 = dH1.sum(0)
    gWs = dY.T @ Xn[:, :n_out]
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3, gWs.ravel()])
    return loss, g


def apply(theta, v_blocks, n_in, hidden, n_out, U=None, act_round=None):
    """M(v)_K = ||v_K|| net(v_K / ||v_K||[, u_K]) for blocks v [E][n]."""
    nrm = np.linalg.norm(v_blocks, axis=1)
    safe = np.where(nrm > 0, nrm, 1.0)
    x = v_blocks / safe[:, None]
    if U is not None:
        x = np.hstack([x, U])
    Y, _ = forward(theta, x, n_in, hidden, n_out, act_round)
    return Y * nrm[:, None]


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) in place; t counts from 1."""
    m[:] = b1 * m + (1 - b1) * g
    v[:] = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    theta -= lr * mh / (np.sqrt(vh) + eps)
