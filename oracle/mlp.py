"""MLP oracle for the learned rewrite picker -- TEST INFRASTRUCTURE ONLY.

Plain numpy float64 forward pass, hand-written backward pass and Adam step of the
picker network: 12 inputs -> 64 -> 64 -> 64 (ReLU) -> 1 output.  The paper names a
learned transformation strategy as future work (Conclusion); nothing here comes from
its text beyond that.  Parameter layout (flat vector, layer by layer):
W1[64][12], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[1][64], b4[1].

bfloat16 mode rounds every parameter to bfloat16 (round to nearest even) before use;
arithmetic stays float64.  Inputs are normalised as (f - mean) / std, targets are
divided by target_scale; the loss is the mean squared error.
"""
from __future__ import annotations

import numpy as np

F, H = 12, 64
SHAPES = [(H, F), (H,), (H, H), (H,), (H, H), (H,), (1, H), (1,)]
NPARAM = sum(int(np.prod(s)) for s in SHAPES)


def unpack(p: np.ndarray) -> list[np.ndarray]:
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(p[o:o + k].reshape(s))
        o += k
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def effective_params(p: np.ndarray, bf16: bool) -> np.ndarray:
    """float64 view of the parameters; bfloat16 mode first rounds them to float32, then
    to bfloat16."""
    if bf16:
        return bf16_round(np.asarray(p, dtype=np.float32))
    return np.asarray(p, dtype=np.float64)


def forward(p, X, mean=None, std=None, bf16=False, keep=False):
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(effective_params(p, bf16))
    X = np.asarray(X, dtype=np.float64)
    mean = np.zeros(F) if mean is None else np.asarray(mean, dtype=np.float64)
    std = np.ones(F) if std is None else np.asarray(std, dtype=np.float64)
    x0 = (X - mean) / std
    z1 = x0 @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ W3.T + b3
    h3 = np.maximum(z3, 0.0)
    y = (h3 @ W4.T + b4)[:, 0]
    if keep:
        return y, (x0, z1, h1, z2, h2, z3, h3)
    return y


def loss_and_grad(p, X, t, mean=None, std=None, target_scale=1.0, bf16=False):
    """Mean squared error of forward(X) against t / target_scale and its gradient with
    respect to every parameter (through the bfloat16-rounded weights in bf16 mode)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(effective_params(p, bf16))
    y, (x0, z1, h1, z2, h2, z3, h3) = forward(p, X, mean, std, bf16, keep=True)
    n = y.size
    tt = np.asarray(t, dtype=np.float64) / target_scale
    r = y - tt
    loss = float(np.mean(r * r))
    dy = (2.0 / n) * r                      # dL/dy
    gW4 = dy[None, :] @ h3                  # (1, H)
    gb4 = np.array([dy.sum()])
    dh3 = dy[:, None] * W4                  # (N, H)
    dz3 = dh3 * (z3 > 0)
    gW3 = dz3.T @ h2
    gb3 = dz3.sum(axis=0)
    dh2 = dz3 @ W3
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ x0
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)])
    return loss, g


def adam_step(p, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int) -> np.ndarray:
    """Kaiming-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for s in SHAPES:
        if len(s) == 2:
            bound = np.sqrt(6.0 / s[1])
            parts.append(rng.uniform(-bound, bound, size=s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts).astype(np.float32)
